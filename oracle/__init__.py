"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct CPU implementations of what the adaptive-region
hot path computes, used to check the CUDA library and nothing else.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does, and the two share
no code (the seeded generators in ``synth/`` feed both).

* ``loops``  -- the four region bodies in float64 C (``oracle/loops.c``).
* ``select`` -- variant ranges, records, labels, exhaustive argmin, regret and
  the depth-limited CART decision tree (Section 2, Section 3.1, Table 1).
* ``mlp``    -- the 3-layer MLP selector: forward, cross-entropy backward and
  Adam in float64 numpy.
"""
from . import loops, select, mlp  # noqa: F401
