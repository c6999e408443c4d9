"""daxpy variants against the float64 oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
V = 15


def _run(v, a, x, y):
    xd, yd = dev(x), dev(y)
    ar.ar_daxpy(v, x.size, a, xd, yd)
    return host(yd)


@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 4097, 1000003, 1 << 20])
def test_all_variants_match_oracle(n):
    a, x, y = synth.daxpy_inputs(1, n)
    ref = loops.daxpy(a, x, y)
    scale = np.abs(a * x) + np.abs(y)
    for v in range(V):
        out = _run(v, a, x, y)
        bad = np.abs(out - ref) > 1e-13 * scale
        assert not bad.any(), (v, n, np.flatnonzero(bad)[:5])


def test_dyadic_inputs_are_exact_in_every_variant():
    r = np.random.Generator(np.random.PCG64(3))
    n = 65537
    x = r.integers(-2**20, 2**20, n) / 2.0**20
    y = r.integers(-2**20, 2**20, n) / 2.0**20
    ref = loops.daxpy(1.5, x, y)
    for v in range(V):
        assert np.array_equal(_run(v, 1.5, x, y), ref), v


def test_a_zero_and_identity_cases_bitwise():
    _, x, y = synth.daxpy_inputs(5, 3001)
    for v in range(V):
        assert np.array_equal(_run(v, 0.0, x, y), y)
        assert np.array_equal(_run(v, 1.0, x, np.zeros_like(x)), x)


def test_empty_and_stream_argument():
    s = torch.cuda.Stream()
    _, x, y = synth.daxpy_inputs(1, 1000)
    xd, yd = dev(x), dev(y)
    ar.ar_daxpy(0, 0, 1.5, xd, yd, stream=s)
    ar.ar_daxpy(8, 1000, 1.5, xd, yd, stream=s)
    s.synchronize()
    assert np.allclose(yd.cpu().numpy(), loops.daxpy(1.5, x, y), rtol=0, atol=1e-15)


def test_region_exhaustive_profile_and_invoke():
    n = 1 << 20
    a, x, y = synth.daxpy_inputs(1, n)
    xd, yd = dev(x), dev(y)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    r = ar.Region("daxpy", 1, "exhaustive,reps=5")
    assert r.add_builtin(ar.AR_LOOP_DAXPY) == V
    r.set_l2_flush(flush, flush.numel())
    args = ar.ArDaxpyArgs(n, a, xd.data_ptr(), yd.data_ptr())
    ms, best = r.profile([n], args)
    assert all(np.isfinite(ms)) and all(t > 0 for t in ms)
    assert len(r.records()) == V * 5
    # profiling ran every variant 6 times in place: y = y0 + 6*15*a*x
    yd.copy_(dev(y))
    v, val = r.invoke([n], args)
    assert v == best and val == float(best)
    assert np.allclose(host(yd), loops.daxpy(a, x, y), rtol=0, atol=1e-14)
