"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random inputs with the shapes and distributions of the
workloads (daxpy vectors, 3D grids, CSR matrices, n-body clouds, mixed call
streams).  It holds none of the method's arithmetic: no loop body, no feature
reduction, no selection logic.  Both the oracle (``oracle/``) and the CUDA
package consume what it returns, so neither needs to import the other.

Random draws use ``numpy.random.Generator(PCG64(seed))`` on the host, or a
seeded ``torch.Generator`` on a device for the large CSR matrices whose host
generation would take minutes (``device=`` argument).  The same call with the
same arguments always returns the same values on the same device kind.
"""
from .gen import (  # noqa: F401
    daxpy_inputs,
    grid_inputs,
    linear_field,
    sine_mode,
    nbody_inputs,
    nbody_batch_sizes,
    nbody_batch_inputs,
    zipf_row_lengths,
    csr_zipf,
    csr_band,
    csr_from_lengths,
    spmv_matrix_params,
    spmv_matrix,
    spmv_x,
    mixed_stream,
    DAXPY_A,
    NBODY_EPS,
)
