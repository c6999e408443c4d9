"""The no-allocation merge-path SpMV entry point against the regular one (GPU).

Some callers cannot allocate device memory (a plug-in whose device memory is
owned by another allocator, a loop that must not pay the synchronisation of
cudaMalloc/cudaFree).  ar_spmv_merge_path_noalloc serves them from a fixed
scratch array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
TOL = 1e-10  # per row: |y - y_ref| <= TOL * sum_k |val_k x_col_k|, as in the SpMV tests


def _regular(rows, nnz, d):
    y = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
    wsb = ar.ar_spmv_workspace_bytes(6, rows, nnz)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ar.ar_spmv(6, rows, nnz, *d, y, ws, wsb)
    return host(y)


def _noalloc(rows, nnz, d):
    y = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
    ar.ar_spmv_merge_path_noalloc(rows, nnz, *d, y)
    return host(y)


@pytest.mark.parametrize("case", [("zipf", 200000, 1.5), ("band", 50000, 129)])
def test_noalloc_matches_regular_entry_point_twice(case):
    kind, rows, p = case
    rp, c, v = synth.csr_zipf(5, rows, p) if kind == "zipf" else synth.csr_band(5, rows, p)
    rp, c, v = rp.numpy(), c.numpy(), v.numpy()
    x = synth.spmv_x(5, rows).numpy()
    nnz = int(rp[-1])
    d = (dev(rp), dev(c), dev(v), dev(x))
    _, absum = loops.spmv_rows(rp, c, v, x, np.arange(rows))
    ref = _regular(rows, nnz, d)
    for _ in range(2):  # two calls in a row share the fixed scratch
        got = _noalloc(rows, nnz, d)
        assert np.all(np.abs(got - ref) <= TOL * absum)


def test_noalloc_rejects_sizes_beyond_capacity():
    big = ar.lib.ar_spmv_merge_path_noalloc(1 << 30, (1 << 31) - 1, 16, 16, 16, 16, 16, None)
    assert big == ar.AR_ERR_ARG
