"""The no-allocation merge-path SpMV entry point against the regular one.

Some callers cannot allocate device memory (a plug-in whose device memory is
owned by another allocator, a loop that must not pay the synchronisation of
cudaMalloc/cudaFree).  ar_spmv_merge_path_noalloc serves them from a fixed
scratch array inside the library.  This file is collected last so that a
run stopping at the first failure has already run every other test.  The
capacity checks run before any device work, so they need no GPU.
"""
import numpy as np
import pytest

import paper_2303_08873_b300 as ar

TOL = 1e-10  # per row: |y - y_ref| <= TOL * sum_k |val_k x_col_k|, as in the SpMV tests
MAX_PATH = 349525 * 4096  # (8 MiB - 8) // 24 blocks of 4096 path items
INT32_MAX = (1 << 31) - 1


def test_noalloc_capacity_constant():
    assert MAX_PATH == ((8 << 20) - 8) // 24 * 4096 == 1431654400


@pytest.mark.parametrize("rows,nnz", [
    (MAX_PATH - INT32_MAX + 1, INT32_MAX),  # rows + nnz = MAX_PATH + 1
    (MAX_PATH + 1, 0),
    ((1 << 63) - 1, 0),                      # a sum with nnz would overflow int64
    ((1 << 63) - 1, INT32_MAX),
    ((1 << 30), INT32_MAX),
])
def test_noalloc_rejects_sizes_beyond_capacity(rows, nnz):
    # dummy non-null pointers: the size check rejects the call before any use
    got = ar.lib.ar_spmv_merge_path_noalloc(rows, nnz, 16, 16, 16, 16, 16, None)
    assert got == ar.AR_ERR_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("case", [("zipf", 200000, 1.5), ("band", 50000, 129)])
def test_noalloc_matches_regular_entry_point_twice(case):
    import torch

    import synth
    from oracle import loops
    from tests.gpu_util import dev, host

    kind, rows, p = case
    rp, c, v = synth.csr_zipf(5, rows, p) if kind == "zipf" else synth.csr_band(5, rows, p)
    rp, c, v = rp.numpy(), c.numpy(), v.numpy()
    x = synth.spmv_x(5, rows).numpy()
    nnz = int(rp[-1])
    d = (dev(rp), dev(c), dev(v), dev(x))
    _, absum = loops.spmv_rows(rp, c, v, x, np.arange(rows))
    y = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
    wsb = ar.ar_spmv_workspace_bytes(6, rows, nnz)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ar.ar_spmv(6, rows, nnz, *d, y, ws, wsb)
    ref = host(y)
    for _ in range(2):  # two calls in a row share the fixed scratch
        y.fill_(np.nan)
        ar.ar_spmv_merge_path_noalloc(rows, nnz, *d, y)
        got = host(y)
        assert np.all(np.abs(got - ref) <= TOL * absum)


@pytest.mark.gpu
def test_noalloc_at_exact_capacity():
    """rows + nnz == MAX_PATH: the last path block ends on the scratch's last
    carry word.  A synthetic matrix (2^24 rows of 84-85 nonzeros, hashed
    columns, dyadic values) built on the device in chunks; ~18 GB resident."""
    import torch

    from oracle import loops

    rows = 1 << 24
    nnz = MAX_PATH - rows
    cuda = torch.device("cuda")
    i = torch.arange(rows + 1, dtype=torch.int64, device=cuda)
    rowptr = ((i * nnz) // rows).to(torch.int32)
    del i
    col = torch.empty(nnz, dtype=torch.int32, device=cuda)
    val = torch.empty(nnz, dtype=torch.float64, device=cuda)
    chunk = 1 << 27
    for k0 in range(0, nnz, chunk):
        k = torch.arange(k0, min(nnz, k0 + chunk), dtype=torch.int64, device=cuda)
        col[k0:k0 + k.numel()] = ((k * 2654435761) % rows).to(torch.int32)
        val[k0:k0 + k.numel()] = ((k * 40503) % 2048 - 1024).to(torch.float64) / 1024.0
        del k
    j = torch.arange(rows, dtype=torch.int64, device=cuda)
    x = ((j * 7) % 1000 - 500).to(torch.float64) / 512.0
    del j
    y_ref = torch.full((rows,), np.nan, dtype=torch.float64, device=cuda)
    wsb = ar.ar_spmv_workspace_bytes(6, rows, nnz)
    ws = torch.empty(wsb, dtype=torch.uint8, device=cuda)
    ar.ar_spmv(6, rows, nnz, rowptr, col, val, x, y_ref, ws, wsb)
    y = torch.full((rows,), np.nan, dtype=torch.float64, device=cuda)
    ar.ar_spmv_merge_path_noalloc(rows, nnz, rowptr, col, val, x, y)
    torch.cuda.synchronize()
    # the same kernels with the same partition: identical to the last bit
    assert torch.equal(y, y_ref)
    # sampled rows, including the last ones, against the oracle
    pick = np.unique(np.r_[np.random.default_rng(9).integers(0, rows, 256), rows - 3, rows - 2, rows - 1])
    rp_h = rowptr.cpu().numpy().astype(np.int64)
    segs = [np.arange(rp_h[r], rp_h[r + 1]) for r in pick]
    idx = torch.from_numpy(np.concatenate(segs)).to(cuda)
    sub_rp = np.r_[0, np.cumsum([len(s) for s in segs])].astype(np.int32)
    sub_c, sub_v = col[idx].cpu().numpy(), val[idx].cpu().numpy()
    ref, absum = loops.spmv_rows(sub_rp, sub_c, sub_v, x.cpu().numpy(), np.arange(len(pick)))
    got = y.cpu().numpy()[pick]
    assert np.all(np.abs(got - ref) <= TOL * absum)
