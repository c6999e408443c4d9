"""CSR SpMV variants and the row-feature reduction against the oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
V = ar.loop_num_variants(2)
DF = [v for v in range(V) if "_df_" in ar.loop_variant_name(2, v)]  # float-pair arithmetic
TOL = 1e-10  # |y - y_ref| <= TOL * sum_k |val_k x_col_k| per row


def _run(v, rp, c, val, x, dev_arrays=None):
    rows = rp.size - 1
    nnz = int(rp[-1])
    d = dev_arrays or (dev(rp), dev(c), dev(val), dev(x))
    y = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
    wsb = ar.ar_spmv_workspace_bytes(v, rows, nnz)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
    ar.ar_spmv(v, rows, nnz, *d, y, ws, wsb)
    return host(y)


def _check_all(rp, c, val, x, what):
    rows = rp.size - 1
    ref = loops.spmv(rp, c, val, x)
    _, absum = loops.spmv_rows(rp, c, val, x, np.arange(rows))
    d = (dev(rp), dev(c), dev(val), dev(x))
    for v in range(V):
        y = _run(v, rp, c, val, x, d)
        bad = ~(np.abs(y - ref) <= TOL * absum)
        assert not bad.any(), (what, ar.loop_variant_name(2, v), np.flatnonzero(bad)[:5])


def _np(t3):
    return [t.numpy() for t in t3]


@pytest.mark.parametrize("rows,s", [(1, 1.5), (1000, 1.5), (3001, 2.2), (20000, 1.7)])
def test_zipf_matrices(rows, s):
    rp, c, val = _np(synth.csr_zipf(10 + rows, rows, s))
    _check_all(rp, c, val, synth.spmv_x(1, rows).numpy(), ("zipf", rows))


@pytest.mark.parametrize("rows,b", [(777, 9), (5000, 129), (3, 7)])
def test_band_matrices(rows, b):
    rp, c, val = _np(synth.csr_band(20 + rows, rows, b))
    _check_all(rp, c, val, synth.spmv_x(2, rows).numpy(), ("band", rows, b))


def test_identity_and_diagonal_bitwise():
    n = 10007
    x = synth.spmv_x(3, n).numpy()
    rp = np.arange(n + 1, dtype=np.int32)
    c = np.arange(n, dtype=np.int32)
    d = np.random.Generator(np.random.PCG64(4)).normal(size=n)
    for v in range(V):
        if v in DF:  # each operand is carried to 2^-46 by its float pair, a product to ~3 * 2^-46
            assert np.all(np.abs(_run(v, rp, c, np.ones(n), x) - x) <= 2.0 ** -45 * np.abs(x)), v
            assert np.all(np.abs(_run(v, rp, c, d, x) - d * x) <= 2.0 ** -43 * np.abs(d * x)), v
        else:
            assert np.array_equal(_run(v, rp, c, np.ones(n), x), x), v
            assert np.array_equal(_run(v, rp, c, d, x), d * x), v


def test_empty_rows_long_rows_and_block_straddles():
    # rows of length 0, 1 and 4096 interleaved; several 4096-long rows in a
    # row so merge-path blocks (4096 path items) start and end inside rows
    rng = np.random.Generator(np.random.PCG64(5))
    lens = np.array([0, 4096, 0, 0, 1, 4096, 4096, 4096, 3, 0, 2049, 4095, 1, 0, 4096] + [0] * 300 +
                    list(rng.integers(0, 40, 3000)) + [4096, 0], dtype=np.int64)
    rows = lens.size
    rp = np.zeros(rows + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    nnz = int(rp[-1])
    cols = rows + 5000
    c = np.concatenate([np.sort(rng.choice(cols, int(L), replace=False)) for L in lens]).astype(np.int32)
    val = rng.normal(size=nnz)
    x = rng.uniform(-1, 1, cols)
    _check_all(rp.astype(np.int32), c, val, x, "mixed")


def test_all_empty_and_single_dense_row():
    rp = np.zeros(65, dtype=np.int32)
    for v in range(V):
        assert np.array_equal(_run(v, rp, np.zeros(0, np.int32), np.zeros(0), np.ones(4)), np.zeros(64))
    n = 4096
    r = np.random.Generator(np.random.PCG64(6))
    _check_all(np.array([0, n], dtype=np.int32), np.arange(n, dtype=np.int32), r.normal(size=n),
               r.uniform(-1, 1, n), "dense row")


def test_operands_outside_the_float_pair_range():
    """Rows holding zeros, values outside [2^-62, 2^62) or products whose
    float sum overflows: the float-pair variants redo those rows in float64,
    every variant matches the oracle."""
    rng = np.random.Generator(np.random.PCG64(9))
    rows, cols = 600, 700
    lens = rng.integers(0, 60, rows)
    lens[:4] = [4096 // 8, 50, 50, 50]
    rp = np.zeros(rows + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    nnz = int(rp[-1])
    c = np.concatenate([np.sort(rng.choice(cols, int(L), replace=False)) for L in lens]).astype(np.int32)
    val = rng.normal(size=nnz)
    x = rng.uniform(-1, 1, cols)
    val[: lens[0]] = 2.0 ** 61                              # row 0: 512 products of 2^122 overflow a float sum
    x[c[: lens[0]]] = 2.0 ** 61
    val[rp[1]] = 1e-25                                      # row 1: a tiny value
    val[rp[2]] = 0.0                                        # row 2: an explicit zero
    val[rp[3]] = -1e25                                      # row 3: a huge value
    x[rng.integers(0, cols, 20)] = 0.0                      # zeros in x
    x[c[rp[5]]] = 3e-30                                     # a tiny x entry
    _check_all(rp.astype(np.int32), c, val, x, "range")


def test_every_variant_is_deterministic():
    rp, c, val = _np(synth.csr_zipf(7, 50000, 1.5))
    x = synth.spmv_x(7, 50000).numpy()
    d = (dev(rp), dev(c), dev(val), dev(x))
    for v in range(V):
        assert np.array_equal(_run(v, rp, c, val, x, d), _run(v, rp, c, val, x, d)), v


@pytest.mark.parametrize("params", [
    {"rows": 10_000_000, "kind": "zipf", "s": 1.5, "band": 0},
    {"rows": 10_000_000, "kind": "band", "s": 0.0, "band": 129},
    {"rows": 1_000_000, "kind": "zipf", "s": 2.5, "band": 0},
])
def test_full_size_sampled_rows(params):
    """Largest matrices of the workload, generated on the device; 3000 sampled
    rows (first, last, random) checked against the oracle."""
    rows = params["rows"]
    rp, c, val = synth.spmv_matrix(31, params, device="cuda")
    x = synth.spmv_x(31, rows, device="cuda")
    nnz = int(rp[-1].item())
    rng = np.random.Generator(np.random.PCG64(rows))
    which = np.unique(np.concatenate([[0, rows - 1], rng.integers(0, rows, 3000)]))
    rph = rp.cpu().numpy().astype(np.int64)
    lens = rph[which + 1] - rph[which]
    idx = torch.from_numpy(np.concatenate([np.arange(rph[w], rph[w + 1]) for w in which])).cuda()
    srp = np.zeros(which.size + 1, dtype=np.int64)
    srp[1:] = np.cumsum(lens)
    sc, sv = c[idx].cpu().numpy(), val[idx].cpu().numpy()
    xh = x.cpu().numpy()
    ref, absum = loops.spmv_rows(srp.astype(np.int32), sc, sv, xh, np.arange(which.size))
    y = torch.empty(rows, dtype=torch.float64, device="cuda")
    wsb = max(ar.ar_spmv_workspace_bytes(var, rows, nnz) for var in range(V))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    wt = torch.from_numpy(which).cuda()
    for v in range(V):
        y.fill_(np.nan)
        ar.ar_spmv(v, rows, nnz, rp, c, val, x, y, ws, wsb)
        got = host(y[wt])
        assert np.all(np.abs(got - ref) <= TOL * absum), (params, ar.loop_variant_name(2, v))


@pytest.mark.parametrize("rows,kind", [(1, "zipf"), (999, "zipf"), (123457, "zipf"), (40000, "band")])
def test_row_features_match_oracle(rows, kind):
    rp = (synth.csr_zipf(3, rows, 1.6)[0] if kind == "zipf" else synth.csr_band(3, rows, 33)[0]).numpy()
    ref = loops.csr_row_stats(rp)
    wsb = ar.ar_csr_features_workspace_bytes(rows)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    out = torch.zeros(5, dtype=torch.float32, device="cuda")
    ar.ar_csr_features(rows, dev(rp), out, ws, wsb)
    got = host(out).astype(np.float64)
    assert got[0] == np.float32(ref[0]) and got[1] == np.float32(ref[1]) and got[4] == ref[4]
    assert got[2] == pytest.approx(ref[2], rel=1e-6)
    assert got[3] == pytest.approx(ref[3], rel=1e-5, abs=1e-6)


def test_gather_floor_is_below_every_variant():
    """ar_spmv_gather_floor does a subset of every variant's memory work (no
    row logic, no float64 arithmetic), so on a power-law matrix it is not
    slower than the fastest variant (mean of 5 runs, 10 % slack for noise)."""
    rows = 2_000_000
    rp, c, v = synth.csr_zipf(31, rows, 1.5, device="cuda")
    x = synth.spmv_x(31, rows, device="cuda")
    nnz = int(rp[-1].item())
    y = torch.empty(rows, dtype=torch.float64, device="cuda")
    sink = torch.empty(1, dtype=torch.int64, device="cuda")
    wsb = max(ar.ar_spmv_workspace_bytes(var, rows, nnz) for var in range(V))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 5

    floor = timed(lambda: ar.ar_spmv_gather_floor(nnz, c, v, x, sink))
    best = min(timed(lambda var=var: ar.ar_spmv(var, rows, nnz, rp, c, v, x, y, ws, wsb)) for var in range(V))
    assert floor <= 1.1 * best, (floor, best)
