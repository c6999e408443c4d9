"""Host-data loops split between the GPU and the host cores (the paper's
co-scheduling and device-selection use cases, Section 3.2, Listings 5 and 3)
against the oracle (GPU): every GPU fraction of [0.0:1.0:0.1], the regions
that choose among them, and the copies of a region execution."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops

pytestmark = pytest.mark.gpu
FRACTIONS = [i * 0.1 for i in range(11)]


def _daxpy_args(n, a, x, y, xd, yd, variant):
    return ar.ArDaxpySplitArgs(n, a, x.data_ptr(), y.data_ptr(), xd.data_ptr(), yd.data_ptr(), variant)


@pytest.mark.parametrize("n", [1, 1000, 1000003])
def test_daxpy_every_fraction_is_bitwise_the_fma_oracle(n):
    a, x, y = synth.daxpy_inputs(21, n)
    ref = loops.daxpy(a, x, y, fma=True)
    hx = torch.from_numpy(x).pin_memory()
    xd, yd = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    for f in FRACTIONS:
        for variant in (0, 8, 14):  # 1, 2 and 4 elements per thread on the GPU part
            hy = torch.from_numpy(y.copy()).pin_memory()
            ar.ar_daxpy_split(f, _daxpy_args(n, a, hx, hy, xd, yd, variant), stream=s)
            assert np.array_equal(hy.numpy(), ref), (f, variant)


@pytest.mark.parametrize("kind", ["zipf", "band"])
def test_spmv_every_fraction_matches_the_oracle(kind):
    rows = 30011
    rp, c, v = synth.csr_zipf(22, rows, 1.6) if kind == "zipf" else synth.csr_band(23, rows, 65)
    rp, c, v = rp.numpy(), c.numpy(), v.numpy()
    x = synth.spmv_x(24, rows).numpy()
    nnz = int(rp[-1])
    ref, absum = loops.spmv_rows(rp, c, v, x, np.arange(rows))
    h = [torch.from_numpy(t).pin_memory() for t in (rp, c, v, x)]
    d = [torch.empty_like(t, device="cuda") for t in h]
    yd = torch.empty(rows, dtype=torch.float64, device="cuda")
    wsb = max(ar.ar_spmv_workspace_bytes(var, rows, nnz) for var in range(ar.loop_num_variants(2)))
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    for f in FRACTIONS:
        for variant in (0, 4, 7, 8):
            hy = torch.full((rows,), np.nan, dtype=torch.float64).pin_memory()
            args = ar.ArSpmvSplitArgs(rows=rows, nnz=nnz, cols=rows, rowptr=h[0].data_ptr(), col=h[1].data_ptr(),
                                      val=h[2].data_ptr(), x=h[3].data_ptr(), y=hy.data_ptr(),
                                      rowptr_dev=d[0].data_ptr(), col_dev=d[1].data_ptr(), val_dev=d[2].data_ptr(),
                                      x_dev=d[3].data_ptr(), y_dev=yd.data_ptr(), workspace=ws.data_ptr(),
                                      workspace_bytes=wsb, gpu_variant=variant)
            ar.ar_spmv_split(f, args)
            assert np.all(np.abs(hy.numpy() - ref) <= 1e-10 * absum), (kind, f, variant)


def test_cosched_and_device_selection_regions_profile_train_and_invoke():
    """The co-scheduling region (11 fractions) and the device-selection
    region (host cores or GPU) profile every variant on host data, train
    their decision trees, and an invocation through the trained model still
    computes daxpy exactly."""
    n = 1 << 20
    a, x, y = synth.daxpy_inputs(25, n)
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.from_numpy(y.copy()).pin_memory()
    xd, yd = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
    args = _daxpy_args(n, a, hx, hy, xd, yd, 6)
    for spec, rng in (("cosched", (0.0, 1.0, 0.1)), ("device", (0.0, 1.0, 1.0))):
        r = ar.Region(spec, 1, "dtree,2,reps=2", 10 ** 9)
        V = r.add_split(ar.AR_LOOP_DAXPY, *rng)
        for m in (1 << 12, 1 << 20):
            args.n = m
            ms, best = r.profile([m], args)
            assert len(ms) == V and all(np.isfinite(ms)) and 0 <= best < V
        r.train()
        args.n = n
        hy.copy_(torch.from_numpy(y))
        v, frac = r.invoke([n], args)
        torch.cuda.synchronize()
        assert frac == r.variant(v)["value"]
        assert np.array_equal(hy.numpy(), loops.daxpy(a, x, y, fma=True)), spec
