"""Host part of the GPU / host split loops (co-scheduling, device selection):
at GPU fraction 0 the whole loop runs on the host cores and touches no
device, so it is checked against the oracle here, on the CPU."""
import numpy as np
import pytest

import paper_2303_08873_b300 as ar
import synth
from oracle import loops


def test_daxpy_split_all_on_host_matches_the_fma_oracle_bitwise():
    a, x, y = synth.daxpy_inputs(12, 100003)
    ref = loops.daxpy(a, x, y, fma=True)
    yy = y.copy()
    args = ar.ArDaxpySplitArgs(x.size, a, x.ctypes.data, yy.ctypes.data, None, None, 0)
    ar.ar_daxpy_split(0.0, args)
    assert np.array_equal(yy, ref)
    assert ar.ar_split_threads() >= 1


def test_spmv_split_all_on_host_matches_the_oracle():
    rp, c, v = (t.numpy() for t in synth.csr_zipf(13, 5000, 1.7))
    x = synth.spmv_x(14, 5000).numpy()
    rows, nnz = rp.size - 1, int(rp[-1])
    ref, absum = loops.spmv_rows(rp, c, v, x, np.arange(rows))
    y = np.full(rows, np.nan)
    args = ar.ArSpmvSplitArgs(rows=rows, nnz=nnz, cols=rows, rowptr=rp.ctypes.data, col=c.ctypes.data,
                              val=v.ctypes.data, x=x.ctypes.data, y=y.ctypes.data, gpu_variant=0)
    ar.ar_spmv_split(0.0, args)
    assert np.all(np.abs(y - ref) <= 1e-10 * absum)


@pytest.mark.parametrize("f", [-0.1, 1.5, float("nan")])
def test_split_rejects_fractions_outside_0_1(f):
    x = np.zeros(4)
    args = ar.ArDaxpySplitArgs(4, 1.0, x.ctypes.data, x.ctypes.data, 64, 64, 0)
    with pytest.raises(ar.ArError) as e:
        ar.ar_daxpy_split(f, args)
    assert e.value.code == ar.AR_ERR_ARG


def test_split_rejects_missing_device_buffers_and_bad_variants():
    x = np.zeros(8)
    with pytest.raises(ar.ArError):  # the GPU part needs device buffers
        ar.ar_daxpy_split(0.5, ar.ArDaxpySplitArgs(8, 1.0, x.ctypes.data, x.ctypes.data, None, None, 0))
    with pytest.raises(ar.ArError):
        ar.ar_daxpy_split(0.0, ar.ArDaxpySplitArgs(8, 1.0, x.ctypes.data, x.ctypes.data, None, None, 15))
    rp = np.array([0, 2, 1], dtype=np.int32)  # rowptr[rows] != nnz
    c = np.zeros(2, dtype=np.int32)
    with pytest.raises(ar.ArError):
        ar.ar_spmv_split(0.0, ar.ArSpmvSplitArgs(rows=2, nnz=2, cols=1, rowptr=rp.ctypes.data, col=c.ctypes.data,
                                                 val=x.ctypes.data, x=x.ctypes.data, y=x.ctypes.data))


def test_split_regions_register_the_paper_ranges():
    r = ar.Region("cosched", 1, "dtree", 10 ** 9)
    assert r.add_split(ar.AR_LOOP_DAXPY) == 11  # [0.0:1.0:0.1] (Listing 5)
    vals = [r.variant(v)["value"] for v in range(11)]
    assert vals == [i * 0.1 for i in range(11)]
    d = ar.Region("device", 1, "dtree", 10 ** 9)
    assert d.add_split(ar.AR_LOOP_SPMV, 0.0, 1.0, 1.0) == 2  # cpu, gpu (Listing 3)
    with pytest.raises(ar.ArError):
        ar.Region("bad", 1, "dtree", 1).add_split(ar.AR_LOOP_JACOBI7)
