"""End-to-end region executions on host data (ar_invoke_host): host -> device
copies, the region's variant, device -> host copies, all on one stream,
checked against the oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [64, 45])
def test_jacobi_region_on_host_buffers(N):
    S = 10
    u0 = synth.grid_inputs(11 + N, N)
    ref = loops.jacobi7(u0, S)
    h_in = torch.from_numpy(u0).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_u0 = torch.empty(u0.shape, dtype=torch.float64, device="cuda")
    d_out, d_work = torch.empty_like(d_u0), torch.empty_like(d_u0)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    r = ar.Region("host-jacobi", 2, "dtree,2", 10 ** 9)
    V = r.add_builtin(ar.AR_LOOP_JACOBI7)
    args = ar.ArJacobi7Args(N, S, d_u0.data_ptr(), d_out.data_ptr(), d_work.data_ptr(), status.data_ptr())
    nbytes = 8 * N ** 3
    s = torch.cuda.Stream()
    seen = []
    for _ in range(V):  # RoundRobin exploration: every variant once
        h_out.fill_(np.nan)
        d_u0.fill_(0.0)  # the input must come from the host copy
        v, _ = r.invoke_host([N, S], args, [(h_in, d_u0, nbytes)], [(h_out, d_out, nbytes)], stream=s)
        s.synchronize()
        seen.append(v)
        assert np.max(np.abs(h_out.numpy() - ref)) <= 1e-13 * np.max(np.abs(ref)), v
    assert sorted(seen) == list(range(V))
    assert int(status[0].item()) == 0
    r.flush_records()
    assert r.counts()[0] == V


def test_daxpy_region_on_host_buffers():
    n = 1000003
    a, x, y = synth.daxpy_inputs(8, n)
    ref = loops.daxpy(a, x, y)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    hres = torch.full_like(hy, np.nan).pin_memory()
    dx, dy = torch.empty(n, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
    r = ar.Region("host-daxpy", 1, "fixed,4", 0)
    r.add_builtin(ar.AR_LOOP_DAXPY)
    args = ar.ArDaxpyArgs(n, a, dx.data_ptr(), dy.data_ptr())
    v, _ = r.invoke_host([n], args, [(hx, dx, 8 * n), (hy, dy, 8 * n)], [(hres, dy, 8 * n)])
    torch.cuda.synchronize()
    assert v == 4
    assert np.all(np.abs(hres.numpy() - ref) <= 1e-13 * (np.abs(a * x) + np.abs(y)))
