"""Executor parity on a batch drawn from the mixed-stream distribution (GPU).

128 calls of `synth.mixed_stream` (loop ~ U{4}, log-uniform sizes; sizes
capped so the test stays short: daxpy n <= 2^22, Jacobi N <= 160, SpMV pool
rows <= 2e5, n-body N <= 32k), each with a seeded random variant, run in one
persistent batch; every call's output is compared with the stand-alone
kernel of the same variant (itself checked against the oracle elsewhere).
"""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth

pytestmark = pytest.mark.gpu
V = {0: 15, 1: 16, 2: 8, 3: 9}


def test_stream_batch_matches_standalone_kernels():
    loops_, sizes = synth.mixed_stream(5, 128)
    rng = np.random.Generator(np.random.PCG64(8))
    pool = [synth.spmv_matrix(5000 + k, {**synth.spmv_matrix_params(5000 + k, rows_max=2e5)}, device="cuda")
            for k in range(8)]
    calls, force, checks, keep = [], [], [], []
    for L, size in zip(loops_.tolist(), sizes.tolist()):
        v = int(rng.integers(0, V[L]))
        c = ar.ArExecCall(loop=L)
        if L == 0:
            n = int(min(size, 1 << 22))
            a, x, y = synth.daxpy_inputs(int(size), n)
            xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
            ref = yd.clone()
            ar.ar_daxpy(v, n, a, xd, ref)
            c.n, c.a, c.in0, c.out0 = n, a, xd.data_ptr(), yd.data_ptr()
            scale = (a * xd).abs() + torch.from_numpy(y).cuda().abs()
            checks.append(lambda yd=yd, ref=ref, s=scale: bool(((yd - ref).abs() <= 1e-13 * s).all()))
            keep += [xd, yd, ref]
        elif L == 1:
            N = int(min(size, 160))
            u0 = torch.from_numpy(synth.grid_inputs(int(size), N)).cuda()
            out, work = torch.empty_like(u0), torch.empty_like(u0)
            ref, rw = torch.empty_like(u0), torch.empty_like(u0)
            st = torch.zeros(2, dtype=torch.int32, device="cuda")
            ar.ar_jacobi7(v, N, 10, u0, ref, rw, st)
            c.n, c.sweeps, c.in0, c.out0, c.out1 = N, 10, u0.data_ptr(), out.data_ptr(), work.data_ptr()
            checks.append(lambda out=out, ref=ref: float((out - ref).abs().max()) <= 1e-13 * float(ref.abs().max()))
            keep += [u0, out, work, ref, rw, st]
        elif L == 2:
            rp, col, val = pool[int(size) % len(pool)]
            rows, nnz = rp.numel() - 1, int(rp[-1].item())
            x = synth.spmv_x(int(size), rows, device="cuda")
            y, ref = torch.empty(rows, dtype=torch.float64, device="cuda"), torch.empty(rows, dtype=torch.float64,
                                                                                          device="cuda")
            wsb = ar.ar_spmv_workspace_bytes(6, rows, nnz)
            ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
            ar.ar_spmv(v, rows, nnz, rp, col, val, x, ref, ws, wsb)
            nb = -(-(rows + nnz) // 4096)
            ews = torch.empty(16 * nb, dtype=torch.uint8, device="cuda")
            c.n, c.nnz = rows, nnz
            c.in0, c.in1, c.in2, c.in3 = rp.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr()
            c.out0, c.out1, c.out1_bytes = y.data_ptr(), ews.data_ptr(), ews.numel()
            # per-row scale of the summation error: sum_k |val_k x_col_k|
            absum = torch.zeros(rows, dtype=torch.float64, device="cuda")
            row_of = torch.repeat_interleave(torch.arange(rows, device="cuda"), rp[1:] - rp[:-1])
            absum.index_add_(0, row_of, (val * x[col.long()]).abs())
            checks.append(lambda y=y, ref=ref, s=absum: bool(((y - ref).abs() <= 1e-10 * s).all()))
            keep += [x, y, ref, ws, ews, absum]
        else:
            N = int(min(size, 32768))
            p = torch.from_numpy(synth.nbody_inputs(int(size), N)).cuda()
            acc, ref = torch.empty_like(p), torch.empty_like(p)
            ar.ar_nbody(v, N, p, ref, synth.NBODY_EPS)
            c.n, c.eps, c.in0, c.out0 = N, synth.NBODY_EPS, p.data_ptr(), acc.data_ptr()
            checks.append(lambda acc=acc, ref=ref: float((acc - ref)[:, :3].norm(dim=1).max())
                          <= 1e-5 * float(ref[:, :3].norm(dim=1).max()))
            keep += [p, acc, ref]
        calls.append(c)
        force.append(v)
    torch.cuda.synchronize()
    n = len(calls)
    table = torch.frombuffer(bytearray(ar.exec_table_bytes(calls)), dtype=torch.uint8).cuda()
    out = [torch.zeros(n, dtype=torch.int32, device="cuda"), torch.zeros(n, dtype=torch.float32, device="cuda"),
           torch.zeros((n, 8), dtype=torch.float32, device="cuda"), torch.zeros(n, dtype=torch.int64, device="cuda"),
           torch.zeros(n, dtype=torch.int64, device="cuda"), torch.zeros(n, dtype=torch.int32, device="cuda")]
    wsb = ar.ar_exec_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    ar.ar_exec_batch(table, n, None, torch.tensor(force, dtype=torch.int32, device="cuda"), *out, ws, wsb)
    torch.cuda.synchronize()
    assert int(out[5].abs().sum()) == 0
    bad = [k for k, ok in enumerate(checks) if not ok()]
    assert not bad, [(k, calls[k].loop, force[k]) for k in bad]
