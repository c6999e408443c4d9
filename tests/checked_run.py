"""Every variant of every loop, the batched n-body and one executor batch at
small sizes (plus three Jacobi calls of N 258-377 that take the executor's
deepest plane chunks), run in the bounds-check build of the library; prints a JSON
line with the check status and the parity of each result against the
oracle.  Run as a child process with AR_CHECKED=1 (tests/test_gpu_checked.py)."""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_2303_08873_b300 as ar  # noqa: E402
import synth  # noqa: E402
from oracle import loops  # noqa: E402
from tests.gpu_util import dev, host  # noqa: E402


def main():
    assert ar.CHECKED, "run with AR_CHECKED=1"
    ar.ar_check_status(clear=True)
    bad = []
    # daxpy: odd length, every variant
    a, x, y = synth.daxpy_inputs(3, 30001)
    ref = loops.daxpy(a, x, y)
    for v in range(15):
        yd = dev(y)
        ar.ar_daxpy(v, x.size, a, dev(x), yd)
        if not np.all(np.abs(host(yd) - ref) <= 1e-13 * (np.abs(a * x) + np.abs(y))):
            bad.append(f"daxpy {v}")
    # Jacobi and heat: even N (3D tensor copies), odd N (2D view), N below a box (smem / ring)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    for N in (20, 37, 40):
        u0 = synth.grid_inputs(N, N)
        jref, href = loops.jacobi7(u0, 3), loops.heat7(u0, 3, 0.125)
        ud = dev(u0)
        for v in range(16):
            for name, fn, r_ in (("jacobi7", lambda o, w: ar.ar_jacobi7(v, N, 3, ud, o, w, st), jref),
                                 ("heat7", lambda o, w: ar.ar_heat7(v, N, 3, 0.125, ud, o, w, st), href)):
                out, work = torch.empty_like(ud), torch.empty_like(ud)
                fn(out, work)
                scale = max(np.max(np.abs(r_)), np.max(np.abs(u0)))
                if np.max(np.abs(host(out) - r_)) > 1e-13 * scale:
                    bad.append(f"{name} N={N} v={v}")
    if int(st[0].item()) != 0:
        bad.append("stencil status")
    # SpMV: power-law rows with empty ones, band rows, every variant
    for rp, c, vv in (synth.csr_zipf(4, 9000, 1.5), synth.csr_band(5, 7000, 65)):
        rp, c, vv = rp.numpy(), c.numpy(), vv.numpy()
        rows, nnz = rp.size - 1, int(rp[-1])
        xs = synth.spmv_x(6, rows).numpy()
        sref, absum = loops.spmv_rows(rp, c, vv, xs, np.arange(rows))
        d = [dev(rp), dev(c), dev(vv), dev(xs)]
        for v in range(ar.loop_num_variants(2)):
            yd = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
            wsb = ar.ar_spmv_workspace_bytes(v, rows, nnz)
            ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
            ar.ar_spmv(v, rows, nnz, *d, yd, ws, wsb)
            if not np.all(np.abs(host(yd) - sref) <= 1e-10 * absum):
                bad.append(f"spmv rows={rows} v={v}")
    # n-body: a small N (cluster split) and a ragged one
    for N in (700, 2049):
        p = synth.nbody_inputs(N, N)
        nref = loops.nbody(p, synth.NBODY_EPS)
        pd = dev(p)
        for v in range(9):
            acc = torch.empty_like(pd)
            ar.ar_nbody(v, N, pd, acc, synth.NBODY_EPS)
            err = np.max(np.linalg.norm(host(acc)[:, :3] - nref, axis=1))
            if err > 1e-4 * np.max(np.linalg.norm(nref, axis=1)):
                bad.append(f"nbody N={N} v={v}")
    # one executor batch: every variant of every loop
    from tests.test_gpu_executor import Batch
    b = Batch()
    force = []
    for v in range(15):
        b.daxpy(20001 + v, 40 + v)
        force.append(v)
    for v in range(16):
        b.jacobi(37 if v % 2 else 40, 3, 60 + v)
        force.append(v)
    for N, v in ((376, 13), (377, 12), (258, 15)):  # 94-plane tiles; last chunks of 94, 1 and 70 planes
        b.jacobi(N, 2, 120 + N)
        force.append(v)
    zipf = synth.csr_zipf(7, 12000, 1.6)
    for v in range(8):
        b.spmv(zipf, 80 + v)
        force.append(v)
    for v in range(9):
        b.nbody(600 + 31 * v, 90 + v)
        force.append(v)
    r = b.run(force=force)
    if not np.all(r["status"] == 0):
        bad.append("executor status")
    for k, ok in enumerate(b.check):
        if not ok():
            bad.append(f"executor call {k}")
    enabled, first, failures = ar.ar_check_status(clear=True)
    print(json.dumps({"enabled": enabled, "first_failure": first, "failures": failures, "bad": bad}), flush=True)


if __name__ == "__main__":
    main()
