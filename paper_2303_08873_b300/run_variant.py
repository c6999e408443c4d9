"""Run one variant of one region body on a seeded synthetic case.

A small driver for profilers (ncu) and quick timing: builds the inputs with
``synth``, launches the variant ``--reps`` times through the C ABI and prints
the mean time per launch (CUDA events) and the algorithmic bandwidth or flop
rate.

  python -m paper_2303_08873_b300.run_variant jacobi7 13 --size 320 --sweeps 1
  python -m paper_2303_08873_b300.run_variant heat7 13 --size 320 --sweeps 10 --alpha 0.125
  python -m paper_2303_08873_b300.run_variant spmv 6 --size 2000000
  python -m paper_2303_08873_b300.run_variant nbody 4 --size 65536
  python -m paper_2303_08873_b300.run_variant daxpy 8 --size 33554432

With ``--exec`` the same call also runs as a one-call batch of the persistent
mixed-stream executor (``ar_exec_batch``, variant forced; an n-body call
carries a partial-sum workspace for up to 64 j chunks) and both rates are
printed.  With ``--floor`` (spmv) the gather-floor measurement kernel
(``ar_spmv_gather_floor``) is timed on the same matrix.  Variant ``all`` runs
every variant of the loop in turn (one line each), e.g. for a per-variant ncu
launch list.
"""
from __future__ import annotations

import argparse
import json

import torch

import paper_2303_08873_b300 as ar
import synth


LOOPS = ["daxpy", "jacobi7", "spmv", "nbody", "heat7"]  # index = loop id


def main():
    p = argparse.ArgumentParser()
    p.add_argument("loop", choices=LOOPS)
    p.add_argument("variant", help="variant index, or 'all' for every variant of the loop in turn")
    p.add_argument("--size", type=int, required=True, help="n (daxpy), N (jacobi7, heat7, nbody) or rows (spmv)")
    p.add_argument("--sweeps", type=int, default=1, help="jacobi7 sweeps / heat7 steps")
    p.add_argument("--alpha", type=float, default=0.125, help="heat7: alpha of the explicit step")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--zipf", type=float, default=1.5, help="Zipf exponent of the spmv row lengths")
    p.add_argument("--band", type=int, default=0, help="spmv: banded matrix of this (odd) width instead of Zipf")
    p.add_argument("--exec", action="store_true", help="also time the call through the executor (one-call batch)")
    p.add_argument("--floor", action="store_true",
                   help="spmv: also time ar_spmv_gather_floor (the memory-side floor) on the same matrix")
    a = p.parse_args()
    if a.exec and a.loop == "heat7":
        raise SystemExit("--exec: the executor runs daxpy, jacobi7, spmv and nbody only")
    L = LOOPS.index(a.loop)
    variants = range(ar.loop_num_variants(L)) if a.variant == "all" else [int(a.variant)]
    dev = torch.device("cuda", 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.loop == "daxpy":
        al, x, y = synth.daxpy_inputs(1, a.size)
        x, y = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        make_run = lambda var: lambda: ar.ar_daxpy(var, a.size, al, x, y)  # noqa: E731
        call = ar.ArExecCall(loop=0, n=a.size, a=al, in0=x.data_ptr(), out0=y.data_ptr())
        work, unit = 24.0 * a.size, "GB/s"
    elif a.loop == "jacobi7":
        u0 = torch.from_numpy(synth.grid_inputs(1000 + a.size, a.size)).to(dev)
        out, wk = torch.empty_like(u0), torch.empty_like(u0)
        st = torch.zeros(2, dtype=torch.int32, device=dev)
        make_run = lambda var: lambda: ar.ar_jacobi7(var, a.size, a.sweeps, u0, out, wk, st)  # noqa: E731
        call = ar.ArExecCall(loop=1, n=a.size, sweeps=a.sweeps, in0=u0.data_ptr(), out0=out.data_ptr(),
                             out1=wk.data_ptr())
        work, unit = 16.0 * a.size ** 3 * a.sweeps, "GB/s"
    elif a.loop == "heat7":
        u0 = torch.from_numpy(synth.grid_inputs(2000 + a.size, a.size)).to(dev)
        out, wk = torch.empty_like(u0), torch.empty_like(u0)
        st = torch.zeros(2, dtype=torch.int32, device=dev)
        make_run = lambda var: lambda: ar.ar_heat7(var, a.size, a.sweeps, a.alpha, u0, out, wk, st)  # noqa: E731
        call = None
        work, unit = 16.0 * a.size ** 3 * a.sweeps, "GB/s"
    elif a.loop == "spmv":
        if a.band:
            rp, c, v = synth.csr_band(31, a.size, a.band, device="cuda")
        else:
            rp, c, v = synth.csr_zipf(31, a.size, a.zipf, device="cuda")
        x = synth.spmv_x(31, a.size, device="cuda")
        y = torch.empty(a.size, dtype=torch.float64, device=dev)
        nnz = int(rp[-1].item())
        wsb = max(ar.ar_spmv_workspace_bytes(var, a.size, nnz) for var in variants)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
        make_run = lambda var: lambda: ar.ar_spmv(var, a.size, nnz, rp, c, v, x, y, ws, wsb)  # noqa: E731
        ews = torch.empty(16 * (-(-(a.size + nnz) // 4096)), dtype=torch.uint8, device=dev)
        call = ar.ArExecCall(loop=2, n=a.size, nnz=nnz, in0=rp.data_ptr(), in1=c.data_ptr(), in2=v.data_ptr(),
                             in3=x.data_ptr(), out0=y.data_ptr(), out1=ews.data_ptr(), out1_bytes=ews.numel())
        work, unit = 12.0 * nnz + 4.0 * (a.size + 1) + 16.0 * a.size, "GB/s"
    else:
        pos = torch.from_numpy(synth.nbody_inputs(4, a.size)).to(dev)
        acc = torch.empty_like(pos)
        make_run = lambda var: lambda: ar.ar_nbody(var, a.size, pos, acc, synth.NBODY_EPS)  # noqa: E731
        part = torch.empty(a.size * 4 * 64, dtype=torch.float32, device=dev)  # partial sums of up to 64 j chunks
        call = ar.ArExecCall(loop=3, n=a.size, eps=synth.NBODY_EPS, in0=pos.data_ptr(), out0=acc.data_ptr(),
                             out1=part.data_ptr(), out1_bytes=part.numel() * 4)
        work, unit = 20.0 * a.size ** 2, "GFLOP/s"

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / a.reps

    for var in variants:
        ms = timed(make_run(var))
        line = {"loop": a.loop, "variant": var, "name": ar.loop_variant_name(L, var), "size": a.size, "ms": ms,
                "rate": work / (ms * 1e-3) / 1e9, "unit": unit}
        if a.floor and a.loop == "spmv":
            sink = torch.empty(1, dtype=torch.int64, device=dev)
            fms = timed(lambda: ar.ar_spmv_gather_floor(nnz, c, v, x, sink))
            line.update({"floor_ms": fms, "floor_rate": work / (fms * 1e-3) / 1e9,
                         "floor_gathers_per_s": nnz / (fms * 1e-3)})
        if a.exec:
            table = torch.frombuffer(bytearray(ar.exec_table_bytes([call])), dtype=torch.uint8).to(dev)
            outs = [torch.zeros(1, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.float32, device=dev),
                    torch.zeros((1, 8), dtype=torch.float32, device=dev),
                    torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev),
                    torch.zeros(1, dtype=torch.int32, device=dev)]
            ewsb = ar.ar_exec_workspace_bytes(1)
            ews_all = torch.empty(ewsb, dtype=torch.uint8, device=dev)
            force = torch.tensor([var], dtype=torch.int32, device=dev)
            ems = timed(lambda: ar.ar_exec_batch(table, 1, None, force, *outs, ews_all, ewsb))
            if int(outs[5][0]) != 0:
                raise SystemExit(f"executor status {int(outs[5][0])}")
            line.update({"exec_ms": ems, "exec_rate": work / (ems * 1e-3) / 1e9})
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
