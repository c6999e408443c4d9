#!/usr/bin/env python3
"""Benchmark of the adaptive-region hot path on B300.

Workload (default): the 7-point 3D Jacobi region, float64, N in
{32, 64, 128, 256, 384, 512}, U[-1, 1] interior, zero Dirichlet ghosts, 10
sweeps per invocation.  The region holds 16 variants (naive, 2.5D smem, TMA,
float-pair TMA x 4 block shapes); a depth-2 decision tree on the features
(N, sweeps) is trained from exhaustive profiling of N x sweeps in {1,5,10,20}
before timing.  One step = one ar_invoke per N (select with the tree, run the
selected variant's 10 sweeps, record the elapsed time): the whole hot path.

Prints ONE JSON line: selected-variant GB/s (algorithmic 16 bytes per point
per sweep), next to the exhaustive-best and fixed-default GB/s, regret, the
roofline of the dominant kernel, the CPU oracle and an end-to-end number
through host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIZES = [32, 64, 128, 256, 384, 512]
SWEEPS = 10
TRAIN_SWEEPS = [1, 5, 10, 20]
BYTES_PER_POINT = 16.0          # one float64 read + one write per point per sweep
FP64_OPS_PER_POINT = 6          # 5 adds + 1 multiply in the native families
METRIC = "selected-variant GB/s (or GFLOP/s) vs exhaustive-best & fixed default; regret %"
FALLBACK_HBM_GBS = 6400.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--workload", default="jacobi7", choices=["jacobi7", "spmv"],
                   help="jacobi7: the headline line; spmv: the learned-selector study (one JSON line)")
    p.add_argument("--train", type=int, default=2000, help="spmv: profiled training matrices")
    p.add_argument("--test", type=int, default=500, help="spmv: held-out test matrices")
    p.add_argument("--rows-max", type=float, default=1e7, help="spmv: largest row count")
    p.add_argument("--epochs", type=int, default=200, help="spmv: MLP epochs")
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def workload_bytes(sizes, sweeps):
    return sum(BYTES_PER_POINT * n ** 3 * sweeps for n in sizes)


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(seconds: float):
    """GB/s of the float64 CPU oracle on a bounded sample of the workload:
    N in {32, 64, 128, 256} at 10 sweeps, repeated until `seconds` elapse."""
    import synth
    from oracle import loops

    grids = {n: synth.grid_inputs(1000 + n, n) for n in (32, 64, 128, 256)}
    t0 = time.perf_counter()
    done = 0.0
    reps = 0
    while True:
        for n, u in grids.items():
            loops.jacobi7(u, SWEEPS)
            done += BYTES_PER_POINT * n ** 3 * SWEEPS
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt / 1e9, "unit": "GB/s", "cores": loops.num_threads(), "kind": "oracle",
            "sample": f"jacobi7 float64 N in (32,64,128,256), 10 sweeps, {reps} passes, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from oracle import loops

    sizes = (32, 64, 128, 256)
    import synth

    grids = {n: synth.grid_inputs(1000 + n, n) for n in sizes}
    for _ in range(args.warmup):
        for n, u in grids.items():
            loops.jacobi7(u, SWEEPS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for n, u in grids.items():
            loops.jacobi7(u, SWEEPS)
    dt = time.perf_counter() - t0
    val = workload_bytes(sizes, SWEEPS) * args.steps / dt / 1e9
    sample = f"jacobi7 float64 N in {sizes}, 10 sweeps per step (bounded sample of N up to 512)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "jacobi7 CPU oracle sample", "sizes": list(sizes),
                                            "sweeps": SWEEPS},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": loops.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks
class Clocks:
    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1].split()[0]))
                mx.append(float(c[2].split()[0]))
            except ValueError:
                continue
            for nm, val in zip(names, c[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    hbm_peak, peak_src = peaks()
    fp64_fma, _ = ar.ar_measure_fma_rates()

    # --- inputs resident in HBM (one u0/out/work triple per size)
    bufs = {}
    for n in SIZES:
        u0 = torch.from_numpy(synth.grid_inputs(1000 + n, n)).to(dev)
        bufs[n] = (u0, torch.empty_like(u0), torch.empty_like(u0))
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    argblocks = {n: ar.ArJacobi7Args(n, SWEEPS, bufs[n][0].data_ptr(), bufs[n][1].data_ptr(),
                                     bufs[n][2].data_ptr(), status.data_ptr()) for n in SIZES}

    # --- profiling + training (untimed): exhaustive over N x sweeps
    region = ar.Region("jacobi7", 2, "dtree,2,reps=5", 10 ** 9)
    V = region.add_builtin(ar.AR_LOOP_JACOBI7)
    region.set_l2_flush(flush, flush.numel())
    table = {}
    t_prof = time.perf_counter()
    for n in SIZES:
        for s in TRAIN_SWEEPS:
            a = ar.ArJacobi7Args(n, s, *[bufs[n][i].data_ptr() for i in range(3)], status.data_ptr())
            ms, best = region.profile([n, s], a, stream=stream)
            table[(n, s)] = (ms, best)
    t_prof = time.perf_counter() - t_prof
    region.train()
    tree = region.tree()
    default = ar.loop_default_variant(ar.AR_LOOP_JACOBI7)
    names = [ar.loop_variant_name(ar.AR_LOOP_JACOBI7, v) for v in range(V)]
    chosen = {n: region.select([n, SWEEPS])[0] for n in SIZES}

    def step():
        for n in SIZES:
            region.invoke([n, SWEEPS], argblocks[n], stream=stream)

    # --- timed region
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    big = SIZES[-1]
    torch.cuda.nvtx.range_push("bench_timed")
    e0.record(stream)
    for t in range(args.steps):
        for n in SIZES:
            if n == big:
                k0[t].record(stream)
            region.invoke([n, SWEEPS], argblocks[n], stream=stream)
            if n == big:
                k1[t].record(stream)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    stream.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    step_bytes = workload_bytes(SIZES, SWEEPS)
    value = step_bytes * args.steps * ws / (ms * 1e-3) / 1e9
    assert int(status[0].item()) == 0, "a bounded wait inside a TMA kernel timed out"

    # --- dominant kernel roofline: the N=512 invocation's sweeps
    big_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k0, k1)) / SWEEPS
    achieved = BYTES_PER_POINT * big ** 3 / (big_ms * 1e-3) / 1e9
    vbig = chosen[big]
    if names[vbig].startswith("jacobi7_df"):
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                "kernel": names[vbig]}
    else:
        alu_gbs = fp64_fma / FP64_OPS_PER_POINT * BYTES_PER_POINT / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_gbs, "unit": "GB/s",
                "frac": achieved / alu_gbs, "traffic": None,
                "peak_source": "float64 issue rate measured by ar_measure_fma_rates x 16 B / 6 FP64 ops per point",
                "kernel": names[vbig], "hbm_frac": achieved / hbm_peak}

    # --- selection quality from the exhaustive table (sweeps = 10)
    per = []
    t_sel = t_best = t_def = 0.0
    for n in SIZES:
        ms_n, best = table[(n, SWEEPS)]
        sel = chosen[n]
        t_sel += ms_n[sel]
        t_best += ms_n[best]
        t_def += ms_n[default]
        per.append({"N": n, "selected": names[sel], "best": names[best], "regret_pct": 100 * (ms_n[sel] / ms_n[best] - 1),
                    "selected_gbs": BYTES_PER_POINT * n ** 3 * SWEEPS / ms_n[sel] / 1e6,
                    "best_gbs": BYTES_PER_POINT * n ** 3 * SWEEPS / ms_n[best] / 1e6,
                    "default_gbs": BYTES_PER_POINT * n ** 3 * SWEEPS / ms_n[default] / 1e6})
    regret = statistics.mean(p["regret_pct"] for p in per)

    # --- end to end through host buffers (pinned), copies inside the timed region
    host_in = {n: bufs[n][0].cpu().pin_memory() for n in SIZES}
    host_out = {n: torch.empty_like(host_in[n]).pin_memory() for n in SIZES}
    e2e_steps = max(3, min(args.steps, 10))
    with torch.cuda.stream(stream):
        for n in SIZES:
            bufs[n][0].copy_(host_in[n], non_blocking=True)
    stream.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(e2e_steps):
            for n in SIZES:
                bufs[n][0].copy_(host_in[n], non_blocking=True)
                region.invoke([n, SWEEPS], argblocks[n], stream=stream)
                host_out[n].copy_(bufs[n][1], non_blocking=True)
    a1.record(stream)
    stream.synchronize()
    e2e_ms = a0.elapsed_time(a1) / e2e_steps
    h2d = sum(8 * n ** 3 for n in SIZES)
    e2e = {"value": step_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d, "ms_per_step": e2e_ms}

    if rank != 0:
        return
    cpu = cpu_oracle_rate(args.cpu_seconds) if ws == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "jacobi7 float64 N in {32,64,128,256,384,512}, 10 sweeps, depth-2 tree on "
                               "(N, sweeps) over 16 variants", "sizes": SIZES, "sweeps": SWEEPS,
                   "parallelism": "replicas" if ws > 1 else "single-gpu",
                   "l2": "inputs larger than L2: six grids, 3.2 GB read+written per step"},
        "selection": {"exhaustive_best_gbs": step_bytes / t_best / 1e6, "default_gbs": step_bytes / t_def / 1e6,
                      "selected_table_gbs": step_bytes / t_sel / 1e6, "regret_pct": regret,
                      "default_variant": names[default], "per_N": per, "tree": tree,
                      "profiling_s": t_prof, "profiled_points": len(table), "variants": V},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * len(SIZES) * SWEEPS,
        "clocks": clk,
        "fp64_fma_per_s": fp64_fma,
    }
    print(json.dumps(line), flush=True)



# ---------------------------------------------------------------- SpMV selector study
SPMV_FEATURES = ("rows", "nnz", "mean", "var", "max")


def spmv_bytes(rows, nnz):
    """Algorithmic bytes of one y = A x: val + col per nonzero, row pointers,
    x read once, y written once."""
    return 12.0 * nnz + 4.0 * (rows + 1) + 8.0 * rows + 8.0 * rows


def run_spmv(args):
    """Config 3: profile `train` seeded matrices (7 variants, 5 reps after a
    warm-up, L2 flushed), train the MLP selector on the device and the depth-2
    tree on the same records, then compare their choices with the exhaustive
    argmin and the fixed default (thread per row) on `test` held-out matrices."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ws = torch.empty(16 << 20, dtype=torch.uint8, device=dev)
    fwsb = ar.ar_csr_features_workspace_bytes(0)
    fws = torch.empty(fwsb, dtype=torch.uint8, device=dev)
    f5 = torch.zeros(5, dtype=torch.float32, device=dev)

    def case(seed):
        prm = synth.spmv_matrix_params(seed, rows_max=args.rows_max)
        rp, c, v = synth.spmv_matrix(seed, prm, device="cuda")
        rows = prm["rows"]
        nnz = int(rp[-1].item())
        x = synth.spmv_x(seed, rows, device="cuda")
        y = torch.empty(rows, dtype=torch.float64, device=dev)
        ar.ar_csr_features(rows, rp, f5, fws, fwsb, stream=stream)
        stream.synchronize()
        feats = f5.cpu().tolist()
        a = ar.ArSpmvArgs(rows, nnz, rp.data_ptr(), c.data_ptr(), v.data_ptr(), x.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), ws.numel())
        return feats, a, (rp, c, v, x, y), rows, nnz

    mlp = ar.Region("spmv-mlp", 5, f"mlp,64,epochs={args.epochs},seed=7", 10 ** 9)
    tree = ar.Region("spmv-dtree", 5, "dtree,2", 10 ** 9)
    exh = ar.Region("spmv-exhaustive", 5, "exhaustive,reps=5")
    V = mlp.add_builtin(ar.AR_LOOP_SPMV)
    tree.add_builtin(ar.AR_LOOP_SPMV)
    exh.add_builtin(ar.AR_LOOP_SPMV)
    for r in (mlp, exh):
        r.set_l2_flush(flush, flush.numel())
    default = ar.loop_default_variant(ar.AR_LOOP_SPMV)
    names = [ar.loop_variant_name(ar.AR_LOOP_SPMV, v) for v in range(V)]

    t0 = time.perf_counter()
    prof_ms = 0.0
    for k in range(args.train):
        feats, a, keep, rows, nnz = case(1000 + k)
        ms, _ = mlp.profile(feats, a, stream=stream)
        prof_ms += 6 * sum(ms)  # warm-up + 5 timed runs of every variant
        del keep
    for f, v, ms in mlp.records():
        tree.add_record(list(f), v, ms)
    t_prof = time.perf_counter() - t0
    t1 = time.perf_counter()
    mlp.train()
    t_mlp = time.perf_counter() - t1
    tree.train()

    per = []
    for k in range(args.test):
        feats, a, keep, rows, nnz = case(3000 + k)
        ms, best = exh.profile(feats, a, stream=stream)
        vm, conf = mlp.select(feats)
        vt, _ = tree.select(feats)
        per.append({"rows": rows, "nnz": nnz, "bytes": spmv_bytes(rows, nnz), "ms": ms, "best": best,
                    "mlp": vm, "conf": conf, "dtree": vt})
        del keep

    def agg(key):
        tsel = [p["ms"][p[key] if key != "default" else default] for p in per]
        reg = [t / p["ms"][p["best"]] - 1.0 for t, p in zip(tsel, per)]
        gbs = sum(p["bytes"] for p in per) / (sum(tsel) * 1e-3) / 1e9
        return {"gbs": gbs, "mean_regret_pct": 100 * statistics.mean(reg),
                "p90_regret_pct": 100 * float(np.percentile(reg, 90)),
                "exact_pct": 100 * statistics.mean(1.0 if (p[key] if key != "default" else default) == p["best"]
                                                   else 0.0 for p in per)}

    best_gbs = sum(p["bytes"] for p in per) / (sum(p["ms"][p["best"]] for p in per) * 1e-3) / 1e9
    res = {"mlp": agg("mlp"), "dtree": agg("dtree"), "default": agg("default")}
    low_conf = sum(1 for p in per if p["conf"] < 0.5)
    line = {
        "metric": METRIC, "value": res["mlp"]["gbs"], "unit": "GB/s", "n_gpus": 1, "dtype": "f64",
        "data": "synthetic", "higher_is_better": True, "vs_baseline": None,
        "config": {"workload": f"spmv float64 CSR, {args.train} training + {args.test} test matrices, rows "
                               f"log-uniform [1e4, {args.rows_max:.0e}], 50% Zipf(s in [1.5,2.5]) / 50% band(7..129)",
                   "features": list(SPMV_FEATURES), "variants": names, "default": names[default]},
        "selection": {"exhaustive_best_gbs": best_gbs, **{k + "_" + m: v for k, d in res.items() for m, v in d.items()},
                      "mlp_low_confidence_calls": low_conf,
                      "best_variant_histogram": {names[v]: sum(1 for p in per if p["best"] == v) for v in range(V)}},
        "cost": {"profiling_wall_s": t_prof, "profiling_gpu_ms": prof_ms, "train_mlp_s": t_mlp,
                 "train_records": len(mlp.records())},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "spmv":
        run_spmv(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
