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
# DRAM bytes (read + write, ncu) of one launch of the SpMV variants on the
# 2e6-row Zipf(1.5) matrix of run_variant (97,990,829 nonzeros)
SPMV_TRAFFIC_2M = {"spmv_df_merge_path": 1200742000.0 + 7975680.0, "spmv_merge_path": 1200358000.0 + 7375360.0,
                   "spmv_vec8": 1212000000.0 + 6400000.0, "spmv_vec16": 1205318000.0 + 7819008.0}
FALLBACK_HBM_GBS = 6400.0
# DRAM bytes (read + write) of one pairs -> pairs sweep of jacobi7_df_32x8 at
# N = 320 (ncu dram__bytes_read.sum + dram__bytes_write.sum, median of the 8
# middle sweeps of a 10-sweep call), scaled to N = 512 by the unknowns; writes
# still dirty in L2 when the kernel ends are not counted by ncu.
DF_PP_TRAFFIC_N320 = 262383232.0 + 216723200.0
HEAT_ALPHA = 0.125              # alpha of the heat workload (stable: <= 1/6)

# The two stencil workloads: the Jacobi region (the headline) and the explicit
# heat step on the same grids.  fp64_ops: float64 operations per point of the
# native families (the "alu" roof); pp_traffic: ncu DRAM bytes of one
# pairs -> pairs sweep at N = 320 per df kernel (see DF_PP_TRAFFIC_N320).
STENCILS = {
    "jacobi7": {"loop": 1, "label": "jacobi7 float64", "fp64_ops": FP64_OPS_PER_POINT,
                "pp_traffic": {"jacobi7_df_32x8": DF_PP_TRAFFIC_N320,
                               "jacobi7_df_32x4": 262181376.0 + 218752000.0}},
    "heat7": {"loop": 4, "label": f"heat7 float64 (alpha = {HEAT_ALPHA})", "fp64_ops": 7,
              "pp_traffic": {"heat7_df_32x8": 262317568.0 + 218154624.0,
                             "heat7_df_32x4": 262190848.0 + 219815424.0}},
}


def stencil_args(ar, kind, n, sweeps, ptrs, status_ptr):
    """The loop's argument block for one call of `sweeps` sweeps (steps)."""
    if kind == "heat7":
        return ar.ArHeat7Args(n, sweeps, HEAT_ALPHA, *ptrs, status_ptr)
    return ar.ArJacobi7Args(n, sweeps, *ptrs, status_ptr)


def stencil_oracle(loops, kind, u, sweeps):
    return loops.heat7(u, sweeps, HEAT_ALPHA) if kind == "heat7" else loops.jacobi7(u, sweeps)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--workload", default="jacobi7",
                   choices=["jacobi7", "heat7", "spmv", "mixed", "daxpy", "nbody", "protocol", "cosched"],
                   help="jacobi7: the headline line; heat7: the same region and grids with the explicit "
                        "heat step; spmv: the learned-selector study; mixed: the persistent mixed-stream "
                        "executor; protocol: K-fold and Online for daxpy, Jacobi and n-body; cosched: GPU / "
                        "host-core splits of loops on host data (each prints one JSON line)")
    p.add_argument("--calls", type=int, default=10000, help="mixed: calls in the stream")
    p.add_argument("--tau", type=float, default=0.5, help="mixed: confidence below which a call is profiled")
    p.add_argument("--train", type=int, default=2000, help="spmv: profiled training matrices")
    p.add_argument("--test", type=int, default=500, help="spmv: held-out test matrices")
    p.add_argument("--rows-max", type=float, default=1e7, help="spmv: largest row count")
    p.add_argument("--epochs", type=int, default=200, help="spmv: MLP epochs")
    p.add_argument("--no-configs", action="store_true",
                   help="jacobi7: skip the bounded records of the other configurations on the line")
    p.add_argument("--kfold", action="store_true",
                   help="spmv: also run the paper's K-fold protocol (K=4, f = 25/50/75 %%, 10 shuffles) and "
                        "Adaptive-100 on all profiled matrices")
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


def max_over_ranks(ms: float, device) -> float:
    """Slowest rank's time: the timed region ends when every replica is done."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(step_bytes: float, steps: int, world: int, ms: float) -> float:
    """Whole-job GB/s: the bytes every replica processed over the slowest
    replica's time (weak scaling: each rank runs the full workload)."""
    return step_bytes * steps * world / (ms * 1e-3) / 1e9


def jacobi_launches(name, N, sweeps):
    """Kernel launches of one ar_jacobi7 / ar_heat7 call: one per sweep, plus
    the catch-up launch of a df call that keeps float pairs between sweeps
    (TMA staging usable: even N at least one box wide)."""
    bx = int(name.split("_")[-1].split("x")[0])
    df_chain = "_df_" in name and N % 2 == 0 and N >= bx + 4 and N >= 10 and sweeps >= 2
    return sweeps + (1 if df_chain else 0)


def workload_bytes(sizes, sweeps):
    return sum(BYTES_PER_POINT * n ** 3 * sweeps for n in sizes)


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(seconds: float, kind: str = "jacobi7"):
    """GB/s of the float64 CPU oracle on a bounded sample of the workload:
    N in {32, 64, 128, 256} at 10 sweeps on all host threads, repeated until
    `seconds` elapse, then N in {32, 64, 128} on one thread for a quarter of
    that (reported as `single_thread`)."""
    import synth
    from oracle import loops

    def rate(sizes, budget):
        grids = {n: synth.grid_inputs(1000 + n, n) for n in sizes}
        t0 = time.perf_counter()
        done, reps = 0.0, 0
        while True:
            for n, u in grids.items():
                stencil_oracle(loops, kind, u, SWEEPS)
                done += BYTES_PER_POINT * n ** 3 * SWEEPS
            reps += 1
            if time.perf_counter() - t0 >= budget:
                break
        dt = time.perf_counter() - t0
        return done / dt / 1e9, reps, dt

    cores = loops.num_threads()
    val, reps, dt = rate((32, 64, 128, 256), seconds)
    loops.set_threads(1)
    try:
        one, reps1, dt1 = rate((32, 64, 128), seconds / 4)
    finally:
        loops.set_threads(cores)
    return {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{STENCILS[kind]['label']} N in (32,64,128,256), 10 sweeps, {reps} passes, {dt:.1f} s "
                      "(the GPU value covers N up to 512)",
            "single_thread": {"value": one, "unit": "GB/s", "cores": 1,
                              "sample": f"N in (32,64,128), 10 sweeps, {reps1} passes, {dt1:.1f} s"},
            "host_cpus": os.cpu_count()}


def jacobi_config(ws, kind="jacobi7"):
    """The stencil workload's `config`, shared by both arms."""
    return {"workload": f"{STENCILS[kind]['label']} N in {{32,64,128,256,384,512}}, 10 sweeps, depth-2 tree on "
                        "(N, sweeps) over 16 variants", "sizes": SIZES, "sweeps": SWEEPS,
            "parallelism": "replicas" if ws > 1 else "single-gpu",
            "l2": "inputs larger than L2: six grids of 1.68 GB in all; each sweep reads and writes "
                  "3.36 GB, 33.6 GB per step"}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    from oracle import loops

    kind = args.workload if args.workload in STENCILS else "jacobi7"
    sizes = (32, 64, 128, 256)
    import synth

    grids = {n: synth.grid_inputs(1000 + n, n) for n in sizes}
    for _ in range(args.warmup):
        for n, u in grids.items():
            stencil_oracle(loops, kind, u, SWEEPS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for n, u in grids.items():
            stencil_oracle(loops, kind, u, SWEEPS)
    dt = time.perf_counter() - t0
    val = workload_bytes(sizes, SWEEPS) * args.steps / dt / 1e9
    sample = f"{STENCILS[kind]['label']} N in {sizes}, 10 sweeps per step (bounded sample of N up to 512)"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": jacobi_config(ws, kind),
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
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
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
def other_configs(args):
    """The other configurations of the workload, each bounded so that the
    default run stays within a few minutes, as compact records for the
    headline line: daxpy (exhaustive selection), SpMV selection (MLP vs tree
    vs default on 300 training and 100 held-out matrices), n-body per N with
    the batched form, the paper's evaluation protocol (K-fold and Online) on
    daxpy, Jacobi and n-body, co-scheduling and device selection on host
    data, and a 2,560-call mixed stream with the confidence fallback."""
    import torch

    out = {}
    t = time.perf_counter()
    d = daxpy_record(50, 5)
    out["daxpy"] = {"value": d["value"], "unit": "GB/s", "selection": d["selection"], "roofline": d["roofline"],
                    "warm_graph": d["warm_graph"], "config": d["config"]["workload"],
                    "wall_s": time.perf_counter() - t}
    out["daxpy"]["selection"].pop("profile_gbs", None)
    torch.cuda.empty_cache()
    t = time.perf_counter()
    sp = spmv_study(300, 100, 1e7, 200)
    sel = sp["selection"]
    out["spmv"] = {"value": sp["value"], "unit": "GB/s", "config": sp["config"]["workload"],
                   "selection": {k: sel[k] for k in ("exhaustive_best_gbs", "mlp_gbs", "dtree_gbs", "default_gbs",
                                                    "mlp_mean_regret_pct", "dtree_mean_regret_pct",
                                                    "default_mean_regret_pct", "mlp_exact_pct",
                                                    "mlp_low_confidence_calls")},
                   "roofline": sp["roofline"], "gather_floor": sp["gather_floor"], "cost": sp["cost"],
                   "wall_s": time.perf_counter() - t}
    torch.cuda.empty_cache()
    t = time.perf_counter()
    nb = nbody_record(3, 2)
    out["nbody"] = {"value": nb["value"], "unit": "GFLOP/s", "config": nb["config"]["workload"],
                    "per_N": nb["selection"]["per_N"], "roofline": nb["roofline"], "batched": nb["batched"],
                    "wall_s": time.perf_counter() - t}
    torch.cuda.empty_cache()
    t = time.perf_counter()
    pr = protocol_record(200)
    out["protocol"] = {"value": pr["value"], "unit": "%", "metric": pr["metric"], "config": pr["config"],
                       "loops": {name: {"adaptive_75": {m: r["kfold_mean_regret_pct"][m]["adaptive_75"]
                                                        for m in r["kfold_mean_regret_pct"]},
                                        "mlp": r["kfold_mean_regret_pct"]["mlp"],
                                        **({"mlp_n_only": r["kfold_mean_regret_pct_n_only"]["mlp"]}
                                           if "kfold_mean_regret_pct_n_only" in r else {}),
                                        "online_mean_regret_pct": r["online"]["mean_regret_pct"]}
                                 for name, r in pr["loops"].items()},
                       "wall_s": time.perf_counter() - t}
    torch.cuda.empty_cache()
    t = time.perf_counter()
    cs = cosched_record()
    out["cosched"] = {"value": cs["value"], "unit": "GB/s", "config": cs["config"],
                      "daxpy": {k: v for k, v in cs["daxpy"].items() if k != "per_n"},
                      "daxpy_best_fraction_per_n": {str(p["n"]): p["best_fraction"] for p in cs["daxpy"]["per_n"]},
                      "spmv": cs["spmv"], "wall_s": time.perf_counter() - t}
    torch.cuda.empty_cache()
    t = time.perf_counter()
    mx = mixed_record(2560, args.tau)
    out["mixed"] = {"value": mx["value"], "unit": "GB/s", "config": mx["config"]["workload"],
                    "stream": mx["stream"], "selection": mx["selection"], "fallback": mx["fallback"],
                    "cost": mx["cost"], "roofline": mx["roofline"], "wall_s": time.perf_counter() - t}
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import paper_2303_08873_b300 as ar
    import synth

    kind = args.workload
    spec = STENCILS[kind]
    loop = spec["loop"]
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
    argblocks = {n: stencil_args(ar, kind, n, SWEEPS, [b.data_ptr() for b in bufs[n]], status.data_ptr())
                 for n in SIZES}

    # --- profiling + training (untimed): exhaustive over N x sweeps
    region = ar.Region(kind, 2, "dtree,2,reps=5", 10 ** 9)
    V = region.add_builtin(loop)
    region.set_l2_flush(flush, flush.numel())
    table = {}
    t_prof = time.perf_counter()
    for n in SIZES:
        for s in TRAIN_SWEEPS:
            a = stencil_args(ar, kind, n, s, [b.data_ptr() for b in bufs[n]], status.data_ptr())
            ms, best = region.profile([n, s], a, stream=stream)
            table[(n, s)] = (ms, best)
    t_prof = time.perf_counter() - t_prof
    region.train()
    tree = region.tree()
    default = ar.loop_default_variant(loop)
    names = [ar.loop_variant_name(loop, v) for v in range(V)]
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
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    step_bytes = workload_bytes(SIZES, SWEEPS)
    value = job_rate(step_bytes, args.steps, ws, ms)
    assert int(status[0].item()) == 0, "a bounded wait inside a TMA kernel timed out"

    # --- dominant kernel roofline: the N=512 invocation's sweeps
    big_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k0, k1)) / SWEEPS
    achieved = BYTES_PER_POINT * big ** 3 / (big_ms * 1e-3) / 1e9
    vbig = chosen[big]
    if "_df_" in names[vbig]:
        pp = spec["pp_traffic"].get(names[vbig])
        traffic = pp * (big / 320.0) ** 3 if pp else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": peak_src,
                "kernel": names[vbig],
                "note": "achieved: the N=512 invocation's time per sweep (10 sweep launches + 1 catch-up); "
                        "traffic: DRAM bytes of one pairs->pairs sweep launch, measured at N=320 and scaled"}
    else:
        alu_gbs = fp64_fma / spec["fp64_ops"] * BYTES_PER_POINT / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": alu_gbs, "unit": "GB/s",
                "frac": achieved / alu_gbs, "traffic": None,
                "peak_source": "float64 issue rate measured by ar_measure_fma_rates x 16 B / "
                               f"{spec['fp64_ops']} FP64 ops per point",
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

    # --- the tree's regret on points it was not trained on: (a) sweeps = 10
    # held out (trained on sweeps 1, 5, 20); (b) leave one N out (trained on
    # the other five sizes, every sweep count)
    def tree_regret(train_keys, test_n):
        rt = ar.Region(f"{kind}-heldout", 2, "dtree,2", 10 ** 9)
        for v in range(V):
            rt.register(names[v], float(v), lambda a_, v_, x_, s_, u_: 0)
        for key in train_keys:
            for v in range(V):
                rt.add_record(list(key), v, table[key][0][v])
        rt.train()
        out = []
        for n in test_n:
            ms_n, best = table[(n, SWEEPS)]
            out.append(100 * (ms_n[rt.select([n, SWEEPS])[0]] / ms_n[best] - 1))
        return out

    held_sweeps = tree_regret([k for k in table if k[1] != SWEEPS], SIZES)
    held_n = [tree_regret([k for k in table if k[0] != n], [n])[0] for n in SIZES]

    # --- the best native float64 variant (families naive, smem, tma) at N = 512
    ms_big = table[(big, SWEEPS)][0]
    v64 = min(range(12), key=lambda v: ms_big[v])
    gbs64 = BYTES_PER_POINT * big ** 3 * SWEEPS / ms_big[v64] / 1e6
    alu64 = fp64_fma / spec["fp64_ops"] * BYTES_PER_POINT / 1e9
    native64 = {"kernel": names[v64], "gbs": gbs64, "alu_roof_gbs": alu64, "alu_frac": gbs64 / alu64,
                "hbm_frac": gbs64 / hbm_peak,
                "note": "best of the native float64 families (naive, smem, tma) at N = 512, 10 sweeps, from the "
                        "profile table; roof: measured float64 FMA issue rate / 6 float64 ops per point x 16 B"}

    # --- the paper's Online mode (Section 4.2): one fresh region per N, default
    # min_train_data (= number of variants), RoundRobin exploration over real
    # invocations, automatic training, then the tree's choice; regret from the
    # exhaustive table above
    online = []
    for n in SIZES:
        ro = ar.Region(f"{kind}-online-{n}", 2, "dtree,2")
        ro.add_builtin(loop)
        explore_ms = 0.0
        calls = 0
        while not ro.info()["trained"]:
            ro.invoke([n, SWEEPS], argblocks[n], stream=stream)
            calls += 1
        stream.synchronize()
        explore_ms = sum(ms_ for _, _, ms_ in ro.records())
        v_on, _ = ro.select([n, SWEEPS])
        ms_n, best = table[(n, SWEEPS)]
        online.append({"N": n, "explore_calls": calls, "selected": names[v_on],
                       "regret_pct": 100 * (ms_n[v_on] / ms_n[best] - 1),
                       "explore_overhead_pct": 100 * (explore_ms / (calls * ms_n[best]) - 1)})

    # --- end to end through the library's host-buffer call (ar_invoke_host):
    # per N and lane its own stream carrying the copy of u0 in, the selected
    # variant's sweeps and the copy of the result out (one cudaMemcpyAsync
    # each way).  Steps alternate between two lanes (own device grids, status
    # arrays and host result buffers), so one step's copies out overlap the
    # next step's copies in on the duplex link, and the streams of different
    # N overlap one grid's copies with another's sweeps
    lanes = 2
    host_in = {n: bufs[n][0].cpu().pin_memory() for n in SIZES}
    lane_bufs = {n: [bufs[n]] + [[torch.empty_like(b) for b in bufs[n]] for _ in range(lanes - 1)] for n in SIZES}
    lane_status = {n: [torch.zeros(2, dtype=torch.int32, device=dev) for _ in range(lanes)] for n in SIZES}
    lane_args = {n: [stencil_args(ar, kind, n, SWEEPS, [b.data_ptr() for b in lane_bufs[n][q]],
                                  lane_status[n][q].data_ptr()) for q in range(lanes)] for n in SIZES}
    host_out = {n: [torch.empty_like(host_in[n]).pin_memory() for _ in range(lanes)] for n in SIZES}
    e2e_steps = max(4, min(args.steps, 10))
    streams = {n: [torch.cuda.Stream(device=dev) for _ in range(lanes)] for n in SIZES}
    order = sorted(SIZES, reverse=True)
    copies = {n: [([(host_in[n], lane_bufs[n][q][0], 8 * n ** 3)], [(host_out[n][q], lane_bufs[n][q][1], 8 * n ** 3)])
                  for q in range(lanes)] for n in SIZES}
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for n in SIZES:
        for q in range(lanes):
            streams[n][q].wait_event(a0)
    for k in range(e2e_steps):
        q = k % lanes
        for n in order:
            region.invoke_host([n, SWEEPS], lane_args[n][q], *copies[n][q], stream=streams[n][q])
    for n in SIZES:
        for q in range(lanes):
            stream.wait_stream(streams[n][q])
    a1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a0.elapsed_time(a1) / e2e_steps
    ref0 = bufs[big][1].cpu()
    for q in range(lanes):
        assert torch.equal(host_out[big][q], ref0), "host result differs from the device result"
    assert all(int(t[0]) == 0 for n in SIZES for t in lane_status[n]), "a status array reports an error"
    h2d = sum(8 * n ** 3 for n in SIZES)
    e2e = {"value": step_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": h2d, "ms_per_step": e2e_ms,
           "note": "ar_invoke_host per N (pinned host u0 in, the region's selected variant, result out), "
                   "steps alternating between two lanes of device grids, one stream per N and lane"}
    del lane_bufs, lane_args, lane_status, host_out, host_in, copies, streams

    configs = None
    if rank == 0 and ws == 1 and kind == "jacobi7" and not args.no_configs:
        del bufs, argblocks, flush
        torch.cuda.empty_cache()
        configs = other_configs(args)

    if rank != 0:
        return
    cpu = cpu_oracle_rate(args.cpu_seconds, kind) if ws == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64 data, f32-pair arithmetic", "data": "synthetic",
        "config": jacobi_config(ws, kind),
        "selection": {"exhaustive_best_gbs": step_bytes / t_best / 1e6, "default_gbs": step_bytes / t_def / 1e6,
                      "selected_table_gbs": step_bytes / t_sel / 1e6, "regret_pct": regret,
                      "default_variant": names[default], "per_N": per, "tree": tree,
                      "online": {"mean_regret_pct": statistics.mean(o["regret_pct"] for o in online),
                                 "per_N": online},
                      "held_out": {"sweeps10_mean_regret_pct": statistics.mean(held_sweeps),
                                   "sweeps10_per_N": held_sweeps,
                                   "leave_one_N_out_mean_regret_pct": statistics.mean(held_n),
                                   "leave_one_N_out_per_N": held_n,
                                   "note": "regret_pct above is in-sample (the tree is trained on all 24 profiled "
                                           "points); here sweeps = 10 is held out, or each N in turn"},
                      "profiling_s": t_prof, "profiled_points": len(table), "variants": V},
        "native_f64": native64,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * sum(jacobi_launches(names[chosen[n]], n, SWEEPS) for n in SIZES),
        "clocks": clk,
        "fp64_fma_per_s": fp64_fma,
    }
    line["config"]["arithmetic"] = (
        "float64 in and out; the df variants the tree selects compute in float pairs (two float32 values, "
        "~2^-46 relative per split value, TwoSum chains, one float64 add per output); the best native float64 "
        "variant is reported under native_f64")
    if configs is not None:
        line["configs"] = configs
    print(json.dumps(line), flush=True)



# ---------------------------------------------------------------- SpMV selector study
SPMV_FEATURES = ("rows", "nnz", "mean", "var", "max")


def spmv_bytes(rows, nnz):
    """Algorithmic bytes of one y = A x: val + col per nonzero, row pointers,
    x read once, y written once."""
    return 12.0 * nnz + 4.0 * (rows + 1) + 8.0 * rows + 8.0 * rows


def run_spmv(args):
    print(json.dumps(spmv_study(args.train, args.test, args.rows_max, args.epochs, kfold=args.kfold)), flush=True)


def kfold_protocol(table, V, F, epochs, shuffles=10, K=4, seed=77, models=("mlp", "dtree", "rfc", "static_best")):
    """The paper's evaluation protocol (Section 4.1): inputs split into K equal
    groups; a fraction f of the groups trains the model and the others test
    it (Adaptive-25/50/75; every group trains and tests across the K
    rotations); repeated over `shuffles` permutations.  Adaptive-100 trains
    and tests on everything; Static,Best is the single variant fastest in
    total over the training groups.  `table` holds (features, per-variant
    mean ms).  Returns mean regret (%) per model and fraction."""
    import paper_2303_08873_b300 as ar

    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(table)

    def fit(kind, idx):
        spec = {"mlp": f"mlp,64,epochs={epochs},seed=7", "dtree": "dtree,2", "rfc": "rfc,10,4"}[kind]
        r = ar.Region("kfold", F, spec, 10 ** 9)
        for v in range(V):
            r.register(f"v{v}", float(v), lambda a, v_, x, s_, u: 0)
        for i in idx:
            f, ms = table[i]
            for v in range(V):
                r.add_record(f, v, ms[v])
        r.train()
        return r

    def regret(model, idx):
        out = []
        for i in idx:
            f, ms = table[i]
            v = model(f)
            out.append(ms[v] / min(ms) - 1.0)
        return 100.0 * statistics.mean(out)

    res = {}
    for kind in models:
        res[kind] = {}
        for frac in (1, 2, 3):
            vals = []
            for _ in range(shuffles):
                perm = rng.permutation(n)
                groups = np.array_split(perm, K)
                for rot in range(K):
                    tr = np.concatenate([groups[(rot + g) % K] for g in range(frac)])
                    te = np.concatenate([groups[(rot + g) % K] for g in range(frac, K)])
                    if kind == "static_best":
                        tot = [sum(table[i][1][v] for i in tr) for v in range(V)]
                        vb = int(np.argmin(tot))
                        vals.append(regret(lambda f, vb=vb: vb, te))
                    else:
                        r = fit(kind, tr)
                        vals.append(regret(lambda f, r=r: r.select(f)[0], te))
            res[kind][f"adaptive_{25 * frac}"] = statistics.mean(vals)
        if kind == "static_best":
            tot = [sum(t[1][v] for t in table) for v in range(V)]
            vb = int(np.argmin(tot))
            res[kind]["adaptive_100"] = regret(lambda f: vb, range(n))
        else:
            r = fit(kind, range(n))
            res[kind]["adaptive_100"] = regret(lambda f, r=r: r.select(f)[0], range(n))
    return res


def spmv_study(n_train, n_test, rows_max, epochs, kfold=False):
    """Config 3: profile `n_train` seeded matrices (8 variants, 5 reps after a
    warm-up, L2 flushed), train the MLP selector on the device and the depth-2
    tree on the same records, then compare their choices with the exhaustive
    argmin and the fixed default (thread per row) on `n_test` held-out
    matrices.  Returns the JSON-ready result."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    fwsb = ar.ar_csr_features_workspace_bytes(0)
    fws = torch.empty(fwsb, dtype=torch.uint8, device=dev)
    f5 = torch.zeros(5, dtype=torch.float32, device=dev)
    sink = torch.empty(1, dtype=torch.int64, device=dev)
    fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def floor_ms(keep, nnz):
        """Mean time of the gather-floor kernel on one matrix (3 runs after a
        warm-up, L2 flushed before each, like the variants' profiles)."""
        _, c, v, x, _, _ = keep
        t = []
        with torch.cuda.stream(stream):
            ar.ar_spmv_gather_floor(nnz, c, v, x, sink, stream=stream)
            for _ in range(3):
                flush.fill_(1)
                fe0.record(stream)
                ar.ar_spmv_gather_floor(nnz, c, v, x, sink, stream=stream)
                fe1.record(stream)
                stream.synchronize()
                t.append(fe0.elapsed_time(fe1))
        return statistics.mean(t)

    def case(seed):
        prm = synth.spmv_matrix_params(seed, rows_max=rows_max)
        rp, c, v = synth.spmv_matrix(seed, prm, device="cuda")
        rows = prm["rows"]
        nnz = int(rp[-1].item())
        x = synth.spmv_x(seed, rows, device="cuda")
        y = torch.empty(rows, dtype=torch.float64, device=dev)
        # the largest workspace any variant needs on this matrix (merge path:
        # 24 B per 4096 path items; binned: 12 B per row): a variant whose
        # launch is refused is marked unusable for the rest of the study
        wsb = max(ar.ar_spmv_workspace_bytes(var, rows, nnz) for var in range(ar.loop_num_variants(ar.AR_LOOP_SPMV)))
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        ar.ar_csr_features(rows, rp, f5, fws, fwsb, stream=stream)
        stream.synchronize()
        feats = f5.cpu().tolist()
        a = ar.ArSpmvArgs(rows, nnz, rp.data_ptr(), c.data_ptr(), v.data_ptr(), x.data_ptr(), y.data_ptr(),
                          ws.data_ptr(), wsb)
        return feats, a, (rp, c, v, x, y, ws), rows, nnz, prm["kind"]

    mlp = ar.Region("spmv-mlp", 5, f"mlp,64,epochs={epochs},seed=7", 10 ** 9)
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
    table = []
    for k in range(n_train):
        feats, a, keep, rows, nnz, _ = case(1000 + k)
        ms, _ = mlp.profile(feats, a, stream=stream)
        prof_ms += 6 * sum(ms)  # warm-up + 5 timed runs of every variant
        table.append((feats, ms))
        del keep
    for f, v, ms in mlp.records():
        tree.add_record(list(f), v, ms)
    t_prof = time.perf_counter() - t0
    t1 = time.perf_counter()
    mlp.train()
    t_mlp = time.perf_counter() - t1
    tree.train()

    per = []
    for k in range(n_test):
        feats, a, keep, rows, nnz, kind = case(3000 + k)
        ms, best = exh.profile(feats, a, stream=stream)
        vm, conf = mlp.select(feats)
        vt, _ = tree.select(feats)
        per.append({"rows": rows, "nnz": nnz, "bytes": spmv_bytes(rows, nnz), "ms": ms, "best": best,
                    "mlp": vm, "conf": conf, "dtree": vt, "floor_ms": floor_ms(keep, nnz), "kind": kind})
        table.append((feats, ms))
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
        "config": {"workload": f"spmv float64 CSR, {n_train} training + {n_test} test matrices, rows "
                               f"log-uniform [1e4, {rows_max:.0e}], 50% Zipf(s in [1.5,2.5]) / 50% band(7..129)",
                   "features": list(SPMV_FEATURES), "variants": names, "default": names[default]},
        "selection": {"exhaustive_best_gbs": best_gbs, **{k + "_" + m: v for k, d in res.items() for m, v in d.items()},
                      "mlp_low_confidence_calls": low_conf,
                      "best_variant_histogram": {names[v]: sum(1 for p in per if p["best"] == v) for v in range(V)}},
        "cost": {"profiling_wall_s": t_prof, "profiling_gpu_ms": prof_ms, "train_mlp_s": t_mlp,
                 "train_records": len(mlp.records()),
                 # exhaustive profiling of one call (warm-up + 5 timed runs of every
                 # variant), and after how many calls the learned selector's one-off
                 # training profiles cost less than profiling every call
                 "exhaustive_per_call_gpu_ms": statistics.mean(6 * sum(p["ms"]) for p in per),
                 "break_even_calls": prof_ms / statistics.mean(6 * sum(p["ms"]) for p in per)},
    }
    hbm_peak, peak_src = peaks()
    # the variant most often fastest on the test set, and its DRAM bytes per
    # launch on the 2e6-row Zipf(1.5) matrix from one ncu capture (~1.20 GB
    # read + ~8 MB written against 1.216 GB algorithmic)
    dom = max(range(V), key=lambda v: sum(1 for p in per if p["best"] == v))
    line["roofline"] = {"bound": "hbm", "achieved": res["mlp"]["gbs"], "peak": hbm_peak, "unit": "GB/s",
                        "frac": res["mlp"]["gbs"] / hbm_peak, "peak_source": peak_src,
                        "traffic": SPMV_TRAFFIC_2M.get(names[dom]),
                        "kernel": names[dom],
                        "note": "achieved: the MLP-selected variants over the test matrices (sum of algorithmic "
                                "bytes / sum of times); traffic: DRAM bytes of one launch of the dominant kernel "
                                "on the 2e6-row Zipf(1.5) matrix"}
    # the memory-side floor of every test matrix (ar_spmv_gather_floor: col and
    # val streamed, x gathered, no row logic, no float64 arithmetic)
    floor_gbs = sum(p["bytes"] for p in per) / (sum(p["floor_ms"] for p in per) * 1e-3) / 1e9
    line["gather_floor"] = {"gbs": floor_gbs, "mlp_frac": res["mlp"]["gbs"] / floor_gbs,
                            "exhaustive_best_frac": best_gbs / floor_gbs,
                            "zipf_mlp_frac": _floor_frac(per, "mlp", lambda p: p["kind"] == "zipf"),
                            "band_mlp_frac": _floor_frac(per, "mlp", lambda p: p["kind"] == "band"),
                            "note": "algorithmic bytes over the time of a kernel that only streams col and val and "
                                    "gathers x[col] (8 in flight per thread): the bound random 8-byte gathers "
                                    "(32-byte sectors) set on power-law matrices"}
    if kfold:
        t2 = time.perf_counter()
        line["kfold_mean_regret_pct"] = kfold_protocol(table, V, 5, epochs)
        line["kfold_wall_s"] = time.perf_counter() - t2
    return line


def _floor_frac(per, key, keep):
    """Selected time's share of the gather floor over the matrices `keep`
    admits (None if none)."""
    sel = [p for p in per if keep(p)]
    if not sel:
        return None
    return sum(p["floor_ms"] for p in sel) / sum(p["ms"][p[key]] for p in sel)


# ---------------------------------------------------------------- mixed stream
LOOPS = ("daxpy", "jacobi7", "spmv", "nbody")
NBODY_FLOPS = 20.0


class Arena:
    """Bump allocator over one device tensor, reset per batch."""

    def __init__(self, t):
        self.t, self.off = t, 0

    def take(self, nbytes):
        o = (self.off + 255) & ~255
        if o + nbytes > self.t.numel() * self.t.element_size():
            raise MemoryError
        self.off = o + nbytes
        return self.t.data_ptr() + o


def mixed_record(n_calls, tau, reps_fb=2, regret_sample=96):
    """Config 5: a stream of `n_calls` region invocations (loop ~ U{4}, sizes
    log-uniform over each loop's range, SpMV from a pool of 32 matrices) run by
    the persistent executor in batches of 256 replayed from one captured CUDA
    graph; per-loop MLPs choose the variants on the device.  Training set and
    fallback both go through the library (ar_exec_fallback): the training
    calls are profiled exhaustively into one region per loop, which is trained
    and uploaded; after every batch the calls whose confidence is below tau
    are profiled the same way (unless their features were profiled before),
    their records join the regions, and the regions are retrained and their
    device models refreshed before the next batch.  Regret is scored on a
    random sample of the stream by exhaustive profiling (5 timed runs)."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    B = ar.AR_EXEC_MAX_CALLS
    loop_ids, sizes = synth.mixed_stream(5, n_calls)
    # pool of SpMV matrices (device-generated), shared inputs; y per call
    pool = []
    for k in range(32):
        prm = synth.spmv_matrix_params(5000 + k)
        rp, c, v = synth.spmv_matrix(5000 + k, prm, device="cuda")
        x = synth.spmv_x(5000 + k, prm["rows"], device="cuda")
        pool.append((prm["rows"], int(rp[-1].item()), rp, c, v, x))
    f64 = torch.empty((64 << 30) // 8, dtype=torch.float64, device=dev).uniform_(-1.0, 1.0)
    f32 = torch.empty((1 << 30) // 4, dtype=torch.float32, device=dev).uniform_(0.5, 1.0)
    scratch = torch.empty((48 << 30) // 8, dtype=torch.float64, device=dev)

    def make_call(loop, size, a64, a32, sc):
        """ArExecCall for one invocation; inputs point into the random arenas,
        outputs into the scratch arena.  Returns (call, algorithmic bytes, flops)."""
        c = ar.ArExecCall(loop=int(loop))
        if loop == 0:
            n = int(size)
            c.n, c.a = n, 1.5
            c.in0, c.out0 = a64.take(8 * n), sc.take(8 * n)
            return c, 24.0 * n, 2.0 * n
        if loop == 1:
            N = int(size)
            c.n, c.sweeps = N, 10
            c.in0, c.out0, c.out1 = a64.take(8 * N ** 3), sc.take(8 * N ** 3), sc.take(8 * N ** 3)
            return c, 16.0 * N ** 3 * 10, 6.0 * N ** 3 * 10
        if loop == 2:
            rows, nnz, rp, cl, v, x = pool[int(size)]
            c.n, c.nnz = rows, nnz
            c.in0, c.in1, c.in2, c.in3 = rp.data_ptr(), cl.data_ptr(), v.data_ptr(), x.data_ptr()
            c.out0 = sc.take(8 * rows)
            nb = -(-(rows + nnz) // 4096)
            c.out1, c.out1_bytes = sc.take(16 * nb), 16 * nb
            return c, spmv_bytes(rows, nnz), 2.0 * nnz
        N = int(size)
        c.n, c.eps = N, synth.NBODY_EPS
        c.in0, c.out0 = a32.take(16 * N), sc.take(16 * N)
        c.out1, c.out1_bytes = sc.take(16 * N * 8), 16 * N * 8  # partial sums of up to 8 j chunks
        return c, 0.0, NBODY_FLOPS * N * N

    def arenas():
        return Arena(f64), Arena(f32), Arena(scratch)

    # executor buffers and one captured graph for a full batch
    table_h = torch.zeros(96 * B, dtype=torch.uint8).pin_memory()
    table_d = torch.zeros(96 * B, dtype=torch.uint8, device=dev)
    o_var = torch.zeros(B, dtype=torch.int32, device=dev)
    o_conf = torch.zeros(B, dtype=torch.float32, device=dev)
    o_feat = torch.zeros((B, 8), dtype=torch.float32, device=dev)
    o_t0 = torch.zeros(B, dtype=torch.int64, device=dev)
    o_t1 = torch.zeros(B, dtype=torch.int64, device=dev)
    o_st = torch.zeros(B, dtype=torch.int32, device=dev)
    h_out = [torch.zeros_like(t, device="cpu").pin_memory() for t in (o_var, o_conf, o_feat, o_t0, o_t1, o_st)]
    wsb = ar.ar_exec_workspace_bytes(B)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    fb_wsb = ar.ar_exec_fallback_workspace_bytes(1 << 24)
    fb_ws = torch.empty(fb_wsb, dtype=torch.uint8, device=dev)

    def run_batch(calls, models=None):
        """Eager batch: returns per-call (variant, conf, features, ns, status)."""
        n = len(calls)
        table_d[:96 * n].copy_(torch.frombuffer(bytearray(ar.exec_table_bytes(calls)), dtype=torch.uint8))
        ar.ar_exec_batch(table_d, n, models, None, o_var, o_conf, o_feat, o_t0, o_t1, o_st, ws, wsb, stream=stream)
        stream.synchronize()
        return (o_var[:n].cpu().numpy(), o_conf[:n].cpu().numpy(), o_feat[:n].cpu().numpy(),
                (o_t1[:n] - o_t0[:n]).cpu().numpy(), o_st[:n].cpu().numpy())

    def new_records_ms(regs, before):
        """Executor ms of the records added since `before` (per-loop counts)."""
        return sum(ms for L in range(4) if regs[L] is not None for _, _, ms in regs[L].records(before[L]))

    def counts(regs):
        return [regs[L].counts()[0] if regs[L] is not None else 0 for L in range(4)]

    nfeat = {0: 1, 1: 3, 2: 5, 3: 1}  # the executor's features per loop (ar_loops.h)
    # --- training: the library's exhaustive profiling of sampled calls per loop
    rng = np.random.Generator(np.random.PCG64(55))
    lo = {0: 2.0 ** 10, 1: 32.0, 3: 1024.0}
    hi = {0: 2.0 ** 24, 1: 512.0, 3: 262144.0}
    train_sizes = {L: [int(np.exp(rng.uniform(np.log(lo[L]), np.log(hi[L])))) for _ in range(24)] for L in (0, 1, 3)}
    train_sizes[2] = list(range(32))
    # daxpy tie=0.03: inside the persistent executor daxpy variants that differ
    # only in block size run alike, and timing noise would otherwise pick
    # among them at random, leaving the MLP unsure; the other loops keep the
    # 0.5 % tie of the paper reading
    regions = [ar.Region(f"mixed-{LOOPS[L]}", nfeat[L], "mlp,64,epochs=400,seed=3" + (",tie=0.03" if L == 0 else ""), 10 ** 9)
               for L in range(4)]
    for L in range(4):
        regions[L].add_exec_variants(L)
    models = ar.ArExecModels()
    models.H = 64
    keep = []
    t0w = time.perf_counter()
    for L in range(4):
        a64, a32, sc = arenas()
        calls = [make_call(L, s_, a64, a32, sc)[0] for s_ in train_sizes[L]]
        feats = run_batch(calls)[2]
        only = [regions[q] if q == L else None for q in range(4)]
        ar.ar_exec_fallback(calls, feats, np.zeros(len(calls), np.float32), 0.5, only, reps_fb, None, False,
                            fb_ws, fb_wsb, stream=stream)
        regions[L].train()
        m = regions[L].mlp()
        th, mu, sd = (torch.from_numpy(m[k]).to(dev) for k in ("theta", "mu", "sd"))
        keep += [th, mu, sd]
        models.F[L], models.V[L] = m["F"], m["V"]
        models.theta[L], models.mu[L], models.sd[L] = th.data_ptr(), mu.data_ptr(), sd.data_ptr()
    train_ms = sum(ms for r in regions for _, _, ms in r.records()) * (reps_fb + 1) / reps_fb
    train_wall = time.perf_counter() - t0w
    train_counts = counts(regions)

    # --- capture one batch graph: table copy, executor, result copies
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        table_d.copy_(table_h, non_blocking=True)
        ar.ar_exec_batch(table_d, B, models, None, o_var, o_conf, o_feat, o_t0, o_t1, o_st, ws, wsb, stream=stream)
        for h, d in zip(h_out, (o_var, o_conf, o_feat, o_t0, o_t1, o_st)):
            h.copy_(d, non_blocking=True)

    batches = [range(s0, min(s0 + B, n_calls)) for s0 in range(0, n_calls, B)]
    # full batches replay the graph; a final partial batch runs eagerly
    lat = {L: [] for L in range(4)}
    byts = flops = 0.0
    low = fb_profiled = 0
    low_by = [0, 0, 0, 0]
    fb_wall = 0.0
    chosen = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    batch_ms = []
    for bi, idx in enumerate(batches):
        a64, a32, sc = arenas()
        calls = []
        for q in idx:
            c, b_, f_ = make_call(loop_ids[q], sizes[q], a64, a32, sc)
            calls.append(c)
            byts += b_
            flops += f_ if loop_ids[q] == 3 else 0.0
        n = len(calls)
        table_h[:96 * n].copy_(torch.frombuffer(bytearray(ar.exec_table_bytes(calls)), dtype=torch.uint8))
        ev0.record(stream)
        if n == B:
            with torch.cuda.stream(stream):  # replay() runs on the current stream
                g.replay()
        else:
            with torch.cuda.stream(stream):
                table_d[:96 * n].copy_(table_h[:96 * n], non_blocking=True)
                ar.ar_exec_batch(table_d, n, models, None, o_var, o_conf, o_feat, o_t0, o_t1, o_st, ws, wsb,
                                 stream=stream)
                for h, d in zip(h_out, (o_var, o_conf, o_feat, o_t0, o_t1, o_st)):
                    h.copy_(d, non_blocking=True)
        ev1.record(stream)
        stream.synchronize()
        batch_ms.append(ev0.elapsed_time(ev1))
        var, conf, feat, t0n, t1n, st = (h.numpy()[:n].copy() for h in h_out)
        assert np.all(st == 0), "executor status"
        for k, q in enumerate(idx):
            L = int(loop_ids[q])
            lat[L].append((int(t1n[k]) - int(t0n[k])) * 1e-3)
            chosen.append((L, int(sizes[q]), int(var[k])))
        # the confidence fallback through the library: profile, record, retrain, refresh the device models
        low += int(np.sum(conf < tau))
        for k, q in enumerate(idx):
            low_by[int(loop_ids[q])] += int(conf[k] < tau)
        tf = time.perf_counter()
        _, cnt = ar.ar_exec_fallback(calls, feat, conf, tau, regions, reps_fb, models, True, fb_ws, fb_wsb,
                                     stream=stream)
        fb_wall += time.perf_counter() - tf
        fb_profiled += cnt
    stream_ms = sum(batch_ms)
    fb_ms = new_records_ms(regions, train_counts) * (reps_fb + 1) / reps_fb
    # --- regret on a sample of the stream: exhaustive profiling (5 timed runs)
    # of each sampled call through the library into fresh regions
    samp = rng.choice(len(chosen), size=min(regret_sample, len(chosen)), replace=False)
    judge = [ar.Region(f"judge-{LOOPS[L]}", nfeat[L], "exhaustive", 10 ** 9) for L in range(4)]
    for L in range(4):
        judge[L].add_exec_variants(L)
    regrets = {L: [] for L in range(4)}
    exh_ms = []
    for q in samp:
        L, size, v = chosen[q]
        c = make_call(L, size, *arenas())[0]
        feats = run_batch([c])[2]
        only = [judge[p] if p == L else None for p in range(4)]
        ar.ar_exec_fallback([c], feats, np.zeros(1, np.float32), 0.5, only, 5, None, False, fb_ws, fb_wsb,
                            stream=stream)
        key = tuple(float(x) for x in np.asarray(feats[0][:nfeat[L]], dtype=np.float32))
        per_v = {}
        for f_, v_, ms_ in judge[L].records():
            if f_ == key:
                per_v.setdefault(v_, []).append(ms_)
        means = [statistics.mean(per_v[w]) for w in range(ar.ar_exec_num_variants(L))]
        regrets[L].append(means[v] / min(means) - 1.0)
        exh_ms.append((reps_fb + 1) * sum(means))  # exhaustive profile of this call at the fallback's reps
    all_reg = [x for L in range(4) for x in regrets[L]]
    hbm_peak, peak_src = peaks()
    _, fp32_fma = ar.ar_measure_fma_rates()
    fp32_roof = fp32_fma / 12.0 * NBODY_FLOPS / 1e9
    mem_gbs = byts / (stream_ms * 1e-3) / 1e9
    nb_gflops = flops / (stream_ms * 1e-3) / 1e9
    exhaustive_all_ms = statistics.mean(exh_ms) * n_calls
    return {
        "metric": METRIC, "value": mem_gbs, "unit": "GB/s", "n_gpus": 1,
        "dtype": "f64 (daxpy, Jacobi, SpMV) / f32 (n-body)", "data": "synthetic", "higher_is_better": True,
        "vs_baseline": None,
        "config": {"workload": f"mixed stream of {n_calls} calls (loop ~ U{{4}}, sizes log-uniform), batches "
                               f"of {B} replayed from one CUDA graph, device MLP selection, confidence fallback "
                               f"below tau = {tau} through ar_exec_fallback ({reps_fb} timed runs per variant)",
                   "batches": len(batches)},
        "stream": {"ms": stream_ms, "memory_loops_gbs": mem_gbs, "nbody_gflops": nb_gflops,
                   "batch_ms_p50": float(np.percentile(batch_ms, 50)),
                   "latency_us": {LOOPS[L]: {"p50": float(np.percentile(lat[L], 50)),
                                             "p99": float(np.percentile(lat[L], 99)), "calls": len(lat[L])}
                                  for L in range(4) if lat[L]},
                   "kernels_per_batch": 3},
        "selection": {"mean_regret_pct": 100 * statistics.mean(all_reg),
                      "per_loop_regret_pct": {LOOPS[L]: 100 * statistics.mean(regrets[L]) for L in range(4)
                                              if regrets[L]},
                      "regret_sample_calls": len(samp),
                      "note": "regret of the variant the device MLP chose when the call ran (before any fallback)"},
        "fallback": {"low_confidence_calls": low, "low_confidence_pct": 100.0 * low / n_calls,
                     "low_confidence_by_loop": {LOOPS[L]: low_by[L] for L in range(4)},
                     "region_tie": {"daxpy": 0.03, "others": 0.005},
                     "profiled_calls": fb_profiled, "answered_from_records": low - fb_profiled,
                     "gpu_ms": fb_ms, "wall_s": fb_wall,
                     "stream_plus_fallback_gbs": byts / ((stream_ms + fb_ms) * 1e-3) / 1e9},
        "cost": {"training_profile_gpu_ms": train_ms, "training_wall_s": train_wall,
                 "fallback_profile_gpu_ms": fb_ms,
                 "exhaustive_every_call_gpu_ms": exhaustive_all_ms,
                 "profiling_cost_ratio": (train_ms + fb_ms) / exhaustive_all_ms,
                 "note": "GPU time of every profiled execution (warm-up included) of the learned method "
                         "(training set + fallbacks) over exhaustive profiling of every call of the stream "
                         "(estimated from the regret sample at the same repetitions)"},
        "roofline": {"bound": "hbm", "achieved": mem_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": mem_gbs / hbm_peak, "peak_source": peak_src, "traffic": None,
                     "kernel": "exec_run (all loops in one launch)",
                     "nbody": {"achieved_gflops": nb_gflops, "peak_gflops": fp32_roof, "frac": nb_gflops / fp32_roof},
                     "machine_frac": mem_gbs / hbm_peak + nb_gflops / fp32_roof},
    }


def run_mixed(args):
    print(json.dumps(mixed_record(args.calls, args.tau)), flush=True)


# ---------------------------------------------------------------- evaluation protocol, all loops
NBODY_GEOM_VARIANTS = (1, 2, 4, 5, 7, 8)  # t128/t256/t512 x unroll 4/8


def nbody_features(ar, N):
    """n-body selector features: N and the waves of the unroll-4 and unroll-8
    variants' launches (grid x cluster / (resident blocks x SMs))."""
    return [float(N)] + [float(np.float32(ar.ar_nbody_geometry(v, int(N))["waves"])) for v in NBODY_GEOM_VARIANTS]


def protocol_record(epochs):
    """The paper's evaluation protocol (Section 4.1: K-fold Adaptive-25/50/75,
    Adaptive-100, Static,Best) and its Online mode (Section 4.2) for daxpy,
    Jacobi and n-body, on profile tables of seeded feature points (the SpMV
    tables are the selector study's: `--workload spmv --kfold`).  Profiles:
    every variant of the stand-alone kernels, 5 timed runs after a warm-up,
    512 MB L2 flush before each.  Online: one fresh region per loop with the
    default min_train_data (= number of variants) and RoundRobin exploration,
    invoked on the table's feature points in a seeded random order; after its
    automatic training its choices are scored against the table's argmin."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    rng = np.random.Generator(np.random.PCG64(4171))
    status = torch.zeros(2, dtype=torch.int32, device=dev)
    # largest inputs, used as prefixes for smaller feature points
    nmax = 1 << 26
    _, x, y = synth.daxpy_inputs(1, nmax)
    xd, yd = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    del x, y
    Nmax = 512
    u0 = torch.from_numpy(synth.grid_inputs(7, Nmax)).to(dev).reshape(-1)
    out, work = torch.empty_like(u0), torch.empty_like(u0)
    Bmax = 1 << 18
    pos = torch.from_numpy(synth.nbody_inputs(4, Bmax)).to(dev)
    acc = torch.empty_like(pos)

    def log_uniform_ints(lo, hi, n):
        # values exact in float32, the features' type inside the runtime
        return sorted({int(np.float32(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))) for _ in range(n)})

    def jacobi_args(f):
        N = int(f[0])
        return ar.ArJacobi7Args(N, int(f[1]), u0.data_ptr(), out.data_ptr(), work.data_ptr(), status.data_ptr())

    loops = {
        "daxpy": (ar.AR_LOOP_DAXPY, [[float(n)] for n in log_uniform_ints(1 << 10, nmax, 64)],
                  lambda f: ar.ArDaxpyArgs(int(f[0]), 1.5, xd.data_ptr(), yd.data_ptr())),
        "jacobi7": (ar.AR_LOOP_JACOBI7,
                    [[float(N), float(rng.choice([1, 5, 10, 20]))] for N in log_uniform_ints(32, Nmax, 48)],
                    jacobi_args),
        # n-body: N and the number of waves each unroll-4 / unroll-8 variant's
        # launch takes (ar_nbody_geometry; a pure function of N and the
        # device): the split rule makes the winner change where these cross 1
        "nbody": (ar.AR_LOOP_NBODY, [nbody_features(ar, n) for n in log_uniform_ints(1 << 10, Bmax, 40)],
                  lambda f: ar.ArNbodyArgs(int(f[0]), pos.data_ptr(), acc.data_ptr(), synth.NBODY_EPS)),
    }
    result = {}
    for name, (L, points, make_args) in loops.items():
        t0 = time.perf_counter()
        F = len(points[0])
        prof = ar.Region(f"protocol-{name}", F, "exhaustive,reps=5", 10 ** 9)
        V = prof.add_builtin(L)
        prof.set_l2_flush(flush, flush.numel())
        table = []
        for f in points:
            ms, _ = prof.profile(f, make_args(f), stream=stream)
            table.append((f, [float(m) for m in ms]))
        t_prof = time.perf_counter() - t0
        assert int(status[0].item()) == 0
        t1 = time.perf_counter()
        kf = kfold_protocol(table, V, F, epochs)
        t_kfold = time.perf_counter() - t1
        kf_n_only = None
        if name == "nbody":  # the same profiles with N as the only feature
            kf_n_only = kfold_protocol([([f[0]], ms) for f, ms in table], V, 1, epochs)
        # Online mode
        ro = ar.Region(f"online-{name}", F, "dtree,2")
        ro.add_builtin(L)
        order = rng.permutation(len(points))
        calls = 0
        while not ro.info()["trained"]:
            f = points[order[calls % len(points)]]
            ro.invoke(f, make_args(f), stream=stream)
            calls += 1
        stream.synchronize()
        best = {tuple(f): min(ms) for f, ms in table}
        msd = {tuple(f): ms for f, ms in table}
        explore = [(tuple(ff[:F]), v, t) for ff, v, t in ro.records()]
        online_regret = statistics.mean(msd[tuple(f)][ro.select(f)[0]] / best[tuple(f)] - 1.0 for f, _ in table)
        names = [ar.loop_variant_name(L, v) for v in range(V)]
        result[name] = {
            "points": len(points), "variants": V, "features": F,
            "kfold_mean_regret_pct": kf,
            **({"kfold_mean_regret_pct_n_only": kf_n_only} if kf_n_only else {}),
            "online": {"explore_calls": calls, "mean_regret_pct": 100 * online_regret,
                       "explore_overhead_pct": 100 * (sum(t for _, _, t in explore) /
                                                      sum(best[tuple(float(x) for x in f)] for f, _, t in explore)
                                                      - 1.0)},
            "best_variant_histogram": {names[v]: sum(1 for _, ms in table if int(np.argmin(ms)) == v)
                                       for v in range(V)},
            "profiling_wall_s": t_prof, "kfold_wall_s": t_kfold}
    line = {"metric": "mean regret % of the selected variant against the exhaustive argmin (paper Section 4.1-4.2)",
            "value": statistics.mean(r["kfold_mean_regret_pct"]["mlp"]["adaptive_75"] for r in result.values()),
            "unit": "%", "n_gpus": 1, "higher_is_better": False, "dtype": "f64 (daxpy, Jacobi) / f32 (n-body)",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": "evaluation protocol: K = 4, f = 25/50/75 %, 10 shuffles, Adaptive-100, "
                                   "Static,Best, Online; daxpy n in [2^10, 2^26] (64 points), Jacobi N in [32, 512] "
                                   "x sweeps in {1,5,10,20} (48), n-body N in [1k, 256k] (40)",
                       "value": "mean over the three loops of the MLP's Adaptive-75 regret",
                       "nbody_features": "N and the waves of the t128/t256/t512 x unroll 4/8 launches "
                                         "(ar_nbody_geometry); kfold_mean_regret_pct_n_only: N alone"},
            "loops": result}
    return line


def run_protocol(args):
    print(json.dumps(protocol_record(args.epochs)), flush=True)


# ---------------------------------------------------------------- host data: co-scheduling, device selection
def cosched_record(reps=5):
    """The paper's co-scheduling use case (Section 3.2, Listing 5; Section
    5.4) and device selection (Listing 3; Section 5.2) on host-resident data:
    daxpy at 12 sizes n log-uniform in [2^14, 2^27] and four SpMV matrices,
    every GPU fraction of [0.0:1.0:0.1] profiled through a split region
    (ar_region_add_split: the GPU part copied in, computed by a CUDA variant
    and copied back while the host cores run the rest; `reps` timed runs
    after a warm-up, wall time by CUDA events around the blocking call).  The
    depth-2 tree on n is scored leave-one-size-out; device selection (host
    cores or GPU, fractions 0 and 1) is trained and scored on the same
    table's two columns."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    nmax = 1 << 27
    rng = np.random.Generator(np.random.PCG64(77))
    sizes = sorted({int(np.float32(round(np.exp(rng.uniform(np.log(2 ** 14), np.log(nmax)))))) for _ in range(12)})
    a, x, y = synth.daxpy_inputs(7, nmax)
    hx, hy = torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()
    del x, y
    xd, yd = torch.empty(nmax, dtype=torch.float64, device=dev), torch.empty(nmax, dtype=torch.float64, device=dev)
    args = ar.ArDaxpySplitArgs(0, a, hx.data_ptr(), hy.data_ptr(), xd.data_ptr(), yd.data_ptr(), 6)
    co = ar.Region("cosched-daxpy", 1, f"dtree,2,reps={reps}", 10 ** 9)
    V = co.add_split(ar.AR_LOOP_DAXPY)
    fr = [co.variant(v)["value"] for v in range(V)]
    t0 = time.perf_counter()
    table = {}
    for n in sizes:
        args.n = n
        ms, _ = co.profile([n], args, stream=stream)
        table[n] = [float(m) for m in ms]
    t_prof = time.perf_counter() - t0

    def tree_choice(train, n, cols):
        r = ar.Region("cosched-fit", 1, "dtree,2", 10 ** 9)
        for v in range(len(cols)):
            r.register(f"v{v}", float(v), lambda a_, v_, x_, s_, u_: 0)
        for m in train:
            for k, v in enumerate(cols):
                r.add_record([m], k, table[m][v])
        r.train()
        return cols[r.select([n])[0]]

    per = []
    for n in sizes:
        ms = table[n]
        best = int(np.argmin(ms))
        loo = tree_choice([m for m in sizes if m != n], n, list(range(V)))
        dev_loo = tree_choice([m for m in sizes if m != n], n, [0, V - 1])
        per.append({"n": n, "best_fraction": fr[best], "gpu_only_ms": ms[V - 1], "cpu_only_ms": ms[0],
                    "best_ms": ms[best], "best_over_gpu_only": ms[V - 1] / ms[best],
                    "tree_loo_fraction": fr[loo], "tree_loo_regret_pct": 100 * (ms[loo] / ms[best] - 1),
                    "device_loo": "gpu" if dev_loo == V - 1 else "cpu",
                    "device_loo_regret_pct": 100 * (ms[dev_loo] / min(ms[0], ms[V - 1]) - 1)})
    tot = {k: sum(table[n][v] for n in sizes) for k, v in (("cpu", 0), ("gpu", V - 1))}
    bytes_ = sum(24.0 * n for n in sizes)
    sel_ms = sum(table[p["n"]][fr.index(p["tree_loo_fraction"])] for p in per)
    best_ms = sum(p["best_ms"] for p in per)
    # SpMV: four matrices, every fraction
    sp = []
    for seed, kind, rows, prm in ((61, "zipf", 200000, 1.5), (62, "zipf", 2000000, 1.8), (63, "band", 1000000, 65),
                                  (64, "band", 4000000, 17)):
        rp, c, v = synth.csr_zipf(seed, rows, prm) if kind == "zipf" else synth.csr_band(seed, rows, prm)
        xs = synth.spmv_x(seed, rows)
        h = [t.pin_memory() for t in (rp, c, v, xs)]
        d = [torch.empty_like(t, device=dev) for t in h]
        nnz = int(rp[-1])
        hys = torch.empty(rows, dtype=torch.float64).pin_memory()
        ysd = torch.empty(rows, dtype=torch.float64, device=dev)
        sargs = ar.ArSpmvSplitArgs(rows=rows, nnz=nnz, cols=rows, rowptr=h[0].data_ptr(), col=h[1].data_ptr(),
                                   val=h[2].data_ptr(), x=h[3].data_ptr(), y=hys.data_ptr(),
                                   rowptr_dev=d[0].data_ptr(), col_dev=d[1].data_ptr(), val_dev=d[2].data_ptr(),
                                   x_dev=d[3].data_ptr(), y_dev=ysd.data_ptr(), gpu_variant=4)
        rs = ar.Region("cosched-spmv", 1, f"exhaustive,reps={reps}")
        rs.add_split(ar.AR_LOOP_SPMV)
        ms, best = rs.profile([rows], sargs, stream=stream)
        sp.append({"kind": kind, "rows": rows, "nnz": nnz, "best_fraction": fr[best],
                   "best_over_gpu_only": ms[V - 1] / ms[best], "cpu_only_over_gpu_only": ms[0] / ms[V - 1],
                   "best_gbs": spmv_bytes(rows, nnz) / (ms[best] * 1e-3) / 1e9})
    return {
        "metric": METRIC, "value": bytes_ / (sel_ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "dtype": "f64",
        "data": "synthetic, host-resident (pinned)", "higher_is_better": True, "vs_baseline": None,
        "config": {"workload": "daxpy on host data, n log-uniform in [2^14, 2^27] (12 sizes), GPU fraction "
                               "[0.0:1.0:0.1] (11 variants), depth-2 tree on n scored leave-one-size-out; device "
                               "selection (fractions 0 / 1); SpMV on 4 matrices", "host_threads": ar.ar_split_threads(),
                   "value": "daxpy algorithmic bytes (24 n) over the tree's leave-one-out choices' time"},
        "daxpy": {"per_n": per, "best_gbs": bytes_ / (best_ms * 1e-3) / 1e9,
                  "gpu_only_gbs": bytes_ / (tot["gpu"] * 1e-3) / 1e9, "cpu_only_gbs": bytes_ / (tot["cpu"] * 1e-3) / 1e9,
                  "tree_loo_mean_regret_pct": statistics.mean(p["tree_loo_regret_pct"] for p in per),
                  "device_loo_mean_regret_pct": statistics.mean(p["device_loo_regret_pct"] for p in per)},
        "spmv": sp, "profiling_wall_s": t_prof}


def run_cosched(args):
    print(json.dumps(cosched_record()), flush=True)


# ---------------------------------------------------------------- daxpy (config 1)
def daxpy_record(steps, warmup):
    """Config 1: daxpy n = 2^20, 15 variants, exhaustive profiling (5 reps after
    a warm-up, L2 flushed before each) picks the argmin -- the plain method, no
    learned model.  Timed: `steps` invocations through the region, each after
    an L2 flush (only the invocation is timed); plus the warm form, 100
    invocations replayed from one CUDA graph with the vectors L2-resident."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    n = 1 << 20
    a, x, y = synth.daxpy_inputs(1, n)
    xd, yd = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    r = ar.Region("daxpy", 1, "exhaustive,reps=5")
    V = r.add_builtin(ar.AR_LOOP_DAXPY)
    r.set_l2_flush(flush, flush.numel())
    args_blk = ar.ArDaxpyArgs(n, a, xd.data_ptr(), yd.data_ptr())
    ms, best = r.profile([n], args_blk, stream=stream)
    default = ar.loop_default_variant(ar.AR_LOOP_DAXPY)
    names = [ar.loop_variant_name(ar.AR_LOOP_DAXPY, v) for v in range(V)]
    bytes_ = 24.0 * n
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            r.invoke([n], args_blk, stream=stream)
        for e0, e1 in ev:
            flush.fill_(1)
            e0.record(stream)
            v, _ = r.invoke([n], args_blk, stream=stream)
            e1.record(stream)
    stream.synchronize()
    t = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_med = statistics.median(t)
    hbm_peak, src = peaks()
    # warm form: 100 invocations of the selected variant in one graph
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(100):
            ar.ar_daxpy(best, n, a, xd, yd, stream=stream)
    with torch.cuda.stream(stream):  # replay() runs on the current stream
        g.replay()
    stream.synchronize()
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    with torch.cuda.stream(stream):
        g.replay()
    w1.record(stream)
    stream.synchronize()
    warm_ms = w0.elapsed_time(w1) / 100
    line = {"metric": METRIC, "value": bytes_ / (t_med * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": 1, "dtype": "f64",
            "data": "synthetic", "higher_is_better": True, "vs_baseline": None, "steps": steps,
            "config": {"workload": "daxpy float64 n = 2^20, a = 1.5, 15 variants, exhaustive profiling (5 reps, "
                                   "L2 flushed) picks the argmin", "l2": "flushed (512 MB) before every timed call"},
            "selection": {"selected": names[v], "exhaustive_best": names[best], "default": names[default],
                          "profile_gbs": {names[k]: bytes_ / (ms[k] * 1e-3) / 1e9 for k in range(V)},
                          "exhaustive_best_gbs": bytes_ / (ms[best] * 1e-3) / 1e9,
                          "default_gbs": bytes_ / (ms[default] * 1e-3) / 1e9,
                          "regret_pct": 100.0 * (ms[v] / ms[best] - 1.0)},
            "roofline": {"bound": "hbm", "achieved": bytes_ / (t_med * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": bytes_ / (t_med * 1e-3) / 1e9 / hbm_peak, "peak_source": src,
                         "note": "25 MB per call: 3.9 us at the HBM roof, comparable to launch latency"},
            "warm_graph": {"us_per_call": warm_ms * 1e3, "gbs": bytes_ / (warm_ms * 1e-3) / 1e9,
                           "note": "x, y resident in L2; 100 calls in one CUDA graph"}}
    return line


def run_daxpy(args):
    print(json.dumps(daxpy_record(args.steps, args.warmup)), flush=True)


# ---------------------------------------------------------------- n-body (config 4)
def nbody_record(steps, warmup):
    """Config 4: all-pairs n-body, N in {1k, 4k, 16k, 64k, 256k}, 9 variants;
    exhaustive profiling per N picks the variant; the timed step invokes the
    selected variant once per N.  Also the batched form (64 systems, sizes
    log-uniform in [1k, 64k]) in one persistent launch."""
    import torch

    import paper_2303_08873_b300 as ar
    import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    Ns = [1024, 4096, 16384, 65536, 262144]
    _, fp32_fma = ar.ar_measure_fma_rates()
    r = ar.Region("nbody", 1, "exhaustive,reps=3")
    V = r.add_builtin(ar.AR_LOOP_NBODY)
    names = [ar.loop_variant_name(ar.AR_LOOP_NBODY, v) for v in range(V)]
    default = ar.loop_default_variant(ar.AR_LOOP_NBODY)
    bufs, blks, per = {}, {}, []
    for N in Ns:
        p = torch.from_numpy(synth.nbody_inputs(4, N)).to(dev)
        acc = torch.empty_like(p)
        bufs[N] = (p, acc)
        blks[N] = ar.ArNbodyArgs(N, p.data_ptr(), acc.data_ptr(), synth.NBODY_EPS)
        ms, best = r.profile([N], blks[N], stream=stream)
        per.append({"N": N, "best": names[best], "best_gflops": NBODY_FLOPS * N * N / (ms[best] * 1e-3) / 1e9,
                    "default_gflops": NBODY_FLOPS * N * N / (ms[default] * 1e-3) / 1e9,
                    "worst_gflops": NBODY_FLOPS * N * N / (max(ms) * 1e-3) / 1e9})
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            for N in Ns:
                r.invoke([N], blks[N], stream=stream)
        e0.record(stream)
        for _ in range(steps):
            for N in Ns:
                if N == Ns[-1]:
                    k0.record(stream)
                r.invoke([N], blks[N], stream=stream)
                if N == Ns[-1]:
                    k1.record(stream)
        e1.record(stream)
    stream.synchronize()
    ms_step = e0.elapsed_time(e1) / steps
    flops = sum(NBODY_FLOPS * N * N for N in Ns)
    big_ms = k0.elapsed_time(k1)
    inter_s = Ns[-1] ** 2 / (big_ms * 1e-3)
    peak_inter = fp32_fma / 12.0  # 12 FP32 lane operations per interaction (6 packed pairs per 2)
    packed_inter = ar.ar_measure_fp32x2_rate() / 12.0  # the same lanes issued as packed pairs
    # batched form
    bodies, offs = synth.nbody_batch_inputs(40)
    bd, od = torch.from_numpy(bodies).to(dev), torch.from_numpy(offs).to(dev)
    ad = torch.empty_like(bd)
    wsb = ar.ar_nbody_batched_workspace_bytes(offs.size - 1)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ar.ar_nbody_batched(offs.size - 1, od, bd, ad, synth.NBODY_EPS, ws, wsb, stream=stream)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(3):
        ar.ar_nbody_batched(offs.size - 1, od, bd, ad, synth.NBODY_EPS, ws, wsb, stream=stream)
    b1.record(stream)
    stream.synchronize()
    bms = b0.elapsed_time(b1) / 3
    sizes = np.diff(offs.astype(np.int64))
    bflops = NBODY_FLOPS * float(np.sum(sizes.astype(np.float64) ** 2))
    line = {"metric": METRIC, "value": flops / (ms_step * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1,
            "dtype": "f32", "data": "synthetic", "higher_is_better": True, "vs_baseline": None,
            "steps": steps, "ms_per_step": ms_step,
            "config": {"workload": "all-pairs n-body float32, eps 1e-2, N in {1k,4k,16k,64k,256k}, 9 variants, "
                                   "exhaustive profiling per N", "flops_per_interaction": NBODY_FLOPS},
            "selection": {"per_N": per},
            "roofline": {"bound": "alu", "achieved": inter_s * NBODY_FLOPS / 1e9, "unit": "GFLOP/s",
                         "peak": peak_inter * NBODY_FLOPS / 1e9, "frac": inter_s / peak_inter,
                         "peak_source": "float32 FMA lane rate (ar_measure_fma_rates) / 12 FP32 lane operations "
                                        "per interaction", "kernel": per[-1]["best"],
                         "packed": {"peak": packed_inter * NBODY_FLOPS / 1e9, "frac": inter_s / packed_inter,
                                    "peak_source": "packed float32 pair FMA lane rate (ar_measure_fp32x2_rate) / "
                                                   "12 FP32 lane operations per interaction"}},
            "batched": {"systems": int(offs.size - 1), "bodies": int(sizes.sum()), "ms": bms,
                        "gflops": bflops / (bms * 1e-3) / 1e9,
                        "roofline_frac": bflops / (bms * 1e-3) / (peak_inter * NBODY_FLOPS)}}
    return line


def run_nbody(args):
    print(json.dumps(nbody_record(args.steps, args.warmup)), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "spmv":
        run_spmv(args)
    elif args.workload == "mixed":
        run_mixed(args)
    elif args.workload == "daxpy":
        run_daxpy(args)
    elif args.workload == "nbody":
        run_nbody(args)
    elif args.workload == "protocol":
        run_protocol(args)
    elif args.workload == "cosched":
        run_cosched(args)
    else:  # the stencil workloads: jacobi7 (default) and heat7
        run_ours(args)


if __name__ == "__main__":
    main()
