"""Persistent mixed-stream executor against the oracle (GPU).

One batch mixes every variant of the four loops (forced variants), so the
phase-major scheduling, the Jacobi sweep dependencies and the merge-path
fix-up phase all run in the same persistent launch.  A second batch lets the
device MLPs choose; a third is replayed from a captured CUDA graph.
"""

import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
EPS = synth.NBODY_EPS


class Batch:
    """Calls with their own device buffers, plus the expected outputs."""

    def __init__(self):
        self.calls, self.keep, self.check = [], [], []

    def daxpy(self, n, seed):
        a, x, y = synth.daxpy_inputs(seed, n)
        xd, yd = dev(x), dev(y)
        self.keep += [xd, yd]
        self.calls.append(ar.ArExecCall(loop=0, n=n, a=a, in0=xd.data_ptr(), out0=yd.data_ptr()))
        ref = loops.daxpy(a, x, y)
        scale = np.abs(a * x) + np.abs(y)
        self.check.append(lambda yd=yd, ref=ref, scale=scale: np.all(np.abs(host(yd) - ref) <= 1e-13 * scale))

    def jacobi(self, N, sweeps, seed, plant=None):
        u0 = synth.grid_inputs(seed, N)
        if plant is not None:
            u0[N // 2, N // 3, N // 4] = plant
        ud = dev(u0)
        out, work = torch.empty_like(ud), torch.empty_like(ud)
        self.keep += [ud, out, work]
        self.calls.append(ar.ArExecCall(loop=1, sweeps=sweeps, n=N, in0=ud.data_ptr(), out0=out.data_ptr(),
                                        out1=work.data_ptr()))
        ref = loops.jacobi7(u0, sweeps)
        self.check.append(lambda out=out, ref=ref: np.max(np.abs(host(out) - ref)) <= 1e-13 * np.max(np.abs(ref)))

    def spmv(self, mat, seed):
        rp, c, v = mat
        rows = rp.numel() - 1
        nnz = int(rp[-1])
        x = synth.spmv_x(seed, rows).numpy()
        d = [t.cuda() for t in (rp, c, v)] + [dev(x)]
        y = torch.full((rows,), np.nan, dtype=torch.float64, device="cuda")
        nb = -(-(rows + nnz) // 4096)
        ws = torch.empty(16 * nb + 16, dtype=torch.uint8, device="cuda")
        self.keep += d + [y, ws]
        self.calls.append(ar.ArExecCall(loop=2, n=rows, nnz=nnz, in0=d[0].data_ptr(), in1=d[1].data_ptr(),
                                        in2=d[2].data_ptr(), in3=d[3].data_ptr(), out0=y.data_ptr(),
                                        out1=ws.data_ptr(), out1_bytes=ws.numel()))
        rph, ch, vh = rp.numpy(), c.numpy(), v.numpy()
        ref, absum = loops.spmv_rows(rph, ch, vh, x, np.arange(rows))
        self.check.append(lambda y=y, ref=ref, absum=absum: np.all(np.abs(host(y) - ref) <= 1e-10 * absum))
        return loops.csr_row_stats(rph)

    def nbody(self, N, seed, negate=None, ws_bytes=0, ws_offset=0):
        """ws_bytes > 0: a partial-sum workspace in out1 (filled with NaN),
        starting ws_offset bytes into its allocation; returned."""
        p = synth.nbody_inputs(seed, N)
        if negate is not None:
            p[negate, 3] *= -1.0
        pd = dev(p)
        acc = torch.full((N, 4), np.nan, dtype=torch.float32, device="cuda")
        self.keep += [pd, acc]
        call = ar.ArExecCall(loop=3, n=N, eps=EPS, in0=pd.data_ptr(), out0=acc.data_ptr())
        ws = None
        if ws_bytes > 0:
            ws = torch.full(((ws_bytes + ws_offset + 3) // 4,), np.nan, dtype=torch.float32, device="cuda")
            self.keep.append(ws)
            call.out1, call.out1_bytes = ws.data_ptr() + ws_offset, ws_bytes
        self.calls.append(call)
        ref = loops.nbody(p, EPS)
        scale = np.max(np.linalg.norm(ref, axis=1))

        def ok(acc=acc, ref=ref, scale=scale):
            a = host(acc)
            return np.max(np.linalg.norm(a[:, :3] - ref, axis=1)) <= 1e-4 * scale and np.all(a[:, 3] == 0)
        self.check.append(ok)
        return ws

    def run(self, force=None, models=None, stream=None):
        n = len(self.calls)
        table = torch.frombuffer(bytearray(ar.exec_table_bytes(self.calls)), dtype=torch.uint8).cuda()
        self.keep.append(table)
        out = {"variant": torch.full((n,), -9, dtype=torch.int32, device="cuda"),
               "conf": torch.zeros(n, dtype=torch.float32, device="cuda"),
               "features": torch.zeros((n, 8), dtype=torch.float32, device="cuda"),
               "t0": torch.zeros(n, dtype=torch.int64, device="cuda"),
               "t1": torch.zeros(n, dtype=torch.int64, device="cuda"),
               "status": torch.full((n,), 99, dtype=torch.int32, device="cuda")}
        wsb = ar.ar_exec_workspace_bytes(n)
        ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        fv = dev(np.asarray(force, dtype=np.int32)) if force is not None else None
        ar.ar_exec_batch(table, n, models, fv, out["variant"], out["conf"], out["features"], out["t0"], out["t1"],
                         out["status"], ws, wsb, stream=stream)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}


def test_every_variant_of_every_loop_in_one_batch():
    b = Batch()
    force = []
    for v in range(15):
        b.daxpy(100003 + v, 10 + v)
        force.append(v)
    for v in range(16):
        b.jacobi(37 if v % 2 else 50, 3, 30 + v)
        force.append(v)
    zipf = synth.csr_zipf(5, 20000, 1.6)
    band = synth.csr_band(6, 9000, 129)
    stats = []
    for v in range(8):
        stats.append(b.spmv(zipf if v % 2 == 0 else band, 50 + v))
        force.append(v)
    for v in range(9):
        b.nbody(1000 + 37 * v, 70 + v)
        force.append(v)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    assert np.array_equal(r["variant"], np.array(force))
    for k, ok in enumerate(b.check):
        assert ok(), (k, b.calls[k].loop, force[k])
    assert np.all(r["t1"] >= r["t0"]) and np.all(r["t0"] > 0)
    # features of the SpMV calls (reduced on the device)
    for k, st in zip(range(31, 39), stats):
        f = r["features"][k]
        assert f[0] == np.float32(st[0]) and f[1] == np.float32(st[1]) and f[4] == st[4]
        assert f[2] == pytest.approx(st[2], rel=1e-6) and f[3] == pytest.approx(st[3], rel=1e-5)
    assert r["features"][0][0] == 100003 and tuple(r["features"][15][:3]) == (50.0, 3.0, 1.0)
    assert tuple(r["features"][16][:3]) == (37.0, 3.0, 0.0)


def test_edge_sizes_of_every_loop_in_one_batch():
    """Sizes at and just past the executor's tile edges (daxpy 16384-element
    tiles, Jacobi plane chunks and the even-N plane ring, SpMV row groups and
    4096-item merge-path blocks, n-body 256/512-body tiles), and the degenerate
    ones (one element, one unknown, one row, one body), every loop and family."""
    b = Batch()
    force = []
    for n, v in [(1, 0), (2, 13), (3, 14), (16383, 1), (16385, 2), (32769, 7), (49152, 5)]:
        b.daxpy(n, 200 + n % 97)
        force.append(v)
    for N, sweeps, v in [(1, 1, 1), (1, 3, 13), (2, 2, 13), (2, 1, 9), (3, 3, 15), (4, 2, 5), (6, 3, 14), (9, 2, 12),
                         (34, 3, 13), (33, 2, 13), (64, 1, 0), (65, 2, 3)]:
        b.jacobi(N, sweeps, 300 + N, None)
        force.append(v)
    tiny = synth.csr_zipf(11, 1, 1.5)
    small = synth.csr_zipf(12, 4099, 1.5)
    band = synth.csr_band(13, 5, 3)
    for k, v in enumerate(range(8)):
        b.spmv([tiny, small, band][k % 3], 400 + k)
        force.append(v)
    for N, v in [(1, 0), (2, 3), (3, 6), (129, 1), (257, 4), (513, 8), (255, 7)]:
        b.nbody(N, 500 + N)
        force.append(v)
    for v in (1, 4, 7):  # negative masses in one tile
        b.nbody(700, 600 + v, negate=slice(300, 303))
        force.append(v)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, b.calls[k].loop, force[k])


def test_float_pair_chain_with_and_without_range_flag():
    """The float-pair Jacobi variants keep pairs between sweeps (float64 in,
    float64 out) and redo the call in float64 from the second phase on when an
    input lies outside the pair range; calls with and without such an input
    share one batch, so the range flag is per call."""
    b = Batch()
    force = []
    for k, (N, sweeps, plant) in enumerate([(40, 1, None), (40, 2, None), (33, 3, None), (50, 6, None),
                                            (40, 1, 1e40), (40, 2, 1e40), (33, 3, 1e-30), (50, 6, -3e39),
                                            (29, 5, 0.0), (64, 4, 2.0 ** -80)]):
        b.jacobi(N, sweeps, 90 + k, plant)
        force.append(12 + k % 4)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, force[k])


def test_jacobi_tensor_copy_tiles():
    """tma and df variants of shapes 32x4 and 32x8 on N >= 36 stage their
    planes by tensor copies through maps the plan kernel makes on the device
    (odd N: through the grid's 2N-wide 2D view): every mode of the pair
    chain, the float64 and float-pair forms, ragged x, y and z tile edges, an
    input outside the pair range, next to calls of the other loops in the
    same batch."""
    b = Batch()
    force = []
    for k, (N, sweeps, v, plant) in enumerate([(36, 1, 8, None), (40, 2, 9, None), (66, 3, 12, None),
                                               (100, 5, 13, None), (70, 10, 13, None), (38, 4, 12, 3e39),
                                               (44, 3, 13, 1e-30), (36, 2, 9, 5e40), (98, 1, 13, None),
                                               (37, 1, 8, None), (41, 2, 9, None), (67, 3, 12, None),
                                               (101, 5, 13, None), (39, 4, 12, 3e39), (45, 3, 13, 1e-30)]):
        b.jacobi(N, sweeps, 700 + k, plant)
        force.append(v)
        b.nbody(600 + 50 * k, 720 + k)
        force.append(k % 9)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, b.calls[k].loop, force[k])


def test_jacobi_deep_tiles():
    """From N ~ 250 up a Jacobi tile spans the deepest chunk, 94 planes, and
    the last chunk takes what is left (N = 376: four full chunks; N = 377: a
    last chunk of one plane; N = 311 / 258 / 257 / 300: 29 / 70 / 69 / 18):
    the tensor-copy tiles on even and odd N, the plane ring (df 128x2), the
    shared-memory family and a call whose input lies outside the pair range."""
    b = Batch()
    force = []
    for k, (N, sweeps, v, plant) in enumerate([(376, 2, 13, None), (377, 3, 12, None), (311, 3, 13, None),
                                               (258, 2, 15, None), (257, 2, 9, None), (300, 1, 5, None),
                                               (310, 3, 13, 1e40)]):
        b.jacobi(N, sweeps, 800 + k, plant)
        force.append(v)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, force[k])


def test_nbody_j_chunks_with_a_partials_workspace():
    """An n-body call with fewer i tiles than the persistent kernel has blocks
    splits its j range over chunks when out1 holds the partial sums (16 N
    bytes per chunk, 16-byte aligned); a second phase adds each body's
    partials in chunk order.  Chunk edges one body past a j tile (N = 129),
    a last chunk shorter than a tile, every variant, a workspace for exactly
    two chunks, a misaligned one and a call that fits in one j tile (neither
    splits: the workspace stays untouched), and calls without a workspace,
    in one batch."""
    b = Batch()
    force, cases = [], []
    big = 64 << 20
    for k, (N, v, wsb, off, splits) in enumerate([
            (129, 1, big, 0, True), (700, 7, big, 0, True), (4099, 2, big, 0, True), (20000, 5, big, 0, True),
            (65536, 7, big, 0, True), (5000, 3, 2 * 16 * 5000, 0, True), (5000, 6, big, 4, False),
            (100, 4, big, 0, False), (3000, 8, 0, 0, False), (1, 0, big, 0, False)]):
        ws = b.nbody(N, 900 + k, ws_bytes=min(wsb, 16 * N * 1024), ws_offset=off)
        force.append(v)
        cases.append((N, ws, off, splits))
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, force[k])
    for N, ws, off, splits in cases:
        if ws is None:
            continue
        first = ws.cpu().numpy()[off // 4: off // 4 + 4 * N]  # partial-sum array of chunk 0
        if splits:
            assert np.all(np.isfinite(first)), N
        else:
            assert np.all(np.isnan(ws.cpu().numpy())), N


def test_merge_path_calls_of_many_blocks():
    """Merge-path calls with thousands of path blocks (more than the
    persistent kernel's blocks, so blocks take several items and the carry
    fix-up spans many): a 500k-row power-law matrix (~6k path blocks), a
    400k-row band-33 matrix (~3.3k) and a small one, float64 and float-pair
    forms, in one batch."""
    b = Batch()
    force = []
    mats = [synth.csr_zipf(41, 500000, 1.5), synth.csr_band(42, 400000, 33), synth.csr_zipf(43, 30000, 1.5)]
    for k, m in enumerate(mats):
        for v in (6, 7):
            b.spmv(m, 1000 + 10 * k + v)
            force.append(v)
    r = b.run(force=force)
    assert np.all(r["status"] == 0)
    for k, ok in enumerate(b.check):
        assert ok(), (k, force[k])


def test_bad_variant_and_loop_are_reported_per_call():
    b = Batch()
    b.daxpy(1000, 1)
    b.daxpy(1000, 2)
    b.calls.append(ar.ArExecCall(loop=7, n=10))
    b.check.append(lambda: True)
    # Jacobi calls with aliased or missing buffers, and an empty one
    u = torch.zeros(8 ** 3, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(u)
    b.keep += [u, w]
    b.calls.append(ar.ArExecCall(loop=1, n=8, sweeps=2, in0=u.data_ptr(), out0=w.data_ptr(), out1=w.data_ptr()))
    b.calls.append(ar.ArExecCall(loop=1, n=8, sweeps=1, in0=u.data_ptr(), out0=u.data_ptr()))
    b.calls.append(ar.ArExecCall(loop=1, n=8, sweeps=3, in0=u.data_ptr(), out0=w.data_ptr()))
    b.calls.append(ar.ArExecCall(loop=1, n=0, sweeps=1))
    b.check += [lambda: True] * 4
    r = b.run(force=[3, 15, 0, 13, 1, 5, 13])
    assert r["status"][0] == 0 and r["status"][1] == ar.AR_ERR_ARG and r["status"][2] == ar.AR_ERR_ARG
    assert list(r["status"][3:6]) == [ar.AR_ERR_ARG] * 3 and r["status"][6] == 0
    assert b.check[0]()


def _trained_models():
    """One MLP per loop, trained on the device from a deterministic cost model
    of the features (no timing involved)."""
    nv = [ar.ar_exec_num_variants(L) for L in range(4)]
    specs = [(1, nv[0], lambda f: int(np.log2(f[0])) % 15),
             (3, nv[1], lambda f: ((int(f[0]) // 40) % 8) * 2 + int(f[2])),
             (5, nv[2], lambda f: 7 if f[2] > 40 else (6 if f[2] > 20 else (1 if f[4] > 1000 else 3))),
             (1, nv[3], lambda f: int(f[0] > 2000) * 4)]
    models = ar.ArExecModels()
    models.H = 64
    keep, regions = [], []
    rng = np.random.Generator(np.random.PCG64(9))
    samples = {0: [[float(2 ** rng.uniform(10, 24))] for _ in range(300)],
               1: [[float(n), 3.0, float(n % 2 == 0)] for n in rng.integers(8, 600, 300)],
               2: [[float(rng.integers(1e3, 1e6)), 1e6, float(rng.uniform(1, 60)), 5.0, float(rng.integers(1, 4096))]
                   for _ in range(300)],
               3: [[float(rng.integers(500, 5000))] for _ in range(300)]}
    for L, (F, V, best) in enumerate(specs):
        r = ar.Region(f"exec{L}", F, "mlp,64,epochs=400,seed=1", 10 ** 9)
        for v in range(V):
            r.register(f"v{v}", float(v), lambda a, v, x, s, u: 0)
        r.set_fake_timer(lambda f, v, best=best: 1.0 if v == best(f) else 2.0)
        for f in samples[L]:
            r.profile(f, reps=1)
        r.train()
        m = r.mlp()
        th, mu, sd = dev(m["theta"]), dev(m["mu"]), dev(m["sd"])
        keep += [th, mu, sd]
        models.F[L], models.V[L] = F, V
        models.theta[L], models.mu[L], models.sd[L] = th.data_ptr(), mu.data_ptr(), sd.data_ptr()
        regions.append(r)
    return models, keep, regions


def test_device_mlp_selection_matches_host_models():
    models, keep, regions = _trained_models()
    b = Batch()
    b.daxpy(70000, 1)
    b.daxpy(3000000, 2)
    b.jacobi(45, 2, 3)
    b.jacobi(130, 1, 4)
    b.spmv(synth.csr_zipf(7, 30000, 1.5), 5)
    b.nbody(1500, 6)
    b.nbody(3000, 7)
    r = b.run(models=models)
    assert np.all(r["status"] == 0)
    for k, call in enumerate(b.calls):
        f = r["features"][k][:regions[call.loop].nf]
        want, conf = regions[call.loop].select(list(f))
        assert r["variant"][k] == want, (k, call.loop)
        assert r["conf"][k] == pytest.approx(conf, abs=1e-4)
        assert b.check[k](), k


def test_graph_capture_and_replay_with_new_table():
    b1, b2 = Batch(), Batch()
    for b, s in ((b1, 0), (b2, 100)):
        b.daxpy(50001, 1 + s)
        b.jacobi(40, 4, 2 + s)
        b.spmv(synth.csr_zipf(3 + s, 5000, 2.0), 4 + s)
        b.nbody(700, 5 + s)
    n = 4
    force = dev(np.array([8, 13, 6, 4], dtype=np.int32))
    table = torch.zeros(96 * n, dtype=torch.uint8, device="cuda")
    host_table = torch.zeros(96 * n, dtype=torch.uint8).pin_memory()
    outs = [torch.zeros(n, dtype=torch.int32, device="cuda"), torch.zeros(n, dtype=torch.float32, device="cuda"),
            torch.zeros((n, 8), dtype=torch.float32, device="cuda"), torch.zeros(n, dtype=torch.int64, device="cuda"),
            torch.zeros(n, dtype=torch.int64, device="cuda"), torch.zeros(n, dtype=torch.int32, device="cuda")]
    wsb = ar.ar_exec_workspace_bytes(n)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    host_table.copy_(torch.frombuffer(bytearray(ar.exec_table_bytes(b1.calls)), dtype=torch.uint8))
    with torch.cuda.graph(g, stream=s):
        table.copy_(host_table, non_blocking=True)
        ar.ar_exec_batch(table, n, None, force, *outs, ws, wsb, stream=s)
    for b in (b1, b2):
        host_table.copy_(torch.frombuffer(bytearray(ar.exec_table_bytes(b.calls)), dtype=torch.uint8))
        with torch.cuda.stream(s):  # replay() runs on the current stream
            g.replay()
        s.synchronize()
        assert np.all(outs[5].cpu().numpy() == 0)
        for k, ok in enumerate(b.check):
            assert ok(), k


def test_bounded_waits_give_up_with_a_status():
    """A wait that nothing satisfies ends after its poll limit with
    AR_ERR_TIMEOUT (a counter nothing raises, an mbarrier phase nothing
    completes); satisfied ones return AR_OK.  Nothing faults or hangs."""
    import time
    st = torch.full((4,), 99, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    for kind in range(4):
        ar.lib.ar_wait_selftest(kind, 1000, st[kind:].data_ptr(), None)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert st.cpu().tolist() == [ar.AR_ERR_TIMEOUT, ar.AR_ERR_TIMEOUT, ar.AR_OK, ar.AR_OK]



def test_plan_kernel_mlp_matches_oracle_forward():
    """The plan kernel's per-call MLP (variant, confidence) against the float64
    oracle forward at the float32-rounded weights and statistics, on the
    features the executor computed for each call."""
    from oracle import mlp

    models, keep, regions = _trained_models()
    b = Batch()
    rng = np.random.Generator(np.random.PCG64(21))
    for n in np.exp(rng.uniform(np.log(1000), np.log(400000), 14)).astype(int):
        b.daxpy(int(n), int(n) % 97)
    for N in (33, 40, 48, 71, 96, 130):
        b.jacobi(N, 2, N)
    for rows, s in ((5000, 1.5), (20000, 2.2), (60000, 1.8)):
        b.spmv(synth.csr_zipf(rows % 13, rows, s), rows % 17)
    b.spmv(synth.csr_band(3, 15000, 33), 8)
    for N in (600, 1500, 2100, 3700):
        b.nbody(N, N % 11)
    r = b.run(models=models)
    assert np.all(r["status"] == 0)
    checked = 0
    for k, call in enumerate(b.calls):
        L = call.loop
        F, V = models.F[L], models.V[L]
        m = regions[L].mlp()
        th32, mu32, sd32 = (np.asarray(m[q], dtype=np.float32) for q in ("theta", "mu", "sd"))
        f32 = r["features"][k][:F].astype(np.float32)
        p, _ = mlp.forward(th32.astype(np.float64), f32[None, :].astype(np.float64), mu32.astype(np.float64),
                           sd32.astype(np.float64), 64, V)
        p = p[0]
        assert abs(float(r["conf"][k]) - p.max()) <= 1e-5, (k, L)
        top2 = np.sort(p)[-2:]
        if top2[1] - top2[0] > 1e-4:
            assert r["variant"][k] == int(np.argmax(p)), (k, L)
            checked += 1
        assert b.check[k](), k
    assert checked >= len(b.calls) // 2


def _fallback_regions(spec):
    regions = []
    for L, nf in enumerate((1, 3, 5, 1)):
        r = ar.Region(f"fb{L}", nf, spec, 10 ** 9)
        r.add_exec_variants(L)
        regions.append(r)
    return regions


def _fallback_batch():
    b = Batch()
    b.daxpy(70001, 3)
    b.jacobi(45, 2, 4)
    b.spmv(synth.csr_zipf(5, 30000, 1.6), 6)
    b.nbody(1500, 7)
    return b


def test_fallback_profiles_low_confidence_calls_into_records():
    """Calls planted below the confidence threshold are profiled through the
    executor: V x reps records each, best = the fastest recorded mean (the
    oracle's label rule), outputs still the loop's result; a second fallback
    on the same features profiles nothing and returns the same choices."""
    from oracle import select

    b = _fallback_batch()
    r = b.run()
    assert np.all(r["status"] == 0)
    regions = _fallback_regions("dtree")
    conf = np.array([0.2, 0.9, 0.3, 0.1], dtype=np.float32)
    reps = 2
    wsb = ar.ar_exec_fallback_workspace_bytes(70001)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    best, cnt = ar.ar_exec_fallback(b.calls, r["features"], conf, 0.5, regions, reps, None, False, ws, wsb)
    assert cnt == 3 and best[1] == -1
    for k, L in ((0, 0), (2, 2), (3, 3)):
        V = ar.ar_exec_num_variants(L)
        recs = regions[L].records()
        assert len(recs) == V * reps
        nf = regions[L].nf
        for f, v, ms in recs:
            assert np.array_equal(np.asarray(f[:nf], dtype=np.float32), r["features"][k][:nf])
            assert ms >= 0
        assert sorted(v for _, v, _ in recs) == sorted(list(range(V)) * reps)
        assert best[k] == select.labels([(tuple(f), v, ms) for f, v, ms in recs])[0][1]
    assert regions[1].counts()[0] == 0
    for k, ok in enumerate(b.check):
        assert ok(), k  # daxpy applied once, the rest recomputed by the best variant
    best2, cnt2 = ar.ar_exec_fallback(b.calls, r["features"], conf, 0.5, regions, reps, None, False, ws, wsb)
    assert cnt2 == 0 and np.array_equal(best, best2)
    assert [rg.counts()[0] for rg in regions] == [15 * reps, 0, 8 * reps, 9 * reps]
    for k, ok in enumerate(b.check):
        assert ok(), k


def test_fallback_retrains_and_refreshes_device_models():
    b = _fallback_batch()
    r = b.run()
    regions = _fallback_regions("mlp,64,epochs=30,seed=2")
    models = ar.ArExecModels()
    models.H = 64
    keep = []
    for L, F in enumerate((1, 3, 5, 1)):
        V = ar.ar_exec_num_variants(L)
        th = torch.zeros(ar.ar_mlp_num_params(F, 64, V), dtype=torch.float32, device="cuda")
        mu = torch.zeros(F, dtype=torch.float32, device="cuda")
        sd = torch.ones(F, dtype=torch.float32, device="cuda")
        keep += [th, mu, sd]
        models.F[L], models.V[L] = F, V
        models.theta[L], models.mu[L], models.sd[L] = th.data_ptr(), mu.data_ptr(), sd.data_ptr()
    wsb = ar.ar_exec_fallback_workspace_bytes(70001)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    conf = np.zeros(4, dtype=np.float32)
    best, cnt = ar.ar_exec_fallback(b.calls, r["features"], conf, 0.5, regions, 1, models, True, ws, wsb)
    assert cnt == 4 and np.all(best >= 0)
    for L in range(4):
        m = regions[L].mlp()
        assert np.array_equal(host(keep[3 * L]), np.asarray(m["theta"], dtype=np.float32))
        assert np.array_equal(host(keep[3 * L + 1]), np.asarray(m["mu"], dtype=np.float32))
        assert np.array_equal(host(keep[3 * L + 2]), np.asarray(m["sd"], dtype=np.float32))
    # the refreshed device models choose what the retrained regions choose
    r2 = b.run(models=models)
    for k, call in enumerate(b.calls):
        want, _ = regions[call.loop].select(list(r2["features"][k][:regions[call.loop].nf]))
        assert r2["variant"][k] == want, k
