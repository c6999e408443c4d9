"""Host logic of the region runtime through the C ABI, on CPU.

CUDA-event timing is replaced by a deterministic cost model
(ar_set_fake_timer) and the variants by host launchers, so these tests need
no GPU.  The runtime's labels and decision trees are compared with the
selection oracle on the same records.
"""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import paper_2303_08873_b300 as ar
from oracle import select

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "variant_ranges.json")))


def _declared_functions():
    names = set()
    for h in ("ar.h", "ar_loops.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|void)\s+(ar_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    declared = _declared_functions()
    assert len(declared) >= 30
    for name in sorted(declared):
        assert hasattr(ar.lib, name), name
    assert declared == set(ar.EXPORTED), declared ^ set(ar.EXPORTED)


def _noop(args, v, value, stream, user):
    return 0


class Calls:
    def __init__(self):
        self.seq = []

    def __call__(self, args, v, value, stream, user):
        self.seq.append(v)
        return 0


def _region(V=4, nf=1, spec="", mtd=0, cost=None):
    r = ar.Region("t", nf, spec, mtd)
    calls = Calls()
    for v in range(V):
        r.register(f"v{v}", float(v), calls)
    r.set_fake_timer(cost or (lambda f, v: 1.0 + v))
    return r, calls


# ------------------------------------------------------------ registration
def test_categorical_variants_enumerate_in_order():
    ex = GOLD["apollo_example"]
    r = ar.Region("vecAdd", ex["num_features"], "DecisionTree,explore=RoundRobin", ex["min_train_data"])
    for name, idx in ex["policies"].items():
        assert r.register(name, float(idx), _noop) == idx
    info = r.info()
    assert info["num_variants"] == ex["num_policies"] and info["min_train_data"] == 10
    assert [r.variant(i)["name"] for i in range(2)] == ["cpu", "gpu"]


@pytest.mark.parametrize("case", GOLD["ranges"])
def test_range_registration_matches_oracle(case):
    r = ar.Region("r", 1)
    n = r.register_range(case["begin"], case["end"], case["step"], _noop)
    want = select.expand_range(case["begin"], case["end"], case["step"])
    assert n == len(want)
    assert [r.variant(i)["value"] for i in range(n)] == want


def test_defaults_min_train_is_variant_count_and_dtree_depth_2():
    r, _ = _region(V=5)
    info = r.info()
    assert info["min_train_data"] == 5 and info["model"] == "dtree"


def test_bad_specs_and_arguments():
    for spec in ("forest", "dtree,0", "mlp,48", "fixed", "dtree,explore=greedy", "reps=0"):
        with pytest.raises(ar.ArError) as e:
            ar.Region("x", 1, spec)
        assert e.value.code == ar.AR_ERR_ARG
    with pytest.raises(ar.ArError):
        ar.Region("x", 9)
    r = ar.Region("x", 1)
    with pytest.raises(ar.ArError):
        r.register_range(5, 1, 1, _noop)


# ------------------------------------------------------------ exploration
def test_round_robin_then_model_selects():
    # variant 0 fastest for small n, variant 2 fastest for large n
    cost = lambda f, v: (1.0 + v) if f[0] < 100 else (3.0 - v)  # noqa: E731
    r, calls = _region(V=3, cost=cost, mtd=6)
    seq = []
    feats = [10, 1000, 10, 1000, 10, 1000]
    for k, n in enumerate(feats):
        v, _ = r.invoke([n])
        seq.append(v)
        assert v == select.round_robin(k, 3)
    assert r.info()["trained"]  # 6 unique (n, v) points reached
    assert r.invoke([20])[0] == 0
    assert r.invoke([5000])[0] == 2
    assert calls.seq == seq + [0, 2]


def test_training_fires_once_on_unique_points_only():
    r, _ = _region(V=2, mtd=3)
    for _ in range(5):
        r.invoke([7])  # only (7,0) and (7,1): 2 unique points
    assert not r.info()["trained"]
    assert r.counts() == (5, 2)
    r.invoke([8])
    assert r.info()["trained"]


def test_policy_always_in_range_property():
    rng = np.random.Generator(np.random.PCG64(0))
    V = 7
    r, _ = _region(V=V, nf=2, cost=lambda f, v: float((int(f[0]) * 31 + v * 17) % 11 + 1), mtd=20)
    for _ in range(200):
        v, _ = r.invoke([float(rng.integers(0, 50)), float(rng.integers(0, 3))])
        assert 0 <= v < V


def test_labels_and_tree_match_oracle_on_random_costs():
    for seed in range(8):
        rng = np.random.Generator(np.random.PCG64(seed))
        V = int(rng.integers(2, 6))
        table = rng.uniform(1.0, 2.0, (4, 3, V))
        cost = lambda f, v: float(table[int(f[0]) % 4, int(f[1]) % 3, v])  # noqa: E731
        r, _ = _region(V=V, nf=2, cost=cost, mtd=10 ** 6)
        for _ in range(150):
            r.invoke([float(rng.integers(0, 4)), float(rng.integers(0, 3))])
        r.train()
        recs = r.records()
        labs = select.labels(recs)
        X = [list(f) for f, _ in labs]
        y = [l for _, l in labs]
        want = select.cart_fit(X, y, max_depth=2)
        assert r.tree() == want
        for x in X:
            assert r.select(x)[0] == select.cart_predict(want, x)


# ------------------------------------------------------------ profiling
def test_profile_exhaustive_argmin_with_ties():
    cost = lambda f, v: [3.0, 1.004, 1.0, 2.0][v]  # noqa: E731
    r, calls = _region(V=4, spec="exhaustive,reps=5", cost=cost)
    ms, best = r.profile([42])
    assert best == select.exhaustive_argmin(ms) == 1  # 1.004 within 0.5 % of 1.0
    assert ms == pytest.approx([3.0, 1.004, 1.0, 2.0])
    assert len(calls.seq) == 4 * 6  # 1 warm-up + 5 timed per variant
    assert r.counts()[0] == 20
    assert r.select([42]) == (1, 1.0)
    with pytest.raises(ar.ArError) as e:
        r.select([43])
    assert e.value.code == ar.AR_ERR_NOMODEL


def test_fixed_model_always_runs_its_variant():
    r, calls = _region(V=3, spec="fixed,2")
    for n in (1, 2, 3):
        assert r.invoke([n])[0] == 2
    assert r.select([9])[0] == 2


# ------------------------------------------------------------ errors
def test_state_and_argument_errors():
    r, _ = _region(V=2)
    with pytest.raises(ar.ArError) as e:
        r.select([1])
    assert e.value.code == ar.AR_ERR_NOMODEL
    with pytest.raises(ar.ArError) as e:
        r.invoke([1, 2])
    assert e.value.code == ar.AR_ERR_STATE
    with pytest.raises(ar.ArError) as e:
        r.invoke([float("nan")])
    assert e.value.code == ar.AR_ERR_ARG
    r.invoke([1])
    with pytest.raises(ar.ArError) as e:
        r.register("late", 9.0, _noop)
    assert e.value.code == ar.AR_ERR_STATE
    # Apollo call order
    with pytest.raises(ar.ArError):
        r.end()
    r.begin()
    with pytest.raises(ar.ArError):
        r.get_policy()  # feature missing
    r.set_feature(3.0)
    with pytest.raises(ar.ArError):
        r.set_feature(4.0)  # too many
    v = r.get_policy()
    assert v == r.get_policy()
    r.end()


def test_failing_launcher_marks_variant_unusable():
    r = ar.Region("f", 1)
    r.register("ok", 0.0, _noop)
    r.register("bad", 1.0, lambda a, v, x, s, u: 7)
    r.register("ok2", 2.0, _noop)
    r.set_fake_timer(lambda f, v: 1.0)
    assert r.invoke([1])[0] == 0
    with pytest.raises(ar.ArError) as e:
        r.invoke([1])
    assert e.value.code == ar.AR_ERR_CUDA
    assert not r.variant(1)["usable"]
    seq = [r.invoke([1])[0] for _ in range(4)]
    assert 1 not in seq


# ------------------------------------------------------------ persistence
def test_save_load_round_trip_and_corruption(tmp_path):
    cost = lambda f, v: (1.0 + v) if f[0] < 100 else (3.0 - v)  # noqa: E731
    r, _ = _region(V=3, cost=cost)
    for n in (10, 1000, 10, 1000, 10, 1000):
        r.invoke([n])
    p = tmp_path / "region.bin"
    r.save(p)
    q, _ = _region(V=3, cost=cost)
    q.load(p)
    assert q.info()["trained"] and q.tree() == r.tree() and q.records() == r.records()
    assert q.select([5000]) == r.select([5000])
    data = bytearray(p.read_bytes())
    data[40] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(data))
    with pytest.raises(ar.ArError) as e:
        q.load(bad)
    assert e.value.code == ar.AR_ERR_IO
    short = tmp_path / "short.bin"
    short.write_bytes(p.read_bytes()[:20])
    with pytest.raises(ar.ArError) as e:
        q.load(short)
    assert e.value.code == ar.AR_ERR_IO
    with pytest.raises(ar.ArError) as e:
        q.load(tmp_path / "missing.bin")
    assert e.value.code == ar.AR_ERR_IO
    w, _ = _region(V=4, cost=cost)
    with pytest.raises(ar.ArError) as e:
        w.load(p)
    assert e.value.code == ar.AR_ERR_STATE
    # the failed loads left q intact
    assert q.tree() == r.tree()


def test_add_record_feeds_training():
    r, _ = _region(V=2, mtd=100)
    for n, best in ((1, 0), (2, 0), (50, 1), (60, 1)):
        r.add_record([n], best, 1.0)
        r.add_record([n], 1 - best, 2.0)
    r.train()
    assert r.select([1.5])[0] == 0 and r.select([55])[0] == 1


def test_loop_tables():
    assert ar.loop_num_variants(ar.AR_LOOP_DAXPY) == 15
    assert ar.loop_default_variant(ar.AR_LOOP_DAXPY) == 6
    assert ar.loop_variant_name(ar.AR_LOOP_DAXPY, 6) == "daxpy_b256_e1"
    assert ar.loop_num_variants(ar.AR_LOOP_JACOBI7) == 16
    assert ar.loop_variant_name(ar.AR_LOOP_JACOBI7, 1) == "jacobi7_naive_32x8"
    r = ar.Region("j", 2)
    assert r.add_builtin(ar.AR_LOOP_JACOBI7) == 16
    assert ar.loop_num_variants(ar.AR_LOOP_HEAT7) == 16
    assert ar.loop_default_variant(ar.AR_LOOP_HEAT7) == 1
    assert ar.loop_variant_name(ar.AR_LOOP_HEAT7, 13) == "heat7_df_32x8"
    assert ar.Region("h", 2).add_builtin(ar.AR_LOOP_HEAT7) == 16
    with pytest.raises(ar.ArError):
        ar.loop_num_variants(17)


def test_kernel_entry_points_validate_before_launch():
    # argument errors are reported without touching the GPU
    with pytest.raises(ar.ArError) as e:
        ar.ar_daxpy(15, 10, 1.0, 16, 32)
    assert e.value.code == ar.AR_ERR_ARG
    assert ar.lib.ar_daxpy(0, 0, 1.0, None, None, None) == 0  # empty: nothing launched
    assert ar.lib.ar_daxpy(1, 4, 1.0, 8, 16, None) == ar.AR_ERR_ARG  # misaligned double2
    assert ar.lib.ar_jacobi7(0, 8, 1, 64, 64, 128, None, None) == ar.AR_ERR_ARG  # aliasing
    assert ar.lib.ar_heat7(0, 8, 1, 0.1, 64, 64, 128, None, None) == ar.AR_ERR_ARG  # aliasing
    for bad in (-0.01, 1.5, float("nan"), float("inf")):  # alpha outside [0, 1]
        assert ar.lib.ar_heat7(0, 8, 1, bad, 64, 128, 192, None, None) == ar.AR_ERR_ARG
    assert ar.lib.ar_heat7(0, 0, 3, 0.1, None, None, None, None, None) == 0  # empty grid
    assert ar.lib.ar_spmv_gather_floor(-1, 8, 8, 8, 8, None) == ar.AR_ERR_ARG
    assert ar.lib.ar_spmv_gather_floor(10, None, 8, 8, 8, None) == ar.AR_ERR_ARG
    assert ar.lib.ar_spmv_gather_floor(0, None, None, None, None, None) == 0  # nothing to stream
    for kind, limit in ((4, 10), (-1, 10), (0, 0), (1, (1 << 24) + 1)):
        assert ar.lib.ar_wait_selftest(kind, limit, 64, None) == ar.AR_ERR_ARG
    assert ar.lib.ar_wait_selftest(0, 10, None, None) == ar.AR_ERR_ARG
    assert ar.lib.ar_measure_fp32x2_rate(None) == ar.AR_ERR_ARG
    assert ar.lib.ar_mlp_num_params(5, 64, 7) == 5 * 64 + 64 + 64 * 64 + 64 + 7 * 64 + 7
    assert ar.lib.ar_mlp_num_params(5, 48, 7) == ar.AR_ERR_ARG


def test_random_forest_matches_oracle_and_needs_both_parameters():
    for bad in ("rfc,5", "rfc,0,2", "rfc,5,0"):
        with pytest.raises(ar.ArError) as e:
            ar.Region("x", 2, bad)
        assert e.value.code == ar.AR_ERR_ARG
    for seed, (nt, depth) in enumerate([(7, 2), (4, 3), (10, 1)]):
        rng = np.random.Generator(np.random.PCG64(40 + seed))
        V = 4
        table = rng.uniform(1.0, 2.0, (5, 4, V))
        cost = lambda f, v: float(table[int(f[0]) % 5, int(f[1]) % 4, v])  # noqa: E731
        r = ar.Region("rf", 2, f"rfc,{nt},{depth},seed={seed + 3}", 10 ** 6)
        for v in range(V):
            r.register(f"v{v}", float(v), _noop)
        r.set_fake_timer(cost)
        for _ in range(120):
            r.invoke([float(rng.integers(0, 5)), float(rng.integers(0, 4))])
        r.train()
        assert r.info()["model"] == "rfc"
        labs = select.labels(r.records())
        X = [list(f) for f, _ in labs]
        y = [lab for _, lab in labs]
        want = select.rfc_fit(X, y, nt, depth, seed + 3)
        assert r.forest() == want
        for x in X:
            v, conf = r.select(x)
            assert (v, conf) == pytest.approx(select.rfc_predict(want, x))


def test_random_forest_save_load(tmp_path):
    r, _ = _region(V=3, spec="rfc,5,2", mtd=6, cost=lambda f, v: (1.0 + v) if f[0] < 100 else (3.0 - v))
    for n in (10, 1000, 10, 1000, 10, 1000, 40, 4000):
        r.invoke([n])
    p = tmp_path / "rf.bin"
    r.save(p)
    q, _ = _region(V=3, spec="rfc,5,2")
    q.load(p)
    assert q.forest() == r.forest() and q.select([5000]) == r.select([5000])


def test_exec_fallback_checks_region_shapes_before_device_work():
    ws = 256  # a dummy device address: every case below returns before any device work
    daxpy_like = ar.Region("fb-shape", 1, "dtree", 10 ** 9)
    daxpy_like.add_builtin(ar.AR_LOOP_JACOBI7)  # 16 variants where daxpy has 15
    bad = [daxpy_like, None, None, None]
    call = ar.ArExecCall(loop=0, n=10)
    with pytest.raises(ar.ArError) as e:
        ar.ar_exec_fallback([call], np.zeros((1, 8)), [0.0], 0.5, bad, 1, None, False, ws, 1 << 20)
    assert e.value.code == ar.AR_ERR_STATE
    wrong_nf = ar.Region("fb-nf", 2, "dtree", 10 ** 9)
    wrong_nf.add_builtin(ar.AR_LOOP_DAXPY)
    with pytest.raises(ar.ArError) as e:
        ar.ar_exec_fallback([call], np.zeros((1, 8)), [0.0], 0.5, [wrong_nf, None, None, None], 1, None, False,
                            ws, 1 << 20)
    assert e.value.code == ar.AR_ERR_STATE
    for reps in (0, 17):
        with pytest.raises(ar.ArError) as e:
            ar.ar_exec_fallback([call], np.zeros((1, 8)), [0.0], 0.5, [None] * 4, reps, None, False, ws, 1 << 20)
        assert e.value.code == ar.AR_ERR_ARG
    with pytest.raises(ar.ArError) as e:  # workspace smaller than the fixed part
        ar.ar_exec_fallback([call], np.zeros((1, 8)), [0.0], 0.5, [None] * 4, 1, None, False, ws, 64)
    assert e.value.code == ar.AR_ERR_ARG


def test_invoke_host_rejects_bad_copy_lists_before_enqueuing():
    r = ar.Region("host-copy", 1, "fixed,0", 0)
    r.register("v0", 0.0, _noop)
    with pytest.raises(ar.ArError) as e:
        r.invoke_host([1.0], None, [(0, 64, 8)], [])  # NULL host pointer with bytes
    assert e.value.code == ar.AR_ERR_ARG
    with pytest.raises(ar.ArError) as e:
        r.invoke_host([1.0], None, [], [(64, 0, 8)])  # NULL device pointer with bytes
    assert e.value.code == ar.AR_ERR_ARG
    with pytest.raises(ar.ArError) as e:
        r.invoke_host([1.0, 2.0], None, [], [])  # wrong feature count
    assert e.value.code == ar.AR_ERR_STATE
    with pytest.raises(ar.ArError) as e:
        r.invoke_host([float("nan")], None, [], [])
    assert e.value.code == ar.AR_ERR_ARG
    assert r.counts() == (0, 0)


def test_normal_build_reports_checks_disabled():
    # the normal build's readers answer without touching the device
    if ar.CHECKED:
        pytest.skip("this process loaded the bounds-check build")
    assert ar.ar_check_status(clear=False) == (False, 0, 0)


def test_tie_option_widens_the_label_ties_to_the_lowest_index():
    times = {0: 1.02, 1: 1.0, 2: 1.01}  # variant 0 within 2 % of the fastest

    def make(spec):
        r = ar.Region("tie", 1, spec, 10 ** 9)
        for v in range(3):
            r.register(f"v{v}", float(v), _noop)
        r.set_fake_timer(lambda f, v: times[v])
        return r

    default, wide = make("exhaustive"), make("exhaustive,tie=0.03")
    assert default.profile([1.0], reps=1)[1] == 1  # the paper reading: 0.5 %
    assert wide.profile([1.0], reps=1)[1] == 0
    for r, want in ((default, 1), (wide, 0)):
        r.train()
        assert r.select([1.0])[0] == want
    for bad in ("dtree,tie=1", "dtree,tie=-0.1", "dtree,tie=x"):
        with pytest.raises(ar.ArError):
            ar.Region("bad", 1, bad, 1)


def test_ar_log_levels_write_region_events_to_stderr():
    import subprocess
    import sys
    import textwrap

    code = textwrap.dedent("""
        import paper_2303_08873_b300 as ar
        r = ar.Region("logged", 1, "dtree", 4)
        for v in range(2):
            r.register(f"v{v}", float(v), lambda a, v, x, s, u: 0)
        r.set_fake_timer(lambda f, v: 1.0 + v)
        r.profile([1.0], reps=1)
        r.profile([2.0], reps=1)
        r.train()
        r.select([1.0])
    """)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for level in ("0", "1", "2"):
        env = dict(os.environ, AR_LOG=level)
        p = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True,
                           timeout=120)
        assert p.returncode == 0, p.stderr
        out[level] = [ln for ln in p.stderr.splitlines() if ln.startswith("[ar] logged:")]
    assert out["0"] == []
    assert any("trained dtree" in ln for ln in out["1"]) and not any("profiled" in ln for ln in out["1"])
    assert any("profiled 2 variants" in ln for ln in out["2"]) and any("selected 0" in ln for ln in out["2"])
