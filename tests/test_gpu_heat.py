"""7-point explicit heat variants against the float64 oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import cone_cube, dev, host

pytestmark = pytest.mark.gpu
V = 16
# max |gpu - ref| <= TOL * max(max |ref|, max |u0|): the update cancels (at
# alpha = 1/6 a lone point's u (1 - 6 alpha) is 0), so the error is measured
# against the operands' scale, which the step never exceeds for alpha <= 1/6
TOL = 1e-13
HEAT = 4     # loop id of the heat stencil


def _run(v, u0, steps, alpha, status="new"):
    """status "new": a fresh int[2] status array (lets the df family keep
    float pairs between steps); None: no status array."""
    N = u0.shape[0]
    ud = dev(u0)
    out = torch.empty_like(ud)
    work = torch.empty_like(ud)
    st = torch.zeros(2, dtype=torch.int32, device="cuda") if isinstance(status, str) else status
    ar.ar_heat7(v, N, steps, alpha, ud, out, work, st)
    if st is not None:
        assert int(st[0].item()) == 0
    return host(out)


def _check(out, ref, what, u0=None):
    err = np.max(np.abs(out - ref))
    scale = max(np.max(np.abs(ref)), np.max(np.abs(u0)) if u0 is not None else 0.0)
    assert err <= TOL * scale, (what, err, scale)


# sizes: odd, tiny, ragged against every tile, >= 132 so the 128x2 boxes run TMA
@pytest.mark.parametrize("N", [1, 2, 7, 33, 50, 134])
@pytest.mark.parametrize("steps,alpha", [(1, 0.1), (2, 1.0 / 6.0), (10, 0.125)])
def test_all_variants_match_oracle(N, steps, alpha):
    u0 = synth.grid_inputs(21, N)
    ref = loops.heat7(u0, steps, alpha)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    for v in range(V):
        _check(_run(v, u0, steps, alpha, status), ref, (ar.loop_variant_name(HEAT, v), N, steps), u0)
        assert int(status[0].item()) == 0
    for v in range(12, 16):  # df family without a status array: float64 between steps
        _check(_run(v, u0, steps, alpha, None), ref, (ar.loop_variant_name(HEAT, v), N, steps, "no status"), u0)


def test_alpha_bounds_and_zero_steps():
    u0 = synth.grid_inputs(22, 36)
    for v in range(V):
        assert np.array_equal(_run(v, u0, 0, 0.1), u0)
        _check(_run(v, u0, 3, 0.0), u0, ("alpha 0", v))
        _check(_run(v, u0, 2, 1.0), loops.heat7(u0, 2, 1.0), ("alpha 1", v), u0)
    for v in range(8):  # float64 families: alpha 0 leaves every value bitwise
        assert np.array_equal(_run(v, u0, 3, 0.0), u0), v


def test_linear_field_interior_and_eigenmode():
    N = 48
    lin = synth.linear_field(N, 3, -2, 5)
    mode = synth.sine_mode(N)
    h = 1.0 / (N + 1)
    lam = 1.0 - 6.0 * 0.15 * (1.0 - np.cos(np.pi * h))
    for v in range(V):
        out = _run(v, lin, 4, 0.15)
        core = (slice(4, N - 4),) * 3
        _check(out[core], lin[core], ("linear", v))
        _check(_run(v, mode, 3, 0.15), lam ** 3 * mode, ("mode", v))


def test_df_range_guard_falls_back_to_float64():
    N = 40
    u0 = synth.grid_inputs(24, N)
    u0[5, 6, 7] = 1e-30
    u0[20, 20, 20] = 3e40
    u0[10, 11, 12] = 0.0
    ref = loops.heat7(u0, 3, 0.125)
    big = np.abs(ref) > 1e3
    for v in range(12, 16):
        for st in ("new", None):
            out = _run(v, u0, 3, 0.125, st)
            _check(out[~big], ref[~big], ("df mixed", v, st), u0[~big])
            assert np.all(np.abs(out[big] - ref[big]) <= 1e-15 * np.abs(ref[big]) * 8)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    _run(13, u0, 3, 0.125, st)
    assert int(st[1].item()) == 1
    u1 = synth.grid_inputs(25, 36)
    u1[3, 3, 3] = np.inf
    u1[20, 3, 3] = np.nan
    ref1 = loops.heat7(u1, 1, 0.1)
    for v in range(V):
        out = _run(v, u1, 1, 0.1)
        assert np.array_equal(np.isnan(out), np.isnan(ref1)), v
        assert np.array_equal(np.isinf(out), np.isinf(ref1)), v
        fin = np.isfinite(ref1)
        _check(out[fin], ref1[fin], ("nonfinite", v), u1[np.isfinite(u1)])


@pytest.mark.parametrize("N", [128, 256, 512])
def test_bench_sizes_sampled(N):
    """Launch configuration of the heat benchmark (10 steps, alpha 1/8):
    sampled outputs against the oracle on their 10-step dependency cube."""
    s, alpha = 10, 0.125
    u0 = synth.grid_inputs(2000 + N, N)
    rng = np.random.Generator(np.random.PCG64(N + 1))
    pts = [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N // 2, N - 1), (N // 3, 0, 1)]
    pts += [tuple(int(c) for c in rng.integers(0, N, 3)) for _ in range(24)]
    refs = []
    for p in pts:
        o, L = cone_cube(N, s, p)
        cube = u0[o[0]:o[0] + L, o[1]:o[1] + L, o[2]:o[2] + L]
        if L < N:
            refs.append(loops.heat7(cube, s, alpha)[p[0] - o[0], p[1] - o[1], p[2] - o[2]])
        else:
            refs.append(loops.heat7(u0, s, alpha)[p])
    refs = np.array(refs)
    scale = max(np.max(np.abs(refs)), np.max(np.abs(u0)))
    ud = dev(u0)
    out = torch.empty_like(ud)
    work = torch.empty_like(ud)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    idx = torch.tensor([(p[0] * N + p[1]) * N + p[2] for p in pts], device="cuda")
    for v in range(V):
        ar.ar_heat7(v, N, s, alpha, ud, out, work, status)
        got = host(out.view(-1)[idx])
        assert np.max(np.abs(got - refs)) <= TOL * scale, (ar.loop_variant_name(HEAT, v), N)


def test_every_variant_is_deterministic():
    u0 = synth.grid_inputs(26, 66)
    for v in range(V):
        assert np.array_equal(_run(v, u0, 4, 0.1), _run(v, u0, 4, 0.1)), v


def test_region_selects_among_heat_variants():
    """The region runtime drives the heat variants like any loop: it explores
    every variant once per feature vector, then its trained tree picks one."""
    N, steps, alpha = 64, 2, 0.125
    u0 = synth.grid_inputs(27, N)
    ud = dev(u0)
    out, work = torch.empty_like(ud), torch.empty_like(ud)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    r = ar.Region("heat", 2, "dtree,2")
    assert r.add_builtin(HEAT) == V
    args = ar.ArHeat7Args(N, steps, alpha, ud.data_ptr(), out.data_ptr(), work.data_ptr(), st.data_ptr())
    seen = set()
    ref = loops.heat7(u0, steps, alpha)
    for _ in range(V + 2):
        v, _ = r.invoke([N, steps], args)
        torch.cuda.synchronize()
        seen.add(v)
        _check(host(out), ref, ("region", v))
    assert seen == set(range(V))


@pytest.mark.parametrize("N", [37, 133])
def test_odd_n_tensor_copies(N):
    u0 = synth.grid_inputs(60 + N, N)
    ref = loops.heat7(u0, 4, 0.125)
    for v in range(8, 16):
        _check(_run(v, u0, 4, 0.125), ref, (ar.loop_variant_name(HEAT, v), N), u0)

