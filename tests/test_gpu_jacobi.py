"""7-point Jacobi variants against the float64 oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import cone_cube, dev, host

pytestmark = pytest.mark.gpu
V = 16
TOL = 1e-13  # max |gpu - ref| <= TOL * max |ref|


def _run(v, u0, sweeps, status="new"):
    """status "new": a fresh int[2] status array (lets the df family keep
    float pairs between sweeps); None: no status array."""
    N = u0.shape[0]
    ud = dev(u0)
    out = torch.empty_like(ud)
    work = torch.empty_like(ud)
    st = torch.zeros(2, dtype=torch.int32, device="cuda") if isinstance(status, str) else status
    ar.ar_jacobi7(v, N, sweeps, ud, out, work, st)
    if st is not None:
        assert int(st[0].item()) == 0
    return host(out)


def _check(out, ref, what):
    err = np.max(np.abs(out - ref))
    scale = np.max(np.abs(ref))
    assert err <= TOL * scale, (what, err, scale)


# sizes: odd, tiny, ragged against every tile, >= 132 so the 128x2 boxes run TMA
@pytest.mark.parametrize("N", [1, 2, 7, 33, 50, 70, 134])
@pytest.mark.parametrize("sweeps", [1, 2, 10])
def test_all_variants_match_oracle(N, sweeps):
    u0 = synth.grid_inputs(2, N)
    ref = loops.jacobi7(u0, sweeps)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    for v in range(V):
        _check(_run(v, u0, sweeps, status), ref, (ar.loop_variant_name(1, v), N, sweeps))
        assert int(status[0].item()) == 0
    for v in range(12, 16):  # df family without a status array: float64 between sweeps
        _check(_run(v, u0, sweeps, None), ref, (ar.loop_variant_name(1, v), N, sweeps, "no status"))


def test_zero_sweeps_copies():
    u0 = synth.grid_inputs(3, 9)
    for v in range(V):
        assert np.array_equal(_run(v, u0, 0), u0)


def test_linear_field_interior_and_eigenmode():
    N = 48
    lin = synth.linear_field(N, 3, -2, 5)
    mode = synth.sine_mode(N)
    for v in range(V):
        out = _run(v, lin, 4)
        core = (slice(4, N - 4),) * 3
        # a linear field is reproduced away from the faces
        _check(out[core], lin[core], ("linear", v))
        _check(_run(v, mode, 3), np.cos(np.pi / (N + 1)) ** 3 * mode, ("mode", v))


def test_df_range_guard_falls_back_to_float64():
    # values the float-pair split cannot carry: tiny, huge, zero, inf and NaN
    N = 40
    u0 = synth.grid_inputs(4, N)
    u0[5, 6, 7] = 1e-30
    u0[20, 20, 20] = 3e40
    u0[10, 11, 12] = 0.0
    u0[30, 1, 1] = -2.5e-25
    ref = loops.jacobi7(u0, 3)
    big = np.abs(ref) > 1e3
    for v in range(12, 16):
        for st in ("new", None):
            out = _run(v, u0, 3, st)
            _check(out[~big], ref[~big], ("df mixed", v, st))
            assert np.all(np.abs(out[big] - ref[big]) <= 1e-15 * np.abs(ref[big]) * 8)
    tiny = synth.grid_inputs(5, 36) * 1e-80
    reft = loops.jacobi7(tiny, 4)
    for v in range(12, 16):
        _check(_run(v, tiny, 4), reft, ("df tiny", v))
    # the first sweep's decision: float64 storage between sweeps when a value
    # leaves the float-pair range, float pairs otherwise
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    _run(13, u0, 3, st)
    assert int(st[1].item()) == 1
    _run(13, synth.grid_inputs(4, N), 3, st)
    assert int(st[1].item()) == 0
    u1 = synth.grid_inputs(6, 36)
    u1[3, 3, 3] = np.inf
    u1[20, 3, 3] = np.nan
    ref1 = loops.jacobi7(u1, 1)
    for v in range(V):
        out = _run(v, u1, 1)
        assert np.array_equal(np.isnan(out), np.isnan(ref1)), v
        assert np.array_equal(np.isinf(out), np.isinf(ref1)), v
        fin = np.isfinite(ref1)
        _check(out[fin], ref1[fin], ("nonfinite", v))


@pytest.mark.parametrize("N", [32, 64, 128, 256, 384, 512])
def test_bench_sizes_sampled(N):
    """Launch configuration of the benchmark: 10 sweeps of U[-1,1] at each N;
    sampled outputs (corners, faces, random) against the oracle on their
    10-sweep dependency cube."""
    s = 10
    u0 = synth.grid_inputs(1000 + N, N)
    rng = np.random.Generator(np.random.PCG64(N))
    pts = [(0, 0, 0), (N - 1, N - 1, N - 1), (0, N // 2, N - 1), (N // 3, 0, 1)]
    pts += [tuple(int(c) for c in rng.integers(0, N, 3)) for _ in range(24)]
    refs = []
    for p in pts:
        o, L = cone_cube(N, s, p)
        cube = u0[o[0]:o[0] + L, o[1]:o[1] + L, o[2]:o[2] + L]
        if L < N:
            refs.append(loops.jacobi7(cube, s)[p[0] - o[0], p[1] - o[1], p[2] - o[2]])
        else:
            refs.append(loops.jacobi7(u0, s)[p])
    refs = np.array(refs)
    scale = np.max(np.abs(refs))
    ud = dev(u0)
    out = torch.empty_like(ud)
    work = torch.empty_like(ud)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    idx = torch.tensor([(p[0] * N + p[1]) * N + p[2] for p in pts], device="cuda")
    for v in range(V):
        ar.ar_jacobi7(v, N, s, ud, out, work, status)
        got = host(out.view(-1)[idx])
        assert np.max(np.abs(got - refs)) <= TOL * scale, (ar.loop_variant_name(1, v), N)


def test_every_variant_is_deterministic():
    u0 = synth.grid_inputs(9, 66)
    for v in range(V):
        assert np.array_equal(_run(v, u0, 4), _run(v, u0, 4)), v


def test_two_sweep_pair_chain_with_flagged_input():
    # 2 sweeps: float64 -> pairs, pairs -> float64, and the catch-up launch
    u0 = synth.grid_inputs(10, 40)
    u0[7, 8, 9] = 1e-200
    ref = loops.jacobi7(u0, 2)
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    for v in range(12, 16):
        _check(_run(v, u0, 2, st), ref, ("flagged 2 sweeps", v))


@pytest.mark.parametrize("N", [37, 71, 135])
@pytest.mark.parametrize("sweeps", [1, 2, 5])
def test_odd_n_tensor_copies(N, sweeps):
    """Odd N >= BX + 4: the tma and df families stage planes through the
    2N-wide view of the grid (two half-boxes per plane, zeroed edges, the last
    grid row loaded by the threads)."""
    u0 = synth.grid_inputs(40 + N, N)
    ref = loops.jacobi7(u0, sweeps)
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    for v in range(8, 16):
        _check(_run(v, u0, sweeps, status), ref, (ar.loop_variant_name(1, v), N, sweeps))
        assert int(status[0].item()) == 0
    for v in range(12, 16):
        _check(_run(v, u0, sweeps, None), ref, (ar.loop_variant_name(1, v), N, sweeps, "no status"))


def test_odd_n_range_guard():
    N = 41
    u0 = synth.grid_inputs(48, N)
    u0[5, 6, 7] = 1e-30
    u0[20, 20, 20] = 3e40
    u0[N - 1, N - 1, N - 1] = 2.5  # the grid's last row, past the 2N-wide view
    ref = loops.jacobi7(u0, 3)
    big = np.abs(ref) > 1e3
    st = torch.zeros(2, dtype=torch.int32, device="cuda")
    for v in range(12, 16):
        out = _run(v, u0, 3, st)
        _check(out[~big], ref[~big], ("odd df mixed", v))
        assert np.all(np.abs(out[big] - ref[big]) <= 1e-15 * np.abs(ref[big]) * 8)

