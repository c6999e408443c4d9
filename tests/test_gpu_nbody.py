"""All-pairs n-body variants (FP32) against the float64 oracle (GPU)."""
import numpy as np
import pytest
import torch

import paper_2303_08873_b300 as ar
import synth
from oracle import loops
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu
V = 9
EPS = synth.NBODY_EPS
TOL = 1e-4  # max_i |a_i - a_ref_i| <= TOL * max_i |a_ref_i|


def _run(v, p):
    pd = dev(p)
    a = torch.full((p.shape[0], 4), np.nan, dtype=torch.float32, device="cuda")
    ar.ar_nbody(v, p.shape[0], pd, a, EPS)
    return host(a)


def _check(acc4, ref, what):
    assert np.all(acc4[:, 3] == 0.0), what
    err = np.max(np.linalg.norm(acc4[:, :3].astype(np.float64) - ref, axis=1))
    scale = np.max(np.linalg.norm(ref, axis=1))
    assert err <= TOL * scale, (what, err, scale)


@pytest.mark.parametrize("N", [1, 2, 100, 1000, 4097])
def test_all_variants_match_oracle(N):
    p = synth.nbody_inputs(4, N)
    ref = loops.nbody(p, EPS)
    for v in range(V):
        a = _run(v, p)
        if N == 1:
            assert np.array_equal(a, np.zeros((1, 4), np.float32)), v
        else:
            _check(a, ref, (ar.loop_variant_name(3, v), N))


def test_two_body_reaction_and_cube_centre():
    two = np.array([[0.25, 0.5, 0.5, 0.75], [0.75, 0.5, 0.5, 0.5]], dtype=np.float32)
    verts = [[x, y, z, 1.0] for x in (0.25, 0.75) for y in (0.25, 0.75) for z in (0.25, 0.75)]
    cube = np.array(verts + [[0.5, 0.5, 0.5, 1.0]], dtype=np.float32)
    for v in range(V):
        a = _run(v, two)
        assert 0.75 * a[0, 0] == pytest.approx(-0.5 * a[1, 0], rel=1e-6)
        _check(a, loops.nbody(two, EPS), ("two", v))
        c = _run(v, cube)
        assert np.max(np.abs(c[-1, :3])) <= 1e-6 * np.max(np.abs(c[:-1, :3]))


def test_signed_and_zero_masses():
    """Negative masses in one tile (the weight keeps the mass's sign); zero
    masses add nothing."""
    N = 3000
    p = synth.nbody_inputs(13, N)
    p[::7, 3] = 0.0
    p[1000:1010, 3] *= -1.0  # one tile of every tile size, and part of one body pair
    ref = loops.nbody(p, EPS)
    for v in range(V):
        _check(_run(v, p), ref, ("signed masses", v))
    q = p.copy()
    q[:, 3] = 0.0
    for v in range(V):
        assert np.array_equal(_run(v, q), np.zeros((N, 4), np.float32)), v


@pytest.mark.parametrize("N", [65536, 262144])
def test_full_size_sampled(N):
    """Workload sizes: 2048 sampled bodies (plus the first and last) against
    the float64 oracle, all variants."""
    p = synth.nbody_inputs(4, N)
    rng = np.random.Generator(np.random.PCG64(N))
    which = np.unique(np.concatenate([[0, N - 1], rng.integers(0, N, 2048)]))
    ref = loops.nbody_rows(p, which, EPS)
    pd = dev(p)
    a = torch.empty((N, 4), dtype=torch.float32, device="cuda")
    for v in range(V):
        ar.ar_nbody(v, N, pd, a, EPS)
        got = host(a)[which]
        _check(got, ref, (ar.loop_variant_name(3, v), N))


def _batched(bodies, offs):
    count = offs.size - 1
    wsb = ar.ar_nbody_batched_workspace_bytes(count)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    a = torch.full((bodies.shape[0], 4), np.nan, dtype=torch.float32, device="cuda")
    ar.ar_nbody_batched(count, dev(offs), dev(bodies), a, EPS, ws, wsb)
    return host(a)


def test_batched_small_full_compare():
    bodies, offs = synth.nbody_batch_inputs(41, count=7, nmin=1, nmax=700)
    a = _batched(bodies, offs)
    for b in range(7):
        sl = slice(offs[b], offs[b + 1])
        if offs[b + 1] - offs[b] > 1:
            _check(a[sl], loops.nbody(bodies[sl], EPS), ("batched", b))


def test_batched_workload_sampled():
    """64 systems, sizes log-uniform in [1k, 64k]: 24 sampled bodies per
    system against the oracle of that system."""
    bodies, offs = synth.nbody_batch_inputs(40)
    a = _batched(bodies, offs)
    rng = np.random.Generator(np.random.PCG64(40))
    for b in range(offs.size - 1):
        sys_p = bodies[offs[b]:offs[b + 1]]
        which = rng.integers(0, sys_p.shape[0], 24)
        ref = loops.nbody_rows(sys_p, which, EPS)
        got = a[offs[b]:offs[b + 1]][which]
        err = np.max(np.linalg.norm(got[:, :3].astype(np.float64) - ref, axis=1))
        assert err <= TOL * np.max(np.linalg.norm(ref, axis=1)) * 4, b


@pytest.mark.parametrize("N", [5000, 70000])
def test_every_variant_is_deterministic(N):
    # 5000 bodies: the j range is split over thread-block clusters and the
    # partials are added in rank order, so repeated runs agree bit for bit
    p = synth.nbody_inputs(12, N)
    for v in range(V):
        assert np.array_equal(_run(v, p), _run(v, p)), v


@pytest.mark.parametrize("N", [16384, 30000])
def test_cluster_split_sizes_match_oracle(N):
    # sizes whose grid of one body per thread underfills the GPU: every tile
    # splits its j range over a cluster (some ranks of the 512 tiles empty)
    p = synth.nbody_inputs(13, N)
    rows = np.arange(0, N, 97)
    ref = loops.nbody_rows(p, rows, EPS)
    scale = np.max(np.linalg.norm(ref, axis=1))
    for v in range(V):
        a = _run(v, p)[rows]
        assert np.all(a[:, 3] == 0.0), v
        err = np.max(np.linalg.norm(a[:, :3].astype(np.float64) - ref, axis=1))
        assert err <= TOL * scale, (ar.loop_variant_name(3, v), N, err, scale)


def test_roofline_denominators_are_plausible():
    # the issue-rate microbenchmarks behind the n-body and float64 roofs:
    # float64 is a small fraction of float32 on B300, and packed float32
    # pairs cannot beat the scalar float32 lane rate by more than noise
    fp64, fp32 = ar.ar_measure_fma_rates()
    packed = ar.ar_measure_fp32x2_rate()
    assert 0 < fp64 < 0.2 * fp32
    assert 0.5 * fp32 < packed < 1.1 * fp32


@pytest.mark.parametrize("N", [1, 1000, 4097, 30000, 65536, 262144])
def test_launch_geometry_follows_the_split_rule(N):
    """ar_nbody_geometry against the rule it reports: two bodies per thread
    once ceil(N / 2T) fills two blocks per SM, else one; the j range split
    over a cluster only below two blocks per SM, never past 8 blocks."""
    for v in range(9):
        T = (128, 256, 512)[v // 3]
        g = ar.ar_nbody_geometry(v, N)
        sms = g["sms"]
        two = -(-N // (2 * T)) >= 2 * sms
        assert g["bodies_per_thread"] == (2 if two else 1)
        assert g["grid"] == -(-N // (T * g["bodies_per_thread"]))
        assert 1 <= g["cluster"] <= min(8, g["grid"]) or (g["cluster"] == 1 and g["grid"] == 1)
        if two:
            assert g["cluster"] == 1
        assert g["resident_per_sm"] >= 1 and g["waves"] > 0
