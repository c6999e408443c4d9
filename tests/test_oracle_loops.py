"""Pins of the float64 loop oracle against closed forms, invariants and
independent library formulations (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import loops


# ------------------------------------------------------------------ daxpy
def test_daxpy_a_zero_leaves_y_bitwise():
    _, x, y = synth.daxpy_inputs(1, 10007)
    assert np.array_equal(loops.daxpy(0.0, x, y), y)


def test_daxpy_y_zero_a_one_gives_x_bitwise():
    _, x, _ = synth.daxpy_inputs(1, 4099)
    assert np.array_equal(loops.daxpy(1.0, x, np.zeros_like(x)), x)


def _dyadic(seed, n):
    r = np.random.Generator(np.random.PCG64(seed))
    kx = r.integers(-2**20, 2**20, n)
    ky = r.integers(-2**20, 2**20, n)
    return kx, ky, kx / 2.0**20, ky / 2.0**20


@pytest.mark.parametrize("fma", [False, True])
def test_daxpy_dyadic_exact(fma):
    kx, ky, x, y = _dyadic(3, 5000)
    out = loops.daxpy(1.5, x, y, fma=fma)
    exact = [float(Fraction(3, 2) * Fraction(int(a), 2**20) + Fraction(int(b), 2**20))
             for a, b in zip(kx, ky)]
    assert np.array_equal(out, np.array(exact))


def test_daxpy_linearity_dyadic():
    _, _, x, y = _dyadic(4, 3000)
    lhs = loops.daxpy(1.5, x, loops.daxpy(0.25, x, y))
    rhs = loops.daxpy(1.75, x, y)
    assert np.array_equal(lhs, rhs)


def test_daxpy_fma_and_plain_agree_to_scaled_bound():
    a, x, y = synth.daxpy_inputs(1, 1 << 16)
    p = loops.daxpy(a, x, y)
    f = loops.daxpy(a, x, y, fma=True)
    scale = np.abs(a * x) + np.abs(y)
    assert np.all(np.abs(p - f) <= 2.3e-16 * scale)


# ------------------------------------------------------------------ Jacobi
def test_jacobi_constant_field_faces_edges_corners():
    # u = 6 everywhere: a point with m in-cube neighbours gets exactly m.
    N = 7
    out = loops.jacobi7(np.full((N, N, N), 6.0), 1)
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    nb = 6 - sum(((c == 0) | (c == N - 1)).astype(int) for c in (i, j, k))
    assert np.array_equal(out, nb.astype(np.float64))


@pytest.mark.parametrize("N,s", [(9, 1), (16, 3), (24, 10)])
def test_jacobi_eigenfunction_closed_form(N, s):
    # sin(x-h) + sin(x+h) = 2 cos(h) sin(x) in each axis, and the zero ghost
    # is sin(0) = sin(pi) = 0, so a sweep multiplies the mode by cos(pi h).
    u0 = synth.sine_mode(N)
    out = loops.jacobi7(u0, s)
    h = 1.0 / (N + 1)
    want = math.cos(math.pi * h) ** s * u0
    assert np.max(np.abs(out - want)) <= 1e-14 * s * np.max(np.abs(u0))


@pytest.mark.parametrize("s", [1, 2, 4])
def test_jacobi_linear_field_exact_away_from_faces(s):
    # A linear field averages to itself; the boundary's influence moves one
    # cell per sweep, so points farther than s from every face stay exact.
    N = 14
    u0 = synth.linear_field(N, 3, -2, 5)
    out = loops.jacobi7(u0, s)
    core = (slice(s, N - s),) * 3
    assert np.array_equal(out[core], u0[core])
    assert not np.array_equal(out, u0)


def _grid_operator(N):
    T = sp.diags([np.ones(N - 1), np.ones(N - 1)], [-1, 1], format="csr")
    I = sp.identity(N, format="csr")
    # unknown (k, j, i) at (k*N + j)*N + i: i is the fastest (last) factor
    return (sp.kron(sp.kron(I, I), T) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(T, I), I)) / 6.0


@pytest.mark.parametrize("N,s", [(5, 1), (8, 4), (11, 3)])
def test_jacobi_matches_kronecker_operator(N, s):
    u0 = synth.grid_inputs(2, N)
    A = _grid_operator(N)
    v = u0.ravel()
    for _ in range(s):
        v = A @ v
    out = loops.jacobi7(u0, s)
    assert np.max(np.abs(out.ravel() - v)) <= 1e-15 * s * np.max(np.abs(u0)) * 4


def test_jacobi_zero_sweeps_is_copy():
    u0 = synth.grid_inputs(2, 6)
    assert np.array_equal(loops.jacobi7(u0, 0), u0)


# ------------------------------------------------------------------ Heat
def test_heat_constant_field_faces_edges_corners():
    # u = 8, alpha = 1/8: u + (m * 8 - 48) / 8 = m + 2 for a point with m
    # in-cube neighbours (every operation exact in float64)
    N = 7
    out = loops.heat7(np.full((N, N, N), 8.0), 1, 0.125)
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    nb = 6 - sum(((c == 0) | (c == N - 1)).astype(int) for c in (i, j, k))
    assert np.array_equal(out, (nb + 2).astype(np.float64))


@pytest.mark.parametrize("N,s,alpha", [(9, 1, 0.1), (16, 3, 1.0 / 6.0), (24, 10, 0.125)])
def test_heat_eigenfunction_closed_form(N, s, alpha):
    # the neighbour sum of the sine mode is 6 cos(pi h) u (one 2 cos(pi h)
    # per axis), so a step multiplies it by 1 - 6 alpha (1 - cos(pi h))
    u0 = synth.sine_mode(N)
    out = loops.heat7(u0, s, alpha)
    h = 1.0 / (N + 1)
    lam = 1.0 - 6.0 * alpha * (1.0 - math.cos(math.pi * h))
    assert np.max(np.abs(out - lam ** s * u0)) <= 1e-14 * s * np.max(np.abs(u0))


@pytest.mark.parametrize("s", [1, 3])
def test_heat_linear_field_unchanged_away_from_faces(s):
    # the discrete Laplacian of an integer linear field is exactly 0
    N = 14
    u0 = synth.linear_field(N, 3, -2, 5)
    out = loops.heat7(u0, s, 0.1)
    core = (slice(s, N - s),) * 3
    assert np.array_equal(out[core], u0[core])
    assert not np.array_equal(out, u0)


@pytest.mark.parametrize("N,s,alpha", [(5, 1, 0.1), (8, 4, 0.15), (11, 3, 1.0 / 7.0)])
def test_heat_matches_kronecker_operator(N, s, alpha):
    u0 = synth.grid_inputs(2, N)
    L = _grid_operator(N) * 6.0 - 6.0 * sp.identity(N ** 3, format="csr")
    v = u0.ravel()
    for _ in range(s):
        v = v + alpha * (L @ v)
    out = loops.heat7(u0, s, alpha)
    assert np.max(np.abs(out.ravel() - v)) <= 1e-15 * s * np.max(np.abs(u0)) * 16


def test_heat_alpha_one_sixth_is_jacobi_and_zero_is_identity():
    u0 = synth.grid_inputs(3, 12)
    a = loops.heat7(u0, 4, 1.0 / 6.0)
    b = loops.jacobi7(u0, 4)
    assert np.max(np.abs(a - b)) <= 1e-15 * 4 * np.max(np.abs(u0)) * 8
    assert np.array_equal(loops.heat7(u0, 3, 0.0), u0)
    assert np.array_equal(loops.heat7(u0, 0, 0.1), u0)


# ------------------------------------------------------------------ SpMV
def test_spmv_identity_bitwise():
    n = 1000
    x = synth.spmv_x(7, n).numpy()
    rowptr = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    assert np.array_equal(loops.spmv(rowptr, col, np.ones(n), x), x)


def test_spmv_diagonal_bitwise():
    n = 777
    x = synth.spmv_x(7, n).numpy()
    d = np.random.Generator(np.random.PCG64(8)).normal(size=n)
    out = loops.spmv(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d, x)
    assert np.array_equal(out, d * x)


def test_spmv_empty_rows_are_zero():
    rowptr = np.array([0, 0, 2, 2, 3, 3], dtype=np.int32)
    col = np.array([0, 4, 2], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0])
    x = np.array([1.0, 10.0, 100.0, 1000.0, 10000.0])
    assert np.array_equal(loops.spmv(rowptr, col, val, x), np.array([0.0, 20001.0, 0.0, 300.0, 0.0]))


def test_spmv_dense_row_within_summation_bound():
    # a 4096-long row against the correctly rounded sum (math.fsum, Shewchuk)
    n = 4096
    r = np.random.Generator(np.random.PCG64(9))
    val = r.normal(size=n)
    x = r.uniform(-1, 1, n)
    out = loops.spmv(np.array([0, n], dtype=np.int32), np.arange(n, dtype=np.int32), val, x)
    prods = val * x  # each product rounded once, as in the oracle
    exact = math.fsum(prods.tolist())
    u = 2.0**-53
    gamma = n * u / (1 - n * u)
    assert abs(out[0] - exact) <= gamma * np.sum(np.abs(prods))


@pytest.mark.parametrize("rows,kind", [(64, "zipf"), (50, "band")])
def test_spmv_matches_dense_matvec(rows, kind):
    if kind == "zipf":
        rp, c, v = synth.csr_zipf(11, rows, 1.7)
    else:
        rp, c, v = synth.csr_band(11, rows, 9)
    rp, c, v = rp.numpy(), c.numpy(), v.numpy()
    x = synth.spmv_x(11, rows).numpy()
    D = sp.csr_matrix((v, c, rp), shape=(rows, rows)).toarray()
    ref = D @ x
    out = loops.spmv(rp, c, v, x)
    absum = np.abs(D) @ np.abs(x)
    assert np.all(np.abs(out - ref) <= 1e-13 * absum + 1e-300)


def test_spmv_rows_subset_matches_full():
    rp, c, v = [t.numpy() for t in synth.csr_zipf(12, 3000, 1.5)]
    x = synth.spmv_x(12, 3000).numpy()
    full = loops.spmv(rp, c, v, x)
    which = np.array([0, 5, 2999, 1234])
    y, a = loops.spmv_rows(rp, c, v, x, which)
    assert np.array_equal(y, full[which])
    assert np.all(a >= np.abs(y))


def test_csr_row_stats_closed_form():
    rowptr = np.array([0, 3, 3, 8, 9], dtype=np.int32)  # lengths 3, 0, 5, 1
    st = loops.csr_row_stats(rowptr)
    assert np.array_equal(st, np.array([4.0, 9.0, 2.25, 3.6875, 5.0]))


# ------------------------------------------------------------------ n-body
def test_nbody_two_body_closed_form_and_reaction():
    p = np.array([[0.25, 0.5, 0.5, 0.75], [0.75, 0.5, 0.5, 0.5]], dtype=np.float32)
    a = loops.nbody(p, 1e-2)
    d, eps = 0.5, 1e-2
    mag = lambda m: m * d / (d * d + eps * eps) ** 1.5  # noqa: E731
    assert a[0, 0] == pytest.approx(mag(0.5), rel=1e-15) and a[0, 0] > 0
    assert a[1, 0] == pytest.approx(-mag(0.75), rel=1e-15)
    assert a[0, 1] == 0.0 and a[0, 2] == 0.0
    # m1 a1 = -m2 a2 exactly here (same |d|, same r2)
    assert 0.75 * a[0, 0] == -0.5 * a[1, 0]


def test_nbody_cube_centre_feels_no_force():
    verts = [[x, y, z, 1.0] for x in (0.25, 0.75) for y in (0.25, 0.75) for z in (0.25, 0.75)]
    p = np.array(verts + [[0.5, 0.5, 0.5, 1.0]], dtype=np.float32)
    a = loops.nbody(p, 1e-2)
    assert np.max(np.abs(a[-1])) <= 1e-15


def test_nbody_momentum_conservation():
    p = synth.nbody_inputs(4, 300)
    a = loops.nbody(p, 1e-2)
    m = p[:, 3].astype(np.float64)
    tot = (m[:, None] * a).sum(axis=0)
    scale = np.sum(m[:, None] * np.abs(a))
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_nbody_mass_scaling_by_two_is_exact():
    p = synth.nbody_inputs(4, 200)
    q = p.copy()
    q[:, 3] *= 2
    assert np.array_equal(loops.nbody(q), 2.0 * loops.nbody(p))


def test_nbody_rows_and_batched_match_full():
    p = synth.nbody_inputs(4, 257)
    full = loops.nbody(p)
    which = np.array([0, 100, 256])
    assert np.array_equal(loops.nbody_rows(p, which), full[which])
    bodies, offs = synth.nbody_batch_inputs(40, count=3, nmin=50, nmax=120)
    acc = loops.nbody_batched(bodies, offs)
    for b in range(3):
        sl = slice(offs[b], offs[b + 1])
        assert np.array_equal(acc[sl], loops.nbody(bodies[sl]))
