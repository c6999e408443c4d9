"""Seeded input generators (no method arithmetic; see package docstring).

Distributions follow the workload descriptions of the build:

* daxpy: x, y ~ U[-1, 1] in float64, a = 1.5.
* 7-point Jacobi: N^3 float64 unknowns ~ U[-1, 1], stored k-major then j then
  i (i fastest); the zero Dirichlet ghosts outside the cube are implicit.
* CSR SpMV: square matrices; row lengths either truncated Zipf(s) on
  [1, min(4096, cols)] or a band of odd total width b; values ~ N(0, 1),
  x ~ U[-1, 1].  Zipf rows take their k distinct columns by stratified
  sampling: [0, cols) is cut into k integer strata and one uniform column is
  drawn in each, which yields distinct, sorted, uniformly spread columns.
* n-body: positions ~ U[0, 1]^3, masses ~ U[0.5, 1], float32, packed as
  (x, y, z, m) per body.
"""
from __future__ import annotations

import math

import numpy as np

DAXPY_A = 1.5
NBODY_EPS = 1e-2


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- daxpy
def daxpy_inputs(seed: int, n: int):
    """Return (a, x, y): float64 vectors of length n, U[-1, 1]; a = 1.5."""
    r = _rng(seed)
    x = r.uniform(-1.0, 1.0, n)
    y = r.uniform(-1.0, 1.0, n)
    return DAXPY_A, x, y


# ---------------------------------------------------------------- Jacobi
def grid_inputs(seed: int, N: int) -> np.ndarray:
    """Return an (N, N, N) float64 grid, U[-1, 1], indexed [k, j, i]."""
    return _rng(seed).uniform(-1.0, 1.0, (N, N, N))


def linear_field(N: int, alpha: int, beta: int, gamma: int) -> np.ndarray:
    """u[k, j, i] = alpha*i + beta*j + gamma*k with 1-based i, j, k (float64)."""
    i = np.arange(1, N + 1, dtype=np.float64)
    return (gamma * i[:, None, None] + beta * i[None, :, None] + alpha * i[None, None, :])


def sine_mode(N: int) -> np.ndarray:
    """u[k, j, i] = sin(pi i h) sin(pi j h) sin(pi k h), h = 1/(N+1), 1-based."""
    h = 1.0 / (N + 1)
    s = np.sin(np.pi * h * np.arange(1, N + 1, dtype=np.float64))
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


# ---------------------------------------------------------------- n-body
def nbody_inputs(seed: int, N: int) -> np.ndarray:
    """Return float32 (N, 4): columns x, y, z ~ U[0,1], m ~ U[0.5, 1]."""
    r = _rng(seed)
    out = np.empty((N, 4), dtype=np.float32)
    out[:, :3] = r.uniform(0.0, 1.0, (N, 3))
    out[:, 3] = r.uniform(0.5, 1.0, N)
    return out


def nbody_batch_sizes(seed: int, count: int = 64, nmin: int = 1024, nmax: int = 65536) -> np.ndarray:
    """Instance sizes, log-uniform on [nmin, nmax], not rounded to tiles."""
    r = _rng(seed)
    u = r.uniform(math.log(nmin), math.log(nmax), count)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), nmin, nmax)


def nbody_batch_inputs(seed: int, count: int = 64, nmin: int = 1024, nmax: int = 65536):
    """Return (bodies float32 (sum N_i, 4), offsets int32 (count+1,))."""
    sizes = nbody_batch_sizes(seed, count, nmin, nmax)
    offs = np.zeros(count + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    bodies = np.concatenate([nbody_inputs((seed, b), int(n)) for b, n in enumerate(sizes)])
    return bodies, offs.astype(np.int32)


# ---------------------------------------------------------------- CSR
def _torch():
    import torch

    return torch


def zipf_row_lengths(seed, rows: int, s: float, cap: int = 4096, cols: int | None = None,
                     device: str = "cpu"):
    """Row lengths k ~ truncated Zipf: P(k) proportional to k^-s, k in [1, min(cap, cols)]."""
    torch = _torch()
    cols = rows if cols is None else cols
    K = min(cap, cols)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 11)
    k = torch.arange(1, K + 1, dtype=torch.float64, device=device)
    w = k.pow(-s)
    cdf = torch.cumsum(w, 0) / w.sum()
    u = torch.rand(rows, generator=g, dtype=torch.float64, device=device)
    lens = torch.searchsorted(cdf, u, right=True) + 1
    return lens.clamp_(1, K)


def csr_from_lengths(lengths, cols: int, kind: str, band: int, g, device):
    """Column indices for given row lengths (see module docstring)."""
    torch = _torch()
    rows = lengths.numel()
    rowptr = torch.zeros(rows + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(lengths, 0)
    nnz = int(rowptr[-1].item())
    row_of = torch.repeat_interleave(torch.arange(rows, device=device), lengths)
    j = torch.arange(nnz, device=device) - rowptr[:-1][row_of]
    if kind == "zipf":
        k = lengths[row_of]
        lo = (j * cols) // k
        hi = ((j + 1) * cols) // k
        u = torch.rand(nnz, generator=g, dtype=torch.float64, device=device)
        col = lo + torch.floor(u * (hi - lo).to(torch.float64)).to(torch.int64)
        col = torch.minimum(col, hi - 1)
    else:
        h = (band - 1) // 2
        col = torch.clamp(row_of - h, min=0) + j
    del row_of, j
    return rowptr, col


def csr_zipf(seed: int, rows: int, s: float, cap: int = 4096, device: str = "cpu"):
    """Square CSR with truncated-Zipf row lengths; returns torch tensors
    (rowptr int32 [rows+1], col int32 [nnz], val float64 [nnz])."""
    torch = _torch()
    lens = zipf_row_lengths(seed, rows, s, cap, rows, device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 17)
    rowptr, col = csr_from_lengths(lens, rows, "zipf", 0, g, device)
    val = torch.randn(col.numel(), generator=g, dtype=torch.float64, device=device)
    return rowptr.to(torch.int32), col.to(torch.int32), val


def csr_band(seed: int, rows: int, band: int, device: str = "cpu"):
    """Square banded CSR of odd total width ``band`` (clipped at the edges)."""
    torch = _torch()
    if band % 2 != 1 or band < 1:
        raise ValueError("band width must be odd and positive")
    h = (band - 1) // 2
    i = torch.arange(rows, device=device)
    lens = torch.minimum(i + h, torch.full_like(i, rows - 1)) - torch.clamp(i - h, min=0) + 1
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 29)
    rowptr, col = csr_from_lengths(lens, rows, "band", band, g, device)
    val = torch.randn(col.numel(), generator=g, dtype=torch.float64, device=device)
    return rowptr.to(torch.int32), col.to(torch.int32), val


def spmv_matrix_params(seed: int, rows_min: float = 1e4, rows_max: float = 1e7):
    """Draw one matrix description: rows log-uniform, 50 % Zipf(s ~ U[1.5, 2.5])
    and 50 % band(b ~ odd U[7, 129])."""
    r = _rng(seed)
    rows = int(math.floor(math.exp(r.uniform(math.log(rows_min), math.log(rows_max)))))
    if r.uniform() < 0.5:
        return {"rows": rows, "kind": "zipf", "s": float(r.uniform(1.5, 2.5)), "band": 0}
    b = 7 + 2 * int(r.integers(0, 62))  # odd in [7, 129]
    return {"rows": rows, "kind": "band", "s": 0.0, "band": b}


def spmv_matrix(seed: int, params: dict | None = None, device: str = "cpu"):
    """Build the matrix of ``spmv_matrix_params(seed)`` (or of ``params``)."""
    p = spmv_matrix_params(seed) if params is None else params
    if p["kind"] == "zipf":
        return csr_zipf(seed, p["rows"], p["s"], device=device)
    return csr_band(seed, p["rows"], p["band"], device=device)


def spmv_x(seed: int, cols: int, device: str = "cpu"):
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 104729 + 3)
    return torch.rand(cols, generator=g, dtype=torch.float64, device=device) * 2.0 - 1.0


# ---------------------------------------------------------------- mixed stream
LOOP_DAXPY, LOOP_JACOBI, LOOP_SPMV, LOOP_NBODY = 0, 1, 2, 3


def mixed_stream(seed: int, ncalls: int, pool: int = 32):
    """Per call: loop id ~ U{0..3}; size log-uniform over the loop's range
    (daxpy n in [2^10, 2^24], Jacobi N in [32, 512], SpMV matrix index in a
    pool of ``pool`` matrices, n-body N in [1k, 256k])."""
    r = _rng(seed)
    loop = r.integers(0, 4, ncalls)
    u = r.uniform(0.0, 1.0, ncalls)
    size = np.zeros(ncalls, dtype=np.int64)
    lo = np.array([2.0 ** 10, 32.0, 0.0, 1024.0])
    hi = np.array([2.0 ** 24, 512.0, 1.0, 262144.0])
    for L in (LOOP_DAXPY, LOOP_JACOBI, LOOP_NBODY):
        m = loop == L
        size[m] = np.floor(np.exp(np.log(lo[L]) + u[m] * (np.log(hi[L]) - np.log(lo[L]))))
    m = loop == LOOP_SPMV
    size[m] = np.minimum((u[m] * pool).astype(np.int64), pool - 1)
    return loop.astype(np.int32), size
