"""Helpers shared by the GPU tests (CPU-side only: no method arithmetic)."""
import numpy as np
import torch


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def cone_cube(N, s, p):
    """Cube origin (per axis) of side L = 2s+1 inside [0, N) whose artificial
    faces are more than s cells from point p, so that s sweeps on the cube give
    the exact value at p (boundary influence moves one cell per sweep)."""
    L = min(N, 2 * s + 1)
    return [min(max(c - s, 0), N - L) for c in p], L
