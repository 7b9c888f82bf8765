"""Shared helpers for the GPU parity tests: seeded inputs on both sides and
error metrics.  The CUDA side is reached only through the C-ABI binding."""
import numpy as np
import torch

import oracle


def oracle_grid(g):
    return oracle.layout(g.L, g.F, g.log2_T, g.nmin_s, g.nmax_s, g.nmin_t, g.nmax_t, g.primes)


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (d if d > 0 else 1.0))


def edge_coords(n, rng):
    """Coordinates with the degenerate cases first: 0, 1, NaN, out of range,
    exact vertices of power-of-two grids, then uniform values."""
    x, y, z, t = (rng.random(n).astype(np.float32) for _ in range(4))
    special = np.array([0.0, 1.0, np.nan, -0.5, 1.5, 0.5, 0.25, 1.0 - 2 ** -24, 2 ** -30, 0.125], dtype=np.float32)
    k = min(n, len(special))
    x[:k] = special[:k]
    y[:k] = special[::-1][:k]
    z[:k] = np.roll(special, 3)[:k]
    t[:k] = np.roll(special, 5)[:k]
    return x, y, z, t
