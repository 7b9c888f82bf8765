"""Pins of the oracle's hash-occupancy statistics (the collision argument of
Sec. 4.2 and the "w/o dec" ablation): per level the distinct touched grid
vertices V, the distinct table entries E they occupy, and the vertices C
that share their entry with another touched vertex."""
from collections import Counter

import numpy as np
import pytest

import oracle


def _brute(g, x, y, z, t):
    """Vertex coordinates from the FP32 products directly, entries from the
    (separately pinned) corner indices, counted with Python sets."""
    n = len(x)
    idx, _ = oracle.corners(g, oracle.Points(x, y, z, t))
    out = []
    for l in range(g.L):
        res = [g.res_s[l]] * 3 + [g.res_t[l]]
        vmap = {}
        for i in range(n):
            p = [min(max(float(v[i]), 0.0), 1.0) for v in (x, y, z, t)]
            i0 = [min(int(np.floor(np.float32(p[d]) * np.float32(res[d]))), res[d] - 1) for d in range(4)]
            for b in range(16):
                v = tuple(i0[d] + ((b >> d) & 1) for d in range(4))
                e = int(idx[i, l, b])
                assert vmap.setdefault(v, e) == e      # a vertex always maps to one entry
        per_entry = Counter(vmap.values())
        out.append([len(vmap), len(per_entry), sum(c for c in per_entry.values() if c >= 2)])
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("cfg,n", [((4, 2, 8, 4, 64, 3, 20), 300), ((3, 2, 6, 2, 9, 2, 5), 500),
                                   ((2, 1, 16, 7, 7, 3, 3), 40)])
def test_counts_equal_brute_force(cfg, n):
    g = oracle.layout(*cfg)
    rng = np.random.default_rng(n)
    x, y, z, t = rng.random((4, n)).astype(np.float32)
    x[:3] = [0.0, 1.0, 0.5]
    assert np.array_equal(oracle.collision_stats(g, oracle.Points(x, y, z, t)), _brute(g, x, y, z, t))


def test_dense_levels_never_collide_and_one_point_touches_16_vertices():
    g = oracle.layout(3, 2, 24, 4, 16, 3, 9)
    assert all(g.dense[:3])
    rng = np.random.default_rng(21)
    x, y, z, t = rng.random((4, 2000)).astype(np.float32)
    s = oracle.collision_stats(g, oracle.Points(x, y, z, t))
    assert np.all(s[:, 0] == s[:, 1]) and np.all(s[:, 2] == 0)
    one = oracle.collision_stats(g, oracle.Points(x[:1], y[:1], z[:1], t[:1]))
    assert np.all(one[:, 0] == 16) and np.all(one[:, 1] == 16)


def test_pigeonhole_and_invariants_on_a_tiny_table():
    g = oracle.layout(4, 2, 4, 8, 256, 4, 64)     # T = 16 entries: every hashed level is crowded
    rng = np.random.default_rng(22)
    n = 3000
    x, y, z, t = rng.random((4, n)).astype(np.float32)
    s = oracle.collision_stats(g, oracle.Points(x, y, z, t))
    for l in range(g.L):
        V, E, C = s[l]
        assert E <= V <= 16 * n and C <= V and (C == 0) == (E == V)
        if not g.dense[l]:
            assert E <= 16 and C >= V - 16
    # more points touch at least as many vertices and entries, and collide at least as much
    s2 = oracle.collision_stats(g, oracle.Points(x[:1000], y[:1000], z[:1000], t[:1000]))
    assert np.all(s2 <= s)
