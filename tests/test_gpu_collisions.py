"""GPU parity of the per-level table occupancy (touched vertices V, occupied
entries E, colliding vertices C): exact integer counts against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import oracle_grid, to_dev

pytestmark = pytest.mark.gpu


def _gpu_stats(dashlib, lay, x, y, z, t, idx=None, n=None, n_dev=None):
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), idx=None if idx is None else to_dev(idx), n=n,
                         n_dev=n_dev)
    return dashlib.dash_hash4d_collision_stats(lay, pts).cpu().numpy()


@pytest.mark.parametrize("grid,n", [(synth.TINY_GRID, 20_000), (synth.PAPER_GRID, 30_000), (synth.PAPER_GRID, 1),
                                    (synth.PAPER_GRID, 0)])
def test_collision_stats_exact(dashlib, grid, n):
    rng = np.random.default_rng(91 + n)
    x, y, z, t = synth.scene_coords(rng, max(n, 1))
    x, y, z, t = (a[:n] for a in (x, y, z, t))
    got = _gpu_stats(dashlib, dashlib.layout_from(grid), x, y, z, t, n=n)
    ref = oracle.collision_stats(oracle_grid(grid), oracle.Points(x, y, z, t, n=n))
    assert np.array_equal(got, ref)


def test_collision_stats_index_list_device_count_and_broadcast_t(dashlib):
    grid = synth.PAPER_GRID
    rng = np.random.default_rng(92)
    n_all = 40_000
    x, y, z, _ = synth.scene_coords(rng, n_all)
    t = np.array([0.3], np.float32)
    idx = np.flatnonzero(synth.bernoulli_mask(rng, n_all)).astype(np.int32)
    live = len(idx) - 1234
    cnt = torch.tensor([live], dtype=torch.int64, device="cuda")
    got = _gpu_stats(dashlib, dashlib.layout_from(grid), x, y, z, t, idx=idx, n=len(idx), n_dev=cnt)
    ref = oracle.collision_stats(oracle_grid(grid), oracle.Points(x, y, z, t, idx=idx[:live], t_stride=0))
    assert np.array_equal(got, ref)


def test_collision_stats_crowded_and_dense_tables(dashlib):
    rng = np.random.default_rng(93)
    x, y, z, t = rng.random((4, 5000)).astype(np.float32)
    crowded = dashlib.dash_hash4d_layout(4, 2, 4, 8, 256, 4, 64)     # 16 entries per hashed level
    g = oracle.layout(4, 2, 4, 8, 256, 4, 64)
    assert np.array_equal(_gpu_stats(dashlib, crowded, x, y, z, t), oracle.collision_stats(g, oracle.Points(x, y, z, t)))
    dense = dashlib.dash_hash4d_layout(3, 2, 24, 4, 16, 3, 9)
    s = _gpu_stats(dashlib, dense, x, y, z, t)
    assert np.all(s[:, 0] == s[:, 1]) and np.all(s[:, 2] == 0)
    assert np.array_equal(s, oracle.collision_stats(oracle.layout(3, 2, 24, 4, 16, 3, 9), oracle.Points(x, y, z, t)))


def test_compaction_reduces_collisions(dashlib):
    """The decomposition's point: the dynamic half occupies fewer entries and
    collides less than all Gaussians (600k-Gaussian scene shape)."""
    grid = synth.PAPER_GRID
    rng = np.random.default_rng(94)
    n_all = 600_000
    x, y, z, t = synth.scene_coords(rng, n_all)
    idx = np.flatnonzero(synth.bernoulli_mask(rng, n_all)).astype(np.int32)
    lay = dashlib.layout_from(grid)
    s_all = _gpu_stats(dashlib, lay, x, y, z, t)
    s_dyn = _gpu_stats(dashlib, lay, x, y, z, t, idx=idx)
    hashed = [l for l in range(grid.L) if not oracle_grid(grid).dense[l]]
    assert np.all(s_dyn[hashed, 2] <= s_all[hashed, 2]) and s_dyn[hashed, 2].sum() < s_all[hashed, 2].sum()
