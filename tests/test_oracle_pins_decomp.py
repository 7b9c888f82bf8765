"""Pins of the oracle's decomposition step (Sec. 4.1, Eqs. 3-4): the 3-D
hash encoder G_3D, the MLPs phi_p / phi_l, and the top-k % threshold that
splits the Gaussians into static and dynamic ones."""
import math

import numpy as np
import pytest
import torch

import oracle


def test_layout3_endpoints_and_dense_rule():
    for L, a, b, lt in ((16, 16, 2048, 19), (8, 2, 512, 14), (4, 4, 32, 10)):
        g = oracle.layout3(L, 2, lt, a, b).as_dict()
        r = g["res_s"]
        assert r[0] == a and r[-1] == b and all(u <= v for u, v in zip(r, r[1:]))
        for l in range(L):
            verts = (r[l] + 1) ** 3
            assert g["dense"][l] == (verts <= 2 ** lt)
            assert g["size"][l] == (verts if verts <= 2 ** lt else 2 ** lt)
    # paper-shaped G_3D: 81^3 = 531,441 > 2^19, so levels 0-4 (N <= 58) are dense
    g = oracle.layout3(16, 2, 19, 16, 2048).as_dict()
    assert g["dense"][:6] == [True] * 5 + [False]


def test_cell3_dense_bijection_and_partition_of_unity():
    g = oracle.layout3(1, 1, 16, 3, 3)
    assert g.dense[0] and g.size[0] == 64
    seen = {}
    for cz in range(3):
        for cy in range(3):
            for cx in range(3):
                idx, w = oracle.cell3(g, 0, np.array([(cx + .5) / 3, (cy + .5) / 3, (cz + .5) / 3], np.float32))
                assert abs(w.sum() - 1) < 1e-12 and np.all(w >= 0)
                for b in range(8):
                    v = (cx + (b & 1), cy + ((b >> 1) & 1), cz + ((b >> 2) & 1))
                    assert seen.setdefault(v, int(idx[b])) == int(idx[b])
    assert sorted(seen.values()) == list(range(64))


def test_cell3_hash_is_bit_packing_with_power_of_two_primes():
    g = oracle.layout3(1, 1, 24, 300, 300, primes=(1, 1 << 9, 1 << 18, 0))
    assert not g.dense[0]  # 301^3 > 2^24
    rng = np.random.default_rng(3)
    for _ in range(100):
        p = rng.random(3).astype(np.float32)
        idx, _ = oracle.cell3(g, 0, p)
        i0 = [min(int(np.floor(np.float32(p[d]) * np.float32(300))), 299) for d in range(3)]
        for b in range(8):
            c = [i0[d] + ((b >> d) & 1) for d in range(3)]
            assert idx[b] == ((c[0] | (c[1] << 9) | (c[2] << 18)) & 0xFFFFFF)


def test_encode3_matches_scipy_trilinear():
    from scipy.interpolate import RegularGridInterpolator
    g = oracle.layout3(1, 1, 16, 8, 8)
    rng = np.random.default_rng(4)
    table = rng.uniform(-1, 1, size=(g.total, 1))
    grid = table[: 9 ** 3, 0].reshape(9, 9, 9)  # [z][y][x]
    ax = np.linspace(0, 1, 9)
    interp = RegularGridInterpolator((ax, ax, ax), grid)
    q = rng.integers(0, 1025, size=(3, 300)) / 1024.0
    f = oracle.encode3(g, *q.astype(np.float32), table)[:, 0]
    assert np.max(np.abs(f - interp(np.stack([q[2], q[1], q[0]], axis=1)))) < 1e-13


def test_decomposition_mlp_matches_torch():
    g = oracle.layout3(4, 2, 12, 4, 32)
    rng = np.random.default_rng(5)
    n, D, H = 200, 8, 16
    x, y, z = rng.random((3, n)).astype(np.float32)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    params = rng.uniform(-0.5, 0.5, H * D + H + 3 * H + 3)
    dp, norm = oracle.decomp_fwd(g, x, y, z, table, H, params)
    f = torch.tensor(oracle.encode3(g, x, y, z, table))
    p = torch.tensor(params)
    W1, b1 = p[:H * D].view(H, D), p[H * D:H * D + H]
    W2, b2 = p[H * D + H:H * D + H + 3 * H].view(3, H), p[-3:]
    ref = torch.nn.functional.linear(torch.relu(torch.nn.functional.linear(f, W1, b1)), W2, b2)
    assert np.max(np.abs(dp - ref.numpy().T)) < 1e-12
    assert np.max(np.abs(norm - torch.linalg.norm(ref, dim=1).numpy())) < 1e-12


@pytest.mark.parametrize("n,k", [(1000, 25.0), (999, 50.0), (10, 0.0), (10, 100.0), (7, 99.0), (1, 50.0)])
def test_topk_mask_invariants(n, k):
    rng = np.random.default_rng(n)
    v = rng.random(n)
    m = math.floor(k * n / 100)
    mask, tau = oracle.topk_mask(v, k)
    assert mask.sum() == min(m, n)               # distinct values: exactly m dynamic
    if 0 < mask.sum() < n:
        assert v[mask == 1].min() > tau >= v[mask == 0].max()


def test_topk_mask_ties_are_static():
    v = np.array([3.0, 2.0, 2.0, 2.0, 1.0, 0.5])
    mask, tau = oracle.topk_mask(v, 50)          # m = 3: tau = 2.0, only 3.0 is above it
    assert tau == 2.0 and list(mask) == [1, 0, 0, 0, 0, 0]


def test_linear_motion_speed_is_the_norm():
    """Eq. 4 makes |dp| the Gaussian's speed: the displacement between any
    two times, divided by their distance, is dp itself, and p(0) = p."""
    g = oracle.layout3(4, 2, 12, 4, 32)
    rng = np.random.default_rng(6)
    n, H = 300, 16
    x, y, z = rng.random((3, n)).astype(np.float32)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    params = rng.uniform(-0.5, 0.5, H * 8 + H + 3 * H + 3)
    dp, norm = oracle.decomp_fwd(g, x, y, z, table, H, params)
    t1 = rng.random(n).astype(np.float32)
    p0 = oracle.linear_motion(x, y, z, np.float32(0.0), dp)
    assert np.array_equal(p0, np.stack([x, y, z]).astype(np.float64))
    p1 = oracle.linear_motion(x, y, z, t1, dp)
    p2 = oracle.linear_motion(x, y, z, np.float32(1.0), dp)
    speed = np.linalg.norm(p2 - p0, axis=0)
    assert np.max(np.abs(speed - norm)) < 1e-12
    assert np.max(np.abs((p1 - p0) - t1.astype(np.float64) * dp)) < 1e-12
    # second difference of a linear trajectory vanishes
    pm = oracle.linear_motion(x, y, z, np.float32(0.5), dp)
    assert np.max(np.abs(p2 - 2 * pm + p0)) < 1e-12


def test_static_loss_special_cases():
    rng = np.random.default_rng(7)
    n = 1000
    mask = (rng.random(n) < 0.5).astype(np.uint8)
    assert abs(oracle.static_loss(np.full(n, 0.75), mask) - 0.75) < 1e-15       # constant speed
    v = rng.random(n)
    assert abs(oracle.static_loss(v, np.zeros(n, np.uint8)) - v.mean()) < 1e-12  # nothing dynamic
    assert oracle.static_loss(v, np.ones(n, np.uint8)) == 0.0                   # nothing static
    for k in (10.0, 50.0, 90.0):                                                 # static speeds lie below tau
        m, tau = oracle.topk_mask(v, k)
        ls = oracle.static_loss(v, m)
        assert v[m == 0].min() <= ls <= tau
        assert abs(ls * (m == 0).sum() + v[m == 1].sum() - v.sum()) < 1e-9


def _decomp_loss(g, x, y, z, table, H, params, d_dp, mask, lam):
    dp, norm = oracle.decomp_fwd(g, x, y, z, table, H, params)
    return float(np.sum(d_dp * dp)) + lam * oracle.static_loss(norm, mask)


def test_decomposition_backward_matches_finite_differences():
    g = oracle.layout3(4, 2, 12, 4, 32)
    rng = np.random.default_rng(8)
    n, D, H = 150, 8, 16
    x, y, z = rng.random((3, n)).astype(np.float32)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    params = rng.uniform(-0.5, 0.5, H * D + H + 3 * H + 3)
    d_dp = rng.standard_normal((3, n))
    _, norm = oracle.decomp_fwd(g, x, y, z, table, H, params)
    mask, _ = oracle.topk_mask(norm, 50.0)
    lam = 0.7
    tg, pg = oracle.decomp_bwd(g, x, y, z, table, H, params, d_dp, mask, lam)
    h = 1e-6
    for j in rng.choice(len(params), size=25, replace=False):
        pp, pm = params.copy(), params.copy()
        pp[j] += h
        pm[j] -= h
        fd = (_decomp_loss(g, x, y, z, table, H, pp, d_dp, mask, lam) -
              _decomp_loss(g, x, y, z, table, H, pm, d_dp, mask, lam)) / (2 * h)
        assert abs(fd - pg[j]) <= 1e-6 * max(1.0, abs(fd)), (j, fd, pg[j])
    touched = np.flatnonzero(np.abs(tg).sum(1) > 0)
    for e in rng.choice(touched, size=20, replace=False):
        for f in range(2):
            tp, tm = table.copy(), table.copy()
            tp[e, f] += h
            tm[e, f] -= h
            fd = (_decomp_loss(g, x, y, z, tp, H, params, d_dp, mask, lam) -
                  _decomp_loss(g, x, y, z, tm, H, params, d_dp, mask, lam)) / (2 * h)
            assert abs(fd - tg[e, f]) <= 1e-6 * max(1.0, abs(fd)), (e, f, fd, tg[e, f])
    # the two terms add up
    tg1, pg1 = oracle.decomp_bwd(g, x, y, z, table, H, params, d_dp, None, 0.0)
    tg2, pg2 = oracle.decomp_bwd(g, x, y, z, table, H, params, None, mask, lam)
    assert np.max(np.abs(tg1 + tg2 - tg)) < 1e-12 and np.max(np.abs(pg1 + pg2 - pg)) < 1e-12
