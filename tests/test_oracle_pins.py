"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics,
not by the oracle itself (arXiv 2507.19141, Sec. 4.2-4.3, Eqs. 7-11).

Each check is chosen so that a plausible slip in the oracle (a dropped level
exponent, a swapped axis, a wrong corner bit, a wrong sign in the smoothness
gradient, a transposed weight) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [int(x) for x in v]
    return out


# ------------------------------------------------------------------ Eq. 7 --

@pytest.mark.parametrize("L,nmin,nmax", [(16, 16, 2048), (16, 8, 150), (4, 16, 128),
                                          (4, 8, 32), (8, 2, 512), (3, 5, 7), (12, 16, 4096)])
def test_layout_endpoints_and_monotone(L, nmin, nmax):
    g = oracle.layout(L, 2, 19, nmin, nmax, nmin, nmax)
    r = list(g.res_s[:L])
    assert r[0] == nmin and r[-1] == nmax
    assert all(a <= b for a, b in zip(r, r[1:]))
    # each level within one unit of the real-valued progression N_min * b^l
    b = math.exp((math.log(nmax) - math.log(nmin)) / (L - 1))
    for l, n in enumerate(r):
        assert abs(n - nmin * b ** l) < 1.0 + 1e-9


def test_layout_single_level():
    g = oracle.layout(1, 2, 10, 12, 12, 3, 3)
    assert g.res_s[0] == 12 and g.res_t[0] == 3


def test_layout_paper_shape_golden():
    gold = _golden("layout_paper_shape.txt")
    g = oracle.layout(16, 2, 19, 16, 2048, 8, 150).as_dict()
    assert g["res_s"] == gold["res_s"]
    assert g["res_t"] == gold["res_t"]
    assert [int(d) for d in g["dense"]] == gold["dense"]
    assert g["size"] == gold["size"]
    assert sum(g["size"]) == gold["used_total"][0]
    # level starts rounded up to a multiple of 8 entries, never overlapping
    for l in range(16):
        assert g["offset"][l] % 8 == 0
        assert g["offset"][l + 1] - g["offset"][l] >= g["size"][l]
        assert g["offset"][l + 1] - g["offset"][l] - g["size"][l] < 8
    t = oracle.layout(4, 2, 14, 16, 128, 8, 32).as_dict()
    assert t["res_s"] == gold["tiny_res_s"] and t["res_t"] == gold["tiny_res_t"]
    assert [int(d) for d in t["dense"]] == gold["tiny_dense"]
    assert sum(t["size"]) == gold["tiny_used_total"][0]


def test_layout_rejects_bad_config():
    with pytest.raises(ValueError):
        oracle.layout(0, 2, 19, 16, 2048, 8, 150)
    with pytest.raises(ValueError):
        oracle.layout(4, 2, 19, 16, 8, 8, 150)


# ------------------------------------------------------ mask compaction --

@pytest.mark.parametrize("n,p", [(0, 0.5), (1, 1.0), (1000, 0.0), (1000, 1.0), (100_003, 0.5),
                                  (77_777, 0.01)])
def test_compaction_is_flatnonzero(n, p):
    rng = np.random.default_rng(n)
    mask = (rng.random(n) < p).astype(np.uint8)
    mask[mask == 1] = rng.integers(1, 256, size=int(mask.sum()), dtype=np.uint8)  # any nonzero byte
    idx, cnt = oracle.compact(mask)
    ref = np.flatnonzero(mask)
    assert cnt == len(ref)
    assert np.array_equal(idx, ref.astype(np.int32))


# ------------------------------------------------------------------ Eq. 8 --

def test_hash_reduces_to_bit_packing_with_power_of_two_primes():
    """With primes (1, 2^8, 2^16, 2^24) and coordinates below 2^8 the XOR of
    Eq. 8 acts on disjoint bit fields, so the hash must equal the packed
    integer cx | cy<<8 | cz<<16 | ct<<24, masked to T-1 = 2^24-1."""
    primes = (1, 1 << 8, 1 << 16, 1 << 24)
    g = oracle.layout(1, 1, 24, 128, 128, 32, 32, primes=primes)
    assert not g.dense[0]  # 129^3 * 33 > 2^24
    rng = np.random.default_rng(5)
    for _ in range(200):
        p = rng.random(4).astype(np.float32)
        idx, w = oracle.cell(g, 0, p)
        i0 = [min(int(np.floor(np.float32(p[d]) * np.float32(128 if d < 3 else 32))),
                  (128 if d < 3 else 32) - 1) for d in range(4)]
        for b in range(16):
            c = [i0[d] + ((b >> d) & 1) for d in range(4)]
            assert idx[b] == ((c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24)) & 0xFFFFFF)


def test_hash_big_integer_brute_force():
    """Eq. 8 evaluated with Python big integers for random cells of hashed
    levels at the paper-shaped configuration."""
    g = oracle.layout(16, 2, 19, 16, 2048, 8, 150)
    rng = np.random.default_rng(6)
    pr = [1, 2654435761, 805459861, 3674653429]
    for _ in range(100):
        l = int(rng.integers(3, 16))
        p = rng.random(4).astype(np.float32)
        idx, _ = oracle.cell(g, l, p)
        res = [g.res_s[l]] * 3 + [g.res_t[l]]
        i0 = [min(int(np.floor(np.float32(p[d]) * np.float32(res[d]))), res[d] - 1) for d in range(4)]
        for b in range(16):
            h = 0
            for d in range(4):
                h ^= ((i0[d] + ((b >> d) & 1)) * pr[d]) % (1 << 32)
            assert idx[b] == h % (1 << 19)


def test_dense_level_is_bijection_onto_table():
    """A dense level indexes its (N_s+1)^3 (N_t+1) vertices one-to-one onto
    [0, T_l): visit every cell, map each corner's vertex to its index."""
    g = oracle.layout(1, 1, 16, 3, 3, 2, 2)
    assert g.dense[0] and g.size[0] == 4 ** 3 * 3
    seen = {}
    for ct in range(2):
        for cz in range(3):
            for cy in range(3):
                for cx in range(3):
                    p = np.array([(cx + .5) / 3, (cy + .5) / 3, (cz + .5) / 3, (ct + .5) / 2], np.float32)
                    idx, _ = oracle.cell(g, 0, p)
                    for b in range(16):
                        v = (cx + (b & 1), cy + ((b >> 1) & 1), cz + ((b >> 2) & 1), ct + ((b >> 3) & 1))
                        assert seen.setdefault(v, int(idx[b])) == int(idx[b])
    assert len(seen) == g.size[0]
    assert sorted(seen.values()) == list(range(g.size[0]))


# ------------------------------------------------------------------ Eq. 9 --

@pytest.mark.parametrize("cfg", [synth.TINY_GRID, synth.PAPER_GRID])
def test_weights_partition_of_unity(cfg):
    g = oracle.layout(cfg.L, cfg.F, cfg.log2_T, cfg.nmin_s, cfg.nmax_s, cfg.nmin_t, cfg.nmax_t)
    rng = np.random.default_rng(7)
    x, y, z, t = synth.uniform_coords(rng, 500)
    x[:4] = [0.0, 1.0, np.nan, -3.0]  # edges, NaN and out-of-range coordinates
    y[:4] = [1.0, 0.0, 2.0, 0.5]
    _, w = oracle.corners(g, oracle.Points(x, y, z, t))
    assert np.all(w >= 0.0) and np.all(w <= 1.0)
    assert np.max(np.abs(w.sum(axis=2) - 1.0)) < 1e-12


def test_vertex_reproduction_exact():
    """At a grid vertex the encoder returns that vertex's table entry exactly
    (power-of-two resolutions make x * N exact)."""
    g = oracle.layout(2, 2, 20, 8, 16, 4, 8)
    assert g.dense[0]
    rng = np.random.default_rng(8)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    # vertices of the coarse level (8, 4); each is also a vertex of the fine (16, 8) one
    k = rng.integers(0, 9, size=(3, 64))
    kt = rng.integers(0, 5, size=64)
    x, y, z = (k / 8.0).astype(np.float32)
    t = (kt / 4.0).astype(np.float32)
    pts = oracle.Points(x, y, z, t)
    f = oracle.encode(g, pts, table)
    idx, w = oracle.corners(g, pts)
    for i in range(64):
        for l in range(2):
            b = int(np.argmax(w[i, l]))
            assert w[i, l, b] == 1.0
            e = g.offset[l] + idx[i, l, b]
            assert np.array_equal(f[i, 2 * l:2 * l + 2], table[e])


def test_multilinear_matches_scipy_regular_grid():
    """A dense level is textbook 4-D multilinear interpolation on a regular
    grid: compare against scipy's RegularGridInterpolator."""
    from scipy.interpolate import RegularGridInterpolator
    g = oracle.layout(1, 1, 20, 8, 8, 4, 4)
    assert g.dense[0]
    R, Rt = 9, 5
    rng = np.random.default_rng(9)
    table = rng.uniform(-1, 1, size=(g.total, 1))
    grid = table[: R * R * R * Rt, 0].reshape(Rt, R, R, R)  # [t][z][y][x], x fastest
    axes = (np.linspace(0, 1, Rt), np.linspace(0, 1, R), np.linspace(0, 1, R), np.linspace(0, 1, R))
    interp = RegularGridInterpolator(axes, grid, method="linear")
    # coordinates on a 1/1024 lattice: x * N is exact in FP32 and in double
    q = rng.integers(0, 1025, size=(4, 400)) / 1024.0
    x, y, z, t = q.astype(np.float32)
    f = oracle.encode(g, oracle.Points(x, y, z, t), table)[:, 0]
    ref = interp(np.stack([q[3], q[2], q[1], q[0]], axis=1))
    assert np.max(np.abs(f - ref)) < 1e-13


def test_trilinear_special_case_at_time_vertex():
    """With t on a temporal vertex the 4-D cell degenerates to a 3-D one:
    the result is trilinear interpolation of that time slice."""
    from scipy.interpolate import RegularGridInterpolator
    g = oracle.layout(1, 1, 20, 8, 8, 4, 4)
    R, Rt = 9, 5
    rng = np.random.default_rng(10)
    table = rng.uniform(-1, 1, size=(g.total, 1))
    grid = table[: R * R * R * Rt, 0].reshape(Rt, R, R, R)
    kt = 3
    ax = np.linspace(0, 1, R)
    interp = RegularGridInterpolator((ax, ax, ax), grid[kt], method="linear")
    q = rng.integers(0, 1025, size=(3, 200)) / 1024.0
    x, y, z = q.astype(np.float32)
    t = np.full(200, kt / 4.0, dtype=np.float32)
    f = oracle.encode(g, oracle.Points(x, y, z, t), table)[:, 0]
    assert np.max(np.abs(f - interp(np.stack([q[2], q[1], q[0]], axis=1)))) < 1e-13


def test_affine_reproduction_two_levels():
    """F=1 tables holding an affine function of the vertex coordinates give
    that affine function at any point (multilinear interpolation is exact on
    affine functions), level by level."""
    g = oracle.layout(2, 1, 22, 5, 11, 3, 7)
    assert g.dense[0] and g.dense[1]
    a = [np.array([0.3, -1.2, 0.7, 2.0]), np.array([-0.4, 0.9, 1.5, -0.6])]
    c = [0.25, -1.0]
    table = np.zeros((g.total, 1))
    for l in range(2):
        Ns, Nt = g.res_s[l], g.res_t[l]
        R = Ns + 1
        for ct in range(Nt + 1):
            for cz in range(R):
                for cy in range(R):
                    for cx in range(R):
                        e = g.offset[l] + cx + R * (cy + R * (cz + R * ct))
                        v = np.array([cx / Ns, cy / Ns, cz / Ns, ct / Nt])
                        table[e, 0] = a[l] @ v + c[l]
    rng = np.random.default_rng(11)
    x, y, z, t = synth.uniform_coords(rng, 300)
    f = oracle.encode(g, oracle.Points(x, y, z, t), table)
    P = np.stack([x, y, z, t], axis=1).astype(np.float64)
    for l in range(2):
        # the encoder sees fl32(x * N) / N, within 2^-24 relative of x
        assert np.max(np.abs(f[:, l] - (P @ a[l] + c[l]))) < 1e-6


def test_encoder_gradient_is_interpolation_weights():
    """The encoder is linear in its tables: with a one-hot upstream gradient
    the table gradient holds exactly the 16 weights at the 16 corners."""
    g = oracle.layout(2, 2, 6, 4, 9, 2, 5)
    rng = np.random.default_rng(12)
    x, y, z, t = synth.uniform_coords(rng, 40)
    pts = oracle.Points(x, y, z, t)
    idx, w = oracle.corners(g, pts)
    for i in range(0, 40, 7):
        for l in range(2):
            for f in range(2):
                d = np.zeros((40, 4))
                d[i, 2 * l + f] = 1.0
                tg = oracle.encode_bwd(g, pts, d)
                ref = np.zeros((g.total, 2))
                for b in range(16):
                    ref[g.offset[l] + idx[i, l, b], f] += w[i, l, b]
                assert np.max(np.abs(tg - ref)) < 1e-15


def test_encoder_gradient_finite_difference():
    g = oracle.layout(2, 2, 5, 3, 6, 2, 4)
    rng = np.random.default_rng(13)
    x, y, z, t = synth.uniform_coords(rng, 30)
    pts = oracle.Points(x, y, z, t)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    dfeat = rng.standard_normal((30, 4))
    tg = oracle.encode_bwd(g, pts, dfeat)
    h = 1e-3  # exact for a linear map up to rounding
    for e in rng.choice(g.total, size=20, replace=False):
        for f in range(2):
            tp = table.copy(); tp[e, f] += h
            tm = table.copy(); tm[e, f] -= h
            fd = ((oracle.encode(g, pts, tp) - oracle.encode(g, pts, tm)) * dfeat).sum() / (2 * h)
            assert abs(fd - tg[e, f]) < 1e-9


# ------------------------------------------------------- decoder (MLP) --

def _torch_mlp(params, D, H, O):
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    o = 0
    parts = []
    for shape in ((H, D), (H,), (H, H), (H,), (O, H), (O,)):
        k = int(np.prod(shape))
        parts.append(p[o:o + k].view(*shape))
        o += k
    return p, parts


@pytest.mark.parametrize("D,H,O", [(8, 64, 10), (32, 64, 10), (5, 7, 3)])
def test_mlp_forward_and_backward_match_torch_autograd(D, H, O):
    rng = np.random.default_rng(D * 100 + H)
    params = rng.uniform(-0.5, 0.5, oracle.mlp_param_count(D, H, O))
    feat = rng.uniform(-1, 1, (50, D))
    dout = rng.standard_normal((O, 50))
    out = oracle.mlp_fwd(D, H, O, params, feat)
    dfeat, pg = oracle.mlp_bwd(D, H, O, params, feat, dout)
    p, (W1, b1, W2, b2, W3, b3) = _torch_mlp(params, D, H, O)
    f = torch.tensor(feat, requires_grad=True)
    ref = torch.nn.functional.linear(
        torch.relu(torch.nn.functional.linear(torch.relu(torch.nn.functional.linear(f, W1, b1)), W2, b2)),
        W3, b3)
    assert np.max(np.abs(out - ref.detach().numpy().T)) < 1e-12
    (ref * torch.tensor(dout.T)).sum().backward()
    assert np.max(np.abs(pg - p.grad.numpy())) < 1e-11
    assert np.max(np.abs(dfeat - f.grad.numpy())) < 1e-11


def test_deform_forward_composes_encoder_mlp_and_eq10():
    cfg = synth.TINY_GRID
    g = oracle.layout(cfg.L, cfg.F, cfg.log2_T, cfg.nmin_s, cfg.nmax_s, cfg.nmin_t, cfg.nmax_t)
    rng = np.random.default_rng(14)
    n_all = 300
    x, y, z, t = synth.uniform_coords(rng, n_all)
    mask = synth.bernoulli_mask(rng, n_all)
    idx, n = oracle.compact(mask)
    pts = oracle.Points(x, y, z, t, idx=idx)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    params = synth.mlp_params(rng, synth.TINY_MLP).astype(np.float64)
    attrs = synth.gaussian_attrs(rng, n_all)
    delta, out = oracle.deform_fwd(g, pts, table, 64, 10, params, attrs_in=attrs)
    feat = oracle.encode(g, pts, table)
    assert np.max(np.abs(delta - oracle.mlp_fwd(8, 64, 10, params, feat))) < 1e-13
    assert np.array_equal(out[:, mask == 0], attrs[:, mask == 0].astype(np.float64))
    assert np.max(np.abs(out[:, idx] - attrs[:, idx] - delta)) < 1e-13


# ------------------------------------------------- Eq. 11 smoothness --

def test_smoothness_closed_form_on_affine_tables():
    """On dense levels holding affine functions a_l . v + c_l, the feature
    difference to the perturbed point is -a_l . e exactly, so
    L_r = sum_e sum_l (a_l . e)^2 for interior points."""
    g = oracle.layout(2, 1, 22, 5, 11, 3, 7)
    a = [np.array([0.3, -1.2, 0.7, 2.0]), np.array([-0.4, 0.9, 1.5, -0.6])]
    table = np.zeros((g.total, 1))
    for l in range(2):
        Ns, Nt = g.res_s[l], g.res_t[l]
        R = Ns + 1
        ii = np.arange(R)
        for ct in range(Nt + 1):
            for cz in range(R):
                for cy in range(R):
                    e = g.offset[l] + ii + R * (cy + R * (cz + R * ct))
                    table[e, 0] = a[l] @ np.array([0, cy / Ns, cz / Ns, ct / Nt]) + a[l][0] * ii / Ns
    rng = np.random.default_rng(15)
    q = rng.integers(64, 960, size=(4, 100)) / 1024.0  # interior, exact in FP32
    x, y, z, t = q.astype(np.float32)
    eps_s = (1 / 2048, 1 / 2048, 1 / 2048)
    eps_t = 1 / 256
    lam = 0.7
    L = oracle.smooth_loss(g, oracle.Points(x, y, z, t), table, lam, eps_s, eps_t)
    es = np.array([1 / 2048, 1 / 2048, 1 / 2048, 0.0])
    et = np.array([0, 0, 0, 1 / 256])
    ref = lam * sum((a[l] @ es) ** 2 + (a[l] @ et) ** 2 for l in range(2))
    assert abs(L - ref) < 1e-6 * ref


def test_full_backward_finite_difference_with_smoothness():
    """dLoss/d(table) and dLoss/d(params) of Loss = sum(ddelta * delta) +
    lambda_r * L_r against central finite differences of the forward."""
    g = oracle.layout(2, 2, 6, 3, 7, 2, 5)
    rng = np.random.default_rng(16)
    n = 24
    x, y, z, t = synth.uniform_coords(rng, n)
    pts = oracle.Points(x, y, z, t)
    D, H, O = 4, 8, 10
    table = rng.uniform(-1, 1, size=(g.total, 2))
    params = rng.uniform(-0.6, 0.6, oracle.mlp_param_count(D, H, O))
    dd = rng.standard_normal((O, n))
    lam, eps_s, eps_t = 0.8, (0.01, -0.02, 0.015), 0.03

    def loss(tab, par):
        dl = oracle.deform_fwd(g, pts, tab, H, O, par)
        return (dl * dd).sum() + oracle.smooth_loss(g, pts, tab, lam, eps_s, eps_t)

    tg, pg, lr = oracle.deform_bwd(g, pts, table, H, O, params, dd, lam, eps_s, eps_t)
    assert abs(lr - oracle.smooth_loss(g, pts, table, lam, eps_s, eps_t)) < 1e-12
    h = 1e-6
    for e in rng.choice(g.total, size=25, replace=False):
        for f in range(2):
            tp = table.copy(); tp[e, f] += h
            tm = table.copy(); tm[e, f] -= h
            fd = (loss(tp, params) - loss(tm, params)) / (2 * h)
            assert abs(fd - tg[e, f]) < 1e-6 * max(1.0, abs(fd))
    for k in rng.choice(len(params), size=40, replace=False):
        pp = params.copy(); pp[k] += h
        pm = params.copy(); pm[k] -= h
        fd = (loss(table, pp) - loss(table, pm)) / (2 * h)
        assert abs(fd - pg[k]) < 1e-5 * max(1.0, abs(fd))
