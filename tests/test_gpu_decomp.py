"""GPU parity of the decomposition step that produces the mask (Sec. 4.1,
Eqs. 3-4): G_3D + phi_p + phi_l norms against the FP64 oracle, and the top-k %
mask bit for bit against the oracle's selection applied to the same FP32
norms (the GPU's), then the whole chain into compaction and deformation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import RELU_MARGIN, rel_err, to_dev

pytestmark = pytest.mark.gpu

G3 = dict(L=16, F=2, log2_T=19, nmin=16, nmax=2048)


def _decomp_inputs(rng, n, tdtype=np.float16):
    g = oracle.layout3(**G3)
    x, y, z, _ = synth.scene_coords(rng, n)
    table = synth.table_values(rng, g.total, 2, tdtype)
    D, H = 32, 64
    params = rng.uniform(-1 / np.sqrt(D), 1 / np.sqrt(D), H * D + H + 3 * H + 3).astype(np.float32)
    return g, (x, y, z), table, params


def _unambiguous(g, x, y, z, table, params, D, margin=RELU_MARGIN):
    """Per Gaussian: True where every hidden pre-activation of phi_p (on the
    oracle's FP64 G_3D encoding, a plain matrix product) is at least
    `margin` from 0, so the GPU and the oracle take the same ReLU decisions
    (the tensor-core backward forms them from hi + lo BF16 splits)."""
    f = oracle.encode3(g, x, y, z, np.asarray(table, np.float64))
    p = np.asarray(params, np.float64)
    W1, b1 = p[:64 * D].reshape(64, D), p[64 * D:64 * D + 64]
    return (np.abs(f @ W1.T + b1) >= margin).all(axis=1)


def _clear_ambiguous(keep, d_dp, mask):
    """Gaussians whose ReLU decisions are ambiguous get no upstream gradient
    and are made dynamic (no Eq. 5 term), on both sides."""
    d_dp[:, ~keep] = 0.0
    if mask is not None:
        m = mask.cpu().numpy().copy()
        m[~keep] = 1
        mask = to_dev(m)
    return d_dp, mask


@pytest.mark.parametrize("tdtype", [np.float16, np.float32])
def test_decomposition_norms_match_oracle(dashlib, tdtype):
    rng = np.random.default_rng(71)
    n = 20_000
    g, (x, y, z), table, params = _decomp_inputs(rng, n, tdtype)
    lay = dashlib.dash_hash3d_layout(**G3)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 3)
    dp, norm = dashlib.dash_decomp_fwd(lay, to_dev(x), to_dev(y), to_dev(z), to_dev(table), mlp)
    rdp, rnorm = oracle.decomp_fwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64))
    assert rel_err(dp.cpu().numpy(), rdp) < 1e-5
    assert rel_err(norm.cpu().numpy(), rnorm) < 1e-5


@pytest.mark.parametrize("n,k", [(1, 50.0), (10, 0.0), (10, 100.0), (1000, 12.5), (1_000_003, 50.0),
                                 (2_000_000, 37.3)])
def test_topk_mask_bit_exact(dashlib, n, k):
    rng = np.random.default_rng(n)
    v = rng.random(n).astype(np.float32) * 3
    mask, tau = dashlib.dash_topk_mask(to_dev(v), k)
    rmask, rtau = oracle.topk_mask(v.astype(np.float64), k)
    assert np.array_equal(mask.cpu().numpy(), rmask)
    assert float(tau.item()) == np.float32(rtau)


@pytest.mark.parametrize("per_gaussian_t", [True, False])
def test_linear_motion_matches_oracle(dashlib, per_gaussian_t):
    """Eq. 4 fused into the decomposition kernel: p(t) = p + t dp."""
    rng = np.random.default_rng(74)
    n = 5_000
    g, (x, y, z), table, params = _decomp_inputs(rng, n)
    x[:7] = [-0.25, 1.5, 0.0, 1.0, 0.5, 2.0, -1.0]        # p(t) uses p as given, the encoder the clamped p
    t = rng.random(n).astype(np.float32) if per_gaussian_t else np.array([0.37], np.float32)
    lay = dashlib.dash_hash3d_layout(**G3)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 3)
    dp, norm, pt = dashlib.dash_decomp_fwd(lay, to_dev(x), to_dev(y), to_dev(z), to_dev(table), mlp, t=to_dev(t))
    rdp, _ = oracle.decomp_fwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64))
    ref = oracle.linear_motion(x, y, z, t, rdp)
    p = np.stack([x, y, z]).astype(np.float64)
    assert rel_err(pt.cpu().numpy() - p, ref - p) < 1e-5
    # and exactly one rounding of t * dp + p on the GPU's own dp
    own = oracle.linear_motion(x, y, z, t, dp.cpu().numpy().astype(np.float64)).astype(np.float32)
    assert np.max(np.abs(pt.cpu().numpy().view(np.int32).astype(np.int64) - own.view(np.int32))) <= 1


@pytest.mark.parametrize("k", [0.0, 20.0, 50.0, 100.0])
def test_static_loss_matches_oracle(dashlib, k):
    """Eq. 5 accumulated while the mask is written (FP64 sums)."""
    rng = np.random.default_rng(75)
    v = (rng.random(300_001) * 2).astype(np.float32)
    ls = torch.empty(1, device="cuda")
    mask, _ = dashlib.dash_topk_mask(to_dev(v), k, static_loss_out=ls)
    m = mask.cpu().numpy()
    ref = oracle.static_loss(v.astype(np.float64), m)
    assert np.array_equal(m, oracle.topk_mask(v.astype(np.float64), k)[0])
    assert abs(float(ls.item()) - ref) <= 1e-6 * max(ref, 1e-30)
    e = torch.empty(0, device="cuda")
    ls.fill_(5.0)
    dashlib.dash_topk_mask(e, k, static_loss_out=ls)
    assert float(ls.item()) == 0.0


def test_topk_mask_with_ties(dashlib):
    rng = np.random.default_rng(72)
    v = rng.integers(0, 50, size=100_000).astype(np.float32) / 7  # many equal values
    for k in (0.5, 10.0, 50.0, 99.9):
        mask, tau = dashlib.dash_topk_mask(to_dev(v), k)
        rmask, rtau = oracle.topk_mask(v.astype(np.float64), k)
        assert np.array_equal(mask.cpu().numpy(), rmask), k
        assert float(tau.item()) == np.float32(rtau)


def test_topk_mask_zeros_of_both_signs(dashlib):
    """Zero norms (either sign) are the smallest keys and never dynamic."""
    v = np.zeros(4096, np.float32)
    v[::3] = -0.0
    v[1::7] = np.linspace(0.5, 2.0, len(v[1::7]), dtype=np.float32)
    for k in (5.0, 14.0, 50.0):
        mask, tau = dashlib.dash_topk_mask(to_dev(v), k)
        rmask, rtau = oracle.topk_mask(v.astype(np.float64), k)
        assert np.array_equal(mask.cpu().numpy(), rmask), k
        assert float(tau.item()) == np.float32(rtau)


def test_decomposition_empty_and_errors(dashlib):
    lay = dashlib.dash_hash3d_layout(**G3)
    e = torch.empty(0, device="cuda")
    dec = dashlib.Mlp(torch.zeros(64 * 32 + 64 + 3 * 64 + 3, device="cuda"), 32, 64, 3)
    _, norm = dashlib.dash_decomp_fwd(lay, e, e, e, torch.zeros(8, device="cuda"), dec)
    assert norm.numel() == 0
    mask, _ = dashlib.dash_topk_mask(e, 50.0)
    assert mask.numel() == 0
    with pytest.raises(dashlib.DashError):
        dashlib.dash_topk_mask(torch.ones(4, device="cuda"), 101.0)
    lay4 = dashlib.layout_from(synth.PAPER_GRID)
    x = torch.rand(16, device="cuda")
    with pytest.raises(dashlib.DashError):   # a 4-D layout is not a G_3D layout
        dashlib.dash_decomp_fwd(lay4, x, x, x, torch.zeros(8, device="cuda"), dec)


def test_decomposition_feeds_compaction_and_deformation(dashlib):
    """decomposition -> top-k mask -> compaction -> fused deformation,
    every stage on the GPU, against the oracle chain fed the GPU's norms."""
    rng = np.random.default_rng(73)
    n_all = 30_000
    g3, (x, y, z), t3, p3 = _decomp_inputs(rng, n_all)
    t = rng.random(n_all).astype(np.float32)
    lay3 = dashlib.dash_hash3d_layout(**G3)
    dec = dashlib.Mlp(to_dev(p3), 32, 64, 3)
    xd, yd, zd, td = to_dev(x), to_dev(y), to_dev(z), to_dev(t)
    _, norm = dashlib.dash_decomp_fwd(lay3, xd, yd, zd, to_dev(t3), dec, want_dp=False)
    mask, _ = dashlib.dash_topk_mask(norm, 30.0)
    idx, cnt = dashlib.dash_compact_dynamic(mask)
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    g4 = oracle.layout(grid.L, grid.F, grid.log2_T, grid.nmin_s, grid.nmax_s, grid.nmin_t, grid.nmax_t)
    table = synth.table_values(rng, g4.total, 2, np.float16)
    params = synth.mlp_params(rng, mlpc)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(xd, yd, zd, td, idx=idx, n=n_all, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 10)
    delta = dashlib.dash_deform_mlp_fwd(lay, pts, to_dev(table), mlp)
    rmask, _ = oracle.topk_mask(norm.cpu().numpy().astype(np.float64), 30.0)
    ridx, rcnt = oracle.compact(rmask)
    assert int(cnt.item()) == rcnt and 0 < rcnt <= int(np.floor(0.3 * n_all))  # fewer only on a tie at tau
    assert np.array_equal(idx[:rcnt].cpu().numpy(), ridx)
    ref = oracle.deform_fwd(g4, oracle.Points(x, y, z, t, idx=ridx), table.astype(np.float64), 64, 10,
                            params.astype(np.float64))
    assert rel_err(delta[:, :rcnt].cpu().numpy(), ref) < 1e-3


@pytest.mark.parametrize("tdtype,with_up,with_ls", [(np.float16, True, True), (np.float32, True, False),
                                                    (np.float16, False, True)])
def test_decomposition_backward_matches_oracle(dashlib, tdtype, with_up, with_ls):
    rng = np.random.default_rng(76)
    n = 9_999
    g, (x, y, z), table, params = _decomp_inputs(rng, n, tdtype)
    lay = dashlib.dash_hash3d_layout(**G3)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 3)
    xd, yd, zd, td = to_dev(x), to_dev(y), to_dev(z), to_dev(table)
    _, norm = dashlib.dash_decomp_fwd(lay, xd, yd, zd, td, mlp)
    mask, _ = dashlib.dash_topk_mask(norm, 40.0)
    d_dp = rng.standard_normal((3, n)).astype(np.float32)
    d_dp, mask = _clear_ambiguous(_unambiguous(g, x, y, z, table, params, 32), d_dp, mask)
    tg = torch.zeros((g.total, 2), device="cuda")
    pg = torch.zeros(params.size, device="cuda")
    dashlib.dash_decomp_bwd(lay, xd, yd, zd, td, mlp, tg, pg, d_dp=to_dev(d_dp) if with_up else None,
                            mask=mask if with_ls else None, lambda_s=0.8 if with_ls else 0.0)
    rtg, rpg = oracle.decomp_bwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64),
                                 d_dp.astype(np.float64) if with_up else None,
                                 mask.cpu().numpy() if with_ls else None, 0.8 if with_ls else 0.0)
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-4
    bounds = np.cumsum([0, 64 * 32, 64, 3 * 64, 3])
    pgn = pg.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert rel_err(pgn[a:b], rpg[a:b]) < 1e-4, (a, b, rel_err(pgn[a:b], rpg[a:b]))


@pytest.mark.parametrize("L,F,tdtype,n", [(16, 1, np.float32, 5_001), (8, 4, np.float16, 3_333),
                                          (4, 8, np.float32, 257), (16, 2, np.float16, 1)])
def test_decomposition_backward_feature_widths(dashlib, L, F, tdtype, n):
    """The two-threads-per-Gaussian backward for F = 1, 4, 8 (and F = 2 with a
    single Gaussian): tile tails, L*F of 16..32, FP16 and FP32 tables."""
    rng = np.random.default_rng(90 + F)
    cfg = dict(L=L, F=F, log2_T=14, nmin=16, nmax=512)
    g = oracle.layout3(**cfg)
    x, y, z, _ = synth.scene_coords(rng, n)
    table = synth.table_values(rng, g.total, F, tdtype)
    D, H = L * F, 64
    params = rng.uniform(-1 / np.sqrt(D), 1 / np.sqrt(D), H * D + H + 3 * H + 3).astype(np.float32)
    lay = dashlib.dash_hash3d_layout(**cfg)
    mlp = dashlib.Mlp(to_dev(params), D, 64, 3)
    xd, yd, zd, td = to_dev(x), to_dev(y), to_dev(z), to_dev(table)
    _, norm = dashlib.dash_decomp_fwd(lay, xd, yd, zd, td, mlp)
    mask, _ = dashlib.dash_topk_mask(norm, 30.0)
    d_dp = rng.standard_normal((3, n)).astype(np.float32)
    d_dp, mask = _clear_ambiguous(_unambiguous(g, x, y, z, table, params, D), d_dp, mask)
    tg = torch.zeros((g.total, F), device="cuda")
    pg = torch.zeros(params.size, device="cuda")
    dashlib.dash_decomp_bwd(lay, xd, yd, zd, td, mlp, tg, pg, d_dp=to_dev(d_dp), mask=mask, lambda_s=0.5)
    rtg, rpg = oracle.decomp_bwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64),
                                 d_dp.astype(np.float64), mask.cpu().numpy(), 0.5)
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-4
    bounds = np.cumsum([0, 64 * D, 64, 3 * 64, 3])
    pgn = pg.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert rel_err(pgn[a:b], rpg[a:b]) < 1e-4, (a, b, rel_err(pgn[a:b], rpg[a:b]))


@pytest.mark.parametrize("n,F,tdtype", [(30_001, 2, np.float16), (4_097, 1, np.float32), (129, 4, np.float16)])
def test_decomposition_backward_forms_agree(dashlib, n, F, tdtype):
    """The tensor-core backward (default) and the CUDA-core one give the
    same gradients up to rounding, and both match the oracle."""
    rng = np.random.default_rng(95 + n)
    L = 32 // F
    cfg = dict(L=L, F=F, log2_T=17, nmin=16, nmax=1024)
    g = oracle.layout3(**cfg)
    x, y, z, _ = synth.scene_coords(rng, n)
    table = synth.table_values(rng, g.total, F, tdtype)
    params = rng.uniform(-1 / np.sqrt(32), 1 / np.sqrt(32), 64 * 32 + 64 + 3 * 64 + 3).astype(np.float32)
    lay = dashlib.dash_hash3d_layout(**cfg)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 3)
    xd, yd, zd, td = to_dev(x), to_dev(y), to_dev(z), to_dev(table)
    _, norm = dashlib.dash_decomp_fwd(lay, xd, yd, zd, td, mlp)
    mask, _ = dashlib.dash_topk_mask(norm, 45.0)
    d_dp = rng.standard_normal((3, n)).astype(np.float32)
    d_dp, mask = _clear_ambiguous(_unambiguous(g, x, y, z, table, params, 32), d_dp, mask)
    out = []
    old = dashlib.dash_get_option(dashlib.OPT_DECOMP_FORM)
    try:
        for form in (0, 1):
            dashlib.dash_set_option(dashlib.OPT_DECOMP_FORM, form)
            tg = torch.zeros((g.total, F), device="cuda")
            pg = torch.zeros(params.size, device="cuda")
            dashlib.dash_decomp_bwd(lay, xd, yd, zd, td, mlp, tg, pg, d_dp=to_dev(d_dp), mask=mask, lambda_s=0.6)
            out.append((tg.cpu().numpy(), pg.cpu().numpy()))
    finally:
        dashlib.dash_set_option(dashlib.OPT_DECOMP_FORM, old)
    dashlib.dash_device_status()
    rtg, rpg = oracle.decomp_bwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64),
                                 d_dp.astype(np.float64), mask.cpu().numpy(), 0.6)
    bounds = np.cumsum([0, 64 * 32, 64, 3 * 64, 3])
    for tg, pg in out:
        assert rel_err(tg, rtg) < 1e-4
        for a, b in zip(bounds[:-1], bounds[1:]):
            assert rel_err(pg[a:b], rpg[a:b]) < 1e-4, (a, b, rel_err(pg[a:b], rpg[a:b]))
    assert rel_err(out[0][0], out[1][0]) < 1e-4 and rel_err(out[0][1], out[1][1]) < 1e-4


@pytest.mark.parametrize("n,L,F,tdtype", [(20_001, 16, 2, np.float16), (3_000, 32, 1, np.float32),
                                          (129, 8, 4, np.float16), (1, 4, 8, np.float32)])
def test_decomposition_forward_forms_agree(dashlib, n, L, F, tdtype):
    """The tensor-core forward (default; three-part BF16 splits, every
    product of total order up to 2 kept) and the CUDA-core forward give the
    same Delta p, norms and Eq. 4 p(t) to FP32 accuracy, and both match the
    oracle."""
    rng = np.random.default_rng(120 + n)
    cfg = dict(L=L, F=F, log2_T=17, nmin=16, nmax=1024)
    g = oracle.layout3(**cfg)
    x, y, z, _ = synth.scene_coords(rng, n)
    t = rng.random(n).astype(np.float32)
    table = synth.table_values(rng, g.total, F, tdtype)
    D = L * F
    params = rng.uniform(-1 / np.sqrt(D), 1 / np.sqrt(D), 64 * D + 64 + 3 * 64 + 3).astype(np.float32)
    lay = dashlib.dash_hash3d_layout(**cfg)
    mlp = dashlib.Mlp(to_dev(params), D, 64, 3)
    out = []
    old = dashlib.dash_get_option(dashlib.OPT_DECOMP_FORM)
    try:
        for form in (0, 1):
            dashlib.dash_set_option(dashlib.OPT_DECOMP_FORM, form)
            res = dashlib.dash_decomp_fwd(lay, to_dev(x), to_dev(y), to_dev(z), to_dev(table), mlp, t=to_dev(t))
            out.append([v.cpu().numpy() for v in res])
    finally:
        dashlib.dash_set_option(dashlib.OPT_DECOMP_FORM, old)
    dashlib.dash_device_status()
    rdp, rnorm = oracle.decomp_fwd(g, x, y, z, table.astype(np.float64), 64, params.astype(np.float64))
    for dp, norm, pt in out:
        assert rel_err(dp, rdp) < 1e-5 and rel_err(norm, rnorm) < 1e-5
        assert rel_err(pt - np.stack([x, y, z]), t * rdp) < 1e-5
    for a, b in zip(out[0], out[1]):
        assert rel_err(a, b) < 1e-5
