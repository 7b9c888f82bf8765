"""GPU parity of the fused deformation path (encoder + tensor-core decoder,
Eqs. 8-10; backward and Eq. 11) against the FP64 oracle through the C ABI.
Targets: outputs within 1e-3 relative error per head, gradients within 1e-2,
each bound holding normwise and for every element against the largest
reference value, with the same table entries touched (gpu_helpers.rel_err)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import edge_coords, oracle_grid, rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu

HEADS = ((0, 3), (3, 7), (7, 10))


def _case(grid, mlpc, n, tdtype, seed, coords=None, n_all=None):
    rng = np.random.default_rng(seed)
    g = oracle_grid(grid)
    if coords is None:
        if n_all is None:
            coords = synth.scene_coords(rng, n)
            idx = None
        else:
            mask = synth.exact_count_mask(rng, n_all, n)
            coords = synth.scene_coords(rng, n_all)
            idx = np.flatnonzero(mask).astype(np.int32)
    else:
        idx = None
    table = synth.table_values(rng, g.total, grid.F, tdtype)
    params = synth.mlp_params(rng, mlpc)
    dd = synth.upstream_grad(rng, mlpc.d_out, n)
    # Gaussians whose ReLU decisions the GPU and the oracle could take
    # differently get no upstream gradient (gpu_helpers.RELU_MARGIN)
    zero_ambiguous(dd, g, oracle.Points(*coords, idx=idx), table, params, mlpc.d_hidden, mlpc.d_out)
    return g, coords, idx, table, params, dd


def _dev_points(dashlib, coords, idx, n):
    x, y, z, t = (to_dev(c) for c in coords)
    return dashlib.Points(x, y, z, t, idx=None if idx is None else to_dev(idx), n=n)


@pytest.mark.parametrize("grid,mlpc,n,tdtype", [
    (synth.TINY_GRID, synth.TINY_MLP, 10_000, np.float32),
    (synth.PAPER_GRID, synth.PAPER_MLP, 20_000, np.float16),
    (synth.PAPER_GRID, synth.PAPER_MLP, 20_000, np.float32),
    (synth.PAPER_GRID, synth.PAPER_MLP, 300, np.float16),      # one ragged tile pair
    (synth.PAPER_GRID, synth.PAPER_MLP, 1, np.float16),
])
def test_fused_forward_parity(dashlib, grid, mlpc, n, tdtype):
    g, coords, idx, table, params, _ = _case(grid, mlpc, n, tdtype, seed=31 + n)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, idx, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    fsave = dashlib.deform_state(dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out), n, "cuda")
    delta = dashlib.dash_deform_mlp_fwd(lay, pts, to_dev(table), mlp, fwd_state=fsave).cpu().numpy()
    ref = oracle.deform_fwd(g, oracle.Points(*coords), table.astype(np.float64), mlpc.d_hidden, mlpc.d_out,
                            params.astype(np.float64))
    for a, b in HEADS:
        assert rel_err(delta[a:b], ref[a:b]) < 1e-3, (a, b, rel_err(delta[a:b], ref[a:b]))
    fh = oracle.encode(g, oracle.Points(*coords), table.astype(np.float64))
    fstate = fsave[:, :2 * mlpc.d_in].contiguous().view(torch.bfloat16)  # BF16 copy of f_h in the state
    assert rel_err(fstate.float().cpu().numpy(), fh) < 8e-3


def test_fused_forward_index_list_apply_and_edges(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(33)
    n_all = 7000
    coords = list(edge_coords(n_all, rng))
    mask = synth.bernoulli_mask(rng, n_all, 0.45)
    mask[:10] = 1  # keep the degenerate coordinates dynamic
    idx = np.flatnonzero(mask).astype(np.int32)
    n = len(idx)
    g = oracle_grid(grid)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    attrs = synth.gaussian_attrs(rng, n_all)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, idx, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    ai = to_dev(attrs)
    ao = ai.clone()
    delta = dashlib.dash_deform_mlp_fwd(lay, pts, to_dev(table), mlp, apply=(ai, ao)).cpu().numpy()
    rdelta, rout = oracle.deform_fwd(g, oracle.Points(*coords, idx=idx), table.astype(np.float64), mlpc.d_hidden,
                                     mlpc.d_out, params.astype(np.float64), attrs_in=attrs)
    for a, b in HEADS:
        assert rel_err(delta[a:b], rdelta[a:b]) < 1e-3
    out = ao.cpu().numpy()
    assert np.array_equal(out[:, mask == 0], attrs[:, mask == 0])  # static Gaussians untouched
    assert np.max(np.abs(out[:, idx] - rout[:, idx])) < 1e-3


def test_fused_forward_device_count(dashlib):
    """The kernel reads the dynamic count from device memory (graph-safe)."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    g, coords, _, table, params, _ = _case(grid, mlpc, 5000, np.float16, seed=34)
    lay = dashlib.layout_from(grid)
    x, y, z, t = (to_dev(c) for c in coords)
    cnt = torch.tensor([3001], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(x, y, z, t, n=5000, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    out = torch.full((10, 5000), 123.0, device="cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, to_dev(table), mlp, delta_out=out)
    o = out.cpu().numpy()
    ref = oracle.deform_fwd(g, oracle.Points(*[c[:3001] for c in coords]), table.astype(np.float64), 64, 10,
                            params.astype(np.float64))
    assert rel_err(o[:, :3001], ref) < 1e-3
    assert np.all(o[:, 3001:] == 123.0)


def test_fused_forward_rejects_unsupported(dashlib):
    grid = synth.PAPER_GRID
    lay = dashlib.layout_from(grid)
    rng = np.random.default_rng(35)
    coords = [to_dev(c) for c in synth.uniform_coords(rng, 10)]
    pts = dashlib.Points(*coords)
    p = torch.zeros(synth.MlpCfg(32, 32, 10).n_params, device="cuda")
    with pytest.raises(dashlib.DashError) as e:
        dashlib.dash_deform_mlp_fwd(lay, pts, torch.zeros((10, 2), device="cuda"), dashlib.Mlp(p, 32, 32, 10))
    assert e.value.status == dashlib.ERR_UNSUPPORTED


def _grad_errors(dashlib, grid, mlpc, n, tdtype, seed, use_saved, smooth=None, n_all=None, coords=None):
    g, coords, idx, table, params, dd = _case(grid, mlpc, n, tdtype, seed, coords=coords, n_all=n_all)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, idx, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    fsave = dashlib.deform_state(dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out), n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=fsave)
    tg = torch.zeros((g.total, grid.F), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    sm = None if smooth is None else (smooth[0], smooth[1], smooth[2], loss)
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=fsave if use_saved else None,
                                smooth=sm)
    lam, es, et = smooth if smooth is not None else (0.0, (0.0, 0.0, 0.0), 0.0)
    rtg, rpg, rl = oracle.deform_bwd(g, oracle.Points(*coords, idx=idx), table.astype(np.float64), mlpc.d_hidden,
                                     mlpc.d_out, params.astype(np.float64), dd.astype(np.float64), lam, es, et)
    D, H, O = mlpc.d_in, mlpc.d_hidden, mlpc.d_out
    bounds = np.cumsum([0, H * D, H, H * H, H, O * H, O])
    pgn = pg.cpu().numpy()
    errs = {"table": rel_err(tg.cpu().numpy(), rtg)}
    for name, a, b in zip(("W1", "b1", "W2", "b2", "W3", "b3"), bounds[:-1], bounds[1:]):
        errs[name] = rel_err(pgn[a:b], rpg[a:b])
    if smooth is not None:
        errs["loss"] = abs(float(loss.item()) - rl) / abs(rl)
    return errs


@pytest.mark.parametrize("grid,mlpc,n,tdtype,use_saved", [
    (synth.TINY_GRID, synth.TINY_MLP, 10_000, np.float32, True),
    (synth.PAPER_GRID, synth.PAPER_MLP, 20_000, np.float16, True),
    (synth.PAPER_GRID, synth.PAPER_MLP, 20_000, np.float16, False),
    (synth.PAPER_GRID, synth.PAPER_MLP, 300, np.float32, True),
])
def test_fused_backward_parity(dashlib, grid, mlpc, n, tdtype, use_saved):
    errs = _grad_errors(dashlib, grid, mlpc, n, tdtype, 41 + n, use_saved)
    assert all(v < 1e-2 for v in errs.values()), errs


def test_fused_backward_with_index_list(dashlib):
    errs = _grad_errors(dashlib, synth.PAPER_GRID, synth.PAPER_MLP, 6000, np.float16, 42, True, n_all=13_000)
    assert all(v < 1e-2 for v in errs.values()), errs


@pytest.mark.parametrize("grid,mlpc,tdtype", [(synth.TINY_GRID, synth.TINY_MLP, np.float32),
                                              (synth.PAPER_GRID, synth.PAPER_MLP, np.float16)])
def test_fused_backward_smoothness_term(dashlib, grid, mlpc, tdtype):
    """Eq. 11 with the paper-shaped perturbations dx = 1/2048, dt = 1/300."""
    smooth = (1.0, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300)
    errs = _grad_errors(dashlib, grid, mlpc, 8000, tdtype, 43, True, smooth=smooth)
    assert all(v < 1e-2 for v in errs.values()), errs


@pytest.mark.parametrize("case", ["index_list", "edge_coords", "coarse_eps"])
def test_fused_backward_smoothness_term_cases(dashlib, case):
    """Eq. 11 where the perturbed points share the hypervoxel of p on some
    levels and not on others: scene points through an index list, the
    degenerate coordinates (0, 1, NaN, out of range, vertices; clamped
    perturbations), and perturbations wide enough to leave the hypervoxel
    on the coarse levels too."""
    smooth = (0.7, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300)
    kw = {}
    if case == "index_list":
        kw = dict(n_all=9_000)
    elif case == "edge_coords":
        kw = dict(coords=edge_coords(3000, np.random.default_rng(48)))
    else:
        smooth = (0.7, (1 / 20, -1 / 30, 1 / 40), -1 / 10)
    errs = _grad_errors(dashlib, synth.PAPER_GRID, synth.PAPER_MLP, 3000, np.float16, 49, True, smooth=smooth, **kw)
    assert all(v < 1e-2 for v in errs.values()), errs


def test_fused_backward_finite_differences(dashlib):
    """Table gradient of Loss = sum(ddelta * delta) + lambda L_r from the GPU
    backward against central differences of the GPU forward (FP32 tables)."""
    grid, mlpc = synth.TINY_GRID, synth.TINY_MLP
    n = 512
    g, coords, _, table, params, dd = _case(grid, mlpc, n, np.float32, 44)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, None, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    ddt = to_dev(dd)
    lam, es, et = 0.5, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300
    tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, ddt, tg, pg, smooth=(lam, es, et, None))
    tgn = tg.cpu().numpy()

    def loss(t):
        delta = dashlib.dash_deform_mlp_fwd(lay, pts, t, mlp).double()
        lr = torch.zeros(1, dtype=torch.float32, device="cuda")
        scratch = torch.zeros_like(tg)
        dashlib.dash_deform_mlp_bwd(lay, pts, t, mlp, torch.zeros_like(ddt), scratch, torch.zeros_like(pg),
                                    smooth=(lam, es, et, lr))
        return float((delta * ddt.double()).sum().item()) + float(lr.item())

    order = np.argsort(-np.abs(tgn).max(axis=1))[:12]
    h = 1e-2
    for e in order:
        for f in range(2):
            tp = tab.clone(); tp[e, f] += h
            tm = tab.clone(); tm[e, f] -= h
            fd = (loss(tp) - loss(tm)) / (2 * h)
            assert abs(fd - tgn[e, f]) < 2e-2 * max(1.0, abs(fd)), (e, f, fd, tgn[e, f])


def test_autograd_function_matches_oracle(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    n = 4000
    g, coords, _, table, params, dd = _case(grid, mlpc, n, np.float32, 45)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, None, n)
    tab = to_dev(table).requires_grad_(True)
    par = to_dev(params).requires_grad_(True)
    delta = dashlib.deform(tab, par, lay, pts)
    (delta * to_dev(dd)).sum().backward()
    rtg, rpg, _ = oracle.deform_bwd(g, oracle.Points(*coords), table.astype(np.float64), 64, 10,
                                    params.astype(np.float64), dd.astype(np.float64))
    assert rel_err(tab.grad.cpu().numpy(), rtg) < 1e-2
    assert rel_err(par.grad.cpu().numpy(), rpg) < 1e-2


@pytest.mark.parametrize("grid,mlpc,tdtype", [(synth.PAPER_GRID, synth.PAPER_MLP, np.float16),
                                              (synth.TINY_GRID, synth.TINY_MLP, np.float32)])
def test_forward_kernel_forms_agree(dashlib, grid, mlpc, tdtype):
    """Every fused-forward form (warp-specialised, 1/2/4 groups per CTA)
    computes the same offsets and state bit for bit."""
    n = 70_001
    g, coords, _, table, params, _ = _case(grid, mlpc, n, tdtype, 46)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, None, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    outs = []
    old = dashlib.dash_get_option(dashlib.OPT_FWD_FORM)
    try:
        for form in (0, 1, 2, 4, 10, 11, 12, 13, 14, 15):
            dashlib.dash_set_option(dashlib.OPT_FWD_FORM, form)
            st = dashlib.deform_state(mlp, n, "cuda")
            d = dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
            outs.append((d.cpu(), st.cpu()))
    finally:
        dashlib.dash_set_option(dashlib.OPT_FWD_FORM, old)
    for d, st in outs[1:]:
        assert torch.equal(d, outs[0][0]) and torch.equal(st, outs[0][1])
    ref = oracle.deform_fwd(g, oracle.Points(*coords), table.astype(np.float64), mlpc.d_hidden, mlpc.d_out,
                            params.astype(np.float64))
    assert rel_err(outs[0][0].numpy(), ref) < 1e-3


@pytest.mark.parametrize("smooth", [None, (0.5, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300)])
def test_backward_kernel_forms_agree(dashlib, smooth):
    """The warp-specialised and the single-group backward give the same
    gradients up to the order of the atomic additions."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    n = 30_001
    g, coords, _, table, params, dd = _case(grid, mlpc, n, np.float16, 47)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, None, n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    res = []
    old = dashlib.dash_get_option(dashlib.OPT_BWD_FORM)
    try:
        # 1: single group; 10, 13, 14: scatter groups taking whole tiles in
        # turn; 0, 11, 12: every group on every tile, each its own share of
        # the levels
        for form in (0, 1, 10, 11, 12, 13, 14):
            dashlib.dash_set_option(dashlib.OPT_BWD_FORM, form)
            tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
            pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
            lo = torch.zeros(1, dtype=torch.float32, device="cuda")
            sm = None if smooth is None else (*smooth, lo)
            dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st, smooth=sm)
            res.append((tg.cpu().numpy(), pg.cpu().numpy(), float(lo.item())))
    finally:
        dashlib.dash_set_option(dashlib.OPT_BWD_FORM, old)
    for other in res[1:]:
        assert rel_err(res[0][0], other[0]) < 1e-5
    if smooth is None:
        for other in res[1:]:
            assert rel_err(res[0][1], other[1]) < 1e-5
    else:
        # with Eq. 11 on, the single-group form recomputes the decoder from a
        # fresh FP32 f_h, the warp-specialised one from the state's BF16 f_h:
        # dW1 = dz1^T f_h differs by that rounding; both must meet the oracle
        assert abs(res[0][2] - res[1][2]) <= 1e-4 * abs(res[1][2])
        lam, es, et = smooth
        rtg, rpg, rl = oracle.deform_bwd(g, oracle.Points(*coords), table.astype(np.float64), 64, 10,
                                         params.astype(np.float64), dd.astype(np.float64), lam, es, et)
        for tg_, pg_, l_ in res:
            assert rel_err(tg_, rtg) < 1e-2 and rel_err(pg_, rpg) < 1e-2 and abs(l_ - rl) < 1e-2 * abs(rl)


@pytest.mark.parametrize("n_all,n,tdtype,grid", [
    (50_000, 20_001, np.float16, synth.PAPER_GRID),   # odd count: the last lane pair has one Gaussian
    (4_000, 1_283, np.float32, synth.PAPER_GRID),
    (2_000, 129, np.float16, synth.TINY_GRID),        # all levels hashed, tail of one row past a tile
    (10, 1, np.float16, synth.PAPER_GRID),
])
def test_backward_scatter_forms_agree_with_oracle(dashlib, n_all, n, tdtype, grid):
    """The lane-paired and the per-lane table-gradient scatter of the
    warp-specialised backward: same sums up to the order of the additions,
    both against the oracle (index list, device count, ragged tails)."""
    mlpc = synth.PAPER_MLP if grid is synth.PAPER_GRID else synth.TINY_MLP
    g, coords, idx, table, params, dd = _case(grid, mlpc, n, tdtype, seed=61 + n, n_all=n_all)
    lay = dashlib.layout_from(grid)
    x, y, z, t = (to_dev(c) for c in coords)
    cnt = torch.tensor([n], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(x, y, z, t, idx=to_dev(idx), n=n, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    res = []
    old = dashlib.dash_get_option(dashlib.OPT_ACCESS_FORM)
    try:
        for form in (0, 1):
            dashlib.dash_set_option(dashlib.OPT_ACCESS_FORM, form)
            tg = torch.zeros((g.total, grid.F), dtype=torch.float32, device="cuda")
            pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
            dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st)
            res.append((tg.cpu().numpy(), pg.cpu().numpy()))
    finally:
        dashlib.dash_set_option(dashlib.OPT_ACCESS_FORM, old)
    assert rel_err(res[0][0], res[1][0]) < 1e-6
    assert np.array_equal(res[0][0] != 0, res[1][0] != 0)  # the same entries touched
    assert rel_err(res[0][1], res[1][1]) < 1e-6
    ref_pts = oracle.Points(*coords, idx=idx)
    rtg, rpg, _ = oracle.deform_bwd(g, ref_pts, table.astype(np.float64), mlpc.d_hidden, mlpc.d_out,
                                    params.astype(np.float64), dd.astype(np.float64))
    for tg_, pg_ in res:
        assert rel_err(tg_, rtg) < 1e-2 and rel_err(pg_, rpg) < 1e-2


@pytest.mark.parametrize("n_all,n,tdtype,grid", [
    (50_000, 20_001, np.float16, synth.PAPER_GRID),
    (4_000, 1_283, np.float32, synth.PAPER_GRID),
    (2_000, 129, np.float32, synth.TINY_GRID),
    (10, 1, np.float16, synth.PAPER_GRID),
])
def test_forward_access_forms_bit_identical(dashlib, n_all, n, tdtype, grid):
    """Lane-paired and per-lane gathers of the warp-specialised forward give
    the same offsets, Eq. 10 update and state bit for bit (index list,
    device count, odd counts), and meet the oracle."""
    mlpc = synth.PAPER_MLP if grid is synth.PAPER_GRID else synth.TINY_MLP
    g, coords, idx, table, params, _ = _case(grid, mlpc, n, tdtype, seed=71 + n, n_all=n_all)
    lay = dashlib.layout_from(grid)
    x, y, z, t = (to_dev(c) for c in coords)
    cnt = torch.tensor([n], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(x, y, z, t, idx=to_dev(idx), n=n, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    attrs = torch.randn((mlpc.d_out, n_all), dtype=torch.float32, device="cuda")
    outs = []
    old = dashlib.dash_get_option(dashlib.OPT_ACCESS_FORM)
    try:
        for form in (0, 1):
            dashlib.dash_set_option(dashlib.OPT_ACCESS_FORM, form)
            st = dashlib.deform_state(mlp, n, "cuda")
            out = attrs.clone()
            d = dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st, apply=(attrs, out))
            outs.append((d.cpu(), st.cpu(), out.cpu()))
    finally:
        dashlib.dash_set_option(dashlib.OPT_ACCESS_FORM, old)
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    ref = oracle.deform_fwd(g, oracle.Points(*coords, idx=idx), table.astype(np.float64), mlpc.d_hidden,
                            mlpc.d_out, params.astype(np.float64))
    assert rel_err(outs[0][0].numpy()[:, :n], ref) < 1e-3


@pytest.mark.parametrize("coord", [False, True])
def test_backward_device_count_broadcast_t(dashlib, coord):
    """Fused forward + backward through an index list whose live length is
    an odd device count below the capacity, with one broadcast timestamp:
    the lane-paired gathers, scatter, coordinate gradient and (without the
    coordinate gradient) the Eq. 11 kernel against the oracle."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(81)
    n_all, cap, live = 9000, 4001, 2999
    g = oracle_grid(grid)
    x, y, z, _ = synth.scene_coords(rng, n_all)
    t = np.array([0.37], dtype=np.float32)
    idx = np.sort(rng.choice(n_all, size=cap, replace=False)).astype(np.int32)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    dd = synth.upstream_grad(rng, mlpc.d_out, cap)
    zero_ambiguous(dd, g, oracle.Points(x, y, z, t, idx=idx[:live], t_stride=0), table, params, 64, 10)
    lay = dashlib.layout_from(grid)
    cnt = torch.tensor([live], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), idx=to_dev(idx), n=cap, n_dev=cnt)
    assert pts.t_stride == 0
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, cap, "cuda")
    delta = dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st).cpu().numpy()
    tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    lam, es, et = (0.0, (0.0,) * 3, 0.0) if coord else (0.6, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300)
    cg = torch.full((4, cap), 7.0, dtype=torch.float32, device="cuda") if coord else None
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st,
                                smooth=None if coord else (lam, es, et, loss), coord_grad=cg)
    opts = oracle.Points(x, y, z, t, idx=idx[:live], t_stride=0)
    ref = oracle.deform_fwd(g, opts, table.astype(np.float64), 64, 10, params.astype(np.float64))
    assert rel_err(delta[:, :live], ref) < 1e-3
    rtg, rpg, rl = oracle.deform_bwd(g, opts, table.astype(np.float64), 64, 10, params.astype(np.float64),
                                     dd[:, :live].astype(np.float64), lam, es, et)
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-2 and rel_err(pg.cpu().numpy(), rpg) < 1e-2
    if coord:
        fh = oracle.encode(g, opts, table.astype(np.float64))
        dfh, _ = oracle.mlp_bwd(32, 64, 10, params.astype(np.float64), fh, dd[:, :live].astype(np.float64))
        rcg = oracle.encode_coord_grad(g, opts, table.astype(np.float64), dfh)
        c = cg.cpu().numpy()
        for ax in range(4):
            assert rel_err(c[ax, :live], rcg[ax]) < 1e-2, ax
        assert np.all(c[:, live:] == 7.0)
    else:
        assert abs(float(loss.item()) - rl) <= 1e-2 * abs(rl)


@pytest.mark.parametrize("n", [1, 2, 129])
def test_fused_backward_tiny_and_ragged(dashlib, n):
    """One Gaussian (a lane pair with one member), one pair, and one past a
    128-row tile: forward and backward (+ Eq. 11) against the oracle."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    errs = _grad_errors(dashlib, grid, mlpc, n, np.float16, 90 + n, True,
                        smooth=(0.5, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300))
    assert all(v < 1e-2 for v in errs.values()), errs


@pytest.mark.parametrize("how", ["host", "device"])
def test_fused_empty_is_a_no_op(dashlib, how):
    """n = 0 on the host, or a device count of 0 under a capacity of 500:
    the forward writes nothing, the backward (with Eq. 11, and again with
    the coordinate gradient) adds nothing, the loss stays 0."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    g, coords, _, table, params, dd = _case(grid, mlpc, 500, np.float16, 95)
    lay = dashlib.layout_from(grid)
    x, y, z, t = (to_dev(c) for c in coords)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    pts = dashlib.Points(x, y, z, t, n=0) if how == "host" else dashlib.Points(x, y, z, t, n=500, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    out = torch.full((10, 500), 5.0, device="cuda")
    st = dashlib.deform_state(mlp, 500, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, delta_out=out, fwd_state=st)
    tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ddev = to_dev(dd)
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, ddev, tg, pg, fwd_state=st,
                                smooth=(1.0, (1 / 2048,) * 3, 1 / 300, loss))
    cg = torch.full((4, 500), 3.0, device="cuda")
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, ddev, tg, pg, fwd_state=st, coord_grad=cg)
    torch.cuda.synchronize()
    assert torch.all(out == 5.0) and torch.all(cg == 3.0)
    assert not torch.any(tg) and not torch.any(pg) and float(loss.item()) == 0.0


@pytest.mark.parametrize("tdtype", [np.float16, np.float32])
@pytest.mark.parametrize("smooth_on", [False, True])
@pytest.mark.parametrize("replicas", [0, 7, 16])
def test_backward_workspace_forms_agree(dashlib, tdtype, smooth_on, replicas):
    """The backward with and without its workspace: the gradient replicas
    of the dense levels (k = 0 / 7 / 16) and, with the Eq. 11 term, the
    hand-over of dL/df_h to the Eq. 11 kernel.  Same gradients up to the
    order of the additions and the same loss, through an index list whose
    device count (2999) is below the capacity (4001, the workspace's row
    stride), into gradient buffers that already hold values; against the
    oracle too; a workspace one byte short is refused."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(97)
    n_all, cap, live = 9000, 4001, 2999
    g = oracle_grid(grid)
    x, y, z, t = synth.scene_coords(rng, n_all)
    idx = np.sort(rng.choice(n_all, size=cap, replace=False)).astype(np.int32)
    table = synth.table_values(rng, g.total, grid.F, tdtype)
    params = synth.mlp_params(rng, mlpc)
    dd_h = synth.upstream_grad(rng, mlpc.d_out, cap)
    zero_ambiguous(dd_h, g, oracle.Points(x, y, z, t, idx=idx[:live]), table, params, 64, 10)
    dd = to_dev(dd_h)
    tg0 = rng.standard_normal((g.total, 2)).astype(np.float32)
    lay = dashlib.layout_from(grid)
    cnt = torch.tensor([live], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), idx=to_dev(idx), n=cap, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, cap, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    es, et = (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300
    lam = 0.8 if smooth_on else 0.0
    old = dashlib.dash_get_option(dashlib.OPT_GRAD_REPLICAS)
    dashlib.dash_set_option(dashlib.OPT_GRAD_REPLICAS, replicas)
    try:
        out = []
        for use_ws in (True, False):
            tg = to_dev(tg0)
            pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
            sm = (lam, es, et, loss)
            ws = None
            if use_ws:
                size = dashlib.dash_deform_bwd_workspace_size(lay, cap, sm)
                assert size > 0 or (replicas < 2 and not smooth_on)
                ws = torch.full((max(size, 1),), 255, dtype=torch.uint8, device="cuda")  # not zeroed
            for _ in range(2):  # a second call adds the same gradients again
                dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd, tg, pg, fwd_state=st, smooth=sm,
                                            ws=ws if use_ws else False)
            out.append((tg.cpu().numpy() - tg0, pg.cpu().numpy(), float(loss.item())))
        (tg1, pg1, l1), (tg2, pg2, l2) = out
        # the buffers started from nonzero values: their differences are
        # compared without the touched-entry check (gpu_helpers.rel_err)
        assert rel_err(tg1, tg2, touched=False) < 1e-5 and rel_err(pg1, pg2) < 1e-6
        assert abs(l1 - l2) <= 1e-6 * max(abs(l2), 1e-30)
        opts = oracle.Points(x, y, z, t, idx=idx[:live])
        rtg, _, rl = oracle.deform_bwd(g, opts, table.astype(np.float64), 64, 10, params.astype(np.float64),
                                       dd[:, :live].cpu().numpy().astype(np.float64), lam, es, et)
        assert rel_err(tg1, 2 * rtg, touched=False) < 1e-2 and abs(l1 - 2 * rl) <= 1e-2 * max(abs(rl), 1e-30)
        size = dashlib.dash_deform_bwd_workspace_size(lay, cap, (lam, es, et, None))
        if size > 0:
            short = torch.empty(size - 1, dtype=torch.uint8, device="cuda")
            with pytest.raises(dashlib.DashError) as e:
                dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd, tg, pg, fwd_state=st,
                                            smooth=(lam, es, et, None), ws=short)
            assert e.value.status == dashlib.ERR_WORKSPACE
    finally:
        dashlib.dash_set_option(dashlib.OPT_GRAD_REPLICAS, old)



def test_backward_replicas_under_contention(dashlib):
    """Gaussians sorted by position with one broadcast t, so neighbouring
    lanes and CTAs reduce into the same coarse entries: the backward with
    the gradient replicas equals the one without (up to the order of the
    additions) and the oracle."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(99)
    n = 40_000
    g = oracle_grid(grid)
    x, y, z, _ = synth.scene_coords(rng, n)
    order = np.lexsort((z, y, x))
    x, y, z = x[order], y[order], z[order]
    t = np.array([0.41], dtype=np.float32)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    dd = synth.upstream_grad(rng, mlpc.d_out, n)
    zero_ambiguous(dd, g, oracle.Points(x, y, z, t, t_stride=0), table, params, 64, 10)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), n=n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    out = []
    for ws in (None, False):
        tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
        pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st, ws=ws)
        out.append(tg.cpu().numpy())
    assert rel_err(out[0], out[1]) < 1e-5
    rtg, _, _ = oracle.deform_bwd(g, oracle.Points(x, y, z, t, t_stride=0), table.astype(np.float64), 64, 10,
                                  params.astype(np.float64), dd.astype(np.float64))
    assert rel_err(out[0], rtg) < 1e-2
    dense = slice(0, int(lay.offset[2]) * 2)  # levels 0-1, the replicated ones
    assert rel_err(out[0].reshape(-1)[dense], rtg.reshape(-1)[dense]) < 1e-2


def test_device_status_after_fused_and_batched_runs(dashlib):
    """The bounded waits of the persistent kernels never give up on valid
    work: after a fused forward + backward and a batched plan the device
    flag words read clear (dash_device_status raises on a set flag)."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    g, coords, _, table, params, dd = _case(grid, mlpc, 3000, np.float16, 101)
    lay = dashlib.layout_from(grid)
    pts = _dev_points(dashlib, coords, None, 3000)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, 3000, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st)
    dashlib.dash_device_status()
    x, y, z, t = (to_dev(c) for c in coords)
    scenes = [{"table": tab, "params": to_dev(params), "x": x, "y": y, "z": z, "timestamps": t[:2].contiguous(),
               "delta_out": torch.empty((2, mlpc.d_out, 3000), device="cuda")}]
    plan = dashlib.BatchPlan(lay, scenes)
    plan.run()
    dashlib.dash_device_status()
    plan.close()
