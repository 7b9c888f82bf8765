"""GPU parity of the input-coordinate gradient d/d(x, y, z, t) (Eq. 9
differentiated through its weights): the encoder-level entry point and the
optional output of the fused backward, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import edge_coords, oracle_grid, rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu


def _per_axis_err(got, ref):
    return max(rel_err(got[a], ref[a]) for a in range(4))


@pytest.mark.parametrize("grid,n,tdtype,broadcast_t,with_idx", [
    (synth.TINY_GRID, 10_000, np.float32, False, False),
    (synth.PAPER_GRID, 20_000, np.float16, False, True),
    (synth.PAPER_GRID, 20_000, np.float32, True, False),
    (synth.PAPER_GRID, 333, np.float16, False, True),
    (synth.PAPER_GRID, 1, np.float16, False, False),
])
def test_encoder_coord_grad_matches_oracle(dashlib, grid, n, tdtype, broadcast_t, with_idx):
    rng = np.random.default_rng(81 + n)
    g = oracle_grid(grid)
    n_all = 2 * n + 7 if with_idx else n
    x, y, z, t = edge_coords(n_all, rng)
    if broadcast_t:
        t = np.array([0.4375], np.float32)
    idx = np.sort(rng.choice(n_all, size=n, replace=False)).astype(np.int32) if with_idx else None
    table = synth.table_values(rng, g.total, grid.F, tdtype)
    dfeat = rng.standard_normal((n, grid.L * grid.F)).astype(np.float32)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), idx=None if idx is None else to_dev(idx), n=n)
    got = dashlib.dash_hash4d_coord_grad(lay, pts, to_dev(table), to_dev(dfeat)).cpu().numpy()
    ref = oracle.encode_coord_grad(g, oracle.Points(x, y, z, t, idx=idx, t_stride=0 if broadcast_t else 1),
                                   table.astype(np.float64), dfeat.astype(np.float64))
    assert _per_axis_err(got, ref) < 1e-5
    assert np.array_equal(got == 0.0, ref == 0.0) or _per_axis_err(got, ref) < 1e-6  # blocked axes are exact zeros


def test_encoder_coord_grad_device_count(dashlib):
    """With a device count only the live prefix is written."""
    grid = synth.PAPER_GRID
    rng = np.random.default_rng(82)
    g = oracle_grid(grid)
    x, y, z, t = synth.scene_coords(rng, 4000)
    table = synth.table_values(rng, g.total, 2, np.float16)
    dfeat = rng.standard_normal((4000, 32)).astype(np.float32)
    cnt = torch.tensor([2500], dtype=torch.int64, device="cuda")
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), n=4000, n_dev=cnt)
    out = torch.full((4, 4000), 7.0, device="cuda")
    dashlib.dash_hash4d_coord_grad(dashlib.layout_from(grid), pts, to_dev(table), to_dev(dfeat), out=out)
    o = out.cpu().numpy()
    ref = oracle.encode_coord_grad(g, oracle.Points(x[:2500], y[:2500], z[:2500], t[:2500]), table.astype(np.float64),
                                   dfeat[:2500].astype(np.float64))
    assert _per_axis_err(o[:, :2500], ref) < 1e-5
    assert np.all(o[:, 2500:] == 7.0)


@pytest.mark.parametrize("form,use_state", [(0, True), (1, True), (0, False)])
def test_fused_backward_coord_grad_matches_oracle(dashlib, form, use_state):
    """d loss / d(x, y, z, t) through decoder and encoder, from the fused
    backward, against oracle encode -> decoder backward -> coordinate gradient."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(83)
    g = oracle_grid(grid)
    n_all, n = 9000, 4000
    x, y, z, t = synth.scene_coords(rng, n_all)
    x[:5] = [0.0, 1.0, -0.2, 1.2, np.nan]
    idx = np.sort(rng.choice(n_all, size=n, replace=False)).astype(np.int32)
    idx[:5] = np.arange(5)
    idx = np.sort(idx)
    table = synth.table_values(rng, g.total, 2, np.float16)
    params = synth.mlp_params(rng, mlpc)
    dd = synth.upstream_grad(rng, mlpc.d_out, n)
    zero_ambiguous(dd, g, oracle.Points(x, y, z, t, idx=idx), table, params, 64, 10)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(to_dev(x), to_dev(y), to_dev(z), to_dev(t), idx=to_dev(idx), n=n)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 10)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    tg = torch.zeros((g.total, 2), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")
    cg = torch.zeros((4, n), device="cuda")
    old = dashlib.dash_get_option(dashlib.OPT_BWD_FORM)
    try:
        dashlib.dash_set_option(dashlib.OPT_BWD_FORM, form)
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st if use_state else None,
                                    coord_grad=cg)
    finally:
        dashlib.dash_set_option(dashlib.OPT_BWD_FORM, old)
    opts = oracle.Points(x, y, z, t, idx=idx)
    feat = oracle.encode(g, opts, table.astype(np.float64))
    dfeat, _ = oracle.mlp_bwd(32, 64, 10, params.astype(np.float64), feat, dd.astype(np.float64))
    ref = oracle.encode_coord_grad(g, opts, table.astype(np.float64), dfeat)
    got = cg.cpu().numpy()
    assert _per_axis_err(got, ref) < 1e-2
    assert np.all(got[0, :5][[2, 3, 4]] == 0.0)   # x outside [0,1] or NaN: the clamp blocks it
    # the table gradient is unchanged by the extra output
    rtg, _, _ = oracle.deform_bwd(g, opts, table.astype(np.float64), 64, 10, params.astype(np.float64),
                                  dd.astype(np.float64))
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-2


def test_fused_backward_coord_grad_rejects_smoothness(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(84)
    g = oracle_grid(grid)
    coords = [to_dev(c) for c in synth.scene_coords(rng, 256)]
    pts = dashlib.Points(*coords)
    mlp = dashlib.Mlp(to_dev(synth.mlp_params(rng, mlpc)), 32, 64, 10)
    tab = to_dev(synth.table_values(rng, g.total, 2, np.float16))
    with pytest.raises(dashlib.DashError) as e:
        dashlib.dash_deform_mlp_bwd(dashlib.layout_from(grid), pts, tab, mlp, torch.zeros((10, 256), device="cuda"),
                                    torch.zeros((g.total, 2), device="cuda"), torch.zeros(mlpc.n_params, device="cuda"),
                                    smooth=(0.1, (1e-3, 1e-3, 1e-3), 1e-3, None),
                                    coord_grad=torch.zeros((4, 256), device="cuda"))
    assert e.value.status == dashlib.ERR_UNSUPPORTED


def test_fused_backward_coord_grad_with_and_without_workspace(dashlib):
    """The coordinate-gradient backward given the binding's default
    workspace and given none: the same table gradients up to the order of
    the additions and the same coordinate gradients (the workspace is not
    used on this path)."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(71)
    n = 6000
    g = oracle_grid(grid)
    coords = synth.scene_coords(rng, n)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    dd = to_dev(synth.upstream_grad(rng, mlpc.d_out, n))
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(*(to_dev(c) for c in coords), n=n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st)
    out = []
    for ws in (None, False):
        tg = torch.zeros((g.total, 2), dtype=torch.float32, device="cuda")
        pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
        cg = torch.zeros((4, n), dtype=torch.float32, device="cuda")
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd, tg, pg, fwd_state=st, coord_grad=cg, ws=ws)
        out.append((tg.cpu().numpy(), cg.cpu().numpy()))
    assert rel_err(out[0][0], out[1][0]) < 1e-5
    assert rel_err(out[0][1], out[1][1]) < 1e-6
