"""Fused deformation forward/backward across the grid and decoder shapes the
library accepts (F in {1, 2, 4, 8}, L*F up to 64, 1 <= O <= 16), in the
warp-specialised and the single-group kernel forms, against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu

SHAPES = [  # L, F, log2_T, N_s range, N_t range, O
    (8, 4, 16, (8, 512), (4, 64), 10),
    (4, 8, 14, (16, 128), (8, 32), 10),
    (16, 1, 18, (16, 1024), (8, 100), 10),
    (32, 2, 18, (4, 2048), (2, 150), 10),
    (3, 1, 12, (5, 40), (3, 9), 16),
    (12, 4, 17, (16, 1024), (8, 120), 3),
]


def _case(shape, n, tdtype, seed):
    L, F, lt, (a, b), (c, d), O = shape
    grid = synth.GridCfg(L=L, F=F, log2_T=lt, nmin_s=a, nmax_s=b, nmin_t=c, nmax_t=d)
    mlpc = synth.MlpCfg(d_in=L * F, d_hidden=64, d_out=O)
    rng = np.random.default_rng(seed)
    g = oracle.layout(L, F, lt, a, b, c, d)
    coords = synth.scene_coords(rng, n)
    table = synth.table_values(rng, g.total, F, tdtype)
    params = synth.mlp_params(rng, mlpc)
    dd = synth.upstream_grad(rng, O, n)
    zero_ambiguous(dd, g, oracle.Points(*coords), table, params, 64, O)
    return grid, mlpc, g, coords, table, params, dd


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"L{s[0]}F{s[1]}O{s[5]}" for s in SHAPES])
def test_fused_forward_and_backward_across_shapes(dashlib, shape, form):
    n = 2333
    tdtype = np.float16 if shape[1] in (2, 4) else np.float32
    grid, mlpc, g, coords, table, params, dd = _case(shape, n, tdtype, seed=100 + SHAPES.index(shape))
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(*(to_dev(c) for c in coords))
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, 64, mlpc.d_out)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    old_f, old_b = dashlib.dash_get_option(dashlib.OPT_FWD_FORM), dashlib.dash_get_option(dashlib.OPT_BWD_FORM)
    try:
        dashlib.dash_set_option(dashlib.OPT_FWD_FORM, form)
        dashlib.dash_set_option(dashlib.OPT_BWD_FORM, form)
        delta = dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st).cpu().numpy()
        tg = torch.zeros((g.total, shape[1]), device="cuda")
        pg = torch.zeros(mlpc.n_params, device="cuda")
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=st)
    finally:
        dashlib.dash_set_option(dashlib.OPT_FWD_FORM, old_f)
        dashlib.dash_set_option(dashlib.OPT_BWD_FORM, old_b)
    opts = oracle.Points(*coords)
    ref = oracle.deform_fwd(g, opts, table.astype(np.float64), 64, mlpc.d_out, params.astype(np.float64))
    assert rel_err(delta[:, :n], ref) < 1e-3
    rtg, rpg, _ = oracle.deform_bwd(g, opts, table.astype(np.float64), 64, mlpc.d_out, params.astype(np.float64),
                                    dd.astype(np.float64))
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-2
    D, H, O = mlpc.d_in, 64, mlpc.d_out
    bounds = np.cumsum([0, H * D, H, H * H, H, O * H, O])
    pgn = pg.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert rel_err(pgn[a:b], rpg[a:b]) < 1e-2, (a, b)
