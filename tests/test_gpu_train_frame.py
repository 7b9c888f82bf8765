"""One training frame through every GPU stage: compaction -> fused
deformation forward with Eq. 10 applied -> splatting -> splatting backward
-> Eq. 10 backward (gather) -> fused deformation backward, against the same
chain in the oracles (renderer autograd at the FP64-deformed attributes,
then the FP64 deformation backward), down to the hash-table and decoder
gradients."""
import numpy as np
import pytest
import torch

import oracle
from oracle import raster as oraster
from paper_2507_19141_gb300 import synth
from gpu_helpers import norm_err, oracle_grid, rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu


def test_apply_backward_gathers_dynamic_rows(dashlib):
    rng = np.random.default_rng(110)
    n_all = 10_001
    mask = synth.bernoulli_mask(rng, n_all, 0.3)
    idx, cnt = dashlib.dash_compact_dynamic(to_dev(mask))
    x = to_dev(rng.random(n_all).astype(np.float32))
    pts = dashlib.Points(x, x, x, x, idx=idx, n=n_all, n_dev=cnt)
    dattrs = rng.standard_normal((10, n_all)).astype(np.float32)
    out = torch.full((10, n_all), 9.0, device="cuda")
    dashlib.dash_deform_apply_bwd(pts, to_dev(dattrs), ddelta=out)
    c = int(cnt.item())
    ridx = np.flatnonzero(mask)
    assert c == len(ridx)
    assert np.array_equal(out[:, :c].cpu().numpy(), dattrs[:, ridx])
    assert np.all(out[:, c:].cpu().numpy() == 9.0)


def test_training_frame_gradients_match_oracle_chain(dashlib):
    rng = np.random.default_rng(111)
    n, w, h = 1200, 112, 80
    cam, g = synth.raster_scene(rng, n, w, h)
    mask = synth.bernoulli_mask(rng, n)
    lo, hi = g["mean"].min(1, keepdims=True), g["mean"].max(1, keepdims=True)
    nc = ((g["mean"] - lo) / (hi - lo)).astype(np.float32)
    t = np.array([0.61], np.float32)
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    gg = oracle_grid(grid)
    table = synth.table_values(rng, gg.total, 2, np.float16)
    params = synth.mlp_params(rng, mlpc)
    params[64 * 32 + 64 + 64 * 64 + 64:] *= 1e-2
    attrs = np.concatenate([g["mean"], g["rot"], g["scale"]], 0).astype(np.float32)
    dimg = rng.standard_normal((3, h, w)).astype(np.float32)
    # GPU
    lay = dashlib.layout_from(grid)
    idx, cnt = dashlib.dash_compact_dynamic(to_dev(mask))
    pts = dashlib.Points(to_dev(nc[0]), to_dev(nc[1]), to_dev(nc[2]), to_dev(t), idx=idx, n=n, n_dev=cnt)
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 10)
    tab = to_dev(table)
    st = dashlib.deform_state(mlp, n, "cuda")
    a_in = to_dev(attrs)
    a_out = a_in.clone()
    dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st, apply=(a_in, a_out))
    G = dashlib.Gaussians(a_out[0:3], a_out[7:10], a_out[3:7], to_dev(g["opacity"]), to_dev(g["sh"]), 3)
    c = dashlib.camera(cam["view"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], w, h, cam["near"], cam["dilation"],
                       cam["campos"], cam["bg"])
    _, ws, cap, _ = dashlib.dash_raster_fwd(c, G)
    d10 = torch.zeros((10, n), device="cuda")           # gradients in the attribute layout x | r | s
    grads = {"mean": d10[0:3], "rot": d10[3:7], "scale": d10[7:10], "opacity": torch.zeros(n, device="cuda"),
             "sh": torch.zeros((n, 16, 3), device="cuda")}
    dashlib.dash_raster_bwd(c, G, to_dev(dimg), ws, cap, grads)
    ddelta = dashlib.dash_deform_apply_bwd(pts, d10)
    tg = torch.zeros((gg.total, 2), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, ddelta, tg, pg, fwd_state=st)
    # oracle chain
    ridx, _ = oracle.compact(mask)
    opts = oracle.Points(nc[0], nc[1], nc[2], t, idx=ridx, t_stride=0)
    _, ref_attrs = oracle.deform_fwd(gg, opts, table.astype(np.float64), 64, 10, params.astype(np.float64), attrs)
    ra = torch.tensor(ref_attrs, requires_grad=True)
    img, _, _ = oraster.render(cam, ra[0:3].T, ra[7:10].T, ra[3:7].T, torch.tensor(g["opacity"].astype(np.float64)),
                               torch.tensor(g["sh"].astype(np.float64)), 3)
    (img * torch.tensor(dimg.astype(np.float64))).sum().backward()
    rdd = ra.grad.numpy()[:, ridx]
    # the renderer's gradient is compared normwise: its discrete decisions
    # (alpha below 1/255, the stop at T < 1e-4) may fall the other way in FP32
    # for a few Gaussians, which changes their whole gradient
    gdd = ddelta[:, :len(ridx)].cpu().numpy()
    assert norm_err(gdd, rdd) < 2e-3
    # the whole chain normwise against the oracle chain
    args = (gg, opts, table.astype(np.float64), 64, 10, params.astype(np.float64))
    ctg, cpg, _ = oracle.deform_bwd(*args, rdd)
    assert norm_err(tg.cpu().numpy(), ctg) < 1e-2
    bounds = np.cumsum([0, 64 * 32, 64, 64 * 64, 64, 10 * 64, 10])
    pgn = pg.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert norm_err(pgn[a:b], cpg[a:b]) < 1e-2, (a, b)
    # the deformation backward element-wise on the upstream gradient the GPU
    # chain produced, with the Gaussians whose ReLU decisions are ambiguous
    # left out (gpu_helpers.RELU_MARGIN): run again on the GPU, and the oracle
    gdd = np.ascontiguousarray(gdd)
    zero_ambiguous(gdd, gg, opts, table, params, 64, 10)
    dd2 = torch.zeros_like(ddelta)
    dd2[:, :len(ridx)] = to_dev(gdd)
    tg2 = torch.zeros_like(tg)
    pg2 = torch.zeros_like(pg)
    dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd2, tg2, pg2, fwd_state=st)
    rtg, rpg, _ = oracle.deform_bwd(*args, gdd.astype(np.float64))
    assert rel_err(tg2.cpu().numpy(), rtg) < 1e-2
    pgn2 = pg2.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert rel_err(pgn2[a:b], rpg[a:b]) < 1e-2, (a, b)
