"""The deformation step and a whole training frame capture into one CUDA
graph (no host synchronisation inside any call) and replay with the same
results as eager execution."""
import numpy as np
import pytest
import torch

from paper_2507_19141_gb300 import synth
from gpu_helpers import oracle_grid, rel_err, to_dev

pytestmark = pytest.mark.gpu


def _capture(fn):
    fn()                                   # warm-up outside the capture (kernel attributes, caches)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g


def test_deformation_step_replays_in_a_graph(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(120)
    n_all = 50_000
    gg = oracle_grid(grid)
    mask = to_dev(synth.bernoulli_mask(rng, n_all))
    x, y, z, t = (to_dev(c) for c in synth.scene_coords(rng, n_all))
    lay = dashlib.layout_from(grid)
    tab = to_dev(synth.table_values(rng, gg.total, 2, np.float16))
    mlp = dashlib.Mlp(to_dev(synth.mlp_params(rng, mlpc)), 32, 64, 10)
    dd = to_dev(synth.upstream_grad(rng, 10, n_all))
    idx = torch.empty(n_all, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    ws = torch.empty(dashlib.dash_compact_workspace_size(n_all), dtype=torch.uint8, device="cuda")
    pts = dashlib.Points(x, y, z, t, idx=idx, n=n_all, n_dev=cnt)
    st = dashlib.deform_state(mlp, n_all, "cuda")
    delta = torch.zeros((10, n_all), device="cuda")
    tg = torch.zeros((gg.total, 2), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")

    def step():
        tg.zero_()
        pg.zero_()
        dashlib.dash_compact_dynamic(mask, idx_out=idx, count_out=cnt, ws=ws)
        dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, delta_out=delta, fwd_state=st)
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd, tg, pg, fwd_state=st)

    step()
    torch.cuda.synchronize()
    e_delta, e_tg, e_pg = delta.clone(), tg.clone(), pg.clone()
    delta.zero_()
    g = _capture(step)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    c = int(cnt.item())
    assert torch.equal(delta[:, :c], e_delta[:, :c])
    assert rel_err(tg.cpu().numpy(), e_tg.cpu().numpy()) < 1e-6     # atomics: order may differ
    assert rel_err(pg.cpu().numpy(), e_pg.cpu().numpy()) < 1e-6


def test_training_frame_replays_in_a_graph(dashlib):
    rng = np.random.default_rng(121)
    n, w, h = 4000, 160, 120
    cam, g = synth.raster_scene(rng, n, w, h)
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    gg = oracle_grid(grid)
    lo, hi = g["mean"].min(1, keepdims=True), g["mean"].max(1, keepdims=True)
    nc = ((g["mean"] - lo) / (hi - lo)).astype(np.float32)
    params = synth.mlp_params(rng, mlpc)
    params[64 * 32 + 64 + 64 * 64 + 64:] *= 1e-2
    lay = dashlib.layout_from(grid)
    mask = to_dev(synth.bernoulli_mask(rng, n))
    tab = to_dev(synth.table_values(rng, gg.total, 2, np.float16))
    mlp = dashlib.Mlp(to_dev(params), 32, 64, 10)
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    cws = torch.empty(dashlib.dash_compact_workspace_size(n), dtype=torch.uint8, device="cuda")
    pts = dashlib.Points(to_dev(nc[0]), to_dev(nc[1]), to_dev(nc[2]), to_dev(np.array([0.4], np.float32)), idx=idx,
                         n=n, n_dev=cnt)
    st = dashlib.deform_state(mlp, n, "cuda")
    a_in = to_dev(np.concatenate([g["mean"], g["rot"], g["scale"]], 0).astype(np.float32))
    a_out = a_in.clone()
    G = dashlib.Gaussians(a_out[0:3], a_out[7:10], a_out[3:7], to_dev(g["opacity"]), to_dev(g["sh"]), 3)
    c = dashlib.camera(cam["view"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], w, h, cam["near"], cam["dilation"],
                       cam["campos"], cam["bg"])
    image = torch.empty((3, h, w), device="cuda")
    _, rws, cap, pairs = dashlib.dash_raster_fwd(c, G, image=image)
    dimg = to_dev(rng.standard_normal((3, h, w)).astype(np.float32))
    d10 = torch.zeros((10, n), device="cuda")
    rgr = {"mean": d10[0:3], "rot": d10[3:7], "scale": d10[7:10], "opacity": torch.zeros(n, device="cuda"),
           "sh": torch.zeros((n, 16, 3), device="cuda")}
    ddelta = torch.zeros((10, n), device="cuda")
    tg = torch.zeros((gg.total, 2), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")

    def frame():
        for v in (d10, rgr["opacity"], rgr["sh"], tg, pg):
            v.zero_()
        dashlib.dash_compact_dynamic(mask, idx_out=idx, count_out=cnt, ws=cws)
        dashlib.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=st, apply=(a_in, a_out))
        dashlib.dash_raster_fwd(c, G, image=image, ws=rws, max_pairs=cap, pairs_needed=pairs)
        dashlib.dash_raster_bwd(c, G, dimg, rws, cap, rgr)
        dashlib.dash_deform_apply_bwd(pts, d10, ddelta=ddelta)
        dashlib.dash_deform_mlp_bwd(lay, pts, tab, mlp, ddelta, tg, pg, fwd_state=st)

    frame()
    torch.cuda.synchronize()
    e_img, e_tg, e_pg, e_d10 = image.clone(), tg.clone(), pg.clone(), d10.clone()
    image.zero_()
    gr = _capture(frame)
    for _ in range(2):
        gr.replay()
    torch.cuda.synchronize()
    assert torch.equal(image, e_img)
    for a, b in ((d10, e_d10), (tg, e_tg), (pg, e_pg)):
        assert rel_err(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
