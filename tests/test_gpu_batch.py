"""GPU checks of the batched persistent form (a12): many scenes with uneven
dynamic counts x many timestamps in one CUDA-graph launch.  Each (scene,
timestamp) must equal the single-scene fused forward bit for bit, and the
FP64 oracle within 1e-3; with the backward, each scene's gradients must
equal the single-scene backward summed over its timestamps (up to the order
of the additions) and the oracle within 1e-2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import oracle_grid, rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu


def _scenes(dashlib, grid, mlpc, counts, Ks, tdtype, seed):
    rng = np.random.default_rng(seed)
    g = oracle_grid(grid)
    out = []
    for n, K in zip(counts, Ks):
        x, y, z, _ = synth.scene_coords(rng, n)
        f = np.sort(rng.choice(300, size=K, replace=False))
        ts = (f / 299).astype(np.float32)
        table = synth.table_values(rng, g.total, grid.F, tdtype)
        params = synth.mlp_params(rng, mlpc)
        out.append({"np": (x, y, z, ts, table, params),
                    "table": to_dev(table), "params": to_dev(params), "x": to_dev(x), "y": to_dev(y),
                    "z": to_dev(z), "timestamps": to_dev(ts),
                    "delta_out": torch.full((K, mlpc.d_out, n), 7.0, device="cuda")})
    return g, out


def test_batched_matches_single_scene_and_oracle(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [5000, 300, 129, 1], [3, 2, 4, 1]
    g, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float16, 51)
    lay = dashlib.layout_from(grid)
    plan = dashlib.BatchPlan(lay, scenes)
    plan.run()
    torch.cuda.synchronize()
    for sc, n, K in zip(scenes, counts, Ks):
        x, y, z, ts, table, params = sc["np"]
        mlp = dashlib.Mlp(sc["params"], mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
        for k in range(K):
            pts = dashlib.Points(sc["x"], sc["y"], sc["z"], sc["timestamps"][k:k + 1].contiguous(), n=n)
            single = dashlib.dash_deform_mlp_fwd(lay, pts, sc["table"], mlp)
            assert torch.equal(sc["delta_out"][k], single), (n, k)
        ref = oracle.deform_fwd(g, oracle.Points(x, y, z, ts[-1:], t_stride=0), table.astype(np.float64),
                                mlpc.d_hidden, mlpc.d_out, params.astype(np.float64))
        assert rel_err(sc["delta_out"][K - 1].cpu().numpy(), ref) < 1e-3
    plan.close()


def test_batched_device_counts_and_graph_replay(dashlib):
    grid, mlpc = synth.TINY_GRID, synth.TINY_MLP
    counts, Ks = [3000, 1000], [2, 3]
    g, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float32, 52)
    lay = dashlib.layout_from(grid)
    plan = dashlib.BatchPlan(lay, scenes, d_in=mlpc.d_in)
    # shrink the live counts on the device, replay the same graph
    plan.counts().copy_(torch.tensor([1500, 0], dtype=torch.int64, device="cuda"))
    plan.run()
    torch.cuda.synchronize()
    d0, d1 = scenes[0]["delta_out"].cpu().numpy(), scenes[1]["delta_out"].cpu().numpy()
    assert np.all(d0[:, :, 1500:] == 7.0) and np.all(d1 == 7.0)
    x, y, z, ts, table, params = scenes[0]["np"]
    for k in range(2):
        ref = oracle.deform_fwd(g, oracle.Points(x[:1500], y[:1500], z[:1500], ts[k:k + 1], t_stride=0),
                                table.astype(np.float64), mlpc.d_hidden, mlpc.d_out, params.astype(np.float64))
        assert rel_err(d0[k, :, :1500], ref) < 1e-3
    # grow them back to the capacity
    plan.counts().copy_(torch.tensor(counts, dtype=torch.int64, device="cuda"))
    plan.run()
    torch.cuda.synchronize()
    assert not np.any(scenes[1]["delta_out"].cpu().numpy() == 7.0)
    plan.close()


def test_batched_autotune_and_cache(dashlib, tmp_path):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [20_000, 7_000], [4, 4]
    _, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float16, 53)
    lay = dashlib.layout_from(grid)
    plan = dashlib.BatchPlan(lay, scenes)
    plan.run()
    torch.cuda.synchronize()
    before = [sc["delta_out"].clone() for sc in scenes]
    cache = tmp_path / "tune.json"
    form = plan.autotune(cache)
    assert 0 <= form < 6 and cache.exists()     # six compiled forward forms
    plan.run()
    torch.cuda.synchronize()
    for sc, b in zip(scenes, before):
        assert torch.equal(sc["delta_out"], b)  # every form computes the same result
    plan2 = dashlib.BatchPlan(lay, scenes)
    assert plan2.autotune(cache) == form     # taken from the cache
    plan.close()
    plan2.close()


def _with_backward(scenes, lay, O, rng, g=None):
    """Upstream gradients and zeroed gradient buffers per scene; given the
    oracle grid g, the (timestamp, Gaussian) pairs whose ReLU decisions are
    ambiguous get a zero upstream gradient (gpu_helpers.RELU_MARGIN)."""
    for sc in scenes:
        K, n = sc["delta_out"].shape[0], sc["x"].numel()
        sc["dd_np"] = rng.standard_normal((K, O, n)).astype(np.float32)
        if g is not None:
            x, y, z, ts, table, params = sc["np"]
            for k in range(K):
                zero_ambiguous(sc["dd_np"][k], g, oracle.Points(x, y, z, ts[k:k + 1], t_stride=0), table, params,
                               64, O)
        sc["ddelta"] = to_dev(sc["dd_np"])
        sc["table_grad"] = torch.zeros((lay.total, 2), dtype=torch.float32, device="cuda")
        sc["mlp_grad"] = torch.zeros(sc["params"].numel(), dtype=torch.float32, device="cuda")


def _single_scene_grads(dashlib, lay, mlpc, sc, n, K, ks=None):
    """The single-scene fused forward + backward at each timestamp, summed."""
    mlp = dashlib.Mlp(sc["params"], mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    tg = torch.zeros_like(sc["table_grad"])
    pg = torch.zeros_like(sc["mlp_grad"])
    for k in (range(K) if ks is None else ks):
        pts = dashlib.Points(sc["x"], sc["y"], sc["z"], sc["timestamps"][k:k + 1].contiguous(), n=n)
        st = dashlib.deform_state(mlp, n, "cuda")
        dashlib.dash_deform_mlp_fwd(lay, pts, sc["table"], mlp, fwd_state=st)
        dashlib.dash_deform_mlp_bwd(lay, pts, sc["table"], mlp, sc["ddelta"][k, :, :n].contiguous(), tg, pg,
                                    fwd_state=st)
    return tg, pg


def test_batched_backward_matches_single_scene_and_oracle(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [5000, 300, 129, 1], [3, 2, 4, 1]
    g, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float16, 54)
    lay = dashlib.layout_from(grid)
    _with_backward(scenes, lay, mlpc.d_out, np.random.default_rng(55), g)
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    plan.run()
    torch.cuda.synchronize()
    for sc, n, K in zip(scenes, counts, Ks):
        mlp = dashlib.Mlp(sc["params"], mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
        for k in range(K):  # the forward is unchanged by the backward
            pts = dashlib.Points(sc["x"], sc["y"], sc["z"], sc["timestamps"][k:k + 1].contiguous(), n=n)
            assert torch.equal(sc["delta_out"][k], dashlib.dash_deform_mlp_fwd(lay, pts, sc["table"], mlp))
        tg, pg = _single_scene_grads(dashlib, lay, mlpc, sc, n, K)
        assert rel_err(sc["table_grad"].cpu().numpy(), tg.cpu().numpy()) < 1e-5, n
        assert rel_err(sc["mlp_grad"].cpu().numpy(), pg.cpu().numpy()) < 1e-5, n
    # the oracle, for the largest scene, summed over its timestamps
    x, y, z, ts, table, params = scenes[0]["np"]
    rtg = np.zeros((g.total, 2))
    rpg = np.zeros(params.size)
    for k in range(Ks[0]):
        oracle.deform_bwd(g, oracle.Points(x, y, z, ts[k:k + 1], t_stride=0), table.astype(np.float64),
                          mlpc.d_hidden, mlpc.d_out, params.astype(np.float64),
                          scenes[0]["dd_np"][k].astype(np.float64), table_grad=rtg, param_grad=rpg)
    assert rel_err(scenes[0]["table_grad"].cpu().numpy(), rtg) < 1e-2
    assert rel_err(scenes[0]["mlp_grad"].cpu().numpy(), rpg) < 1e-2
    plan.close()


def test_batched_backward_device_counts_and_replay(dashlib):
    """Live counts below the capacity (one scene empty) replayed through the
    captured graph: only live Gaussians contribute; a second replay adds the
    same gradients again."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [3001, 700, 400], [2, 3, 1]
    _, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float32, 56)
    lay = dashlib.layout_from(grid)
    _with_backward(scenes, lay, mlpc.d_out, np.random.default_rng(57))
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    live = [1999, 0, 400]
    plan.counts().copy_(torch.tensor(live, dtype=torch.int64, device="cuda"))
    plan.run()
    plan.run()
    torch.cuda.synchronize()
    for sc, n, K in zip(scenes, live, Ks):
        if n == 0:
            assert not torch.any(sc["table_grad"]) and not torch.any(sc["mlp_grad"])
            continue
        tg, pg = _single_scene_grads(dashlib, lay, mlpc, sc, n, K)
        assert rel_err(sc["table_grad"].cpu().numpy(), 2 * tg.cpu().numpy()) < 1e-5, n
        assert rel_err(sc["mlp_grad"].cpu().numpy(), 2 * pg.cpu().numpy()) < 1e-5, n
    plan.close()


def test_batched_backward_rejects_unsupported(dashlib):
    """F = 4 tables have no batched backward: plan creation reports it."""
    grid = synth.GridCfg(L=4, F=4, log2_T=14, nmin_s=16, nmax_s=128, nmin_t=8, nmax_t=32)
    mlpc = synth.MlpCfg(d_in=16, d_hidden=64, d_out=10)
    _, scenes = _scenes(dashlib, grid, mlpc, [100], [1], np.float32, 58)
    lay = dashlib.layout_from(grid)
    _with_backward(scenes, lay, mlpc.d_out, np.random.default_rng(59))
    with pytest.raises(dashlib.DashError):
        dashlib.BatchPlan(lay, scenes, d_in=16, backward=True)
    dashlib.BatchPlan(lay, scenes, d_in=16).close()  # the forward alone is supported


def test_batched_backward_autotune_keeps_gradients(dashlib, tmp_path):
    """Tuning the backward forms runs the backward several times; the
    caller's gradient buffers must come out as they went in, and the chosen
    forms must compute the same gradients."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [20_000, 3_000], [3, 2]
    _, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float16, 60)
    lay = dashlib.layout_from(grid)
    _with_backward(scenes, lay, mlpc.d_out, np.random.default_rng(61))
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    plan.run()
    torch.cuda.synchronize()
    once = [(sc["table_grad"].clone(), sc["mlp_grad"].clone()) for sc in scenes]
    cache = tmp_path / "tune.json"
    code = plan.autotune(cache)
    torch.cuda.synchronize()
    assert 0 <= code % 16 < 6 and 0 <= code // 16 < 5 and cache.exists()  # 6 forward, 5 backward forms
    for sc, (tg, pg) in zip(scenes, once):
        assert torch.equal(sc["table_grad"], tg) and torch.equal(sc["mlp_grad"], pg)
        sc["table_grad"].zero_()
        sc["mlp_grad"].zero_()
    plan.run()
    torch.cuda.synchronize()
    for sc, (tg, pg) in zip(scenes, once):
        assert rel_err(sc["table_grad"].cpu().numpy(), tg.cpu().numpy()) < 1e-5
        assert rel_err(sc["mlp_grad"].cpu().numpy(), pg.cpu().numpy()) < 1e-5
    plan2 = dashlib.BatchPlan(lay, scenes, backward=True)
    assert plan2.autotune(cache) == code     # taken from the cache
    fwd_only = dashlib.BatchPlan(lay, scenes)
    assert fwd_only.autotune(cache) < 16     # its own entry, forward forms only
    plan.close()
    plan2.close()
    fwd_only.close()


@pytest.mark.parametrize("k", [0, 5])
def test_batched_backward_replica_counts_agree(dashlib, k):
    """Batched plans created with k gradient replicas per scene (0 = none,
    5 = an odd count) give the gradients of the default plan (8) up to the
    order of the additions."""
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    counts, Ks = [7000, 2500], [2, 3]
    _, scenes = _scenes(dashlib, grid, mlpc, counts, Ks, np.float16, 62)
    lay = dashlib.layout_from(grid)
    _with_backward(scenes, lay, mlpc.d_out, np.random.default_rng(63))
    old = dashlib.dash_get_option(dashlib.OPT_GRAD_REPLICAS)
    out = []
    try:
        for kk in (old, k):
            dashlib.dash_set_option(dashlib.OPT_GRAD_REPLICAS, kk)
            for sc in scenes:
                sc["table_grad"].zero_()
                sc["mlp_grad"].zero_()
            plan = dashlib.BatchPlan(lay, scenes, backward=True)
            plan.run()
            torch.cuda.synchronize()
            out.append([(sc["table_grad"].cpu().numpy(), sc["mlp_grad"].cpu().numpy()) for sc in scenes])
            plan.close()
    finally:
        dashlib.dash_set_option(dashlib.OPT_GRAD_REPLICAS, old)
    for (tg1, pg1), (tg2, pg2) in zip(*out):
        assert rel_err(tg2, tg1) < 1e-5 and rel_err(pg2, pg1) < 1e-6
