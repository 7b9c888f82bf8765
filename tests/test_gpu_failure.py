"""Failure detection without a GPU fault.

(1) A bounded device-side wait made to run out: dash_selftest_wait waits on
an mbarrier that nothing arrives at, gives up after a short poll bound and
sets its flag; dash_device_status must report DASH_ERR_TIMEOUT once, clear
it, and the context must stay usable (a fused forward afterwards still
matches the oracle).
(2) Host fault injection: every CUDA runtime call that plan creation makes
is failed in turn (dash_debug_fail_cuda_call); each attempt must return
DASH_ERR_CUDA with the injected call named, hand back no plan, and leave no
device memory behind.  Nothing here faults, traps or hangs a GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_19141_gb300 import synth
from gpu_helpers import oracle_grid, rel_err, to_dev, zero_ambiguous

pytestmark = pytest.mark.gpu


def _small_forward_matches_oracle(dashlib, seed):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(seed)
    n = 3000
    coords = synth.scene_coords(rng, n)
    g = oracle_grid(grid)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(*(to_dev(c) for c in coords), n=n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    delta = dashlib.dash_deform_mlp_fwd(lay, pts, to_dev(table), mlp).cpu().numpy()
    ref = oracle.deform_fwd(g, oracle.Points(*coords), table.astype(np.float64), mlpc.d_hidden, mlpc.d_out,
                            params.astype(np.float64))
    assert rel_err(delta, ref) < 1e-3


def test_bounded_wait_runs_out_and_is_reported(dashlib):
    dashlib.dash_device_status()                       # nothing pending
    dashlib.dash_selftest_wait(1000)
    with pytest.raises(dashlib.DashError) as e:
        dashlib.dash_device_status()
    assert e.value.status == dashlib.ERR_TIMEOUT
    assert "gave up" in str(e.value)
    dashlib.dash_device_status()                       # reported once, then cleared
    _small_forward_matches_oracle(dashlib, 131)        # the context is still usable
    dashlib.dash_device_status()
    with pytest.raises(dashlib.DashError) as e:
        dashlib.dash_selftest_wait(0)                  # bound outside [1, 2^22]
    assert e.value.status == dashlib.ERR_INVALID_ARG


def _plan_scenes(dashlib, lay, grid, mlpc, rng):
    g = oracle_grid(grid)
    scenes = []
    for n, K in ((1500, 2), (700, 3)):
        x, y, z, _ = synth.scene_coords(rng, n)
        ts = np.sort(rng.random(K)).astype(np.float32)
        scenes.append({"table": to_dev(synth.table_values(rng, g.total, grid.F, np.float16)),
                       "params": to_dev(synth.mlp_params(rng, mlpc)), "x": to_dev(x), "y": to_dev(y),
                       "z": to_dev(z), "timestamps": to_dev(ts),
                       "delta_out": torch.zeros((K, mlpc.d_out, n), device="cuda"),
                       "ddelta": to_dev(rng.standard_normal((K, mlpc.d_out, n)).astype(np.float32)),
                       "table_grad": torch.zeros((g.total, grid.F), device="cuda"),
                       "mlp_grad": torch.zeros(mlpc.n_params, device="cuda")})
    return scenes


def test_every_cuda_call_of_plan_creation_failing_in_turn(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    lay = dashlib.layout_from(grid)
    scenes = _plan_scenes(dashlib, lay, grid, mlpc, np.random.default_rng(132))
    # a clean creation: count its checked runtime calls (its gradient
    # replicas, 21 MB per scene at this grid, would show any leak)
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    plan.close()
    dashlib.dash_debug_fail_cuda_call(0)
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    calls = dashlib.dash_debug_cuda_call_count()
    plan.close()
    assert calls >= 5
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    try:
        for k in range(1, calls + 1):
            dashlib.dash_debug_fail_cuda_call(k)
            with pytest.raises(dashlib.DashError) as e:
                dashlib.BatchPlan(lay, scenes, backward=True)
            dashlib.dash_debug_fail_cuda_call(0)
            assert e.value.status == dashlib.ERR_CUDA, k
            assert "injected failure" in str(e.value), (k, str(e.value))
    finally:
        dashlib.dash_debug_fail_cuda_call(0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (4 << 20), (free0, free1)   # no replica set (21 MB a scene) left behind
    # the hook is disarmed: a plan works again and matches the single-scene path
    plan = dashlib.BatchPlan(lay, scenes, backward=True)
    plan.run()
    torch.cuda.synchronize()
    sc = scenes[0]
    mlp = dashlib.Mlp(sc["params"], mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    pts = dashlib.Points(sc["x"], sc["y"], sc["z"], sc["timestamps"][1:2].contiguous(), n=sc["x"].numel())
    assert torch.equal(sc["delta_out"][1], dashlib.dash_deform_mlp_fwd(lay, pts, sc["table"], mlp))
    plan.close()


def test_injected_failure_in_the_fused_backward_and_status(dashlib):
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(133)
    n = 2000
    coords = synth.scene_coords(rng, n)
    g = oracle_grid(grid)
    table = to_dev(synth.table_values(rng, g.total, grid.F, np.float16))
    params = synth.mlp_params(rng, mlpc)
    lay = dashlib.layout_from(grid)
    pts = dashlib.Points(*(to_dev(c) for c in coords), n=n)
    mlp = dashlib.Mlp(to_dev(params), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    st = dashlib.deform_state(mlp, n, "cuda")
    dashlib.dash_deform_mlp_fwd(lay, pts, table, mlp, fwd_state=st)
    dd_h = synth.upstream_grad(rng, mlpc.d_out, n)
    zero_ambiguous(dd_h, g, oracle.Points(*coords), table.cpu().numpy(), params, mlpc.d_hidden, mlpc.d_out)
    dd = to_dev(dd_h)
    tg = torch.zeros((g.total, grid.F), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")
    try:
        dashlib.dash_debug_fail_cuda_call(1)   # its first checked runtime call
        with pytest.raises(dashlib.DashError) as e:
            dashlib.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=st)
        assert e.value.status == dashlib.ERR_CUDA and "injected failure" in str(e.value)
        dashlib.dash_debug_fail_cuda_call(1)   # the status call's stream synchronisation
        with pytest.raises(dashlib.DashError) as e:
            dashlib.dash_device_status()
        assert e.value.status == dashlib.ERR_CUDA and "cudaStreamSynchronize" in str(e.value)
    finally:
        dashlib.dash_debug_fail_cuda_call(0)
    dashlib.dash_device_status()
    tg.zero_()
    pg.zero_()
    dashlib.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=st)
    rtg, rpg, _ = oracle.deform_bwd(g, oracle.Points(*coords), table.cpu().numpy().astype(np.float64),
                                    mlpc.d_hidden, mlpc.d_out, params.astype(np.float64),
                                    dd.cpu().numpy().astype(np.float64))
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-2
