"""The error of every output of the precision and differentiation forms
against the FP64 oracle, at the benchmark's configuration (2M Gaussians,
1M dynamic, paper-shaped grid, FP16 tables, BF16 decoder weights): the
encoder's f_h, the three heads, the Eq. 10 update, the table gradients
(FP32 buffers), each decoder parameter block, and the Eq. 11 loss and
gradients.  The oracle evaluates a random sample of the dynamic Gaussians
(forward) and, by linearity, the backward of an upstream gradient that is
zero outside a sample.  Each error is printed (pytest -s) and checked
against the targets: 1e-3 for outputs, 1e-2 for gradients, each both
normwise and per element (|got - ref| <= tol * max|ref|)."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import elem_err, norm_err, oracle_grid, rel_err, relu_clear

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _report(name, got, ref):
    """Prints the normwise and element-wise errors and returns rel_err (the
    larger of the two, infinite if the touched entries differ)."""
    got = np.asarray(got, dtype=np.float64)
    m = float(np.max(np.abs(got - ref))) if got.size else 0.0
    print(f"precision | {name:28s} | normwise {norm_err(got, ref):.3e} | element-wise {elem_err(got, ref):.3e}"
          f" | max abs {m:.3e}")
    return rel_err(got, ref)


def test_precision_of_every_output(dashlib):
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.Workload(seed=2, n_all=bench.N_ALL, n_dyn=bench.N_DYN, device=torch.device("cuda"))
    wl.compact()
    wl.forward()
    torch.cuda.synchronize()
    g = oracle_grid(wl.grid)
    x, y, z, t = wl.coords_h
    ref_idx = np.flatnonzero(wl.mask_h).astype(np.int32)
    tab64, par64 = wl.table_h.astype(np.float64), wl.params_h.astype(np.float64)
    H, O, D = wl.mlpc.d_hidden, wl.mlpc.d_out, wl.mlpc.d_in
    rng = np.random.default_rng(63)

    # forward: f_h (encoder, FP32 out), heads, Eq. 10 on a sample
    sample = np.sort(rng.choice(wl.n_dyn, size=20_000, replace=False))
    pts = oracle.Points(x, y, z, t, idx=ref_idx[sample])
    sel = torch.from_numpy(ref_idx[sample]).cuda()
    dpts = dashlib.Points(wl.x, wl.y, wl.z, wl.t, idx=sel, n=len(sample))
    fh = dashlib.dash_hash4d_fwd(wl.layout, dpts, wl.table, torch.float32).cpu().numpy()
    assert _report("f_h (encoder, FP32)", fh, oracle.encode(g, pts, tab64)) < 1e-6
    ref = oracle.deform_fwd(g, pts, tab64, H, O, par64)
    got = wl.delta[:, :wl.n_dyn].cpu().numpy()[:, sample]
    for name, a, b in (("head dx", 0, 3), ("head dr", 3, 7), ("head ds", 7, 10)):
        assert _report(name, got[a:b], ref[a:b]) < 1e-3
    rows = ref_idx[sample]
    out = wl.attrs_out.cpu().numpy()[:, rows]
    assert _report("Eq. 10 x', r', s'", out, wl.attrs_h[:, rows].astype(np.float64) + ref) < 1e-3

    # backward by linearity: upstream gradient on a sample only
    bsample = np.sort(rng.choice(wl.n_dyn, size=2000, replace=False))
    # only Gaussians whose ReLU decisions are unambiguous in FP32 and FP64
    bsample = bsample[relu_clear(g, oracle.Points(x, y, z, t, idx=ref_idx[bsample]), wl.table_h, wl.params_h, H, O)]
    bpts = oracle.Points(x, y, z, t, idx=ref_idx[bsample])
    dd = np.zeros((O, wl.n_dyn), dtype=np.float32)
    dd[:, bsample] = wl.ddelta_h[:, bsample]
    wl.ddelta.zero_()
    wl.ddelta[:, :wl.n_dyn] = torch.from_numpy(dd).cuda()
    wl.table_grad.zero_()
    wl.mlp_grad.zero_()
    wl.backward()
    torch.cuda.synchronize()
    rtg, rpg, _ = oracle.deform_bwd(g, bpts, tab64, H, O, par64, wl.ddelta_h[:, bsample].astype(np.float64))
    assert _report("table gradient", wl.table_grad.cpu().numpy(), rtg) < 1e-2
    bounds = np.cumsum([0, H * D, H, H * H, H, O * H, O])
    pg = wl.mlp_grad.cpu().numpy()
    for name, a, b in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), bounds[:-1], bounds[1:]):
        assert _report(name, pg[a:b], rpg[a:b]) < 1e-2

    # differentiation form: Eq. 11 with dx = 1/2048, dt = 1/300 over the sampled
    # Gaussians (a compact index list of them, the upstream gradient zero)
    lam, es, et = 1.0, (1 / 2048,) * 3, 1 / 300
    spts = dashlib.Points(wl.x, wl.y, wl.z, wl.t, idx=torch.from_numpy(ref_idx[bsample]).cuda(), n=len(bsample))
    st = dashlib.deform_state(wl.mlp, len(bsample), "cuda")
    dashlib.dash_deform_mlp_fwd(wl.layout, spts, wl.table, wl.mlp, fwd_state=st)
    tg = torch.zeros_like(wl.table_grad)
    pgs = torch.zeros_like(wl.mlp_grad)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    dashlib.dash_deform_mlp_bwd(wl.layout, spts, wl.table, wl.mlp, torch.zeros((O, len(bsample)), device="cuda"),
                                tg, pgs, fwd_state=st, smooth=(lam, es, et, loss))
    rtg2, _, rl = oracle.deform_bwd(g, bpts, tab64, H, O, par64, np.zeros((O, len(bsample))), lam, es, et)
    assert _report("Eq. 11 loss lambda L_r", [float(loss.item())], [rl]) < 1e-3
    assert _report("Eq. 11 table gradient", tg.cpu().numpy(), rtg2) < 1e-2
