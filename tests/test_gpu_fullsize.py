"""Parity at the benchmark's full size and launch configuration: 2M
Gaussians with exactly 1M dynamic, paper-shaped grid, FP16 tables, BF16
decoder, the same kernels and shapes bench.py times.

The oracle cannot run 1M Gaussians in seconds, so the checks use what it can
compute: compaction in full (NumPy), the offsets and the Eq. 10 update on a
random sample, and the gradients through linearity -- with the upstream
gradient zero outside a sample, the full-size backward must produce exactly
the sample's decoder and table gradients."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import oracle_grid, rel_err, relu_clear

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def full(dashlib):
    sys.path.insert(0, ROOT)
    import bench
    wl = bench.Workload(seed=2, n_all=bench.N_ALL, n_dyn=bench.N_DYN, device=torch.device("cuda"))
    return wl


def test_fullsize_compaction_forward_and_eq10(full):
    wl = full
    wl.compact()
    wl.forward()
    torch.cuda.synchronize()
    ref_idx = np.flatnonzero(wl.mask_h).astype(np.int32)
    assert int(wl.count.item()) == len(ref_idx) == wl.n_dyn
    assert np.array_equal(wl.idx[:wl.n_dyn].cpu().numpy(), ref_idx)
    rng = np.random.default_rng(61)
    sample = np.sort(rng.choice(wl.n_dyn, size=3000, replace=False))
    g = oracle_grid(wl.grid)
    x, y, z, t = wl.coords_h
    ref = oracle.deform_fwd(g, oracle.Points(x, y, z, t, idx=ref_idx[sample]), wl.table_h.astype(np.float64),
                            wl.mlpc.d_hidden, wl.mlpc.d_out, wl.params_h.astype(np.float64))
    got = wl.delta[:, :wl.n_dyn].cpu().numpy()[:, sample]
    for a, b in ((0, 3), (3, 7), (7, 10)):
        assert rel_err(got[a:b], ref[a:b]) < 1e-3
    rows = ref_idx[sample]
    out = wl.attrs_out.cpu().numpy()[:, rows]
    assert np.max(np.abs(out - (wl.attrs_h[:, rows].astype(np.float64) + ref))) < 1e-3
    static = np.flatnonzero(wl.mask_h == 0)[:5000]
    assert np.array_equal(wl.attrs_out.cpu().numpy()[:, static], wl.attrs_h[:, static])


def test_fullsize_backward_by_linearity(full):
    wl = full
    wl.compact()
    wl.forward()
    rng = np.random.default_rng(62)
    sample = np.sort(rng.choice(wl.n_dyn, size=2000, replace=False))
    ref_idx = np.flatnonzero(wl.mask_h).astype(np.int32)
    g = oracle_grid(wl.grid)
    x, y, z, t = wl.coords_h
    # only Gaussians whose ReLU decisions are unambiguous in FP32 and FP64
    sample = sample[relu_clear(g, oracle.Points(x, y, z, t, idx=ref_idx[sample]), wl.table_h, wl.params_h,
                               wl.mlpc.d_hidden, wl.mlpc.d_out)]
    dd = np.zeros((wl.mlpc.d_out, wl.n_dyn), dtype=np.float32)
    dd[:, sample] = wl.ddelta_h[:, sample]
    wl.ddelta.zero_()
    wl.ddelta[:, :wl.n_dyn] = torch.from_numpy(dd).cuda()
    wl.table_grad.zero_()
    wl.mlp_grad.zero_()
    wl.backward()
    torch.cuda.synchronize()
    rtg, rpg, _ = oracle.deform_bwd(g, oracle.Points(x, y, z, t, idx=ref_idx[sample]),
                                    wl.table_h.astype(np.float64), wl.mlpc.d_hidden, wl.mlpc.d_out,
                                    wl.params_h.astype(np.float64), wl.ddelta_h[:, sample].astype(np.float64))
    assert rel_err(wl.table_grad.cpu().numpy(), rtg) < 1e-2
    D, H, O = wl.mlpc.d_in, wl.mlpc.d_hidden, wl.mlpc.d_out
    bounds = np.cumsum([0, H * D, H, H * H, H, O * H, O])
    pg = wl.mlp_grad.cpu().numpy()
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert rel_err(pg[a:b], rpg[a:b]) < 1e-2
