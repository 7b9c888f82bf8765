"""The bounds-checked build (libdash_debug.so, compiled with -DDASH_DEBUG).

With dash_debug_set_point_rows(rows) the kernels check every point row they
read (an index-list entry) against [0, rows) BEFORE the access; a row outside
it sets a device flag, the point reads as (0, 0, 0, 0), its Eq. 10 update
and its gathered dL/d(delta) row are not written, and the next
dash_device_status reports DASH_ERR_BOUNDS.  So the results must equal the
oracle's on the same index list with each bad row's point replaced by the
origin, and nothing outside the valid rows may change.  Nothing faults: the
bad rows are never dereferenced.

The debug library runs in a child process started with DASH_LIBRARY=debug,
which loads libdash_debug.so only (checked through /proc/self/maps); the
release library answers DASH_ERR_UNSUPPORTED."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OK_LINE = "bounds-checked build: all checks passed"


def test_bounds_checked_build(dashlib):
    env = dict(os.environ, DASH_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert OK_LINE in r.stdout


def test_release_library_has_no_bounds_checks(dashlib):
    assert dashlib.LIB_PATH.endswith(os.path.join("_build", "libdash.so"))
    with pytest.raises(dashlib.DashError) as e:
        dashlib.dash_debug_set_point_rows(10)
    assert e.value.status == dashlib.ERR_UNSUPPORTED


# ------------------------------------------------------------ the child --
HEADS = ((0, 3), (3, 7), (7, 10))


def _expect_bounds(dash):
    try:
        dash.dash_device_status()
    except dash.DashError as e:
        assert e.status == dash.ERR_BOUNDS, e
        return
    raise AssertionError("no DASH_ERR_BOUNDS reported")


def _substituted(coords, idx, rows):
    """Compact coordinates (x, y, z, t) of the index list, each row outside
    [0, rows) replaced by the origin: what the checked kernels compute on."""
    ok = (idx >= 0) & (idx < rows)
    safe = np.where(ok, idx, 0)
    return [np.where(ok, c[safe], np.float32(0.0)).astype(np.float32) for c in coords], ok


def _child():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch

    import oracle
    from paper_2507_19141_gb300 import dash, synth
    from gpu_helpers import oracle_grid, rel_err, to_dev, zero_ambiguous

    assert dash.LIB_PATH.endswith("libdash_debug.so"), dash.LIB_PATH
    maps = open("/proc/self/maps").read()
    assert "libdash_debug.so" in maps
    assert os.path.join("_build", "libdash.so") not in maps, "the release library is loaded too"

    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    H, O = mlpc.d_hidden, mlpc.d_out
    g = oracle_grid(grid)
    rng = np.random.default_rng(171)
    n_all = 9000
    coords = synth.scene_coords(rng, n_all)
    mask = synth.bernoulli_mask(rng, n_all, 0.4)
    mask[:64] = 0     # rows an index of n_all (or -1) would reach in the
    mask[-64:] = 0    # neighbouring attribute stay static, so must not change
    idx_good = np.flatnonzero(mask).astype(np.int32)
    n = len(idx_good)
    table = synth.table_values(rng, g.total, grid.F, np.float16)
    params = synth.mlp_params(rng, mlpc)
    attrs = synth.gaussian_attrs(rng, n_all)
    lay = dash.layout_from(grid)
    dev = [to_dev(c) for c in coords]
    tab = to_dev(table)
    mlp = dash.Mlp(to_dev(params), mlpc.d_in, H, O)

    def run_forward(idx):
        pts = dash.Points(*dev, idx=to_dev(idx), n=len(idx))
        feat = dash.dash_hash4d_fwd(lay, pts, tab).cpu().numpy()
        ai = to_dev(attrs)
        ao = ai.clone()
        fsave = dash.deform_state(mlp, len(idx), "cuda")
        delta = dash.dash_deform_mlp_fwd(lay, pts, tab, mlp, fwd_state=fsave, apply=(ai, ao)).cpu().numpy()
        return pts, feat, delta, ao.cpu().numpy(), fsave

    def check_forward(idx, feat, delta, out, rows):
        sub, ok = _substituted(coords, idx, rows)
        opts = oracle.Points(*sub)
        assert rel_err(feat, oracle.encode(g, opts, table.astype(np.float64))) < 1e-4
        rdelta = oracle.deform_fwd(g, opts, table.astype(np.float64), H, O, params.astype(np.float64))
        for a, b in HEADS:
            assert rel_err(delta[a:b], rdelta[a:b]) < 1e-3, (a, b, rel_err(delta[a:b], rdelta[a:b]))
        good = idx[ok]
        untouched = np.ones(n_all, dtype=bool)
        untouched[good] = False
        assert np.array_equal(out[:, untouched], attrs[:, untouched])   # only valid rows written
        want = attrs[:, good].astype(np.float64) + rdelta[:, ok]
        assert np.max(np.abs(out[:, good] - want)) < 1e-3

    # 1. checks off (the default): a valid list runs and reports nothing
    pts, feat, delta, out, _ = run_forward(idx_good)
    dash.dash_device_status()
    check_forward(idx_good, feat, delta, out, n_all)

    # 2. checks on, valid list: no false report, same results
    dash.dash_debug_set_point_rows(n_all)
    pts, feat, delta, out, _ = run_forward(idx_good)
    dash.dash_device_status()
    check_forward(idx_good, feat, delta, out, n_all)

    # 3. checks on, rows out of range in the list (first, inside, last)
    idx_bad = idx_good.copy()
    idx_bad[0] = n_all                  # one past the end
    idx_bad[37] = -1
    idx_bad[n // 2] = n_all + 123_457   # far past the end
    idx_bad[-1] = np.iinfo(np.int32).max
    pts, feat, delta, out, fsave = run_forward(idx_bad)
    _expect_bounds(dash)
    dash.dash_device_status()           # reported once, then cleared
    check_forward(idx_bad, feat, delta, out, n_all)

    # the fused backward on the same list: gradients equal the oracle's with
    # the bad points at the origin
    sub, ok = _substituted(coords, idx_bad, n_all)
    opts = oracle.Points(*sub)
    dd = synth.upstream_grad(rng, O, n)
    zero_ambiguous(dd, g, opts, table, params, H, O)
    tg = torch.zeros((g.total, grid.F), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    dash.dash_deform_mlp_bwd(lay, pts, tab, mlp, to_dev(dd), tg, pg, fwd_state=fsave)
    _expect_bounds(dash)
    rtg, rpg, _ = oracle.deform_bwd(g, opts, table.astype(np.float64), H, O, params.astype(np.float64),
                                    dd.astype(np.float64))
    assert rel_err(tg.cpu().numpy(), rtg) < 1e-2
    assert rel_err(pg.cpu().numpy(), rpg) < 1e-2

    # the Eq. 10 gather of dL/d(delta): bad rows keep what the buffer held
    dattrs = rng.standard_normal((O, n_all)).astype(np.float32)
    ddelta = torch.full((O, n), 7.0, dtype=torch.float32, device="cuda")
    dash.dash_deform_apply_bwd(pts, to_dev(dattrs), ddelta=ddelta)
    _expect_bounds(dash)
    got = ddelta.cpu().numpy()
    assert np.array_equal(got[:, ok], dattrs[:, idx_bad[ok]])
    assert np.all(got[:, ~ok] == 7.0)

    # 4. the context is still usable and the checks can be switched off
    dash.dash_debug_set_point_rows(-1)
    pts, feat, delta, out, _ = run_forward(idx_good)
    dash.dash_device_status()
    check_forward(idx_good, feat, delta, out, n_all)
    try:
        dash.dash_debug_set_point_rows(-2)
        raise AssertionError("rows = -2 accepted")
    except dash.DashError as e:
        assert e.status == dash.ERR_INVALID_ARG
    print(OK_LINE)


if __name__ == "__main__":
    _child()
