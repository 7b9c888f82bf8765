"""CPU-side checks of the C ABI: libdash.so builds, loads without a GPU,
exports every function include/dash.h declares, and its host-side Eq. 7
layout equals the oracle's (two independent implementations)."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2507_19141_gb300 import build as dash_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(dash_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = dash_build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_debug_library_exports_the_same_abi(lib):
    """libdash_debug.so (the -DDASH_DEBUG bounds-checked build) exports every
    declared function; only it accepts dash_debug_set_point_rows (host-only
    calls, no GPU needed)."""
    assert os.path.exists(dash_build.DEBUG_LIB), dash_build.DEBUG_LIB
    dbg = ctypes.CDLL(dash_build.DEBUG_LIB)
    missing = [n for n in _declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing
    dbg.dash_debug_set_point_rows.argtypes = [ctypes.c_int64]
    lib.dash_debug_set_point_rows.argtypes = [ctypes.c_int64]
    assert dbg.dash_debug_set_point_rows(1000) == 0
    assert dbg.dash_debug_set_point_rows(-2) == -1      # DASH_ERR_INVALID_ARG
    assert dbg.dash_debug_set_point_rows(-1) == 0
    assert lib.dash_debug_set_point_rows(1000) == -2    # DASH_ERR_UNSUPPORTED in the release build


def test_binding_names_match_the_abi():
    from paper_2507_19141_gb300 import dash
    declared = set(_declared_functions())
    assert set(dash.exported_symbols()) <= declared
    for n in declared:
        assert hasattr(dash._lib, n)


def test_every_declared_function_has_a_same_named_wrapper():
    from paper_2507_19141_gb300 import dash
    missing = [n for n in _declared_functions() if not callable(getattr(dash, n, None))]
    assert not missing, missing
    assert dash.dash_status_string(0) == "DASH_OK"


def test_status_strings_and_version(lib):
    lib.dash_status_string.restype = ctypes.c_char_p
    assert lib.dash_status_string(0) == b"DASH_OK"
    assert lib.dash_status_string(-3) == b"DASH_ERR_WORKSPACE"
    assert lib.dash_version() >= 100


@pytest.mark.parametrize("cfg", [(16, 2, 19, 16, 2048, 8, 150), (4, 2, 14, 16, 128, 8, 32), (1, 1, 10, 5, 5, 3, 3),
                                 (8, 4, 16, 4, 300, 2, 60), (32, 1, 24, 2, 8192, 2, 512), (3, 8, 12, 7, 9, 1, 2)])
def test_host_layout_equals_oracle(cfg):
    from paper_2507_19141_gb300 import dash
    L, F, lt, a, b, c, d = cfg
    got = dash.dash_hash4d_layout(L, F, lt, a, b, c, d).as_dict()
    ref = oracle.layout(L, F, lt, a, b, c, d).as_dict()
    assert got == ref


def test_host_layout_rejects_bad_arguments():
    from paper_2507_19141_gb300 import dash
    with pytest.raises(dash.DashError) as e:
        dash.dash_hash4d_layout(33, 2, 19, 16, 2048, 8, 150)
    assert e.value.status == dash.ERR_UNSUPPORTED
    with pytest.raises(dash.DashError) as e:
        dash.dash_hash4d_layout(4, 3, 19, 16, 2048, 8, 150)
    assert e.value.status == dash.ERR_UNSUPPORTED
    with pytest.raises(dash.DashError) as e:
        dash.dash_hash4d_layout(4, 2, 19, 16, 8, 8, 150)
    assert e.value.status == dash.ERR_INVALID_ARG


@pytest.mark.parametrize("cfg", [(16, 2, 19, 16, 2048), (4, 2, 12, 4, 32), (1, 1, 10, 7, 7), (8, 4, 14, 2, 512)])
def test_host_layout3_equals_oracle(cfg):
    from paper_2507_19141_gb300 import dash
    L, F, lt, a, b = cfg
    lay = dash.dash_hash3d_layout(L, F, lt, a, b)
    assert lay.dims == 3
    got = lay.as_dict()
    ref = oracle.layout3(L, F, lt, a, b).as_dict()
    got["res_t"] = ref["res_t"]  # unused by a 3-D layout
    assert got == ref


def test_replica_workspace_size():
    """Replicas cover the leading dense levels of at most 2^17 entries
    (levels 0 and 1 of the three dense ones at the paper shape): k copies of
    each level's FP32 [entries][2] rows, 256-byte aligned; the Eq. 11
    hand-over adds L * F * n floats."""
    from paper_2507_19141_gb300 import dash, synth
    lay = dash.layout_from(synth.PAPER_GRID)
    old = dash.dash_get_option(dash.OPT_GRAD_REPLICAS)
    try:
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, 8)
        rows = [-(-int(lay.size[l]) * 2 // 64) * 64 for l in range(2)]
        assert all(bool(lay.dense[l]) for l in range(3)) and not lay.dense[3]
        assert lay.size[1] <= 1 << 17 < lay.size[2]
        rep = 4 * 8 * (rows[0] + rows[1])
        assert dash.dash_deform_bwd_workspace_size(lay, 1000) == rep
        sm = (1.0, (0.0, 0.0, 0.0), 0.0, None)
        assert dash.dash_deform_bwd_workspace_size(lay, 1000, sm) == -(-rep // 256) * 256 + 32 * 1000 * 4
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, 3)
        assert dash.dash_deform_bwd_workspace_size(lay, 1000) == 4 * 3 * (rows[0] + rows[1])
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, 0)
        assert dash.dash_deform_bwd_workspace_size(lay, 1000) == 0
        with pytest.raises(dash.DashError):
            dash.dash_set_option(dash.OPT_GRAD_REPLICAS, 65)
    finally:
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, old)


def test_replica_workspace_edge_layouts():
    """No replicas where no leading level is dense (the tiny grid's level 0
    has 44,217 vertices > T = 2^14, so every level is hashed) or F != 2; the
    Eq. 11 hand-over alone then sizes the workspace; the replicas do not
    depend on n."""
    from paper_2507_19141_gb300 import dash, synth
    tiny = dash.layout_from(synth.TINY_GRID)
    assert not any(bool(tiny.dense[l]) for l in range(tiny.L))
    sm = (1.0, (0.0, 0.0, 0.0), 0.0, None)
    assert dash.dash_deform_bwd_workspace_size(tiny, 5000) == 0
    assert dash.dash_deform_bwd_workspace_size(tiny, 5000, sm) == 4 * 2 * 5000 * 4
    f4 = dash.dash_hash4d_layout(4, 4, 14, 16, 128, 8, 32)
    assert dash.dash_deform_bwd_workspace_size(f4, 5000, sm) == 0
    paper = dash.layout_from(synth.PAPER_GRID)
    assert dash.dash_deform_bwd_workspace_size(paper, 0) == dash.dash_deform_bwd_workspace_size(paper, 10)
    assert dash.dash_deform_bwd_workspace_size(paper, 0, sm) % 256 == 0


@pytest.mark.parametrize("cfg", [(16, 2, 19, 16, 2048, 8, 150), (8, 2, 20, 8, 512, 4, 64), (12, 2, 17, 4, 1024, 2, 40),
                                 (3, 2, 22, 16, 64, 8, 16)])
@pytest.mark.parametrize("k", [2, 5, 16])
def test_replica_plan_follows_the_layout(cfg, k):
    """Replicas cover exactly the leading run of dense levels of at most
    2^17 entries (at most 4 levels), k copies each, rows rounded up to 64
    floats: the size the library reports equals this count for layouts with
    1 to 4 such levels."""
    from paper_2507_19141_gb300 import dash
    lay = dash.dash_hash4d_layout(*cfg)
    old = dash.dash_get_option(dash.OPT_GRAD_REPLICAS)
    try:
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, k)
        floats = 0
        for l in range(min(lay.L, 4)):
            if not lay.dense[l] or lay.size[l] > 1 << 17:
                break
            floats += k * (-(-int(lay.size[l]) * 2 // 64) * 64)
        assert dash.dash_deform_bwd_workspace_size(lay, 777) == 4 * floats
    finally:
        dash.dash_set_option(dash.OPT_GRAD_REPLICAS, old)
