"""Thin Python binding of libdash (include/dash.h): the DASH 4D-hash
deformation path of arXiv 2507.19141, Sec. 4.2-4.3.

Functions carry the C entry points' names and only marshal arguments:
torch tensors in, device pointers and the current CUDA stream out.  Every
step of the path runs in libdash's CUDA kernels; there is no Python or CPU
fallback.  Importing this module fails loudly if libdash.so is missing.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DASH_LIBRARY=debug selects the bounds-checked build (libdash_debug.so,
# compiled with -DDASH_DEBUG); a process loads one of the two, never both.
LIB_PATH = (os.path.join(_HERE, "_build_debug", "libdash_debug.so") if os.environ.get("DASH_LIBRARY") == "debug"
            else os.path.join(_HERE, "_build", "libdash.so"))

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); "
                      "run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

MAX_LEVELS = 32
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_CUDA, ERR_BOUNDS, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
F32, F16, BF16 = 0, 1, 2
_DTYPE_CODE = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}
PRIMES = (1, 2654435761, 805459861, 3674653429)


class DashError(RuntimeError):
    def __init__(self, status, fn):
        self.status = status
        msg = _lib.dash_last_error().decode()
        super().__init__(f"{fn}: {_lib.dash_status_string(status).decode()}: {msg}")


# ------------------------------------------------------------------ structs --
class dash_hash4d_cfg(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("F", ctypes.c_int32), ("log2_T", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("nmin_s", ctypes.c_double), ("nmax_s", ctypes.c_double),
                ("nmin_t", ctypes.c_double), ("nmax_t", ctypes.c_double), ("primes", ctypes.c_uint32 * 4)]


class dash_layout(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("F", ctypes.c_int32), ("log2_T", ctypes.c_int32),
                ("dims", ctypes.c_int32), ("primes", ctypes.c_uint32 * 4),
                ("res_s", ctypes.c_int32 * MAX_LEVELS), ("res_t", ctypes.c_int32 * MAX_LEVELS),
                ("dense", ctypes.c_int32 * MAX_LEVELS), ("size", ctypes.c_int64 * MAX_LEVELS),
                ("offset", ctypes.c_int64 * (MAX_LEVELS + 1))]

    @property
    def total(self) -> int:
        return int(self.offset[self.L])

    def as_dict(self) -> dict:
        L = self.L
        return {"L": L, "F": self.F, "log2_T": self.log2_T, "res_s": list(self.res_s[:L]),
                "res_t": list(self.res_t[:L]), "dense": [bool(v) for v in self.dense[:L]],
                "size": list(self.size[:L]), "offset": list(self.offset[:L + 1])}


class dash_points(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("t", ctypes.c_void_p),
                ("t_stride", ctypes.c_int64), ("idx", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("n_dev", ctypes.c_void_p)]


class dash_mlp(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_int32), ("d_hidden", ctypes.c_int32), ("d_out", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("params", ctypes.c_void_p)]


class dash_apply(ctypes.Structure):
    _fields_ = [("attrs_in", ctypes.c_void_p), ("attrs_out", ctypes.c_void_p), ("n_all", ctypes.c_int64)]


class dash_smooth(ctypes.Structure):
    _fields_ = [("lambda_r", ctypes.c_float), ("eps_s", ctypes.c_float * 3), ("eps_t", ctypes.c_float),
                ("loss_out", ctypes.c_void_p)]


class dash_camera(ctypes.Structure):
    _fields_ = [("view", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_plane", ctypes.c_float), ("dilation", ctypes.c_float),
                ("campos", ctypes.c_float * 3), ("bg", ctypes.c_float * 3)]


class dash_gaussians(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("rot", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("sh_degree", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("n", ctypes.c_int64)]


class dash_gaussian_grads(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("rot", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class dash_batch_scene(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("params", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("timestamps", ctypes.c_void_p),
                ("delta_out", ctypes.c_void_p), ("n", ctypes.c_int64), ("K", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ddelta", ctypes.c_void_p), ("fwd_state", ctypes.c_void_p),
                ("table_grad", ctypes.c_void_p), ("mlp_grad", ctypes.c_void_p)]


class dash_batch_desc(ctypes.Structure):
    _fields_ = [("layout", ctypes.c_void_p), ("table_dtype", ctypes.c_int32), ("d_in", ctypes.c_int32),
                ("d_hidden", ctypes.c_int32), ("d_out", ctypes.c_int32), ("n_scenes", ctypes.c_int32),
                ("scenes", ctypes.c_void_p), ("with_backward", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_SIGS = {
    "dash_status_string": ([_I], ctypes.c_char_p),
    "dash_last_error": ([], ctypes.c_char_p),
    "dash_version": ([], _I),
    "dash_set_option": ([_I, _I], _I),
    "dash_device_status": ([_P], _I),
    "dash_selftest_wait": ([_I64, _P], _I),
    "dash_debug_fail_cuda_call": ([_I64], _I),
    "dash_debug_cuda_call_count": ([], _I64),
    "dash_debug_set_point_rows": ([_I64], _I),
    "dash_probe_threads": ([_I], _I),
    "dash_probe_rate": ([_I, _P, _SZ, _I, _P, _P, _P], _I),
    "dash_get_option": ([_I], _I),
    "dash_hash4d_layout": ([_P, _P], _I),
    "dash_compact_workspace_size": ([_I64], _SZ),
    "dash_compact_dynamic": ([_P, _I64, _P, _P, _P, _SZ, _P], _I),
    "dash_compact_dynamic_noalloc": ([_P, _I64, _P, _P, _P], _I),
    "dash_hash4d_indices": ([_P, _P, _P, _P, _P], _I),
    "dash_hash4d_fwd": ([_P, _P, _P, _I, _P, _I, _P], _I),
    "dash_hash4d_bwd": ([_P, _P, _P, _P, _P], _I),
    "dash_hash4d_bwd_half": ([_P, _P, _P, _P, _P], _I),
    "dash_hash4d_coord_grad": ([_P, _P, _P, _I, _P, _P, _P], _I),
    "dash_collision_workspace_size": ([_P, _I64], _SZ),
    "dash_raster_workspace_size": ([_P, _I64, _I64], _SZ),
    "dash_raster_fwd": ([_P, _P, _P, _P, _SZ, _I64, _P, _P], _I),
    "dash_raster_bwd": ([_P, _P, _P, _P, _SZ, _I64, _P, _P], _I),
    "dash_hash4d_collision_stats": ([_P, _P, _P, _P, _SZ, _P], _I),
    "dash_deform_state_size": ([_P], _SZ),
    "dash_deform_bwd_workspace_size": ([_P, _I64, _P], _SZ),
    "dash_deform_apply_bwd": ([_P, _I, _P, _I64, _P, _P], _I),
    "dash_deform_mlp_fwd": ([_P, _P, _P, _I, _P, _P, _P, _P, _P], _I),
    "dash_deform_mlp_bwd": ([_P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P], _I),
    "dash_batch_plan_create": ([_P, _P], _I),
    "dash_batch_counts": ([_P], ctypes.c_void_p),
    "dash_batch_run": ([_P, _P], _I),
    "dash_batch_form": ([_P], _I),
    "dash_batch_autotune": ([_P, ctypes.c_char_p, _P], _I),
    "dash_batch_plan_destroy": ([_P], _I),
    "dash_hash3d_layout": ([_P, _P], _I),
    "dash_decomp_fwd": ([_P, _P, _P, _P, _I64, _P, _I, _P, _P, _P, _P, _I64, _P, _P], _I),
    "dash_topk_workspace_size": ([], _SZ),
    "dash_decomp_bwd_workspace_size": ([], _SZ),
    "dash_decomp_bwd": ([_P, _P, _P, _P, _I64, _P, _I, _P, _P, _P, ctypes.c_float, _P, _P, _P, _SZ, _P], _I),
    "dash_topk_mask": ([_P, _I64, ctypes.c_double, _P, _P, _P, _P, _SZ, _P], _I),
    "dash_plain_hash4d_fwd": ([_P, _P, _P, _P, _P], _I),
    "dash_plain_hash4d_bwd": ([_P, _P, _P, _P, _P], _I),
    "dash_plain_mlp_fwd": ([_P, _P, _I64, _P, _P, _P], _I),
    "dash_plain_mlp_bwd_workspace_size": ([_P, _I64], _SZ),
    "dash_plain_mlp_bwd": ([_P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P], _I),
}
for _name, (_args, _ret) in _SIGS.items():
    _f = getattr(_lib, _name, None)
    if _f is not None:
        _f.argtypes = _args
        _f.restype = _ret


def _check(status, fn):
    if status != OK:
        raise DashError(status, fn)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def exported_symbols():
    return [n for n in _SIGS if hasattr(_lib, n)]


# ------------------------------------------------------------ utilities --
def dash_version() -> int:
    return int(_lib.dash_version())


def dash_status_string(status: int) -> str:
    return _lib.dash_status_string(int(status)).decode()


def dash_last_error() -> str:
    """Message of the last failing call on this host thread."""
    return _lib.dash_last_error().decode()


OPT_FWD_FORM = 1
OPT_BWD_FORM = 2
OPT_ACCESS_FORM = 3
OPT_GRAD_REPLICAS = 4
OPT_DECOMP_FORM = 5


def dash_device_status() -> None:
    """Raises DashError (ERR_TIMEOUT) if a bounded device-side wait of a
    persistent kernel gave up since the last call (synchronises the current
    stream)."""
    _check(_lib.dash_device_status(_stream()), "dash_device_status")


def dash_selftest_wait(polls: int = 1000) -> None:
    """Launches the wait self-test on the current stream: a bounded wait on an
    mbarrier nothing arrives at, which runs out after `polls` polls and sets
    a flag that the next dash_device_status reports as ERR_TIMEOUT."""
    _check(_lib.dash_selftest_wait(int(polls), _stream()), "dash_selftest_wait")


def dash_debug_fail_cuda_call(n: int) -> None:
    """Host fault injection: the n-th checked CUDA runtime call from now on
    is not made and fails (n = 0 disarms); restarts the call count."""
    _check(_lib.dash_debug_fail_cuda_call(int(n)), "dash_debug_fail_cuda_call")


def dash_debug_set_point_rows(rows: int) -> None:
    """Bounds-checked build only: the length of the point arrays that point
    row indices are checked against (-1 = unchecked)."""
    _check(_lib.dash_debug_set_point_rows(int(rows)), "dash_debug_set_point_rows")


def dash_debug_cuda_call_count() -> int:
    """Checked CUDA runtime calls since the last dash_debug_fail_cuda_call."""
    return int(_lib.dash_debug_cuda_call_count())


PROBE_RED8, PROBE_RED16, PROBE_RED8_PAIRED, PROBE_GATHER4, PROBE_GATHER4_PAIRED = 1, 2, 3, 4, 5


def dash_probe_rate(kind: int, buf: torch.Tensor, iters: int, sink=None) -> int:
    """Launches one rate probe over the float32 device buffer buf on the
    current stream; returns the number of lane operations it issued."""
    assert buf.is_cuda and buf.dtype == torch.float32 and buf.is_contiguous()
    if kind in (PROBE_GATHER4, PROBE_GATHER4_PAIRED):
        need = int(_lib.dash_probe_threads(kind))
        assert sink is not None and sink.is_cuda and sink.dtype == torch.float32 and sink.numel() >= need, \
            f"sink: {need} float32 on the device"
    ops = ctypes.c_int64(0)
    _check(_lib.dash_probe_rate(kind, _ptr(buf), buf.numel() * 4, int(iters), _ptr(sink), ctypes.byref(ops),
                                _stream()), "dash_probe_rate")
    return int(ops.value)


def dash_probe_threads(kind: int) -> int:
    return int(_lib.dash_probe_threads(kind))


def dash_set_option(option: int, value: int) -> None:
    _check(_lib.dash_set_option(option, value), "dash_set_option")


def dash_get_option(option: int) -> int:
    v = int(_lib.dash_get_option(option))
    if v < 0:
        raise DashError(v, "dash_get_option")
    return v


def dash_hash4d_layout(L, F, log2_T, nmin_s, nmax_s, nmin_t, nmax_t, primes=PRIMES) -> dash_layout:
    """Eq. 7 level layout (host call)."""
    cfg = dash_hash4d_cfg(L, F, log2_T, 0, float(nmin_s), float(nmax_s), float(nmin_t), float(nmax_t),
                          (ctypes.c_uint32 * 4)(*primes))
    out = dash_layout()
    _check(_lib.dash_hash4d_layout(ctypes.byref(cfg), ctypes.byref(out)), "dash_hash4d_layout")
    return out


def layout_from(grid) -> dash_layout:
    """Layout from any object with L, F, log2_T, nmin_s, nmax_s, nmin_t, nmax_t, primes."""
    return dash_hash4d_layout(grid.L, grid.F, grid.log2_T, grid.nmin_s, grid.nmax_s, grid.nmin_t, grid.nmax_t,
                              grid.primes)


class Points:
    """Device coordinates (float32 CUDA tensors x, y, z of all Gaussians, t per
    Gaussian or a 1-element tensor broadcast), optional int32 index list and
    optional device int64 count (n is then a capacity)."""

    def __init__(self, x, y, z, t, idx=None, n=None, n_dev=None):
        for v in (x, y, z, t):
            assert v.is_cuda and v.dtype == torch.float32 and v.is_contiguous()
        if idx is not None:
            assert idx.is_cuda and idx.dtype == torch.int32 and idx.is_contiguous()
        if n_dev is not None:
            assert n_dev.is_cuda and n_dev.dtype == torch.int64
        self.x, self.y, self.z, self.t, self.idx, self.n_dev = x, y, z, t, idx, n_dev
        if n is None:
            n = idx.numel() if idx is not None else x.numel()
        self.n = int(n)
        self.t_stride = 0 if (t.numel() == 1 and x.numel() != 1) else 1
        self.c = dash_points(x.data_ptr(), y.data_ptr(), z.data_ptr(), t.data_ptr(), self.t_stride,
                             None if idx is None else idx.data_ptr(), self.n,
                             None if n_dev is None else n_dev.data_ptr())

    @property
    def device(self):
        return self.x.device


class Mlp:
    """Decoder description: packed FP32 parameters (a CUDA tensor this object
    keeps alive) and the widths D -> H -> H -> O."""

    def __init__(self, params: torch.Tensor, d_in: int, d_hidden: int, d_out: int):
        assert params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()
        two_layer = d_out == 3 and params.numel() == d_hidden * d_in + d_hidden + 3 * d_hidden + 3
        assert two_layer or params.numel() == mlp_param_count(d_in, d_hidden, d_out)
        self.params = params
        self.d_in, self.d_hidden, self.d_out = d_in, d_hidden, d_out
        self.c = dash_mlp(d_in, d_hidden, d_out, 0, params.data_ptr())


def mlp_param_count(d_in, d_hidden, d_out) -> int:
    return d_hidden * d_in + d_hidden + d_hidden * d_hidden + d_hidden + d_out * d_hidden + d_out


# ------------------------------------------------------- a1: compaction --
def dash_compact_workspace_size(n: int) -> int:
    return int(_lib.dash_compact_workspace_size(n))


def _check_compact_outputs(mask, idx_out, count_out):
    """The kernels write mask.numel() indices and one count: refuse buffers
    that could not hold them before anything is launched."""
    assert idx_out.device == mask.device and idx_out.dtype == torch.int32 and idx_out.is_contiguous(), \
        "idx_out: contiguous int32 on the mask's device"
    assert idx_out.numel() >= mask.numel(), f"idx_out holds {idx_out.numel()} < {mask.numel()} entries"
    assert count_out.device == mask.device and count_out.dtype == torch.int64 and count_out.numel() >= 1, \
        "count_out: int64 on the mask's device"


def dash_compact_dynamic(mask: torch.Tensor, idx_out=None, count_out=None, ws=None):
    """Ascending dynamic index list of a uint8 device mask; returns (idx int32 [n] buffer, count int64 [1])."""
    assert mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()
    n = mask.numel()
    dev = mask.device
    idx_out = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if idx_out is None else idx_out
    count_out = torch.empty(1, dtype=torch.int64, device=dev) if count_out is None else count_out
    _check_compact_outputs(mask, idx_out, count_out)
    need = dash_compact_workspace_size(n)
    ws = torch.empty(need, dtype=torch.uint8, device=dev) if ws is None else ws
    assert ws.device == dev and ws.dtype == torch.uint8 and ws.is_contiguous(), \
        "ws: contiguous uint8 on the mask's device"
    _check(_lib.dash_compact_dynamic(_ptr(mask), n, _ptr(idx_out), _ptr(count_out), _ptr(ws), ws.numel(),
                                     _stream()), "dash_compact_dynamic")
    return idx_out, count_out


def dash_compact_dynamic_noalloc(mask: torch.Tensor, idx_out: torch.Tensor, count_out: torch.Tensor):
    """Like dash_compact_dynamic, with the library's built-in scratch array
    instead of a workspace; the caller passes the (pre-allocated) outputs."""
    assert mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()
    _check_compact_outputs(mask, idx_out, count_out)
    _check(_lib.dash_compact_dynamic_noalloc(_ptr(mask), mask.numel(), _ptr(idx_out), _ptr(count_out), _stream()),
           "dash_compact_dynamic_noalloc")
    return idx_out, count_out


# ---------------------------------------------------------------- encoder --
def dash_hash4d_indices(layout: dash_layout, pts: Points, want_weights=True):
    idx = torch.empty((pts.n, layout.L, 16), dtype=torch.int32, device=pts.device)
    w = torch.empty((pts.n, layout.L, 16), dtype=torch.float32, device=pts.device) if want_weights else None
    _check(_lib.dash_hash4d_indices(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(idx), _ptr(w), _stream()),
           "dash_hash4d_indices")
    return idx, w


def dash_hash4d_fwd(layout: dash_layout, pts: Points, table: torch.Tensor, feat_dtype=torch.float32, out=None):
    out = torch.empty((pts.n, layout.L * layout.F), dtype=feat_dtype, device=pts.device) if out is None else out
    _check(_lib.dash_hash4d_fwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(table), _DTYPE_CODE[table.dtype],
                                _ptr(out), _DTYPE_CODE[out.dtype], _stream()), "dash_hash4d_fwd")
    return out


def dash_hash4d_bwd(layout: dash_layout, pts: Points, dfeat: torch.Tensor, table_grad: torch.Tensor):
    assert dfeat.dtype == torch.float32 and table_grad.dtype == torch.float32
    _check(_lib.dash_hash4d_bwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(dfeat), _ptr(table_grad),
                                _stream()), "dash_hash4d_bwd")
    return table_grad


def dash_hash4d_bwd_half(layout: dash_layout, pts: Points, dfeat: torch.Tensor, table_grad: torch.Tensor):
    """FP16-gradient variant of dash_hash4d_bwd (F = 2); table_grad float16 [offset[L]][2]."""
    assert dfeat.dtype == torch.float32 and table_grad.dtype == torch.float16
    _check(_lib.dash_hash4d_bwd_half(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(dfeat), _ptr(table_grad),
                                     _stream()), "dash_hash4d_bwd_half")
    return table_grad


# ------------------------------------------------------------ plain form --
def dash_hash4d_coord_grad(layout: dash_layout, pts: Points, table: torch.Tensor, dfeat: torch.Tensor, out=None):
    """d(sum dfeat . G_4D(p)) / d(x, y, z, t) per compact point, SoA [4][n] FP32."""
    out = torch.zeros((4, pts.n), dtype=torch.float32, device=pts.device) if out is None else out
    _check(_lib.dash_hash4d_coord_grad(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(table), _DTYPE_CODE[table.dtype],
                                       _ptr(dfeat), _ptr(out), _stream()), "dash_hash4d_coord_grad")
    return out


def dash_collision_workspace_size(layout: dash_layout, n: int) -> int:
    return int(_lib.dash_collision_workspace_size(ctypes.byref(layout), n))


def dash_hash4d_collision_stats(layout: dash_layout, pts: Points, out=None, ws=None):
    """Per level (V, E, C): touched vertices, occupied entries, colliding
    vertices, as a device int64 tensor [L][3]."""
    out = torch.empty((layout.L, 3), dtype=torch.int64, device=pts.device) if out is None else out
    if ws is None:
        ws = torch.empty(dash_collision_workspace_size(layout, pts.n), dtype=torch.uint8, device=pts.device)
    _check(_lib.dash_hash4d_collision_stats(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(out), _ptr(ws), ws.numel(),
                                            _stream()), "dash_hash4d_collision_stats")
    return out


def dash_plain_hash4d_fwd(layout, pts, table, out=None):
    assert table.dtype == torch.float32
    out = torch.empty((pts.n, layout.L * layout.F), dtype=torch.float32, device=pts.device) if out is None else out
    _check(_lib.dash_plain_hash4d_fwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(table), _ptr(out), _stream()),
           "dash_plain_hash4d_fwd")
    return out


def dash_plain_hash4d_bwd(layout, pts, dfeat, table_grad):
    _check(_lib.dash_plain_hash4d_bwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(dfeat), _ptr(table_grad),
                                      _stream()), "dash_plain_hash4d_bwd")
    return table_grad


def dash_plain_mlp_fwd(mlp: Mlp, feat, n=None, n_dev=None, out=None):
    n = feat.shape[0] if n is None else n
    out = torch.empty((mlp.d_out, n), dtype=torch.float32, device=feat.device) if out is None else out
    _check(_lib.dash_plain_mlp_fwd(ctypes.byref(mlp.c), _ptr(feat), n, _ptr(n_dev), _ptr(out), _stream()),
           "dash_plain_mlp_fwd")
    return out


def dash_plain_mlp_bwd_workspace_size(mlp: Mlp, n: int) -> int:
    return int(_lib.dash_plain_mlp_bwd_workspace_size(ctypes.byref(mlp.c), n))


def dash_plain_mlp_bwd(mlp: Mlp, feat, ddelta, mlp_grad, n=None, n_dev=None, dfeat=None, ws=None):
    n = feat.shape[0] if n is None else n
    dfeat = torch.empty((n, mlp.d_in), dtype=torch.float32, device=feat.device) if dfeat is None else dfeat
    need = dash_plain_mlp_bwd_workspace_size(mlp, n)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=feat.device) if ws is None else ws
    _check(_lib.dash_plain_mlp_bwd(ctypes.byref(mlp.c), _ptr(feat), n, _ptr(n_dev), _ptr(ddelta), _ptr(dfeat),
                                   _ptr(mlp_grad), _ptr(ws), ws.numel(), _stream()), "dash_plain_mlp_bwd")
    return dfeat


# ------------------------------------------------------------ fused form --
def dash_deform_state_size(mlp: Mlp) -> int:
    return int(_lib.dash_deform_state_size(ctypes.byref(mlp.c)))


def deform_state(mlp: Mlp, n: int, device) -> torch.Tensor:
    """Buffer for the per-Gaussian forward state (uint8 [n][state_size])."""
    return torch.empty((n, dash_deform_state_size(mlp)), dtype=torch.uint8, device=device)


def dash_deform_mlp_fwd(layout, pts, table, mlp: Mlp, delta_out=None, fwd_state=None, apply=None):
    """apply: optional (attrs_in [O][n_all], attrs_out [O][n_all]) float32 pair for Eq. 10."""
    delta_out = torch.empty((mlp.d_out, pts.n), dtype=torch.float32, device=pts.device) if delta_out is None else delta_out
    ap = None
    if apply is not None:
        ai, ao = apply
        ap = dash_apply(ai.data_ptr(), ao.data_ptr(), ai.shape[1])
    _check(_lib.dash_deform_mlp_fwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(table), _DTYPE_CODE[table.dtype],
                                    ctypes.byref(mlp.c), _ptr(delta_out), _ptr(fwd_state),
                                    None if ap is None else ctypes.byref(ap), _stream()), "dash_deform_mlp_fwd")
    return delta_out


def dash_deform_apply_bwd(pts: Points, dattrs: torch.Tensor, ddelta=None):
    """Gathers the dynamic rows of dattrs SoA [O][n_all] into ddelta SoA [O][pts.n]."""
    O, n_all = dattrs.shape
    ddelta = torch.zeros((O, pts.n), dtype=torch.float32, device=dattrs.device) if ddelta is None else ddelta
    _check(_lib.dash_deform_apply_bwd(ctypes.byref(pts.c), O, _ptr(dattrs), n_all, _ptr(ddelta), _stream()),
           "dash_deform_apply_bwd")
    return ddelta


def _smooth_struct(smooth):
    if smooth is None:
        return None
    lam, es, et, lo = smooth
    return dash_smooth(float(lam), (ctypes.c_float * 3)(*es), float(et), None if lo is None else lo.data_ptr())


def dash_deform_bwd_workspace_size(layout, n, smooth=None) -> int:
    """smooth: the (lambda_r, eps_s, eps_t, loss_out) tuple the backward will get, or None."""
    sm = _smooth_struct(smooth)
    return int(_lib.dash_deform_bwd_workspace_size(ctypes.byref(layout), int(n),
                                                   None if sm is None else ctypes.byref(sm)))


def dash_deform_mlp_bwd(layout, pts, table, mlp: Mlp, ddelta, table_grad, mlp_grad, fwd_state=None, smooth=None,
                        coord_grad=None, ws=None):
    """smooth: optional (lambda_r, (eps_x, eps_y, eps_z), eps_t, loss_out float32 [1] tensor or None).
    coord_grad: optional float32 [4][n] CUDA tensor receiving d loss / d(x, y, z, t).
    ws: a uint8 CUDA tensor of dash_deform_bwd_workspace_size bytes (gradient replicas and, with
    the Eq. 11 term, the dL/df_h hand-over), None to allocate one where it is used (a forward
    state given, F = 2), or False for the forms without it."""
    sm = _smooth_struct(smooth)
    if ws is None and fwd_state is not None and layout.F == 2:
        size = dash_deform_bwd_workspace_size(layout, pts.n, smooth)
        ws = torch.empty(size, dtype=torch.uint8, device=table.device) if size > 0 else False
    if ws is False:
        ws = None
    _check(_lib.dash_deform_mlp_bwd(ctypes.byref(layout), ctypes.byref(pts.c), _ptr(table), _DTYPE_CODE[table.dtype],
                                    ctypes.byref(mlp.c), _ptr(ddelta), _ptr(fwd_state), _ptr(table_grad),
                                    _ptr(mlp_grad), None if sm is None else ctypes.byref(sm), _ptr(coord_grad),
                                    _ptr(ws), 0 if ws is None else ws.numel() * ws.element_size(), _stream()),
           "dash_deform_mlp_bwd")


# ------------------------------------- decomposition producing the mask --
def dash_hash3d_layout(L, F, log2_T, nmin, nmax, primes=PRIMES) -> dash_layout:
    """3-D layout of the position encoder G_3D (host call)."""
    cfg = dash_hash4d_cfg(L, F, log2_T, 0, float(nmin), float(nmax), 1.0, 1.0, (ctypes.c_uint32 * 4)(*primes))
    out = dash_layout()
    _check(_lib.dash_hash3d_layout(ctypes.byref(cfg), ctypes.byref(out)), "dash_hash3d_layout")
    return out


def dash_decomp_fwd(layout3: dash_layout, x, y, z, table, mlp: "Mlp", dp_out=None, norm_out=None, want_dp=True,
                    t=None, pt_out=None):
    """(dp SoA [3][n] or None, norm [n]) of Eq. 3's positional deformation;
    with t (CUDA float32 [n] or [1]) returns (dp, norm, p(t) SoA [3][n]) of Eq. 4."""
    n = x.numel()
    if want_dp and dp_out is None:
        dp_out = torch.empty((3, n), dtype=torch.float32, device=x.device)
    norm_out = torch.empty(n, dtype=torch.float32, device=x.device) if norm_out is None else norm_out
    t_stride = 0
    if t is not None:
        assert t.is_cuda and t.dtype == torch.float32 and t.numel() in (1, n)
        t_stride = 0 if (t.numel() == 1 and n != 1) else 1
        pt_out = torch.empty((3, n), dtype=torch.float32, device=x.device) if pt_out is None else pt_out
    _check(_lib.dash_decomp_fwd(ctypes.byref(layout3), _ptr(x), _ptr(y), _ptr(z), n, _ptr(table),
                                _DTYPE_CODE[table.dtype], ctypes.byref(mlp.c), _ptr(dp_out if want_dp else None),
                                _ptr(norm_out), _ptr(t), t_stride, _ptr(pt_out if t is not None else None),
                                _stream()), "dash_decomp_fwd")
    dp = dp_out if want_dp else None
    return (dp, norm_out) if t is None else (dp, norm_out, pt_out)


def dash_decomp_bwd_workspace_size() -> int:
    return int(_lib.dash_decomp_bwd_workspace_size())


def dash_decomp_bwd(layout3: dash_layout, x, y, z, table, mlp: "Mlp", table_grad, mlp_grad, d_dp=None, mask=None,
                    lambda_s=0.0, ws=None):
    """Accumulates the G_3D table and decoder gradients of sum d_dp . dp + lambda_s L_s."""
    ws = torch.empty(dash_decomp_bwd_workspace_size(), dtype=torch.uint8, device=x.device) if ws is None else ws
    _check(_lib.dash_decomp_bwd(ctypes.byref(layout3), _ptr(x), _ptr(y), _ptr(z), x.numel(), _ptr(table),
                                _DTYPE_CODE[table.dtype], ctypes.byref(mlp.c), _ptr(d_dp), _ptr(mask), float(lambda_s),
                                _ptr(table_grad), _ptr(mlp_grad), _ptr(ws), ws.numel(), _stream()), "dash_decomp_bwd")
    return table_grad, mlp_grad


def dash_topk_workspace_size() -> int:
    return int(_lib.dash_topk_workspace_size())


def dash_topk_mask(values: torch.Tensor, k_percent: float, mask_out=None, tau_out=None, ws=None, static_loss_out=None):
    """(mask uint8 [n], tau float32 [1]): dynamic iff value > tau, tau the top-k % threshold.
    With static_loss_out (CUDA float32 [1]) also Eq. 5's L_s there."""
    n = values.numel()
    mask_out = torch.empty(n, dtype=torch.uint8, device=values.device) if mask_out is None else mask_out
    tau_out = torch.empty(1, dtype=torch.float32, device=values.device) if tau_out is None else tau_out
    if ws is None:
        ws = torch.empty(dash_topk_workspace_size(), dtype=torch.uint8, device=values.device)
    _check(_lib.dash_topk_mask(_ptr(values), n, float(k_percent), _ptr(mask_out), _ptr(tau_out), _ptr(static_loss_out),
                               _ptr(ws), ws.numel(), _stream()), "dash_topk_mask")
    return mask_out, tau_out


# ----------------------------------------------- splatting renderer ------
def camera(view, fx, fy, cx, cy, width, height, near=0.2, dilation=0.3, campos=(0.0, 0.0, 0.0),
           bg=(0.0, 0.0, 0.0)) -> dash_camera:
    """view: 16 floats, row-major world -> camera matrix."""
    v = [float(a) for a in view]
    assert len(v) == 16
    return dash_camera((ctypes.c_float * 16)(*v), fx, fy, cx, cy, int(width), int(height), near, dilation,
                       (ctypes.c_float * 3)(*campos), (ctypes.c_float * 3)(*bg))


class Gaussians:
    """Device SoA attributes (float32 CUDA tensors): mean [3][n], scale [3][n],
    rot [4][n] (w, x, y, z), opacity [n], sh [n][16][3]; kept alive here."""

    def __init__(self, mean, scale, rot, opacity, sh, sh_degree=3):
        n = mean.shape[1]
        for t_, shape in ((mean, (3, n)), (scale, (3, n)), (rot, (4, n)), (opacity, (n,)), (sh, (n, 16, 3))):
            assert t_.is_cuda and t_.dtype == torch.float32 and t_.is_contiguous() and tuple(t_.shape) == shape
        self.mean, self.scale, self.rot, self.opacity, self.sh = mean, scale, rot, opacity, sh
        self.n = n
        self.c = dash_gaussians(mean.data_ptr(), scale.data_ptr(), rot.data_ptr(), opacity.data_ptr(), sh.data_ptr(),
                                int(sh_degree), 0, n)


def dash_raster_workspace_size(cam: dash_camera, n: int, max_pairs: int) -> int:
    return int(_lib.dash_raster_workspace_size(ctypes.byref(cam), n, max_pairs))


def dash_raster_fwd(cam: dash_camera, g: Gaussians, image=None, ws=None, max_pairs=None, pairs_needed=None):
    """Renders [3][H][W]; returns (image, ws, max_pairs, pairs_needed).  Without
    max_pairs the capacity starts at 64 n + 4096 and the call is repeated with
    the needed capacity if the view exceeds it (one host synchronisation)."""
    dev = g.mean.device
    image = torch.empty((3, cam.height, cam.width), dtype=torch.float32, device=dev) if image is None else image
    pairs_needed = torch.zeros(1, dtype=torch.int64, device=dev) if pairs_needed is None else pairs_needed
    grow = max_pairs is None
    max_pairs = 64 * g.n + 4096 if max_pairs is None else int(max_pairs)
    while True:
        need = dash_raster_workspace_size(cam, g.n, max_pairs)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        _check(_lib.dash_raster_fwd(ctypes.byref(cam), ctypes.byref(g.c), _ptr(image), _ptr(ws), ws.numel(),
                                    max_pairs, _ptr(pairs_needed), _stream()), "dash_raster_fwd")
        if not grow:
            return image, ws, max_pairs, pairs_needed
        p = int(pairs_needed.item())
        if p <= max_pairs:
            return image, ws, max_pairs, pairs_needed
        max_pairs = p


def dash_raster_bwd(cam: dash_camera, g: Gaussians, dimage, ws, max_pairs: int, grads: dict):
    """Accumulates into grads (dict of float32 CUDA tensors mean, scale, rot,
    opacity, sh shaped like the attributes)."""
    gr = dash_gaussian_grads(*(grads[k].data_ptr() for k in ("mean", "scale", "rot", "opacity", "sh")))
    _check(_lib.dash_raster_bwd(ctypes.byref(cam), ctypes.byref(g.c), _ptr(dimage), _ptr(ws), ws.numel(), int(max_pairs),
                                ctypes.byref(gr), _stream()), "dash_raster_bwd")
    return grads


# ----------------------------------------------------- a12: batched form --
def dash_batch_plan_create(desc: dash_batch_desc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib.dash_batch_plan_create(ctypes.byref(desc), ctypes.byref(h)), "dash_batch_plan_create")
    return h


def dash_batch_counts(plan) -> int:
    """Device address of the plan's int64 live counts [n_scenes]."""
    return int(_lib.dash_batch_counts(plan))


def dash_batch_run(plan) -> None:
    _check(_lib.dash_batch_run(plan, _stream()), "dash_batch_run")


def dash_batch_form(plan) -> int:
    return int(_lib.dash_batch_form(plan))


def dash_batch_autotune(plan, cache_path=None) -> int:
    p = None if cache_path is None else str(cache_path).encode()
    _check(_lib.dash_batch_autotune(plan, p, _stream()), "dash_batch_autotune")
    return dash_batch_form(plan)


def dash_batch_plan_destroy(plan) -> None:
    _check(_lib.dash_batch_plan_destroy(plan), "dash_batch_plan_destroy")


class BatchPlan:
    """Owner of a dash_batch_plan.  scenes: list of dicts with CUDA tensors
    table, params, x, y, z, timestamps [K], delta_out [K][O][n]; with
    backward=True also ddelta [K][O][n] (upstream gradient), table_grad and
    mlp_grad (FP32, accumulated), and fwd_state [K][n][state size] uint8,
    allocated here when absent (the plan keeps references to all of them)."""

    def __init__(self, layout: dash_layout, scenes, d_in=32, d_hidden=64, d_out=10, backward=False):
        self.layout = layout
        self.scenes = scenes
        arr = (dash_batch_scene * len(scenes))()
        dt = None
        stride = int(_lib.dash_deform_state_size(ctypes.byref(dash_mlp(d_in, d_hidden, d_out, 0, None)))) \
            if backward else 0
        for i, sc in enumerate(scenes):
            dt = _DTYPE_CODE[sc["table"].dtype]
            n, K = sc["x"].numel(), sc["timestamps"].numel()
            bw = [None, None, None, None]
            if backward:
                if sc.get("fwd_state") is None:
                    sc["fwd_state"] = torch.empty((K, n, stride), dtype=torch.uint8, device=sc["x"].device)
                bw = [sc["ddelta"].data_ptr(), sc["fwd_state"].data_ptr(), sc["table_grad"].data_ptr(),
                      sc["mlp_grad"].data_ptr()]
            arr[i] = dash_batch_scene(sc["table"].data_ptr(), sc["params"].data_ptr(), sc["x"].data_ptr(),
                                      sc["y"].data_ptr(), sc["z"].data_ptr(), sc["timestamps"].data_ptr(),
                                      sc["delta_out"].data_ptr(), n, K, 0, *bw)
        self._arr = arr
        desc = dash_batch_desc(ctypes.addressof(layout), dt, d_in, d_hidden, d_out, len(scenes),
                               ctypes.addressof(arr), 1 if backward else 0, 0)
        self.handle = dash_batch_plan_create(desc)

    def counts(self) -> torch.Tensor:
        """The plan's live per-scene counts as an int64 CUDA tensor view
        [n_scenes]; stream-ordered writes to it are seen by the next run."""
        return _device_view_i64(dash_batch_counts(self.handle), len(self.scenes))

    def run(self) -> None:
        dash_batch_run(self.handle)

    def form(self) -> int:
        return dash_batch_form(self.handle)

    def autotune(self, cache_path=None) -> int:
        return dash_batch_autotune(self.handle, cache_path)

    def close(self) -> None:
        if self.handle:
            h, self.handle = self.handle, None
            dash_batch_plan_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view_i64(ptr: int, n: int) -> torch.Tensor:
    """An int64 CUDA tensor aliasing n values at a device address owned by libdash."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


# ------------------------------------------------------------- autograd --
class DashDeform(torch.autograd.Function):
    """delta = D(G_4D(x)) for the dynamic Gaussians (Sec. 4.2), differentiable
    with respect to the hash tables and the decoder parameters.

    forward runs dash_deform_mlp_fwd (keeping the per-Gaussian state); backward
    runs dash_deform_mlp_bwd.  With `smooth = (lambda_r, eps_s, eps_t,
    loss_out)` the backward also adds the gradient of lambda_r * L_r (Eq. 11)
    and accumulates its value into loss_out.  The table gradient is computed
    in FP32: with `table_grad` (an FP32 buffer shaped like the table) it is
    accumulated there and None is returned for the table; otherwise it is
    returned in the table's dtype."""

    @staticmethod
    def forward(ctx, table, params, layout, pts, dims, smooth=None, table_grad=None):
        mlp = Mlp(params, *dims)
        fsave = deform_state(mlp, pts.n, table.device)
        delta = dash_deform_mlp_fwd(layout, pts, table, mlp, fwd_state=fsave)
        ctx.save_for_backward(table, params, fsave)
        ctx.layout, ctx.pts, ctx.dims, ctx.smooth, ctx.table_grad = layout, pts, dims, smooth, table_grad
        return delta

    @staticmethod
    def backward(ctx, ddelta):
        table, params, fsave = ctx.saved_tensors
        mlp = Mlp(params, *ctx.dims)
        tg = ctx.table_grad
        if tg is None:
            tg = torch.zeros(table.shape, dtype=torch.float32, device=table.device)
        pg = torch.zeros_like(params)
        dash_deform_mlp_bwd(ctx.layout, ctx.pts, table, mlp, ddelta.contiguous().float(), tg, pg,
                            fwd_state=fsave, smooth=ctx.smooth)
        gtab = None if ctx.table_grad is not None else tg.to(table.dtype)
        return gtab, pg, None, None, None, None, None


def deform(table, params, layout, pts, dims=(32, 64, 10), smooth=None, table_grad=None):
    """Differentiable deformation offsets SoA [O][n] (see DashDeform)."""
    return DashDeform.apply(table, params, layout, pts, tuple(dims), smooth, table_grad)
