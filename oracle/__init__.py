"""FP64 CPU oracle for the DASH 4D-hash deformation path (arXiv 2507.19141,
Sec. 4.2-4.3, Eqs. 7-11).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package.  The
product library never imports it, and it imports nothing from the product.

The arithmetic lives in ``dash_oracle.c`` (plain C, double precision, one
Gaussian and one corner at a time); this module only compiles it with the host
C compiler and marshals NumPy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dash_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libdash_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 32


class Grid(ctypes.Structure):
    """Mirror of ``orc_grid``: the level layout of Eq. 7 plus the hash primes."""

    _fields_ = [
        ("L", ctypes.c_int32),
        ("F", ctypes.c_int32),
        ("log2_T", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("primes", ctypes.c_uint32 * 4),
        ("res_s", ctypes.c_int32 * MAX_LEVELS),
        ("res_t", ctypes.c_int32 * MAX_LEVELS),
        ("dense", ctypes.c_int32 * MAX_LEVELS),
        ("size", ctypes.c_int64 * MAX_LEVELS),
        ("offset", ctypes.c_int64 * (MAX_LEVELS + 1)),
    ]

    @property
    def total(self) -> int:
        return int(self.offset[self.L])

    def as_dict(self) -> dict:
        L = self.L
        return {
            "L": L,
            "F": self.F,
            "log2_T": self.log2_T,
            "res_s": list(self.res_s[:L]),
            "res_t": list(self.res_t[:L]),
            "dense": [bool(v) for v in self.dense[:L]],
            "size": list(self.size[:L]),
            "offset": list(self.offset[: L + 1]),
        }


def build(force: bool = False) -> str:
    """Compiles ``dash_oracle.c`` into a shared library (host gcc, -O2)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        # -ffp-contract=off: no fused multiply-add, every product rounds as written
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(build()))
    return _lib


def compile_variant(src_path: str, out_path: str) -> str:
    """Compiles another copy of the oracle source (the mutation tests plant
    mistakes in copies to show the pins catch them)."""
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", out_path, src_path,
                    "-lm"], check=True)
    return out_path


def configure(lib):
    """Declares the argument and result types of the oracle entry points on a loaded library."""
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    i32 = ctypes.c_int
    G = ctypes.POINTER(Grid)
    lib.orc_layout.argtypes = [G, i32, i32, i32, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, P]
    lib.orc_layout.restype = i32
    lib.orc_compact.argtypes = [P, i64, P]
    lib.orc_compact.restype = i64
    lib.orc_cell.argtypes = [G, i32, P, P, P]
    lib.orc_cell.restype = None
    pts = [P, P, P, P, i64, P, i64]
    lib.orc_corners.argtypes = [G] + pts + [P, P]
    lib.orc_corners.restype = None
    lib.orc_encode.argtypes = [G] + pts + [P, P]
    lib.orc_encode.restype = None
    lib.orc_encode_bwd.argtypes = [G] + pts + [P, P]
    lib.orc_encode_bwd.restype = None
    lib.orc_mlp_param_count.argtypes = [i32, i32, i32]
    lib.orc_mlp_param_count.restype = i64
    lib.orc_mlp_fwd.argtypes = [i32, i32, i32, P, P, i64, P]
    lib.orc_mlp_fwd.restype = i32
    lib.orc_mlp_bwd.argtypes = [i32, i32, i32, P, P, i64, P, P, P]
    lib.orc_mlp_bwd.restype = i32
    lib.orc_deform_fwd.argtypes = [G] + pts + [P, i32, i32, P, P, P, P, i64]
    lib.orc_deform_fwd.restype = i32
    lib.orc_deform_bwd.argtypes = [G] + pts + [P, i32, i32, P, P, P, P, ctypes.c_float, P,
                                               ctypes.c_float]
    lib.orc_deform_bwd.restype = ctypes.c_double
    lib.orc_smooth_loss.argtypes = [G] + pts + [P, ctypes.c_float, P, ctypes.c_float]
    lib.orc_smooth_loss.restype = ctypes.c_double
    lib.orc_layout3.argtypes = [G, i32, i32, i32, ctypes.c_double, ctypes.c_double, P]
    lib.orc_layout3.restype = i32
    lib.orc_cell3.argtypes = [G, i32, P, P, P]
    lib.orc_cell3.restype = None
    lib.orc_encode3.argtypes = [G, P, P, P, i64, P, P]
    lib.orc_encode3.restype = None
    lib.orc_decomp_fwd.argtypes = [G, P, P, P, i64, P, i32, P, P, P]
    lib.orc_decomp_fwd.restype = i32
    lib.orc_topk_mask.argtypes = [P, i64, ctypes.c_double, P]
    lib.orc_topk_mask.restype = ctypes.c_double
    lib.orc_encode_coord_grad.argtypes = [G, P, P, P, P, i64, P, i64, P, P, P]
    lib.orc_encode_coord_grad.restype = None
    lib.orc_collision_stats.argtypes = [G, P, P, P, P, i64, P, i64, P]
    lib.orc_collision_stats.restype = i32
    lib.orc_decomp_bwd.argtypes = [G, P, P, P, i64, P, i32, P, P, P, ctypes.c_double, P, P]
    lib.orc_decomp_bwd.restype = i32
    lib.orc_linear_motion.argtypes = [P, P, P, P, i64, P, i64, P]
    lib.orc_linear_motion.restype = None
    lib.orc_static_loss.argtypes = [P, P, i64]
    lib.orc_static_loss.restype = ctypes.c_double
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


DEFAULT_PRIMES = (1, 2654435761, 805459861, 3674653429)


def layout(L, F, log2_T, nmin_s, nmax_s, nmin_t, nmax_t, primes=DEFAULT_PRIMES) -> Grid:
    """Eq. 7 level layout (resolutions, dense/hashed decision, offsets)."""
    g = Grid()
    pr = np.asarray(primes, dtype=np.uint32)
    rc = _load().orc_layout(ctypes.byref(g), L, F, log2_T, float(nmin_s), float(nmax_s),
                            float(nmin_t), float(nmax_t), _ptr(pr))
    if rc != 0:
        raise ValueError("invalid hash-grid configuration")
    return g


def compact(mask: np.ndarray):
    """Ascending list of the Gaussians whose mask is set, and its length."""
    m = _c(mask, np.uint8)
    idx = np.zeros(max(len(m), 1), dtype=np.int32)
    cnt = _load().orc_compact(_ptr(m), len(m), _ptr(idx))
    return idx[:cnt].copy(), int(cnt)


class Points:
    """FP32 coordinates of the compact point set (x, y, z, t), optional index
    list into the full arrays, t either per point (t_stride=1) or one scalar
    broadcast to all (t_stride=0)."""

    def __init__(self, x, y, z, t, idx=None, t_stride=1, n=None):
        self.x = _c(x, np.float32)
        self.y = _c(y, np.float32)
        self.z = _c(z, np.float32)
        self.t = _c(t, np.float32)
        self.idx = _c(idx, np.int32)
        self.t_stride = int(t_stride)
        if n is None:
            n = len(self.idx) if self.idx is not None else len(self.x)
        self.n = int(n)

    def args(self):
        return [_ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.t), self.t_stride,
                _ptr(self.idx), self.n]


def cell(g: Grid, l: int, p):
    """Corner indices (level-local) and weights of one point at level l."""
    pf = np.asarray(p, dtype=np.float32)
    idx = np.zeros(16, dtype=np.uint32)
    w = np.zeros(16, dtype=np.float64)
    _load().orc_cell(ctypes.byref(g), l, _ptr(pf), _ptr(idx), _ptr(w))
    return idx, w


def corners(g: Grid, pts: Points):
    idx = np.zeros((pts.n, g.L, 16), dtype=np.uint32)
    w = np.zeros((pts.n, g.L, 16), dtype=np.float64)
    _load().orc_corners(ctypes.byref(g), *pts.args(), _ptr(idx), _ptr(w))
    return idx, w


def encode(g: Grid, pts: Points, table) -> np.ndarray:
    tab = _c(table, np.float64)
    assert tab.size == g.total * g.F
    out = np.zeros((pts.n, g.L * g.F), dtype=np.float64)
    _load().orc_encode(ctypes.byref(g), *pts.args(), _ptr(tab), _ptr(out))
    return out


def encode_bwd(g: Grid, pts: Points, dfeat, table_grad=None) -> np.ndarray:
    d = _c(dfeat, np.float64)
    tg = np.zeros((g.total, g.F), dtype=np.float64) if table_grad is None else table_grad
    assert tg.dtype == np.float64 and tg.flags.c_contiguous
    _load().orc_encode_bwd(ctypes.byref(g), *pts.args(), _ptr(d), _ptr(tg))
    return tg


def encode_coord_grad(g: Grid, pts: Points, table, dfeat) -> np.ndarray:
    """d(sum dfeat . G_4D(p)) / d(x, y, z, t) per compact point, SoA [4][n]."""
    tab = _c(table, np.float64)
    d = _c(dfeat, np.float64)
    out = np.zeros((4, pts.n), dtype=np.float64)
    _load().orc_encode_coord_grad(ctypes.byref(g), *pts.args(), _ptr(tab), _ptr(d), _ptr(out))
    return out


def collision_stats(g: Grid, pts: Points) -> np.ndarray:
    """Per level [V, E, C]: distinct touched vertices, distinct entries they
    occupy, touched vertices sharing their entry with another (int64 [L][3])."""
    out = np.zeros((g.L, 3), dtype=np.int64)
    if _load().orc_collision_stats(ctypes.byref(g), *pts.args(), _ptr(out)) != 0:
        raise MemoryError("collision statistics: out of host memory")
    return out


def mlp_param_count(D, H, O) -> int:
    return int(_load().orc_mlp_param_count(D, H, O))


def mlp_fwd(D, H, O, params, feat) -> np.ndarray:
    p = _c(params, np.float64)
    f = _c(feat, np.float64)
    n = f.shape[0]
    out = np.zeros((O, n), dtype=np.float64)
    if _load().orc_mlp_fwd(D, H, O, _ptr(p), _ptr(f), n, _ptr(out)) != 0:
        raise ValueError("unsupported MLP shape")
    return out


def mlp_bwd(D, H, O, params, feat, dout, param_grad=None):
    p = _c(params, np.float64)
    f = _c(feat, np.float64)
    d = _c(dout, np.float64)
    n = f.shape[0]
    dfeat = np.zeros((n, D), dtype=np.float64)
    pg = np.zeros(mlp_param_count(D, H, O), dtype=np.float64) if param_grad is None else param_grad
    if _load().orc_mlp_bwd(D, H, O, _ptr(p), _ptr(f), n, _ptr(d), _ptr(dfeat), _ptr(pg)) != 0:
        raise ValueError("unsupported MLP shape")
    return dfeat, pg


def deform_fwd(g: Grid, pts: Points, table, H, O, params, attrs_in=None):
    """Returns delta SoA [O][n] and, with attrs_in [O][n_all] (float32), the
    Eq. 10 result attrs_out (float64, static rows copied from attrs_in)."""
    tab = _c(table, np.float64)
    p = _c(params, np.float64)
    delta = np.zeros((O, pts.n), dtype=np.float64)
    ai = _c(attrs_in, np.float32)
    ao = None
    n_all = 0
    if ai is not None:
        n_all = ai.shape[1]
        ao = ai.astype(np.float64)
    rc = _load().orc_deform_fwd(ctypes.byref(g), *pts.args(), _ptr(tab), H, O, _ptr(p),
                                _ptr(delta), _ptr(ai), _ptr(ao), n_all)
    if rc != 0:
        raise ValueError("unsupported MLP shape")
    return (delta, ao) if ai is not None else delta


def deform_bwd(g: Grid, pts: Points, table, H, O, params, ddelta, lambda_r=0.0,
               eps_s=(0.0, 0.0, 0.0), eps_t=0.0, table_grad=None, param_grad=None):
    """Returns (table_grad [total][F], param_grad [P], lambda_r * L_r)."""
    tab = _c(table, np.float64)
    p = _c(params, np.float64)
    dd = _c(ddelta, np.float64)
    D = g.L * g.F
    tg = np.zeros((g.total, g.F), dtype=np.float64) if table_grad is None else table_grad
    pg = np.zeros(mlp_param_count(D, H, O), dtype=np.float64) if param_grad is None else param_grad
    es = np.asarray(eps_s, dtype=np.float32)
    loss = _load().orc_deform_bwd(ctypes.byref(g), *pts.args(), _ptr(tab), H, O, _ptr(p),
                                  _ptr(dd), _ptr(tg), _ptr(pg), float(lambda_r), _ptr(es),
                                  float(eps_t))
    return tg, pg, float(loss)


def smooth_loss(g: Grid, pts: Points, table, lambda_r, eps_s, eps_t) -> float:
    tab = _c(table, np.float64)
    es = np.asarray(eps_s, dtype=np.float32)
    return float(_load().orc_smooth_loss(ctypes.byref(g), *pts.args(), _ptr(tab),
                                         float(lambda_r), _ptr(es), float(eps_t)))


# ------------------------------------------------ decomposition (Sec. 4.1) --
def layout3(L, F, log2_T, nmin, nmax, primes=DEFAULT_PRIMES) -> Grid:
    """3-D level layout of G_3D (Eq. 7 progression, (N+1)^3 dense vertices)."""
    g = Grid()
    pr = np.asarray(primes, dtype=np.uint32)
    if _load().orc_layout3(ctypes.byref(g), L, F, log2_T, float(nmin), float(nmax), _ptr(pr)) != 0:
        raise ValueError("invalid hash-grid configuration")
    return g


def cell3(g: Grid, l: int, p):
    pf = np.asarray(p, dtype=np.float32)
    idx = np.zeros(8, dtype=np.uint32)
    w = np.zeros(8, dtype=np.float64)
    _load().orc_cell3(ctypes.byref(g), l, _ptr(pf), _ptr(idx), _ptr(w))
    return idx, w


def encode3(g: Grid, x, y, z, table) -> np.ndarray:
    xs, ys, zs = (_c(v, np.float32) for v in (x, y, z))
    tab = _c(table, np.float64)
    n = len(xs)
    out = np.zeros((n, g.L * g.F), dtype=np.float64)
    _load().orc_encode3(ctypes.byref(g), _ptr(xs), _ptr(ys), _ptr(zs), n, _ptr(tab), _ptr(out))
    return out


def decomp_fwd(g: Grid, x, y, z, table, H, params):
    """Returns (dp SoA [3][n], norm [n]) of Eqs. 3-4's positional deformation."""
    xs, ys, zs = (_c(v, np.float32) for v in (x, y, z))
    tab = _c(table, np.float64)
    p = _c(params, np.float64)
    n = len(xs)
    dp = np.zeros((3, n), dtype=np.float64)
    norm = np.zeros(n, dtype=np.float64)
    if _load().orc_decomp_fwd(ctypes.byref(g), _ptr(xs), _ptr(ys), _ptr(zs), n, _ptr(tab), H, _ptr(p), _ptr(dp),
                              _ptr(norm)) != 0:
        raise ValueError("unsupported MLP shape")
    return dp, norm


def decomp_bwd(g: Grid, x, y, z, table, H, params, d_dp=None, mask=None, lambda_s=0.0):
    """(table_grad [total][F], param_grad) of sum d_dp . dp + lambda_s L_s."""
    xs, ys, zs = (_c(v, np.float32) for v in (x, y, z))
    tab = _c(table, np.float64)
    p = _c(params, np.float64)
    dd = _c(d_dp, np.float64)
    m = _c(mask, np.uint8)
    tg = np.zeros((g.total, g.F), dtype=np.float64)
    pg = np.zeros(len(p), dtype=np.float64)
    if _load().orc_decomp_bwd(ctypes.byref(g), _ptr(xs), _ptr(ys), _ptr(zs), len(xs), _ptr(tab), H, _ptr(p), _ptr(dd),
                              _ptr(m), float(lambda_s), _ptr(tg), _ptr(pg)) != 0:
        raise ValueError("unsupported MLP shape")
    return tg, pg


def linear_motion(x, y, z, t, dp):
    """Eq. 4: p(t) = p + t dp, SoA [3][n]; t has n values or one."""
    xs, ys, zs = (_c(v, np.float32) for v in (x, y, z))
    ts = _c(np.atleast_1d(t), np.float32)
    d = _c(dp, np.float64)
    n = len(xs)
    out = np.zeros((3, n), dtype=np.float64)
    _load().orc_linear_motion(_ptr(xs), _ptr(ys), _ptr(zs), _ptr(ts), 0 if len(ts) == 1 and n != 1 else 1,
                              _ptr(d), n, _ptr(out))
    return out


def static_loss(norm, mask) -> float:
    """Eq. 5: mean |dp| over the static Gaussians (mask 0)."""
    v = _c(norm, np.float64)
    m = _c(mask, np.uint8)
    return float(_load().orc_static_loss(_ptr(v), _ptr(m), len(v)))


def topk_mask(values, k_percent):
    """(mask uint8 [n], tau): dynamic iff value > tau, tau the (m+1)-th largest, m = floor(k n / 100)."""
    v = _c(values, np.float64)
    mask = np.zeros(max(len(v), 1), dtype=np.uint8)
    tau = _load().orc_topk_mask(_ptr(v), len(v), float(k_percent), _ptr(mask))
    return mask[:len(v)].copy(), float(tau)
