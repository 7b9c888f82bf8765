"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's datasets (Neural 3D Video, Technicolor; arXiv 2507.19141 Sec. 5.1)
are not available, so every input is drawn here from fixed seeds with the
shapes and value distributions of those workloads: normalised 4-D coordinates
of dynamic Gaussians, a static/dynamic mask, FP16/FP32 hash tables, BF16 MLP
weights and upstream gradients.

This module only draws numbers.  It holds none of the method's arithmetic, and
both the CUDA path's tests and the CPU oracle take their inputs from it.
Values that the GPU stores at reduced precision (FP16 tables, BF16 weights) are
rounded here, once, so both sides see bit-identical parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PRIMES = (1, 2654435761, 805459861, 3674653429)


@dataclass(frozen=True)
class GridCfg:
    """Hash-grid hyper-parameters of Sec. 4.2: levels L, features per level F,
    hashed-table size 2^log2_T, coarsest/finest spatial and temporal resolutions."""

    L: int = 16
    F: int = 2
    log2_T: int = 19
    nmin_s: float = 16.0
    nmax_s: float = 2048.0
    nmin_t: float = 8.0
    nmax_t: float = 150.0
    primes: tuple = PRIMES


@dataclass(frozen=True)
class MlpCfg:
    d_in: int = 32
    d_hidden: int = 64
    d_out: int = 10

    @property
    def n_params(self) -> int:
        D, H, O = self.d_in, self.d_hidden, self.d_out
        return H * D + H + H * H + H + O * H + O


TINY_GRID = GridCfg(L=4, F=2, log2_T=14, nmin_s=16, nmax_s=128, nmin_t=8, nmax_t=32)
TINY_MLP = MlpCfg(d_in=8)
PAPER_GRID = GridCfg()
PAPER_MLP = MlpCfg()


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Rounds float32 values to the nearest BF16-representable float32 (ties to even)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def uniform_coords(rng, n):
    """x, y, z, t ~ U[0,1] (float32)."""
    return tuple(rng.random(n).astype(np.float32) for _ in range(4))


def scene_coords(rng, n):
    """x, y, z ~ N(0.5, 0.15) clipped to [0,1]; t ~ U[0,1] (float32)."""
    xyz = [np.clip(rng.normal(0.5, 0.15, n), 0.0, 1.0).astype(np.float32) for _ in range(3)]
    t = rng.random(n).astype(np.float32)
    return xyz[0], xyz[1], xyz[2], t


def bernoulli_mask(rng, n, p=0.5):
    return (rng.random(n) < p).astype(np.uint8)


def exact_count_mask(rng, n, k):
    """A mask with exactly k set entries at uniformly random positions."""
    m = np.zeros(n, dtype=np.uint8)
    m[rng.choice(n, size=k, replace=False)] = 1
    return m


def table_values(rng, total_entries, F, dtype):
    """Hash-table features ~ U[-1,1], stored as `dtype` (np.float16 / np.float32)."""
    return rng.uniform(-1.0, 1.0, size=(total_entries, F)).astype(dtype)


def mlp_params(rng, mlp: MlpCfg, bf16: bool = True):
    """Packed W1 [H][D], b1, W2 [H][H], b2, W3 [O][H], b3 ~ U[-1/sqrt(fan_in), +],
    float32, rounded to BF16-representable values when `bf16`."""
    D, H, O = mlp.d_in, mlp.d_hidden, mlp.d_out
    parts = []
    for fan_out, fan_in in ((H, D), (H, H), (O, H)):
        k = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-k, k, size=fan_out * fan_in))
        parts.append(rng.uniform(-k, k, size=fan_out))
    p = np.concatenate(parts).astype(np.float32)
    return bf16_round(p) if bf16 else p


def upstream_grad(rng, O, n):
    """dL/d(delta) ~ N(0,1), SoA [O][n] float32."""
    return rng.standard_normal((O, n)).astype(np.float32)


def gaussian_attrs(rng, n_all):
    """Canonical Gaussian attributes for Eq. 10, SoA [10][n_all] float32:
    position (3), rotation quaternion (4), log-scale (3)."""
    pos = rng.uniform(-1.0, 1.0, size=(3, n_all))
    q = rng.standard_normal((4, n_all))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    s = rng.uniform(-5.0, -2.0, size=(3, n_all))
    return np.concatenate([pos, q, s]).astype(np.float32)


@dataclass
class Workload:
    grid: GridCfg
    mlp: MlpCfg
    coords: tuple            # x, y, z, t of all Gaussians (float32, length n_all)
    mask: np.ndarray | None  # uint8 [n_all] or None (all dynamic)
    table_dtype: type
    seed: int
    extra: dict = field(default_factory=dict)


def tiny(seed=0, n=10_000):
    """Plain FP32 case: N=10k, xyzt ~ U[0,1], L=4, F=2, T=2^14, 16->128, 8->32, MLP 8-64-64-10."""
    rng = np.random.default_rng(seed)
    coords = uniform_coords(rng, n)
    return Workload(TINY_GRID, TINY_MLP, coords, None, np.float32, seed)


def paper_plain(seed=1, n_all=600_000):
    """Paper-shaped plain FP32: 600k Gaussians, Bernoulli(0.5) mask, scene coordinates."""
    rng = np.random.default_rng(seed)
    mask = bernoulli_mask(rng, n_all)
    coords = scene_coords(rng, n_all)
    return Workload(PAPER_GRID, PAPER_MLP, coords, mask, np.float32, seed)


def precision(seed=2, n_dyn=1_000_000, n_all=None):
    """Precision form: n_dyn dynamic Gaussians (of n_all, mask with exactly n_dyn set when
    n_all is given), FP16 tables, BF16 MLP, scene coordinates."""
    rng = np.random.default_rng(seed)
    if n_all is None:
        coords = scene_coords(rng, n_dyn)
        mask = None
    else:
        mask = exact_count_mask(rng, n_all, n_dyn)
        coords = scene_coords(rng, n_all)
    return Workload(PAPER_GRID, PAPER_MLP, coords, mask, np.float16, seed)


def batched(seed=4, scenes=8, timestamps=64, n_lo=50_000, n_hi=2_000_000, frames=300):
    """Batched form: per-scene dynamic counts log-uniform in [n_lo, n_hi], `timestamps`
    distinct sorted frames of a `frames`-frame sequence per scene, t = frame/(frames-1)."""
    rng = np.random.default_rng(seed)
    counts = [int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))) for _ in range(scenes)]
    ts = []
    for _ in range(scenes):
        f = np.sort(rng.choice(frames, size=timestamps, replace=False))
        ts.append((f / (frames - 1)).astype(np.float32))
    return counts, ts, rng


def raster_scene(rng, n, width, height, sh_degree=3, depth=(2.0, 8.0), spread=0.6, scale=(0.004, 0.04)):
    """Gaussians in front of a camera (float32 arrays): means with depth
    z ~ U[depth] and x, y ~ U[-spread z, spread z]; scales log-uniform in
    [scale] times z; random quaternions (w, x, y, z); opacity ~ U[0.05, 0.95];
    SH coefficients [n][16][3] ~ N(0, 0.25) beyond degree 0 and a degree-0
    term giving colours ~ U[0, 1].  The camera (dict) sits at campos with a
    small rotation about y; fx = fy = 0.8 width."""
    z = rng.uniform(*depth, n)
    x = rng.uniform(-spread, spread, n) * z
    y = rng.uniform(-spread, spread, n) * z * height / width
    mean_cam = np.stack([x, y, z])
    theta = 0.1
    Rv = np.array([[math.cos(theta), 0.0, math.sin(theta)], [0.0, 1.0, 0.0], [-math.sin(theta), 0.0, math.cos(theta)]])
    tv = np.array([0.05, -0.03, 0.2])
    mean = Rv.T @ (mean_cam - tv[:, None])          # world positions whose camera coordinates are mean_cam
    sc = np.exp(rng.uniform(np.log(scale[0]), np.log(scale[1]), (3, n))) * z[None, :]
    q = rng.standard_normal((4, n))
    opacity = rng.uniform(0.05, 0.95, n)
    sh = rng.standard_normal((n, 16, 3)) * 0.25
    sh[:, 0, :] = (rng.uniform(0.0, 1.0, (n, 3)) - 0.5) * 2.0 * math.sqrt(math.pi)
    if sh_degree < 3:
        sh[:, (sh_degree + 1) ** 2:, :] = 0.0
    view = np.eye(4)
    view[:3, :3] = Rv
    view[:3, 3] = tv
    cam = {"view": view.reshape(-1).tolist(), "fx": 0.8 * width, "fy": 0.8 * width, "cx": width / 2,
           "cy": height / 2, "width": width, "height": height, "near": 0.2, "dilation": 0.3,
           "campos": (-Rv.T @ tv).tolist(), "bg": [0.1, 0.15, 0.2]}
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return cam, {"mean": f32(mean), "scale": f32(sc), "rot": f32(q), "opacity": f32(opacity), "sh": f32(sh)}
