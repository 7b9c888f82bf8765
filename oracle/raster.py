"""FP64 CPU oracle of the 3D Gaussian splatting renderer the deformed
Gaussians are drawn with (Sec. 3: Eq. 1, the covariance factorisation and its
screen-space projection, spherical-harmonics colour, Eq. 2 alpha blending).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs may import this module; the product never does.  It is
plain PyTorch on the CPU in float64; its gradients come from autograd of the
forward written here, so the backward needs no separate derivation.

Readings (the paper defers the renderer to 3DGS and states none of these):
  - camera: world -> camera by a 4x4 matrix V (row-major, acting on column
    vectors); pinhole projection u = fx x/z + cx, v = fy y/z + cy in pixel
    units; pixel (i, j) is evaluated at (i, j); Gaussians with z <= near are
    not drawn.
  - Sigma = R S S^T R^T with R from the normalised quaternion (w, x, y, z) and
    S = diag(scale); Sigma' = J V_r Sigma V_r^T J^T with J the Jacobian of
    the projection at the camera-space mean (no clamping of x/z, y/z), plus
    `dilation` on the diagonal (a screen-space low-pass; 0.3 in 3DGS);
    Gaussians with det(Sigma') <= 0 are not drawn.
  - Eq. 1 on the screen: alpha = min(0.99, sigma exp(-0.5 d^T Sigma'^-1 d)),
    d = mean' - pixel; contributions with alpha < 1/255 or a positive exponent
    are skipped.
  - extent: r = ceil(3 sqrt(lambda_max(Sigma'))); a Gaussian is considered only
    for the 16x16 pixel tiles its square [u - r, u + r] x [v - r, v + r]
    overlaps; tiles [floor((u - r)/16), floor((u + r)/16)], clipped.
  - order: ascending camera depth z, ties by Gaussian index.
  - Eq. 2 front to back with T the transmittance; blending stops before the
    first Gaussian that would take T below 1e-4; the background colour is
    added with the final T.
  - colour: real spherical harmonics up to degree 3 (orthonormal on the
    sphere, no Condon-Shortley phase) at the unit direction from the camera
    centre to the mean, plus 0.5, clamped below at 0.
"""
from __future__ import annotations

import math

import torch

TILE = 16
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """[n, 4] quaternions (w, x, y, z), any norm -> [n, 3, 3] rotations."""
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Real orthonormal spherical harmonics at unit directions d [n, 3]:
    [n, (degree+1)^2], ordered by degree then m = -l..l."""
    x, y, z = d.unbind(1)
    pi = math.pi
    out = [torch.full_like(x, 0.5 / math.sqrt(pi))]
    if degree >= 1:
        k = math.sqrt(3 / (4 * pi))
        out += [k * y, k * z, k * x]
    if degree >= 2:
        a = 0.5 * math.sqrt(15 / pi)
        out += [a * x * y, a * y * z, 0.25 * math.sqrt(5 / pi) * (3 * z * z - 1), a * x * z,
                0.25 * math.sqrt(15 / pi) * (x * x - y * y)]
    if degree >= 3:
        out += [0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
                0.5 * math.sqrt(105 / pi) * x * y * z,
                0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
                0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
                0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
                0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
                0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y)]
    return torch.stack(out, 1)


def screen_cov(cam: dict, mean, scale, rot):
    """Sigma' = J V_r R S S^T R^T V_r^T J^T before the dilation, [n, 2, 2]."""
    V = torch.as_tensor(cam["view"], dtype=torch.float64).reshape(4, 4)
    Vr, Vt = V[:3, :3], V[:3, 3]
    t = mean @ Vr.T + Vt
    tx, ty, tz = t.unbind(1)
    fx, fy = cam["fx"], cam["fy"]
    M = quat_to_rotmat(rot) * scale[:, None, :]
    zero = torch.zeros_like(tz)
    J = torch.stack([torch.stack([fx / tz, zero, -fx * tx / (tz * tz)], -1),
                     torch.stack([zero, fy / tz, -fy * ty / (tz * tz)], -1)], 1)
    T = J @ Vr
    return T @ (M @ M.transpose(1, 2)) @ T.transpose(1, 2)


def project(cam: dict, mean, scale, rot, opacity, sh, sh_degree: int):
    """Per-Gaussian screen quantities (differentiable): dict of mean2d [n, 2],
    conic [n, 3] (a, b, c of Sigma'^-1), opacity [n], color [n, 3], depth [n],
    radius [n] (int), visible [n] (bool)."""
    V = torch.as_tensor(cam["view"], dtype=torch.float64).reshape(4, 4)
    t = mean @ V[:3, :3].T + V[:3, 3]
    tx, ty, tz = t.unbind(1)
    fx, fy = cam["fx"], cam["fy"]
    S2 = screen_cov(cam, mean, scale, rot)
    a = S2[:, 0, 0] + cam["dilation"]
    b = S2[:, 0, 1]
    c = S2[:, 1, 1] + cam["dilation"]
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], 1)
    mid = 0.5 * (a + c)
    lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.0))
    radius = torch.ceil(3.0 * torch.sqrt(lam.detach())).to(torch.int64)
    u = fx * tx / tz + cam["cx"]
    v = fy * ty / tz + cam["cy"]
    campos = torch.as_tensor(cam["campos"], dtype=torch.float64)
    dirs = mean - campos
    dirs = dirs / dirs.norm(dim=1, keepdim=True)
    K = (sh_degree + 1) ** 2
    rgb = (sh[:, :K, :] * sh_basis(dirs, sh_degree)[:, :, None]).sum(1) + 0.5
    color = torch.clamp(rgb, min=0.0)
    visible = (tz.detach() > cam["near"]) & (det.detach() > 0)
    return {"mean2d": torch.stack([u, v], 1), "conic": conic, "opacity": opacity, "color": color,
            "depth": tz, "radius": radius, "visible": visible}


def tile_rect(cam: dict, mean2d, radius):
    """[n, 4] tile ranges x0, y0, x1, y1 (exclusive ends) of each square extent."""
    tx_n = (cam["width"] + TILE - 1) // TILE
    ty_n = (cam["height"] + TILE - 1) // TILE
    u, v = mean2d.detach().unbind(1)
    r = radius.to(torch.float64)
    x0 = torch.clamp(torch.floor((u - r) / TILE), 0, tx_n).to(torch.int64)
    x1 = torch.clamp(torch.floor((u + r) / TILE) + 1, 0, tx_n).to(torch.int64)
    y0 = torch.clamp(torch.floor((v - r) / TILE), 0, ty_n).to(torch.int64)
    y1 = torch.clamp(torch.floor((v + r) / TILE) + 1, 0, ty_n).to(torch.int64)
    return torch.stack([x0, y0, x1, y1], 1)


def render(cam: dict, mean, scale, rot, opacity, sh, sh_degree: int):
    """Image [3, H, W] (differentiable w.r.t. all Gaussian inputs), final
    transmittance [H, W] and the number of Gaussians blended per pixel."""
    p = project(cam, mean, scale, rot, opacity, sh, sh_degree)
    W_, H_ = cam["width"], cam["height"]
    bg = torch.as_tensor(cam["bg"], dtype=torch.float64)
    rect = tile_rect(cam, p["mean2d"], p["radius"])
    ok = p["visible"] & (rect[:, 0] < rect[:, 2]) & (rect[:, 1] < rect[:, 3])
    n = mean.shape[0]
    depth = p["depth"].detach()
    order = sorted((i for i in range(n) if bool(ok[i])), key=lambda i: (float(depth[i]), i))
    rl = rect.tolist()
    final_T = torch.ones(H_, W_, dtype=torch.float64)
    count = torch.zeros(H_, W_, dtype=torch.int64)
    image = [[None] * ((W_ + TILE - 1) // TILE) for _ in range((H_ + TILE - 1) // TILE)]
    for ty in range((H_ + TILE - 1) // TILE):
        for tx in range((W_ + TILE - 1) // TILE):
            ids = [i for i in order if rl[i][0] <= tx < rl[i][2] and rl[i][1] <= ty < rl[i][3]]
            px = torch.arange(tx * TILE, min(tx * TILE + TILE, W_), dtype=torch.float64)
            py = torch.arange(ty * TILE, min(ty * TILE + TILE, H_), dtype=torch.float64)
            gy, gx = torch.meshgrid(py, px, indexing="ij")
            gx, gy = gx.reshape(-1), gy.reshape(-1)
            if not ids:
                image[ty][tx] = bg[:, None].expand(3, gx.numel())
                continue
            idx = torch.tensor(ids)
            m2 = p["mean2d"][idx]
            con = p["conic"][idx]
            dx = m2[None, :, 0] - gx[:, None]
            dy = m2[None, :, 1] - gy[:, None]
            power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy
            alpha = torch.clamp(p["opacity"][idx][None, :] * torch.exp(power), max=ALPHA_MAX)
            take = (power.detach() <= 0) & (alpha.detach() >= ALPHA_MIN)
            a = torch.where(take, alpha, torch.zeros_like(alpha))
            one_minus = 1.0 - a
            T_incl = torch.cumprod(one_minus, dim=1)
            T_excl = torch.cat([torch.ones_like(T_incl[:, :1]), T_incl[:, :-1]], 1)
            # Eq. 2 stops before the first Gaussian that would take T below 1e-4
            alive = T_incl.detach() >= T_MIN
            alive = torch.cumprod(alive.to(torch.int64), dim=1).to(torch.bool)
            w = torch.where(alive, a * T_excl, torch.zeros_like(a))
            rgb = w @ p["color"][idx]                                     # [pix, 3]
            last = alive.sum(1)                                           # alive is a prefix
            Tf = torch.gather(torch.cat([torch.ones_like(T_incl[:, :1]), T_incl], 1), 1, last[:, None])[:, 0]
            image[ty][tx] = (rgb + Tf[:, None] * bg[None, :]).T
            pos = (gy.long(), gx.long())
            final_T[pos] = Tf.detach()
            count[pos] = (alive & take).sum(1)
    out = []
    for ty in range(len(image)):
        band = torch.cat([image[ty][tx].reshape(3, -1, min(TILE, W_ - tx * TILE)) for tx in range(len(image[ty]))], 2)
        out.append(band)
    full = torch.cat(out, 1)
    return full, final_T, count
