"""Pins of the renderer oracle (Sec. 3: Eq. 1, Sigma = R S S^T R^T, the
screen-space covariance, spherical-harmonics colour, Eq. 2)."""
import math

import numpy as np
import pytest
import torch

from oracle import raster


def _cam(w=64, h=48, **kw):
    c = {"view": np.eye(4).reshape(-1).tolist(), "fx": 60.0, "fy": 62.0, "cx": w / 2, "cy": h / 2, "width": w,
         "height": h, "near": 0.2, "dilation": 0.3, "campos": [0.0, 0.0, 0.0], "bg": [0.1, 0.2, 0.3]}
    c.update(kw)
    return c


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64))


def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(1)
    q = rng.standard_normal((50, 4)) * rng.uniform(0.1, 3, (50, 1))
    R = raster.quat_to_rotmat(_t(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()       # scipy takes (x, y, z, w)
    assert np.max(np.abs(R - ref)) < 1e-12


def test_covariance_eigen_and_screen_projection_by_finite_differences():
    rng = np.random.default_rng(2)
    n = 20
    mean = np.c_[rng.uniform(-1, 1, (n, 2)), rng.uniform(2, 6, n)]
    scale = rng.uniform(0.01, 0.3, (n, 3))
    q = rng.standard_normal((n, 4))
    theta = 0.3
    V = np.eye(4)
    V[:3, :3] = [[math.cos(theta), 0, math.sin(theta)], [0, 1, 0], [-math.sin(theta), 0, math.cos(theta)]]
    V[:3, 3] = [0.1, -0.2, 0.5]
    cam = _cam(view=V.reshape(-1).tolist())
    R = raster.quat_to_rotmat(_t(q))
    Sigma = R @ torch.diag_embed(_t(scale) ** 2) @ R.transpose(1, 2)
    ev = torch.linalg.eigvalsh(Sigma).numpy()
    assert np.max(np.abs(np.sort(ev, 1) - np.sort(scale ** 2, 1))) < 1e-13
    S2 = raster.screen_cov(cam, _t(mean), _t(scale), _t(q)).numpy()

    def pix(m):                                     # pinhole projection of a world point
        c = V[:3, :3] @ m + V[:3, 3]
        return np.array([cam["fx"] * c[0] / c[2] + cam["cx"], cam["fy"] * c[1] / c[2] + cam["cy"]])

    h = 1e-6
    for i in range(n):
        Jfd = np.stack([(pix(mean[i] + h * e) - pix(mean[i] - h * e)) / (2 * h) for e in np.eye(3)], 1)
        ref = Jfd @ Sigma[i].numpy() @ Jfd.T
        assert np.max(np.abs(S2[i] - ref)) < 1e-6 * max(1.0, np.abs(ref).max())


def test_sh_basis_is_orthonormal_on_the_sphere():
    from scipy.special import roots_legendre
    ct, wt = roots_legendre(24)                     # exact for polynomials of degree < 48 in cos(theta)
    phi = np.arange(48) * 2 * np.pi / 48            # exact for trigonometric degree < 48
    C, P = np.meshgrid(ct, phi, indexing="ij")
    st = np.sqrt(1 - C ** 2)
    d = np.stack([st * np.cos(P), st * np.sin(P), C], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(48, 2 * np.pi / 48)[None, :]).reshape(-1)
    Y = raster.sh_basis(_t(d), 3).numpy()
    G = (Y * w[:, None]).T @ Y
    assert np.max(np.abs(G - np.eye(16))) < 1e-12


def _scene(means, scales, opac, colors, quat=None):
    n = len(means)
    sh = np.zeros((n, 16, 3))
    sh[:, 0, :] = (np.asarray(colors) - 0.5) * 2 * math.sqrt(math.pi)   # degree 0 only: rgb = colors
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if quat is None else quat
    return _t(means), _t(scales), _t(q), _t(opac), _t(sh)


def test_single_and_two_gaussians_closed_form():
    cam = _cam()
    # mean projects exactly onto pixel (40, 20): u = fx x / z + cx
    z = 4.0
    x, y = (40 - cam["cx"]) * z / cam["fx"], (20 - cam["cy"]) * z / cam["fy"]
    img, T, cnt = raster.render(cam, *_scene([[x, y, z]], [[0.05] * 3], [0.6], [[0.9, 0.4, 0.2]]), 3)
    bg = np.array(cam["bg"])
    assert np.max(np.abs(img[:, 20, 40].numpy() - (0.6 * np.array([0.9, 0.4, 0.2]) + 0.4 * bg))) < 1e-12
    assert abs(float(T[20, 40]) - 0.4) < 1e-12 and int(cnt[20, 40]) == 1
    # two at the same pixel; the nearer one is given second: order is by depth, not input
    z2 = 6.0
    x2, y2 = (40 - cam["cx"]) * z2 / cam["fx"], (20 - cam["cy"]) * z2 / cam["fy"]
    img, T, cnt = raster.render(cam, *_scene([[x2, y2, z2], [x, y, z]], [[0.05] * 3] * 2, [0.5, 0.6],
                                             [[0.0, 1.0, 0.0], [0.9, 0.4, 0.2]]), 3)
    want = 0.6 * np.array([0.9, 0.4, 0.2]) + 0.4 * 0.5 * np.array([0.0, 1.0, 0.0]) + 0.4 * 0.5 * bg
    assert np.max(np.abs(img[:, 20, 40].numpy() - want)) < 1e-12 and int(cnt[20, 40]) == 2


def test_anisotropic_gaussian_follows_eq1():
    """One rotated, elongated Gaussian: every pixel near it equals
    alpha c + (1 - alpha) bg with alpha from Eq. 1 evaluated on the
    independently inverted screen covariance."""
    cam = _cam(w=64, h=64, cx=32.0, cy=32.0)
    mean = np.array([[0.1, -0.05, 3.0]])
    scale = np.array([[0.25, 0.04, 0.08]])
    quat = np.array([[0.9, 0.1, 0.3, 0.2]])
    img, _, _ = raster.render(cam, *_scene(mean, scale, [0.8], [[0.7, 0.3, 0.5]], quat=quat), 3)
    S2 = raster.screen_cov(cam, _t(mean), _t(scale), _t(quat)).numpy()[0] + cam["dilation"] * np.eye(2)
    Sinv = np.linalg.inv(S2)
    u = cam["fx"] * mean[0, 0] / mean[0, 2] + cam["cx"]
    v = cam["fy"] * mean[0, 1] / mean[0, 2] + cam["cy"]
    bg, col = np.array(cam["bg"]), np.array([0.7, 0.3, 0.5])
    checked = 0
    for py in range(int(v) - 6, int(v) + 7):
        for px in range(int(u) - 6, int(u) + 7):
            d = np.array([u - px, v - py])
            a = min(0.99, 0.8 * np.exp(-0.5 * d @ Sinv @ d))
            if a < 1 / 255 + 1e-9:
                continue
            assert np.max(np.abs(img[:, py, px].numpy() - (a * col + (1 - a) * bg))) < 1e-12
            checked += 1
    assert checked > 50


def test_clamp_skip_and_early_termination():
    cam = _cam()
    zs = [3.0, 4.0, 5.0]
    means = [[(40 - cam["cx"]) * z / cam["fx"], (20 - cam["cy"]) * z / cam["fy"], z] for z in zs]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    img, T, cnt = raster.render(cam, *_scene(means, [[0.05] * 3] * 3, [1.0, 1.0, 1.0], cols), 3)
    # alpha clamps to 0.99; T after two is 1e-4 (kept), the third would go below 1e-4 (stopped)
    want = 0.99 * np.array([1, 0, 0]) + 0.01 * 0.99 * np.array([0, 1, 0]) + 1e-4 * np.array(cam["bg"])
    assert np.max(np.abs(img[:, 20, 40].numpy() - want)) < 1e-12 and int(cnt[20, 40]) == 2
    img, T, cnt = raster.render(cam, *_scene(means[:1], [[0.05] * 3], [1.0 / 300], cols[:1]), 3)
    assert np.max(np.abs(img[:, 20, 40].numpy() - np.array(cam["bg"]))) < 1e-15 and int(cnt[20, 40]) == 0


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    n = 6
    cam = _cam(w=48, h=32, campos=[0.05, -0.02, -0.1])
    means = np.c_[rng.uniform(-0.4, 0.4, (n, 2)), rng.uniform(2.5, 4.0, n)]
    scales = rng.uniform(0.04, 0.12, (n, 3))
    quat = rng.standard_normal((n, 4))
    opac = rng.uniform(0.3, 0.8, n)
    sh = rng.standard_normal((n, 16, 3)) * 0.2
    wimg = _t(rng.standard_normal((3, 32, 48)))
    params = [_t(means), _t(scales), _t(quat), _t(opac), _t(sh)]
    for p in params:
        p.requires_grad_(True)
    img, _, _ = raster.render(cam, *params, 3)
    (img * wimg).sum().backward()
    for k, p in enumerate(params):
        flat = p.detach().reshape(-1)
        g = p.grad.reshape(-1)
        for j in rng.choice(flat.numel(), size=min(6, flat.numel()), replace=False):
            vals = []
            for s in (1, -1):
                q = [a.detach().clone() for a in params]
                q[k].reshape(-1)[j] += s * 1e-6
                vals.append(float((raster.render(cam, *q, 3)[0] * wimg).sum()))
            fd = (vals[0] - vals[1]) / 2e-6
            assert abs(fd - float(g[j])) <= 1e-5 * max(1.0, abs(fd)), (k, j, fd, float(g[j]))
