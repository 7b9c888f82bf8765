"""The renderer oracle's pins must catch plausible mistakes: each case plants
one in a copy of oracle/raster.py, loads the copy as a module, points the
pins at it and requires at least one pin to fail."""
import importlib.util

import pytest

import test_oracle_pins_raster as pins
from oracle import raster

MUTATIONS = [
    ("rotation matrix transposed",
     "torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),",
     "torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], -1),",
     ["test_rotation_matches_scipy"]),
    ("Jacobian's depth column with the wrong sign",
     "J = torch.stack([torch.stack([fx / tz, zero, -fx * tx / (tz * tz)], -1),",
     "J = torch.stack([torch.stack([fx / tz, zero, fx * tx / (tz * tz)], -1),",
     ["test_covariance_eigen_and_screen_projection_by_finite_differences"]),
    ("scale not squared in the covariance",
     "M = quat_to_rotmat(rot) * scale[:, None, :]",
     "M = quat_to_rotmat(rot) * scale[:, None, :].sqrt()",
     ["test_covariance_eigen_and_screen_projection_by_finite_differences"]),
    ("degree-2 constant wrong",
     "a = 0.5 * math.sqrt(15 / pi)",
     "a = 0.5 * math.sqrt(5 / pi)",
     ["test_sh_basis_is_orthonormal_on_the_sphere"]),
    ("blending weighted by the transmittance after the Gaussian",
     "w = torch.where(alive, a * T_excl, torch.zeros_like(a))",
     "w = torch.where(alive, a * T_incl, torch.zeros_like(a))",
     ["test_single_and_two_gaussians_closed_form"]),
    ("back-to-front order",
     "key=lambda i: (float(depth[i]), i))",
     "key=lambda i: (-float(depth[i]), i))",
     ["test_single_and_two_gaussians_closed_form"]),
    ("no 0.99 clamp on alpha",
     "alpha = torch.clamp(p[\"opacity\"][idx][None, :] * torch.exp(power), max=ALPHA_MAX)",
     "alpha = p[\"opacity\"][idx][None, :] * torch.exp(power)",
     ["test_clamp_skip_and_early_termination"]),
    ("early termination test on the transmittance before the Gaussian",
     "alive = T_incl.detach() >= T_MIN",
     "alive = T_excl.detach() >= T_MIN",
     ["test_clamp_skip_and_early_termination"]),
    ("conic off-diagonal sign flipped",
     "conic = torch.stack([c / det, -b / det, a / det], 1)",
     "conic = torch.stack([c / det, b / det, a / det], 1)",
     ["test_anisotropic_gaussian_follows_eq1"]),
    ("exponent missing the factor one half",
     "power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy",
     "power = -(con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy",
     ["test_anisotropic_gaussian_follows_eq1"]),
]


def _mutant(tmp_path, old, new):
    src = open(raster.__file__).read()
    assert old in src, f"mutation anchor not found: {old}"
    path = tmp_path / "raster_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("raster_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_raster_pins_catch_planted_mistake(tmp_path, monkeypatch, name, old, new, checks):
    monkeypatch.setattr(pins, "raster", _mutant(tmp_path, old, new))
    caught = []
    for fname in checks:
        try:
            getattr(pins, fname)()
        except (AssertionError, ValueError, RuntimeError):
            caught.append(fname)
    assert caught, f"no pin caught: {name}"


def test_unmutated_copy_passes(tmp_path, monkeypatch):
    monkeypatch.setattr(pins, "raster", _mutant(tmp_path, "TILE = 16", "TILE = 16"))
    for _, _, _, checks in MUTATIONS:
        for fname in checks:
            getattr(pins, fname)()
