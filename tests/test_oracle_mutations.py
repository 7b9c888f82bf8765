"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of the oracle's C source (a dropped exponent, a swapped
axis, a wrong sign, a transposed operand, ...), compiles that copy on the CPU,
points the oracle binding at it, and requires at least one pin to fail."""
import ctypes

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_pins_collisions as pins_coll
import test_oracle_pins_coord as pins_coord
import test_oracle_pins_decomp as pins_decomp
from paper_2507_19141_gb300 import synth

MUTATIONS = [
    ("Eq. 7 level exponent dropped",
     "return (int32_t)floor(nmin * pow(b, (double)l) + 1e-9);",
     "return (int32_t)floor(nmin * b + 1e-9);",
     [("test_layout_paper_shape_golden", {})]),
    ("Eq. 7 rounding guard dropped",
     "return (int32_t)floor(nmin * pow(b, (double)l) + 1e-9);",
     "return (int32_t)floor(nmin * pow(b, (double)l));",
     [("test_layout_endpoints_and_monotone", dict(L=8, nmin=2, nmax=512)),
      ("test_layout_endpoints_and_monotone", dict(L=12, nmin=16, nmax=4096))]),
    ("temporal axis given the spatial resolution",
     "int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_t[l]};",
     "int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_s[l]};",
     [("test_hash_big_integer_brute_force", {})]),
    ("lower corner rounded instead of floored",
     "int64_t c = (int64_t)floor(pos);",
     "int64_t c = (int64_t)floor(pos + 0.5);",
     [("test_weights_partition_of_unity", dict(cfg=synth.TINY_GRID)), ("test_multilinear_matches_scipy_regular_grid", {})]),
    ("corner weights swapped",
     "wb *= up ? frac[d] : (1.0 - frac[d]);",
     "wb *= up ? (1.0 - frac[d]) : frac[d];",
     [("test_multilinear_matches_scipy_regular_grid", {}), ("test_vertex_reproduction_exact", {})]),
    ("y and z corner bits swapped",
     "int up = (b >> d) & 1;",
     "int up = (b >> (d == 1 ? 2 : (d == 2 ? 1 : d))) & 1;",
     [("test_hash_reduces_to_bit_packing_with_power_of_two_primes", {})]),
    ("Eq. 8 XOR replaced by addition",
     "h ^= ((uint64_t)c[d] * (uint64_t)g->primes[d]) & 0xFFFFFFFFull;",
     "h += ((uint64_t)c[d] * (uint64_t)g->primes[d]) & 0xFFFFFFFFull;",
     [("test_hash_big_integer_brute_force", {})]),
    ("dense stride N instead of N + 1",
     "int64_t R = res[0] + 1;",
     "int64_t R = res[0];",
     [("test_dense_level_is_bijection_onto_table", {})]),
    ("features stored feature-major",
     "f_h[l * F + f] = acc;",
     "f_h[f * g->L + l] = acc;",
     [("test_vertex_reproduction_exact", {})]),
    ("compaction keeps only mask bytes equal to 1",
     "if (mask[i] != 0) idx_out[count++] = (int32_t)i;",
     "if (mask[i] == 1) idx_out[count++] = (int32_t)i;",
     [("test_compaction_is_flatnonzero", dict(n=100_003, p=0.5))]),
    ("second ReLU dropped",
     "h2[j] = a > 0.0 ? a : 0.0;",
     "h2[j] = a;",
     [("test_mlp_forward_and_backward_match_torch_autograd", dict(D=8, H=64, O=10))]),
    ("W2 transposed in back-propagation",
     "for (int j = 0; j < H; ++j) a += m->W2[(size_t)j * H + k] * dz2[j];",
     "for (int j = 0; j < H; ++j) a += m->W2[(size_t)k * H + j] * dz2[j];",
     [("test_mlp_forward_and_backward_match_torch_autograd", dict(D=8, H=64, O=10))]),
    ("Eq. 10 subtracts the offset",
     "(double)attrs_in[j * n_all + gi] + o[j];",
     "(double)attrs_in[j * n_all + gi] - o[j];",
     [("test_deform_forward_composes_encoder_mlp_and_eq10", {})]),
    ("Eq. 11 gradient of the perturbed point with the wrong sign",
     "dq[k] = -scale * diff;",
     "dq[k] = scale * diff;",
     [("test_full_backward_finite_difference_with_smoothness", {})]),
    ("Eq. 11 gradient missing the factor 2",
     "const double scale = 2.0 * (double)lambda_r / (double)(n > 0 ? n : 1);",
     "const double scale = (double)lambda_r / (double)(n > 0 ? n : 1);",
     [("test_full_backward_finite_difference_with_smoothness", {})]),
    ("Eq. 5 divides by all Gaussians instead of the static ones",
     "return n_s > 0 ? sum / (double)n_s : 0.0;",
     "return n_s > 0 ? sum / (double)n : 0.0;",
     [("decomp:test_static_loss_special_cases", {})]),
    ("Eq. 4 moves along dp by (1 - t)",
     "out[d * n + i] = p[d] + ti * dp[d * n + i];",
     "out[d * n + i] = p[d] + (1.0 - ti) * dp[d * n + i];",
     [("decomp:test_linear_motion_speed_is_the_norm", {})]),
    ("top-k threshold taken one rank too low",
     "tau = s[m];",
     "tau = s[m + 1 < n ? m + 1 : m];",
     [("decomp:test_topk_mask_invariants", dict(n=1000, k=25.0)), ("decomp:test_topk_mask_ties_are_static", {})]),
    ("decomposition backward: L_s term divided by n instead of N_s",
     "g_dp[c] += lambda_s * dp[c] / ((double)n_s * norm);",
     "g_dp[c] += lambda_s * dp[c] / ((double)n * norm);",
     [("decomp:test_decomposition_backward_matches_finite_differences", {})]),
    ("decomposition backward: ReLU mask dropped",
     "dz1[j] = z1[j] > 0.0 ? a : 0.0;",
     "dz1[j] = a;",
     [("decomp:test_decomposition_backward_matches_finite_differences", {})]),
    ("decomposition backward: W1 transposed for the feature gradient",
     "for (int j = 0; j < H; ++j) a += W1[(size_t)j * D + k] * dz1[j];",
     "for (int j = 0; j < H; ++j) a += W1[(size_t)(j % D) * D + (k % D)] * dz1[j];",
     [("decomp:test_decomposition_backward_matches_finite_differences", {})]),
    ("G_3D dense stride N instead of N + 1",
     "int64_t R = N + 1;",
     "int64_t R = N;",
     [("decomp:test_cell3_dense_bijection_and_partition_of_unity", {})]),
    ("coordinate gradient: weight derivative with the wrong sign",
     "double dw = ((b >> d) & 1) ? 1.0 : -1.0;",
     "double dw = ((b >> d) & 1) ? -1.0 : 1.0;",
     [("coord:test_affine_tables_give_the_closed_form", {})]),
    ("coordinate gradient: chain factor N_l dropped",
     "grad[d] += s_b * dw * (double)res[d];",
     "grad[d] += s_b * dw;",
     [("coord:test_affine_tables_give_the_closed_form", {})]),
    ("coordinate gradient: t scaled by the spatial resolution",
     "const int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_t[l]};",
     "const int64_t res[4] = {g->res_s[l], g->res_s[l], g->res_s[l], g->res_s[l]};",
     [("coord:test_central_differences_are_exact_on_dyadic_inputs", dict(broadcast_t=False))]),
    ("coordinate gradient: own axis weight kept in the product",
     "if (e == d) continue;",
     "if (e == d) dw *= 1.0;",
     [("coord:test_affine_tables_give_the_closed_form", {})]),
    ("coordinate gradient: clamp does not block",
     "dcoord[d * n + i] = inside ? grad[d] : 0.0;",
     "dcoord[d * n + i] = grad[d];",
     [("coord:test_clamp_blocks_the_gradient_outside_the_unit_interval", {})]),
    ("collisions: a shared entry counted once too few",
     "if (r - k >= 2) C += r - k;",
     "if (r - k >= 2) C += r - k - 1;",
     [("coll:test_counts_equal_brute_force", dict(cfg=(4, 2, 8, 4, 64, 3, 20), n=300))]),
    ("collisions: vertex id with stride N instead of N + 1",
     "const int64_t R = res[0] + 1;",
     "const int64_t R = res[0];",
     [("coll:test_counts_equal_brute_force", dict(cfg=(3, 2, 6, 2, 9, 2, 5), n=500))]),
    ("collisions: the temporal corner bit ignored",
     "for (int d = 0; d < 4; ++d) c[d] = i0[d] + ((b >> d) & 1);",
     "for (int d = 0; d < 4; ++d) c[d] = i0[d] + (d < 3 ? ((b >> d) & 1) : 0);",
     [("coll:test_dense_levels_never_collide_and_one_point_touches_16_vertices", {})]),
    ("Eq. 11 temporal perturbation applied to x",
     "const float e_t[4] = {0.f, 0.f, 0.f, eps_t};",
     "const float e_t[4] = {eps_t, 0.f, 0.f, 0.f};",
     [("test_smoothness_closed_form_on_affine_tables", {})]),
]


def _pin(fname):
    if fname.startswith("decomp:"):
        return getattr(pins_decomp, fname[len("decomp:"):])
    if fname.startswith("coord:"):
        return getattr(pins_coord, fname[len("coord:"):])
    if fname.startswith("coll:"):
        return getattr(pins_coll, fname[len("coll:"):])
    return getattr(pins, fname)


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name, old, new, checks):
    src = open(oracle._SRC).read()
    assert old in src, f"mutation anchor not found: {old}"
    (tmp_path / "mutant.c").write_text(src.replace(old, new))
    lib = oracle.configure(ctypes.CDLL(oracle.compile_variant(str(tmp_path / "mutant.c"),
                                                              str(tmp_path / "mutant.so"))))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fname, kwargs in checks:
        try:
            _pin(fname)(**kwargs)
        except (AssertionError, ValueError):
            caught.append(fname)
    assert caught, f"no pin caught: {name}"


def test_unmutated_copy_passes_the_same_checks(tmp_path, monkeypatch):
    """Control: the same procedure on an unchanged copy fails nothing."""
    src = open(oracle._SRC).read()
    (tmp_path / "copy.c").write_text(src)
    lib = oracle.configure(ctypes.CDLL(oracle.compile_variant(str(tmp_path / "copy.c"), str(tmp_path / "copy.so"))))
    monkeypatch.setattr(oracle, "_lib", lib)
    for _, _, _, checks in MUTATIONS:
        for fname, kwargs in checks:
            _pin(fname)(**kwargs)
