"""The error metric every float parity assertion of the GPU tests goes
through (gpu_helpers.rel_err), checked on the CPU: a few lost, duplicated or
stray table-gradient reductions in an array the size of the paper-shaped
table gradient (7,339,136 entries x 2 features) must fail a 1e-2 bound that
the normwise error alone would pass."""
import numpy as np

from gpu_helpers import elem_err, norm_err, rel_err, touched_mismatch

ENTRIES = 7_339_136


def _grad(seed=0, touched=0.6):
    """A table-gradient-like array: a random share of entries touched, values
    of both signs with a heavy tail (coarse entries collect many updates)."""
    rng = np.random.default_rng(seed)
    g = np.zeros((ENTRIES, 2))
    hit = rng.random(ENTRIES) < touched
    g[hit] = rng.standard_normal((int(hit.sum()), 2)) * rng.exponential(1.0, (int(hit.sum()), 1))
    return g


def test_identical_arrays_have_zero_error():
    g = _grad()
    assert rel_err(g, g.copy()) == 0.0 and touched_mismatch(g, g) == 0


def test_one_duplicated_corner_fails_elementwise_not_normwise():
    ref = _grad(1)
    got = ref.copy()
    k = int(np.argmax(np.abs(ref[:, 0])))
    got[k, 0] *= 1.05          # one reduction counted twice on the largest entry
    assert norm_err(got, ref) < 1e-2     # averaged away over 7.3M entries
    assert elem_err(got, ref) > 1e-2
    assert rel_err(got, ref) > 1e-2


def test_lost_reductions_change_the_touched_set():
    ref = _grad(2)
    got = ref.copy()
    lost = np.flatnonzero(ref[:, 0])[:3]
    got[lost] = 0.0            # three entries whose only reductions were dropped
    assert norm_err(got, ref) < 1e-2
    assert touched_mismatch(got, ref) >= 3
    assert rel_err(got, ref) == float("inf")


def test_stray_reduction_into_an_untouched_entry():
    ref = _grad(3)
    got = ref.copy()
    k = int(np.flatnonzero(ref[:, 1] == 0)[0])
    got[k, 1] = 1e-3 * np.max(np.abs(ref))   # a partner's corner scattered to the wrong entry
    assert elem_err(got, ref) < 1e-2
    assert rel_err(got, ref) == float("inf")


def test_underflowed_entries_below_the_floor_are_not_counted():
    ref = _grad(4)
    got = ref.copy()
    k = int(np.flatnonzero(ref[:, 0])[0])
    ref[k, 0] = 1e-9 * np.max(np.abs(ref))   # a product of tiny weights, zero in the other precision
    got[k, 0] = 0.0
    assert touched_mismatch(got, ref) == 0
    assert rel_err(got, ref) < 1e-6


def test_heads_are_bounded_per_element():
    rng = np.random.default_rng(5)
    ref = rng.standard_normal((3, 20_000))
    got = ref + 1e-6 * rng.standard_normal(ref.shape)
    assert rel_err(got, ref) < 1e-3
    got[1, 12345] += 5e-3 * np.max(np.abs(ref))   # one wrong Gaussian of 20k
    assert norm_err(got, ref) < 1e-3 < rel_err(got, ref)
