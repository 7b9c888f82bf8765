"""Shared helpers for the GPU parity tests: seeded inputs on both sides and
error metrics.  The CUDA side is reached only through the C-ABI binding."""
import numpy as np
import torch

import oracle


def oracle_grid(g):
    return oracle.layout(g.L, g.F, g.log2_T, g.nmin_s, g.nmax_s, g.nmin_t, g.nmax_t, g.primes)


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def norm_err(got, ref):
    """Normwise relative error ||got - ref||_2 / ||ref||_2 over the whole array."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (d if d > 0 else 1.0))


def elem_err(got, ref):
    """Element-wise error max_i |got_i - ref_i| / max_i |ref_i|: one wrong
    element of a large array shows here at full size, where the normwise
    error would average it away."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.size == 0:
        return 0.0
    d = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(got - ref)) / (d if d > 0 else 1.0))


def touched_mismatch(got, ref, floor=1e-6):
    """Entries that one side left at zero and the other did not.  A table
    gradient entry is nonzero exactly where some corner with a nonzero weight
    and a nonzero upstream value reduced into it, so a lost or a stray
    reduction changes this set; entries below floor * max|ref| on both sides
    are not counted (an exact cancellation in one precision and not in the
    other, or an underflowed product of tiny weights)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.size == 0:
        return 0
    s = floor * float(np.max(np.abs(ref)))
    big = np.maximum(np.abs(got), np.abs(ref)) > s
    return int(np.count_nonzero(((got != 0) != (ref != 0)) & big))


def is_table_shaped(a):
    """A hash-table (gradient) array: [entries][F], F in {1, 2, 4, 8}."""
    return a.ndim == 2 and a.shape[1] in (1, 2, 4, 8) and a.shape[0] >= 1024


def rel_err(got, ref, touched=None):
    """The error every float parity assertion bounds: the larger of the
    normwise and the element-wise relative errors, so `rel_err < tol`
    asserts |got_i - ref_i| <= tol * max|ref| for every element and the
    normwise bound.  For table-shaped arrays (is_table_shaped: the table
    gradients) it is also infinite when the sets of touched (nonzero)
    entries differ (touched_mismatch).  touched=True / False forces that
    check on or off; off for differences of buffers that started from
    nonzero values (a sum that rounds back to its starting value reads as
    zero there).  Decoder-parameter blocks are not checked for it: one of
    their entries can hold a single small product, which the backward's BF16
    operands may round differently from FP64 without being a lost term."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape and got.size == ref.size:
        got = got.reshape(ref.shape)
    if touched is None:
        touched = is_table_shaped(ref)
    if touched and touched_mismatch(got, ref):
        return float("inf")
    return max(norm_err(got, ref), elem_err(got, ref))


# Smallest |pre-activation| of a decoder hidden unit for which the GPU and
# the oracle are sure to take the same ReLU decision.  The GPU forms each
# pre-activation from hi + lo BF16 splits of FP32 activations (relative error
# <= 2^-17 per operand: about 2e-5 absolute at this decoder's scale) and
# stores the decisions for the backward; the oracle decides in FP64.  A unit
# within that distance of 0 may switch in one precision and not the other,
# which changes that Gaussian's whole backward (a full-size difference that
# no tolerance separates from a lost reduction).  Element-wise gradient
# checks therefore give such Gaussians a zero upstream gradient on both sides.
RELU_MARGIN = 1e-4


def relu_clear(g, pts, table, params, H, O, margin=RELU_MARGIN):
    """Per point of the oracle point set `pts`: True where every hidden
    pre-activation of the decoder (Linear-ReLU-Linear-ReLU on the oracle's
    FP64 encoding) is at least `margin` from 0, so both sides take the same
    ReLU decisions.  params: packed W1 [H][D], b1, W2 [H][H], b2, W3, b3."""
    f = oracle.encode(g, pts, np.asarray(table, dtype=np.float64))
    D = f.shape[1]
    p = np.asarray(params, dtype=np.float64)
    W1 = p[:H * D].reshape(H, D)
    b1 = p[H * D:H * D + H]
    W2 = p[H * D + H:H * D + H + H * H].reshape(H, H)
    b2 = p[H * D + H + H * H:H * D + 2 * H + H * H]
    z1 = f @ W1.T + b1
    z2 = np.maximum(z1, 0.0) @ W2.T + b2
    return (np.abs(z1) >= margin).all(axis=1) & (np.abs(z2) >= margin).all(axis=1)


def zero_ambiguous(dd, g, pts, table, params, H, O, margin=RELU_MARGIN):
    """Sets to zero, in place, the upstream-gradient columns dd[:, i] of the
    points of `pts` whose ReLU decisions are ambiguous (relu_clear); columns
    beyond the point count are left as they are.  Returns how many were
    zeroed."""
    clear = relu_clear(g, pts, table, params, H, O, margin)
    dd[:, :len(clear)][:, ~clear] = 0.0
    return int((~clear).sum())


def edge_coords(n, rng):
    """Coordinates with the degenerate cases first: 0, 1, NaN, out of range,
    exact vertices of power-of-two grids, then uniform values."""
    x, y, z, t = (rng.random(n).astype(np.float32) for _ in range(4))
    special = np.array([0.0, 1.0, np.nan, -0.5, 1.5, 0.5, 0.25, 1.0 - 2 ** -24, 2 ** -30, 0.125], dtype=np.float32)
    k = min(n, len(special))
    x[:k] = special[:k]
    y[:k] = special[::-1][:k]
    z[:k] = np.roll(special, 3)[:k]
    t[:k] = np.roll(special, 5)[:k]
    return x, y, z, t
