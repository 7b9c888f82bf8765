"""Pins of the oracle's input-coordinate gradient d/d(x, y, z, t) of the 4-D
encoder (Eq. 9 differentiated through its quadrilinear weights)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _affine_table(g, rng):
    """Dense levels only: entry (cx, cy, cz, ct) of level l holds
    A_l[f] . (cx/N_s, cy/N_s, cz/N_s, ct/N_t) + c_l[f].  Multilinear
    interpolation reproduces an affine function exactly."""
    table = np.zeros((g.total, g.F))
    A = rng.uniform(-2, 2, size=(g.L, g.F, 4))
    c = rng.uniform(-1, 1, size=(g.L, g.F))
    for l in range(g.L):
        assert g.dense[l]
        ns, nt = g.res_s[l], g.res_t[l]
        R = ns + 1
        ct, cz, cy, cx = np.meshgrid(np.arange(nt + 1), np.arange(R), np.arange(R), np.arange(R), indexing="ij")
        v = np.stack([cx / ns, cy / ns, cz / ns, ct / nt], axis=-1).reshape(-1, 4)   # x fastest
        table[g.offset[l]:g.offset[l] + v.shape[0]] = v @ A[l].T + c[l]
    return table, A


def test_affine_tables_give_the_closed_form():
    g = oracle.layout(3, 2, 24, 4, 16, 3, 9)
    rng = np.random.default_rng(11)
    table, A = _affine_table(g, rng)
    n = 400
    x, y, z, t = rng.random((4, n)).astype(np.float32)
    x[:4] = [0.0, 1.0, 0.25, 0.5]          # vertices and the upper edge
    t[4:6] = [1.0, 0.0]
    dfeat = rng.standard_normal((n, g.L * g.F))
    got = oracle.encode_coord_grad(g, oracle.Points(x, y, z, t), table, dfeat)
    want = np.einsum("nlf,lfd->dn", dfeat.reshape(n, g.L, g.F), A)
    assert np.max(np.abs(got - want)) < 1e-11


def test_constant_tables_have_zero_gradient():
    g = oracle.layout(4, 2, 12, 5, 300, 3, 60)
    rng = np.random.default_rng(12)
    table = np.full((g.total, 2), 0.7)
    x, y, z, t = rng.random((4, 200)).astype(np.float32)
    d = oracle.encode_coord_grad(g, oracle.Points(x, y, z, t), table, rng.standard_normal((200, 8)))
    assert np.max(np.abs(d)) < 1e-10


def _stays_in_cell(v, h, N):
    """[v - h, v + h] * N inside the closed hypervoxel the oracle selects for v."""
    pos, lo, hi = v * N, (v - h) * N, (v + h) * N
    c = min(int(pos), N - 1)   # floor of a non-negative rational
    return v - h >= 0 and v + h <= 1 and lo >= c and hi <= c + 1


def _loss(g, x, y, z, t, table, dfeat):
    return float(np.sum(dfeat * oracle.encode(g, oracle.Points(x, y, z, t), table)))


@pytest.mark.parametrize("broadcast_t", [False, True])
def test_central_differences_are_exact_on_dyadic_inputs(broadcast_t):
    """Coordinates odd/2^13, step 2^-14, resolutions below 2^10: every product
    x * N is exact in FP32, and along one axis the encoding is linear inside
    a hypervoxel, so the central difference equals the derivative up to FP64
    rounding wherever the step stays in the cell at every level."""
    g = oracle.layout(4, 2, 12, 5, 700, 3, 200)   # coarse levels dense, fine levels hashed
    assert not g.dense[3] and g.dense[0]
    rng = np.random.default_rng(13)
    table = rng.uniform(-1, 1, size=(g.total, 2))
    h = Fraction(1, 2 ** 14)
    res = [[g.res_s[l]] * 3 + [g.res_t[l]] for l in range(g.L)]
    tested = 0
    for _ in range(400):
        q = [Fraction(int(2 * rng.integers(1, 2 ** 12) - 1), 2 ** 13) for _ in range(4)]
        ok = [all(_stays_in_cell(q[d], h, res[l][d]) for l in range(g.L)) for d in range(4)]
        if not any(ok):
            continue
        dfeat = rng.standard_normal((1, g.L * g.F))
        p = [np.array([float(v)], np.float32) for v in q]
        grad = oracle.encode_coord_grad(g, oracle.Points(*p), table, dfeat)[:, 0]
        for d in range(4):
            if not ok[d]:
                continue
            up = [a.copy() for a in p]
            dn = [a.copy() for a in p]
            up[d][0] = np.float32(float(q[d] + h))
            dn[d][0] = np.float32(float(q[d] - h))
            fd = (_loss(g, *up, table, dfeat) - _loss(g, *dn, table, dfeat)) / (2 * float(h))
            assert abs(fd - grad[d]) <= 1e-9 * max(1.0, abs(fd)), (d, fd, grad[d])
            tested += 1
    assert tested >= 100
    if broadcast_t:
        # one t shared by all points: the derivative of the total is the sum of the shares
        n = 64
        qs = [np.array([(2 * rng.integers(1, 2 ** 12) - 1) / 2 ** 13 for _ in range(n)], np.float32)
              for _ in range(3)]
        for _ in range(50):
            tq = Fraction(int(2 * rng.integers(1, 2 ** 12) - 1), 2 ** 13)
            if all(_stays_in_cell(tq, h, res[l][3]) for l in range(g.L)):
                break
        assert all(_stays_in_cell(tq, h, res[l][3]) for l in range(g.L))
        dfeat = rng.standard_normal((n, g.L * g.F))
        tt = np.array([float(tq)], np.float32)
        share = oracle.encode_coord_grad(g, oracle.Points(*qs, tt, t_stride=0), table, dfeat)[3]
        lu = float(np.sum(dfeat * oracle.encode(g, oracle.Points(*qs, np.array([float(tq + h)], np.float32),
                                                                 t_stride=0), table)))
        ld = float(np.sum(dfeat * oracle.encode(g, oracle.Points(*qs, np.array([float(tq - h)], np.float32),
                                                                 t_stride=0), table)))
        assert abs((lu - ld) / (2 * float(h)) - share.sum()) <= 1e-9 * max(1.0, abs(share.sum()))


def test_clamp_blocks_the_gradient_outside_the_unit_interval():
    g = oracle.layout(2, 2, 16, 4, 8, 2, 4)
    rng = np.random.default_rng(14)
    table, A = _affine_table(g, rng)
    x = np.array([-0.5, 1.5, np.nan, 0.3, 1.0], np.float32)
    y = np.array([0.2, 0.2, 0.2, -1e-7, 0.0], np.float32)
    z = np.full(5, 0.6, np.float32)
    t = np.array([0.1, 2.0, 0.5, 0.5, 1.0], np.float32)
    dfeat = rng.standard_normal((5, 4))
    d = oracle.encode_coord_grad(g, oracle.Points(x, y, z, t), table, dfeat)
    want = np.einsum("nlf,lfd->dn", dfeat.reshape(5, 2, 2), A)
    raw = np.stack([x, y, z, t])
    inside = (raw >= 0) & (raw <= 1)           # NaN compares false
    assert np.all(d[~inside] == 0.0)
    assert np.max(np.abs(d[inside] - want[inside])) < 1e-11
