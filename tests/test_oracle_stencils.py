"""Pins of the oracle's discrete operators against the paper and mathematics."""
import itertools

import numpy as np
import pytest

from oracle.stencils import lhs_stencil, rhs_stencil, midpoint_lagrange, full_weighting


def _by_distance(w):
    """Weight per Manhattan distance class (centre, face, edge, corner) of a 3^3 stencil."""
    out = {}
    for idx, v in np.ndenumerate(w):
        d = sum(abs(i - 1) for i in idx)
        out.setdefault(d, set()).add(round(float(v), 15))
    return out


def test_lhs_weights_match_figure_stencils():
    # Fig. stencils prints the weights: (1/h^2){-6, 1}, (1/6h^2){-24, 2, 1}, (1/30h^2){-128, 14, 3, 1}
    assert _by_distance(lhs_stencil(2)) == {0: {-6.0}, 1: {1.0}, 2: {0.0}, 3: {0.0}}
    w4 = _by_distance(lhs_stencil(4) * 6)
    assert w4 == {0: {-24.0}, 1: {2.0}, 2: {1.0}, 3: {0.0}}
    w6 = _by_distance(lhs_stencil(6) * 30)
    assert {k: {round(v, 9) for v in s} for k, s in w6.items()} == {0: {-128.0}, 1: {14.0}, 2: {3.0}, 3: {1.0}}


def test_rhs_weights_sum_to_one_and_are_symmetric():
    for M in (2, 4, 6):
        R = rhs_stencil(M)
        assert abs(R.sum() - 1.0) < 1e-15
        for perm in itertools.permutations(range(3)):
            assert np.array_equal(R, R.transpose(perm))
        assert np.array_equal(R, R[::-1, ::-1, ::-1])
    R6 = rhs_stencil(6)
    # centre, face, edge, axis +-2 of R^6 (a consequence of Eq. mehrstellen_discr6)
    assert np.isclose(R6[2, 2, 2], 67 / 120, atol=1e-15)
    assert np.isclose(R6[2, 2, 3], 1 / 18, atol=1e-15)
    assert np.isclose(R6[2, 3, 3], 1 / 90, atol=1e-15)
    assert np.isclose(R6[2, 2, 4], -1 / 240, atol=1e-15)
    assert np.isclose(R6[3, 3, 3], 0.0, atol=1e-15)


def _monomials(deg):
    return [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a) for c in range(deg + 1 - a - b)]


def _lap_monomial(x, y, z, a, b, c):
    def d2(t, p):
        return p * (p - 1) * t ** (p - 2) if p >= 2 else 0.0 * t
    return d2(x, a) * y ** b * z ** c + x ** a * d2(y, b) * z ** c + x ** a * y ** b * d2(z, c)


@pytest.mark.parametrize("M", [2, 4, 6])
def test_mehrstellen_exact_on_polynomials(M):
    """Delta^M_h u = R^M_h (nabla^2 u) holds exactly for polynomials of degree <= M + 1."""
    h = 0.37
    L = lhs_stencil(M) / h ** 2
    R = rhs_stencil(M)
    off = np.arange(-2, 3) * h
    X, Y, Z = np.meshgrid(off + 0.3, off - 0.2, off + 0.1, indexing="ij")  # [z][y][x] meaning below
    for a, b, c in _monomials(M + 1):
        u = X ** a * Y ** b * Z ** c
        f = _lap_monomial(X, Y, Z, a, b, c)
        lhs = float(np.sum(L * u[1:4, 1:4, 1:4]))
        rhs = float(np.sum(R * f))
        scale = max(1.0, abs(lhs))
        assert abs(lhs - rhs) < 1e-11 * scale, (M, a, b, c, lhs, rhs)


@pytest.mark.parametrize("M", [2, 4, 6])
def test_mehrstellen_truncation_order(M):
    """Local truncation error of Delta^M u - R^M f on a smooth function scales as h^M."""
    def err(h):
        off = np.arange(-2, 3) * h
        Z, Y, X = np.meshgrid(off + 0.31, off + 0.17, off + 0.05, indexing="ij")
        u = np.sin(X) * np.cos(2 * Y) * np.exp(0.5 * Z)
        f = (-1 - 4 + 0.25) * u
        return abs(np.sum(lhs_stencil(M) / h ** 2 * u[1:4, 1:4, 1:4]) - np.sum(rhs_stencil(M) * f))
    e1, e2 = err(0.1), err(0.05)
    order = np.log2(e1 / e2)
    assert abs(order - M) < 0.3, order


def test_lagrange_midpoint_weights():
    assert np.allclose(midpoint_lagrange(4) * 16, [-1, 9, 9, -1], atol=1e-14)
    assert np.allclose(midpoint_lagrange(6) * 256, [3, -25, 150, 150, -25, 3], atol=1e-12)
    assert np.allclose(midpoint_lagrange(8) * 2048, [-5, 49, -245, 1225, 1225, -245, 49, -5], atol=1e-10)
    for I in (4, 6, 8):
        w = midpoint_lagrange(I)
        x = np.arange(I) - (I - 1) / 2
        for p in range(I):
            assert abs(np.dot(w, x ** p) - (1.0 if p == 0 else 0.0)) < 1e-13
        # degree I is not reproduced
        assert abs(np.dot(w, x ** I)) > 1e-3


def test_full_weighting():
    W = full_weighting()
    assert abs(W.sum() - 1) < 1e-15
    assert W[1, 1, 1] == 8 / 64 and W[0, 0, 0] == 1 / 64 and W[1, 1, 0] == 4 / 64
