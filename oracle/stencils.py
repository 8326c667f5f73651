"""Discrete operators, built from the paper's difference-operator notation.

Every stencil is assembled from the one-dimensional operators the paper
writes (delta^2 = [1 -2 1], delta^4 = delta^2 delta^2) by tensor products,
so a reader can compare each line with the equation it comes from.

Arrays are indexed ``[z][y][x]``; a (2w+1)^3 stencil has its centre at
index (w, w, w).
"""
from fractions import Fraction

import numpy as np

D2 = np.array([1.0, -2.0, 1.0])            # delta^2, Sec. 3.2
D4 = np.convolve(D2, D2)                   # delta^4 = [1 -4 6 -4 1]
ID3 = np.array([0.0, 1.0, 0.0])
ID5 = np.array([0.0, 0.0, 1.0, 0.0, 0.0])


def _tensor(opz, opy, opx):
    return np.einsum("i,j,k->ijk", opz, opy, opx)


def _embed(op, width):
    """Centre a 1-D stencil in a vector of length 2*width+1."""
    out = np.zeros(2 * width + 1)
    w = (len(op) - 1) // 2
    out[width - w:width + w + 1] = op
    return out


def _d2(axis, width=1):
    """delta^2 along ``axis`` (0=x, 1=y, 2=z) as a (2w+1)^3 array."""
    ops = [_embed(ID3, width)] * 3
    ops = list(ops)
    ops[axis] = _embed(D2, width)
    return _tensor(ops[2], ops[1], ops[0])


def _d2d2(a, b, width=1):
    ops = [_embed(ID3, width)] * 3
    ops = list(ops)
    ops[a] = _embed(D2, width)
    ops[b] = _embed(D2, width)
    return _tensor(ops[2], ops[1], ops[0])


def lhs_stencil(M):
    """Unit-spacing weights of Delta^M_h; multiply by 1/h^2.

    M = 2: Eq. cross_discr2, (delta_x^2 + delta_y^2 + delta_z^2).
    M = 4: Eq. mehrstellen_discr4 LHS, adds (1/6)(dx2 dy2 + dy2 dz2 + dz2 dx2).
    M = 6: Eq. mehrstellen_discr6 LHS, adds (1/30) dx2 dy2 dz2.
    """
    L = _d2(0) + _d2(1) + _d2(2)
    if M >= 4:
        L = L + (_d2d2(0, 1) + _d2d2(1, 2) + _d2d2(2, 0)) / 6.0
    if M >= 6:
        L = L + _tensor(D2, D2, D2) / 30.0
    if M not in (2, 4, 6):
        raise ValueError("order must be 2, 4 or 6")
    return L


def rhs_stencil(M):
    """Weights of R^M_h on a 5^3 cube (dimensionless; f* = R^M f).

    M = 2: identity (Eq. cross_discr2 has no RHS operator).
    M = 4: Eq. mehrstellen_discr4 RHS, 1 + (1/12)(dx2 + dy2 + dz2).
    M = 6: Eq. mehrstellen_discr6 RHS, adds (1/90)(dx2 dy2 + dy2 dz2 + dz2 dx2)
           - (1/240)(dx4 + dy4 + dz4).  The printed middle term reads
           "delta_y delta_z^2"; it is read as delta_y^2 delta_z^2 (the only
           reading that is symmetric and sixth-order accurate).
    """
    R = _tensor(ID5, ID5, ID5)
    if M >= 4:
        R = R + (_d2(0, 2) + _d2(1, 2) + _d2(2, 2)) / 12.0
    if M >= 6:
        R = R + (_d2d2(0, 1, 2) + _d2d2(1, 2, 2) + _d2d2(2, 0, 2)) / 90.0
        d4 = [_embed(D4, 2), _embed(ID5, 2)]
        R = R - (_tensor(d4[1], d4[1], d4[0]) + _tensor(d4[1], d4[0], d4[1])
                 + _tensor(d4[0], d4[1], d4[1])) / 240.0
    if M not in (2, 4, 6):
        raise ValueError("order must be 2, 4 or 6")
    return R


def rhs_width(M):
    """Ghost layers of f that R^M needs (Sec. 3.2: width two for M = 6)."""
    return {2: 0, 4: 1, 6: 2}[M]


def midpoint_lagrange(I):
    """Weights of the I-point Lagrange interpolant at a midpoint.

    Ghost reconstruction at resolution jumps uses polynomial interpolation
    of order I = M + 2 (Sec. 2.1).  Nodes sit at offsets m - (I-1)/2,
    m = 0..I-1, around the midpoint; exact rational arithmetic.
    """
    xs = [Fraction(2 * m - (I - 1), 2) for m in range(I)]
    w = []
    for m in range(I):
        num = Fraction(1)
        for l in range(I):
            if l != m:
                num *= (0 - xs[l]) / (xs[m] - xs[l])
        w.append(num)
    return np.array([float(v) for v in w])


def full_weighting():
    """Residual restriction: tensor product of (1/4)[1 2 1] (Sec. 3.1)."""
    fw = np.array([1.0, 2.0, 1.0]) / 4.0
    return _tensor(fw, fw, fw)
