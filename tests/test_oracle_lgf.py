"""Pins of the oracle's lattice Green's function and free-space convolution."""
import itertools

import numpy as np
import pytest

from oracle.lgf import lgf_table, free_space_solve, direct_sum, apply_lhs_unit, lgf_at
from oracle.stencils import lhs_stencil, rhs_stencil
from oracle.closed_forms import gaussian_potential, manufactured_unb

# Watson's integral for the simple cubic lattice (G.N. Watson, 1939):
# W = (1/pi^3) int_0^pi int_0^pi int_0^pi dk / (3 - cos k1 - cos k2 - cos k3) = 1.516386059151978...
# For the 7-point operator L (centre -6), G[0] = -W / 2 / 3 = -W/6.
WATSON_SC = 1.516386059151978


def _full(G):
    n = G.shape[0] - 1
    idx = np.abs(np.arange(-n, n + 1))
    return G[np.ix_(idx, idx, idx)]


def test_watson_constant(lgf_cache):
    G = lgf_cache(2, 24)
    assert abs(G[0, 0, 0] - (-WATSON_SC / 6)) < 1e-14


@pytest.mark.parametrize("M", [2, 4, 6])
def test_lgf_inverts_operator(lgf_cache, M):
    """L G = delta at every point of the tabulated cube whose stencil is inside it."""
    G = lgf_cache(M, 24)
    LG = apply_lhs_unit(M, _full(G))
    c = LG.shape[0] // 2
    LG[c, c, c] -= 1.0
    assert np.abs(LG).max() < 1e-13


@pytest.mark.parametrize("M", [2, 4, 6])
def test_lgf_symmetry(lgf_cache, M):
    G = lgf_cache(M, 24)
    for perm in itertools.permutations(range(3)):
        assert np.abs(G - G.transpose(perm)).max() < 1e-14


@pytest.mark.parametrize("M,tol", [(2, 2e-3), (4, 1e-5), (6, 1e-5)])
def test_lgf_far_field(lgf_cache, M, tol):
    """G[n] -> -1 / (4 pi |n|) (continuum Green's function) far from the origin."""
    G = lgf_cache(M, 24)
    for n in [(20, 0, 0), (14, 14, 0), (12, 12, 12), (20, 7, 3)]:
        r = np.sqrt(sum(v * v for v in n))
        assert abs(4 * np.pi * r * G[n] + 1.0) < tol


def test_lgf_quadrature_converged():
    """The tabulation does not move when the panels are refined (nmax = 40)."""
    from oracle import lgf as mod
    G1 = lgf_table(6, 40)
    old = mod.quadrature_panels
    try:
        mod.quadrature_panels = lambda n: (2 * old(n)[0], 2 * old(n)[1])
        G2 = lgf_table(6, 40)
    finally:
        mod.quadrature_panels = old
    assert np.abs(G1 - G2).max() < 2e-15


@pytest.mark.parametrize("M", [2, 6])
def test_fft_convolution_equals_direct_sum(lgf_cache, M):
    """Zero-padded FFT convolution == brute-force direct Green's summation (16^3 sources)."""
    rng = np.random.default_rng(5)
    f0 = rng.normal(size=(16, 16, 16))
    G = lgf_cache(M, 17)
    u = free_space_solve(f0, G, 0.1)
    tgt = np.array([(z, y, x) for z in (-1, 0, 7, 16) for y in (-1, 3, 15, 16) for x in (-1, 0, 9, 16)])
    ref = direct_sum(f0, G, 0.1, tgt)
    got = u[tgt[:, 0] + 1, tgt[:, 1] + 1, tgt[:, 2] + 1]
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_free_space_field_satisfies_discrete_equation(lgf_cache):
    """L_h u = f at every target node whose stencil lies in the computed cube."""
    rng = np.random.default_rng(1)
    f0 = rng.normal(size=(12, 10, 14))
    G = lgf_cache(4, 15)
    h = 0.05
    u = free_space_solve(f0, G, h)
    Lu = apply_lhs_unit(4, u) / h ** 2
    assert np.abs(Lu - f0).max() < 1e-12 * np.abs(f0).max()


def _uniform_error(M, n0, G, fn_u, fn_f, lo=0.0, L=1.0):
    h = L / n0
    x = lo + np.arange(n0 + 4) * h - 2 * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = fn_f(X, Y, Z)
    fstar = np.zeros((n0 + 4 - 4,) * 3)
    R = rhs_stencil(M)
    for (a, b, c), w in np.ndenumerate(R):
        fstar += w * f[a:a + n0, b:b + n0, c:c + n0]
    u = free_space_solve(fstar, G, h)[1:-1, 1:-1, 1:-1]
    uref = fn_u(X[2:-2, 2:-2, 2:-2], Y[2:-2, 2:-2, 2:-2], Z[2:-2, 2:-2, 2:-2])
    return np.abs(u - uref).max() / np.abs(uref).max()


@pytest.mark.parametrize("M", [2, 4, 6])
def test_gaussian_erf_potential_order(lgf_cache, M):
    """Single-level free-space solve of a centred Gaussian converges as h^M to the erf potential."""
    c, s, a = (0.5, 0.5, 0.5), 0.08, 1.0

    def fu(x, y, z):
        return gaussian_potential(x, y, z, c, s, a)

    def ff(x, y, z):
        return a * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    e = [_uniform_error(M, n0, lgf_cache(M, n0 + 1), fu, ff) for n0 in (24, 48)]
    order = np.log2(e[0] / e[1])
    assert order > M - 0.35, (e, order)


def test_manufactured_unbounded_solution(lgf_cache):
    """Sec. 4.2 manufactured u = u_unb(x) u_unb(y) u_unb(z): 6th-order error is small and decreasing."""
    def fu(x, y, z):
        return manufactured_unb(x, y, z)[0]

    def ff(x, y, z):
        return manufactured_unb(x, y, z)[1]
    e = [_uniform_error(6, n0, lgf_cache(6, n0 + 1), fu, ff) for n0 in (32, 64)]
    assert e[1] < 2e-4 and e[1] < e[0] / 20, e


def test_manufactured_second_derivative_by_finite_differences():
    """u_unb'' of the closed form equals a fourth-order central difference of u_unb (step 1e-3)."""
    from oracle.closed_forms import u_unb, u_unb_dd
    x = np.linspace(0.05, 0.95, 37)
    d = 1e-3
    fd = (-u_unb(x + 2 * d) + 16 * u_unb(x + d) - 30 * u_unb(x) + 16 * u_unb(x - d) - u_unb(x - 2 * d)) / (12 * d * d)
    assert np.abs(fd - u_unb_dd(x)).max() < 1e-5 * np.abs(u_unb_dd(x)).max()
    assert np.all(u_unb(np.array([-0.1, 0.0, 1.0, 1.3])) == 0.0)
