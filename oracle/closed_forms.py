"""Analytic free-space potentials (pins for the oracle).

With the paper's sign convention (Eq. 1: nabla^2 u = f, u -> 0 at infinity):

* Gaussian f = A exp(-r^2 / (2 s^2)):
      u(r) = -A s^3 sqrt(pi/2) erf(r / (sqrt(2) s)) / r,   u(0) = -A s^2.
* compact bump f = A (1 - r^2/R^2)^5 (r < R): by Gauss's law
      u'(r) = m(r) / r^2,  m(r) = int_0^r s^2 f(s) ds,  u(inf) = 0,
  which integrates to the polynomial below (derived by hand from the two
  integrals; checked numerically in the tests).
* the manufactured product of Sec. 4.2 (Eq. for u_unb):
      u = u_unb(x) u_unb(y) u_unb(z),  u_unb(x) = exp[10 (1 - 1/(1 - (2x-1)^2))]
  on (0,1), zero outside; f = u'' u u + u u'' u + u u u''.
"""
import numpy as np
from scipy.special import erf


def gaussian_potential(x, y, z, centre, sigma, amp):
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    s = sigma
    small = r < 1e-8 * s
    rs = np.where(small, 1.0, r)
    val = -amp * s ** 3 * np.sqrt(np.pi / 2) * erf(rs / (np.sqrt(2) * s)) / rs
    return np.where(small, -amp * s * s, val)


def bump_potential(x, y, z, centre, R, amp):
    """Potential of A (1 - r^2/R^2)^5, r < R (polynomial inside, -m/r outside)."""
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    t = np.minimum(r / R, 1.0)
    # m(r) = A R^3 P(t),  P(t) = int_0^t s^2 (1 - s^2)^5 ds
    c = [1, -5, 10, -10, 5, -1]              # (1 - s^2)^5 = sum c_j s^{2j}
    P = sum(cj * t ** (2 * j + 3) / (2 * j + 3) for j, cj in enumerate(c))
    Ptot = sum(cj / (2 * j + 3) for j, cj in enumerate(c))
    # inside: u(r) = u(R) - int_r^R m(s)/s^2 ds, with u(R) = -A R^2 Ptot
    # int_t^1 P(s)/s^2 ds = sum c_j/((2j+3)(2j+2)) (1 - t^{2j+2})
    Q = sum(cj / ((2 * j + 3) * (2 * j + 2)) * (1 - t ** (2 * j + 2)) for j, cj in enumerate(c))
    inside = -amp * R * R * (Ptot + Q)
    rs = np.where(r > 0, r, 1.0)
    outside = -amp * R ** 3 * Ptot / rs
    return np.where(r < R, inside, outside)


def u_unb(x):
    x = np.asarray(x, float)
    out = np.zeros_like(x)
    m = (x > 0) & (x < 1)
    q = 2 * x[m] - 1
    out[m] = np.exp(10 * (1 - 1 / (1 - q * q)))
    return out


def u_unb_dd(x):
    """Second derivative of u_unb."""
    x = np.asarray(x, float)
    out = np.zeros_like(x)
    m = (x > 0) & (x < 1)
    q = 2 * x[m] - 1
    a = 1 - q * q
    # u = exp(10 - 10/a), a = 1 - q^2, q = 2x - 1, dq/dx = 2
    # du/dq = u * (-20 q / a^2); d2u/dq2 = u * [(20 q / a^2)^2 - 20/a^2 - 80 q^2 / a^3]
    u = np.exp(10 * (1 - 1 / a))
    d2 = u * ((20 * q / a ** 2) ** 2 - 20 / a ** 2 - 80 * q * q / a ** 3)
    out[m] = 4 * d2
    return out


def manufactured_unb(x, y, z):
    """(u, f) of the three-unbounded manufactured solution of Sec. 4.2."""
    ux, uy, uz = u_unb(x), u_unb(y), u_unb(z)
    f = u_unb_dd(x) * uy * uz + ux * u_unb_dd(y) * uz + ux * uy * u_unb_dd(z)
    return ux * uy * uz, f
