"""Lattice Green's function of the multigrid operator and the free-space
convolution on the uniform level 0.

Sec. 2.2: the FFT solver convolves with the lattice Green's function G[n]
of the finite-difference operator L, i.e. L G = delta.  Sec. 3.3: that kernel
must be the LGF of the *multigrid* operator, otherwise the multigrid solver
stops converging.  The paper gives no formula for the three-unbounded LGF, so
this module evaluates the defining Fourier integral directly:

    G[n] = (2 pi)^-3  int_{[-pi,pi]^3} cos(k.n) / sigma(k) dk,

sigma being the symbol of the unit-spacing LHS stencil.  With
s_i = 4 sin^2(k_i / 2) the symbols of Eq. cross_discr2 and
Eq. mehrstellen_discr4/6 are

    sigma_2 = -(s1 + s2 + s3)
    sigma_4 = sigma_2 + (s1 s2 + s2 s3 + s3 s1) / 6
    sigma_6 = sigma_4 - s1 s2 s3 / 30.

Each is affine in s3 = 2 - 2 cos k3: sigma = -(c0 + c1 s3), so the k3
integral is the classical one

    (1/2pi) int cos(n3 k3) / (alpha - beta cos k3) dk3 = rho^|n3| / sqrt(alpha^2 - beta^2),
    alpha = c0 + 2 c1, beta = 2 c1, rho = beta / (alpha + sqrt(alpha^2 - beta^2)),

leaving a 2-D integral over [0, pi]^2 whose only singularity (1/|k_perp| at
the origin) is removed by the Duffy map (k1, k2) = (u, u v) on each of the
two triangles.  The remaining smooth integrand is summed with composite
Gauss-Legendre rules (numpy's ``leggauss`` nodes on equal panels).
"""
import numpy as np

from .stencils import lhs_stencil


def _composite_gl(q, a, b, panels):
    x, w = np.polynomial.legendre.leggauss(q)
    edges = np.linspace(a, b, panels + 1)
    xs, ws = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (hi - lo) * x + 0.5 * (hi + lo))
        ws.append(0.5 * (hi - lo) * w)
    return np.concatenate(xs), np.concatenate(ws)


def quadrature_panels(nmax):
    """Panel counts (u on [0, pi], v on [0, 1]) of 32-point rules for |n| <= nmax."""
    return 8 + nmax // 16, 4 + nmax // 32


def symbol_coefficients(M, s1, s2):
    """(c0, c1) with sigma_M = -(c0 + c1 s3); see the module docstring."""
    if M == 2:
        return s1 + s2, np.ones_like(s1)
    c0 = s1 + s2 - s1 * s2 / 6.0
    c1 = 1.0 - (s1 + s2) / 6.0
    if M == 6:
        c1 = c1 + s1 * s2 / 30.0
    return c0, c1


def lgf_table(M, nmax, q=32):
    """G[n1, n2, n3] for 0 <= n_i <= nmax (one octant; G is even in each n_i).

    Array index order [n1][n2][n3]; G is symmetric under any permutation of
    (n1, n2, n3), so the axis naming does not matter.
    """
    pu, pv = quadrature_panels(nmax)
    u, wu = _composite_gl(q, 0.0, np.pi, pu)
    v, wv = _composite_gl(q, 0.0, 1.0, pv)
    k1 = u[:, None] * np.ones_like(v)[None, :]
    k2 = u[:, None] * v[None, :]
    s1 = 4.0 * np.sin(k1 / 2) ** 2
    s2 = 4.0 * np.sin(k2 / 2) ** 2
    c0, c1 = symbol_coefficients(M, s1, s2)
    sq = np.sqrt(c0 * (c0 + 4.0 * c1))          # sqrt(alpha^2 - beta^2) = sqrt((alpha-beta)(alpha+beta))
    rho = 2.0 * c1 / (c0 + 2.0 * c1 + sq)
    W = wu[:, None] * wv[None, :] * u[:, None] / sq   # Duffy Jacobian u
    n = np.arange(nmax + 1)
    Wp = np.empty(W.shape + (nmax + 1,))
    rp = np.ones_like(rho)
    for n3 in range(nmax + 1):
        Wp[:, :, n3] = W * rp
        rp = rp * rho
    # B[i, n2, n3] = sum_j cos(n2 u_i v_j) W_ij rho_ij^n3
    C2 = np.cos(n[None, :, None] * k2[:, None, :])            # [i, n2, j]
    B = np.matmul(C2, Wp)                                      # [i, n2, n3]
    C1 = np.cos(n[:, None] * u[None, :])                       # [n1, i]
    A = np.einsum("ai,ibc->abc", C1, B)                        # triangle k2 <= k1
    G = -(A + A.transpose(1, 0, 2)) / np.pi ** 2               # + triangle k1 <= k2
    return G


def lgf_at(G, dz, dy, dx):
    """G at integer offsets of any sign (arrays broadcast)."""
    return G[np.abs(dz), np.abs(dy), np.abs(dx)]


def apply_lhs_unit(M, U):
    """Unit-spacing LHS stencil applied at the interior of a 3-D array (one layer lost)."""
    w = lhs_stencil(M)
    nz, ny, nx = U.shape
    out = np.zeros((nz - 2, ny - 2, nx - 2))
    for (a, b, c), wt in np.ndenumerate(w):
        if wt != 0.0:
            out += wt * U[a:a + nz - 2, b:b + ny - 2, c:c + nx - 2]
    return out


def free_space_solve(f0, G, h):
    """u = h^2 (G * f0) on the target cube [-1, N]^3 of a uniform level.

    Sec. 2.2 (Hockney-Eastwood zero padding): ``f0`` [Nz, Ny, Nx] lives on
    nodes 0..N-1 and vanishes elsewhere; the linear convolution is exact on
    targets -1..N when the periodic length is at least 2N + 1; this function
    uses 2N + 2.  The h^2 factor comes from L_h = L / h^2 with G the LGF of
    the unit-spacing L.  Returns [Nz+2, Ny+2, Nx+2] with index 0 <-> node -1.
    """
    N = f0.shape
    P = [2 * s + 2 for s in N]
    ker = np.empty(P)
    idx = [np.where(np.arange(p) <= p // 2, np.arange(p), np.arange(p) - p) for p in P]
    ker[...] = lgf_at(G, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :])
    src = np.zeros(P)
    src[:N[0], :N[1], :N[2]] = f0
    conv = np.fft.irfftn(np.fft.rfftn(src) * np.fft.rfftn(ker), s=P, axes=(0, 1, 2))
    tz = np.arange(-1, N[0] + 1) % P[0]
    ty = np.arange(-1, N[1] + 1) % P[1]
    tx = np.arange(-1, N[2] + 1) % P[2]
    return h * h * conv[np.ix_(tz, ty, tx)]


def direct_sum(f0, G, h, targets=None):
    """Brute-force u[t] = h^2 sum_s G[t - s] f0[s] (for small grids).

    ``targets`` is an int array [m, 3] of (z, y, x) node indices; default
    is the whole cube [-1, N]^3 in the layout of :func:`free_space_solve`.
    """
    N = f0.shape
    sz, sy, sx = np.nonzero(np.ones(N, bool))
    fv = f0.reshape(-1)
    if targets is None:
        grid = np.stack(np.meshgrid(np.arange(-1, N[0] + 1), np.arange(-1, N[1] + 1),
                                    np.arange(-1, N[2] + 1), indexing="ij"), -1).reshape(-1, 3)
    else:
        grid = np.asarray(targets)
    out = np.empty(len(grid))
    for t, (z, y, x) in enumerate(grid):
        out[t] = h * h * np.dot(lgf_at(G, z - sz, y - sy, x - sx), fv)
    if targets is None:
        return out.reshape(N[0] + 2, N[1] + 2, N[2] + 2)
    return out
