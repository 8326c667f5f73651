"""Gradient of the converged solve: f-bar = dL/df for L = <w, u_leaf>.

The converged solution is a linear map of f (every stage of Alg. 1 and of the
ghost rules of Sec. 2.1 is linear).  It factors as

    f*     = B f                                   (Sec. 3.2: f* = R^M f, with f ghosts)
    0      = res(x, f*) = c(f*) - K x              (composite system, oracle.composite)
    u_leaf = E(x, f*)                              (leaf values; level 0 from the convolution)

so  dL/df = B^T (E_f^T w + c^T lambda)  with  K^T lambda = E_x^T w.

Each factor is written here as the chain of elementary linear operations the
forward code performs (injection into covered blocks, ghost filling, stencil
application, zero-padded convolution), and its transpose is the reverse chain
of the elementary transposes.  No forward state is needed: the maps do not
depend on it.  The transposes are pinned by dot-product identities and the
gradient by central finite differences in tests/test_oracle_adjoint.py.
"""
import numpy as np
from scipy.sparse.linalg import LinearOperator, gmres

from .forest import NBR26
from .lgf import free_space_solve, lgf_at
from .multigrid import OracleSolver


# ---------------------------------------------------------------------------- elementary transposes
def inject_T(s: OracleSolver, fields, k):
    """Transpose of fields[k-1][covered] := fields[k][coincident nodes]."""
    n = s.n
    h = n // 2
    g = (fields[k].shape[1] - n) // 2
    gc = (fields[k - 1].shape[1] - n) // 2
    kids = s._children(k - 1)
    for P in np.nonzero(~s.fo.levels[k - 1].is_leaf)[0]:
        for o in range(8):
            ox, oy, oz = (o & 1) * h, ((o >> 1) & 1) * h, ((o >> 2) & 1) * h
            src = (P, slice(gc + oz, gc + oz + h), slice(gc + oy, gc + oy + h), slice(gc + ox, gc + ox + h))
            fields[k][kids[P, o], g:g + n:2, g:g + n:2, g:g + n:2] += fields[k - 1][src]
            fields[k - 1][src] = 0.0


def ghost_fill_T(s: OracleSolver, fields, k):
    """Transpose of OracleSolver.ghost_fill(fields, k, ...) (outside-domain values dropped).

    The forward first injects level k into the covered nodes of level k-1,
    then overwrites every halo node with a linear combination of interior
    values; the transpose scatters each halo adjoint back to those interior
    values, clears the halo adjoint, then applies the injection transpose.
    """
    A = fields[k]
    n = s.n
    g = (A.shape[1] - n) // 2
    dst = {-1: slice(0, g), 0: slice(g, g + n), 1: slice(g + n, 2 * g + n)}
    src = {-1: slice(n, n + g), 0: slice(g, g + n), 1: slice(g, 2 * g)}
    nbr = s._neighbours[k]
    need = np.zeros(A.shape[0], bool)
    for j, (dx, dy, dz) in enumerate(NBR26):
        has = np.nonzero(nbr[:, j] >= 0)[0]
        if len(has):
            np.add.at(A, (nbr[has, j], src[dz], src[dy], src[dx]), A[has][:, dst[dz], dst[dy], dst[dx]])
        need |= nbr[:, j] == -1
    if np.any(need):
        blocks = np.nonzero(need)[0]
        Tbar = np.zeros((len(blocks),) + A.shape[1:])
        for j, (dx, dy, dz) in enumerate(NBR26):
            sel = np.nonzero(nbr[blocks, j] == -1)[0]
            if len(sel):
                Tbar[sel, dst[dz], dst[dy], dst[dx]] = A[blocks[sel], dst[dz], dst[dy], dst[dx]]
        _interp_T(s, fields, k, blocks, g, Tbar)
    # the forward overwrote every halo node: clear the halo adjoint
    inner = np.zeros(A.shape, bool)
    inner[:, g:g + n, g:g + n, g:g + n] = True
    A[~inner] = 0.0
    if k >= 1:
        inject_T(s, fields, k)


def _interp_T(s: OracleSolver, fields, k, blocks, g, Tbar):
    """Transpose of OracleSolver._interp_from_coarse: scatter Tbar into level k-1 interiors."""
    n = s.n
    lvc = s.fo.levels[k - 1]
    Ac = fields[k - 1]
    gc = (Ac.shape[1] - n) // 2
    C = n // 2 + 9
    P = s._prolong_matrix(g)
    t = np.einsum("zc,bzyx->bcyx", P, Tbar)
    t = np.einsum("yd,bcyx->bcdx", P, t)
    patch = np.einsum("xe,bcdx->bcde", P, t)
    coords = s.fo.levels[k].coords[blocks]
    c0 = coords * (n // 2) - 4
    q = c0[:, :, None] + np.arange(C)[None, None, :]
    qb, ql = q // n, q % n
    blk = lvc.map[qb[:, 2][:, :, None, None], qb[:, 1][:, None, :, None], qb[:, 0][:, None, None, :]]
    lz, ly, lx = ql[:, 2], ql[:, 1], ql[:, 0]
    np.add.at(Ac, (blk, gc + lz[:, :, None, None], gc + ly[:, None, :, None], gc + lx[:, None, None, :]), patch)


def stencil_T(s: OracleSolver, k, lam, blocks, weights, g):
    """Transpose of out[b] = sum_w w A[b][shifted] on the interior of ``blocks`` (A has halo g)."""
    n = s.n
    w = weights
    r = (w.shape[0] - 1) // 2
    S = n + 2 * g
    out = np.zeros((len(blocks), S, S, S))
    for (a, b, c), wt in np.ndenumerate(w):
        if wt != 0.0:
            out[:, g - r + a:g - r + a + n, g - r + b:g - r + b + n, g - r + c:g - r + c + n] += wt * lam
    return out


def conv_T(s: OracleSolver, ubar_cube):
    """Transpose of u = h0^2 (G * f0) from sources [0, N)^3 to targets [-1, N]^3.

    ubar_cube [N+2]^3 (index 0 <-> node -1) -> f0bar [N]^3; the kernel is
    even, so this is the same convolution with source and target regions
    exchanged (periodic length 2N + 2 holds every difference in [-N, N+1]).
    """
    fo = s.fo
    Nz, Ny, Nx = fo.n0[2], fo.n0[1], fo.n0[0]
    N = (Nz, Ny, Nx)
    Pd = [2 * v + 2 for v in N]
    idx = [np.where(np.arange(p) <= p // 2, np.arange(p), np.arange(p) - p) for p in Pd]
    ker = lgf_at(s.G, idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :])
    src = np.zeros(Pd)
    src[:N[0] + 2, :N[1] + 2, :N[2] + 2] = ubar_cube          # index i <-> node i - 1
    conv = np.fft.irfftn(np.fft.rfftn(src) * np.fft.rfftn(ker), s=Pd, axes=(0, 1, 2))
    return fo.h0 ** 2 * conv[1:N[0] + 1, 1:N[1] + 1, 1:N[2] + 1]


def _level0_window_T(s: OracleSolver, U0bar):
    """Transpose of the write of the target cube into every level-0 block window."""
    fo, n = s.fo, s.n
    N = fo.n0
    cube = np.zeros((N[2] + 2, N[1] + 2, N[0] + 2))
    for b, c in enumerate(fo.levels[0].coords):
        z, y, x = c[2] * n, c[1] * n, c[0] * n
        cube[z:z + n + 2, y:y + n + 2, x:x + n + 2] += U0bar[b]
    return cube


def _level0_source_blocks(s, dense):
    fo, n = s.fo, s.n
    out = np.zeros((fo.levels[0].nb, n, n, n))
    for b, c in enumerate(fo.levels[0].coords):
        z, y, x = c[2] * n, c[1] * n, c[0] * n
        out[b] = dense[z:z + n, y:y + n, x:x + n]
    return out


# ---------------------------------------------------------------------------- the gradient
class OracleAdjoint:
    """Exact gradient of the converged composite solution (see module docstring)."""

    def __init__(self, solver: OracleSolver):
        self.s = solver
        fo = solver.fo
        self.fo = fo
        n = fo.n
        self.n = n
        self.leaf_sel = [np.nonzero(lv.is_leaf)[0] for lv in fo.levels]
        self.cov0 = np.nonzero(~fo.levels[0].is_leaf)[0]
        self.sizes = [len(self.leaf_sel[k]) * n ** 3 for k in range(1, fo.max_level + 1)]
        self.nx = sum(self.sizes) + len(self.cov0) * n ** 3

    # ---- res^T: residual-space lambda -> (x-bar, f*-bar per level)
    def res_T(self, lam):
        s, fo, n = self.s, self.fo, self.n
        L = fo.max_level
        Ub = [np.zeros_like(A) for A in s.U]
        fsb = [np.zeros_like(A) for A in s.F]
        off = 0
        lam_r = {}
        for k in range(1, L + 1):
            m = self.sizes[k - 1]
            lam_r[k] = lam[off:off + m].reshape(-1, n, n, n)
            off += m
        lam_c = lam[off:].reshape(-1, n, n, n)
        h0 = fo.h0
        # c0 rows: (conv_cov - U0[cov]) / h0^2
        conv_cov_bar = lam_c / h0 ** 2
        Ub[0][self.cov0, 1:1 + n, 1:1 + n, 1:1 + n] -= lam_c / h0 ** 2
        # leaf rows: f*_k - L_k U[k]
        for k in range(1, L + 1):
            leaf = self.leaf_sel[k]
            fsb[k][leaf] += lam_r[k]
            Ub[k][leaf] -= stencil_T(s, k, lam_r[k], leaf, s.wL, 1) / fo.h(k) ** 2
        # ghost fills of levels L..1 (each preceded by its injection), reversed
        for k in range(1, L + 1):
            ghost_fill_T(s, Ub, k)
        # the copy of the level-0 covered values taken before the ghost fills
        Ub[0][self.cov0, 1:1 + n, 1:1 + n, 1:1 + n] += conv_cov_bar
        # level-0 field = window of the convolution of F0 = f*_0 (leaves) + s (covered)
        F0bar = _level0_source_blocks(s, conv_T(s, _level0_window_T(s, Ub[0])))
        leaf0 = self.leaf_sel[0]
        fsb[0][leaf0] += F0bar[leaf0]
        sbar = F0bar[self.cov0]
        # injections of levels L..2 at the start, reversed
        for k in range(2, L + 1):
            inject_T(s, Ub, k)
        xbar = [Ub[k][self.leaf_sel[k], 1:1 + n, 1:1 + n, 1:1 + n].reshape(-1) for k in range(1, L + 1)]
        xbar.append(sbar.reshape(-1))
        return np.concatenate(xbar), fsb

    def K_T(self, lam):
        xb, _ = self.res_T(lam)
        return -xb

    # ---- E^T: leaf adjoint w -> (x-bar, f*-bar)
    def E_T(self, w_leaf):
        s, fo, n = self.s, self.fo, self.n
        L = fo.max_level
        wl = [np.zeros((lv.nb, n, n, n)) for lv in fo.levels]
        for i, (lev, b) in enumerate(fo.leaf_slot):
            wl[lev][b] = w_leaf[i]
        xbar = [wl[k][self.leaf_sel[k]].reshape(-1) for k in range(1, L + 1)]
        U0bar = np.zeros_like(s.U[0])
        U0bar[:, 1:1 + n, 1:1 + n, 1:1 + n] = wl[0]       # only leaf blocks carry w
        F0bar = _level0_source_blocks(s, conv_T(s, _level0_window_T(s, U0bar)))
        fsb = [np.zeros_like(A) for A in s.F]
        leaf0 = self.leaf_sel[0]
        fsb[0][leaf0] = F0bar[leaf0]
        xbar.append(F0bar[self.cov0].reshape(-1))
        return np.concatenate(xbar), fsb

    # ---- B^T: f*-bar (per level, leaf blocks) -> f-bar (leaf layout)
    def B_T(self, fsb):
        s, fo, n = self.s, self.fo, self.n
        L = fo.max_level
        Rb = [np.zeros_like(A) for A in s.fraw]
        for k in range(L + 1):
            leaf = self.leaf_sel[k]
            if len(leaf):
                Rb[k][leaf] += stencil_T(s, k, fsb[k][leaf], leaf, s.wR, 2)
        for k in range(L, -1, -1):
            ghost_fill_T(s, Rb, k)
        for k in range(0, L):
            inject_T(s, Rb, k + 1)
        return np.stack([Rb[l][b, 2:2 + n, 2:2 + n, 2:2 + n] for l, b in fo.leaf_slot])

    # ---- the gradient
    def gradient(self, w_leaf, rtol=1e-13, precondition=True):
        xw, fsb_e = self.E_T(w_leaf)
        A = LinearOperator((self.nx, self.nx), matvec=self.K_T, dtype=float)
        lam, info = gmres(A, xw, rtol=rtol, atol=0.0, restart=400, maxiter=50)
        self.info = info
        _, fsb_c = self.res_T(lam)
        fsb = [a + b for a, b in zip(fsb_e, fsb_c)]
        return self.B_T(fsb)
