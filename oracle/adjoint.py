"""Gradient of the converged solve: f-bar = dL/df for L = <w, u_leaf>.

The converged solution is a linear map of f (every stage of Alg. 1 and of the
ghost rules of Sec. 2.1 is linear).  It factors as

    f*     = B f                                   (Sec. 3.2: f* = R^M f, with f ghosts)
    0      = res(x, f*) = c(f*) - K x              (composite system, oracle.composite)
    u_leaf = E(x, f*)                              (leaf values; level 0 from the convolution)

so  dL/df = B^T (E_f^T w + c^T lambda)  with  K^T lambda = E_x^T w.

K^T lambda = E_x^T w is solved two ways: by plain GMRES (``gradient``, the
independent route) and by the transposed V-cycle inside an iterative
refinement loop (``gradient_ir``, the method the GPU path follows).  One
V-cycle of Alg. 1 started from u = 0 on the correction equation K e = r is a
linear map e = M r; its transpose M^T is the same chain of operations
(smoothing, residual, restriction, coarse solve, correction) transposed one by
one and run in reverse order (Gauss-Seidel colours 7..0, full weighting <->
trilinear interpolation, ghost filling <-> scatter of the ghost adjoints).
Since I - M^T K^T = (I - K M)^T has the spectrum of the forward cycle's error
propagator, lambda <- lambda + M^T (E_x^T w - K^T lambda) contracts at the
forward V-cycle's rate, whereas M itself is a poor preconditioner for K^T (the
composite operator is far from symmetric at resolution jumps).

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
from .stencils import full_weighting


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


# ---------------------------------------------------------------------------- V-cycle transposes
def smooth_T(s: OracleSolver, Ub, Fb, k):
    """Transpose of OracleSolver.smooth(k): colours 7..0, each colour's update transposed.

    The forward colour step overwrites u at the nodes of colour c with
    (h^2 f - sum_q w_q u_q) / w_c; nodes of one colour are never neighbours,
    so the transpose sends the adjoint of each such node to f (h^2 / w_c) and
    to its neighbours (-w_q / w_c), then clears it.
    """
    n = s.n
    U, F = Ub[k], Fb[k]
    h2 = s.fo.h(k) ** 2
    wc = s.wL[1, 1, 1]
    offs = [(a - 1, b - 1, c - 1, w) for (a, b, c), w in np.ndenumerate(s.wL)
            if w != 0.0 and (a, b, c) != (1, 1, 1)]
    for col in range(7, -1, -1):
        cx, cy, cz = col & 1, (col >> 1) & 1, (col >> 2) & 1
        t = U[:, 1 + cz:1 + n:2, 1 + cy:1 + n:2, 1 + cx:1 + n:2].copy()
        U[:, 1 + cz:1 + n:2, 1 + cy:1 + n:2, 1 + cx:1 + n:2] = 0.0
        F[:, cz::2, cy::2, cx::2] += (h2 / wc) * t
        for dz, dy, dx, w in offs:
            U[:, 1 + cz + dz:1 + n + dz:2, 1 + cy + dy:1 + n + dy:2, 1 + cx + dx:1 + n + dx:2] -= (w / wc) * t


def residual_T(s: OracleSolver, Ub, Fb, Rb, k):
    """Transpose of R_k = F_k - L_k U_k on every level-k block."""
    nb = Ub[k].shape[0]
    Fb[k] += Rb[k]
    Ub[k] -= stencil_T(s, k, Rb[k], np.arange(nb), s.wL, 1) / s.fo.h(k) ** 2
    Rb[k][...] = 0.0


def restrict_T(s: OracleSolver, Ub, Fb, Rb, Hb, k, off0b):
    """Transpose of OracleSolver.restrict(k) (injection of u, full weighting of r, FAS, snapshot).

    off0b receives the adjoint of the level-0 offset (k == 1 only).
    """
    fo, n = s.fo, s.n
    h = n // 2
    lvc = fo.levels[k - 1]
    kids = s._children(k - 1)
    covered = np.nonzero(~lvc.is_leaf)[0]
    # uhat_{k-1} = u_{k-1} (whole level)
    Ub[k - 1][:, 1:1 + n, 1:1 + n, 1:1 + n] += Hb[k - 1]
    Hb[k - 1][...] = 0.0
    # f_{k-1} += L u_{k-1} on the covered blocks
    if len(covered):
        Ub[k - 1][covered] += stencil_T(s, k - 1, Fb[k - 1][covered], covered, s.wL, 1) / fo.h(k - 1) ** 2
    ghost_fill_T(s, Ub, k - 1)
    # f_{k-1} = FW(r_k) (injection where the 27-point window leaves Omega_k)
    mask, base = s._dense(np.zeros_like(Rb[k]), k, np.nan)
    Dbar = np.zeros(mask.shape)
    W = full_weighting()
    for P in covered:
        B = lvc.coords[P]
        lo = 2 * B[::-1] * n - 1 - base
        win = mask[lo[0]:lo[0] + 2 * n + 1, lo[1]:lo[1] + 2 * n + 1, lo[2]:lo[2] + 2 * n + 1]
        full = np.ones((n, n, n), bool)
        for (a, b, c), w in np.ndenumerate(W):
            full &= ~np.isnan(win[a:a + 2 * n:2, b:b + 2 * n:2, c:c + 2 * n:2])
        fb = Fb[k - 1][P]
        wbar = Dbar[lo[0]:lo[0] + 2 * n + 1, lo[1]:lo[1] + 2 * n + 1, lo[2]:lo[2] + 2 * n + 1]
        for (a, b, c), w in np.ndenumerate(W):
            wbar[a:a + 2 * n:2, b:b + 2 * n:2, c:c + 2 * n:2] += w * np.where(full, fb, 0.0)
        wbar[1:1 + 2 * n:2, 1:1 + 2 * n:2, 1:1 + 2 * n:2] += np.where(full, 0.0, fb)
        Fb[k - 1][P] = 0.0
    for b, c in enumerate(fo.levels[k].coords):
        o = c * n - base[::-1]
        Rb[k][b] += Dbar[o[2]:o[2] + n, o[1]:o[1] + n, o[0]:o[0] + n]
    # u_{k-1}[covered] = injection of u_k (+ offset at level 0)
    for j, P in enumerate(covered):
        if k == 1:
            off0b[j] += Ub[0][P, 1:1 + n, 1:1 + n, 1:1 + n]
        for o in range(8):
            ox, oy, oz = (o & 1) * h, ((o >> 1) & 1) * h, ((o >> 2) & 1) * h
            Ub[k][kids[P, o], 1:1 + n:2, 1:1 + n:2, 1:1 + n:2] += \
                Ub[k - 1][P, 1 + oz:1 + oz + h, 1 + oy:1 + oy + h, 1 + ox:1 + ox + h]
        Ub[k - 1][P, 1:1 + n, 1:1 + n, 1:1 + n] = 0.0


def coarse_solve_T(s: OracleSolver, Ub, Fb):
    """Transpose of OracleSolver.coarse_solve: u_0 (with its exterior ring) overwritten by h0^2 G * f_0."""
    Fb[0] += _level0_source_blocks(s, conv_T(s, _level0_window_T(s, Ub[0])))
    Ub[0][...] = 0.0


def prolong_correct_T(s: OracleSolver, Ub, Hb, k):
    """Transpose of u_k += trilinear(u_{k-1} - uhat_{k-1})."""
    n = s.n
    h = n // 2
    shape, base = s._dense(np.zeros((s.fo.levels[k - 1].nb, n, n, n)), k - 1, 0.0)
    Dbar = np.zeros(shape.shape)
    T = np.zeros((n, h + 1))
    for i in range(n):
        if i % 2 == 0:
            T[i, i // 2] = 1.0
        else:
            T[i, (i - 1) // 2] = 0.5
            T[i, (i + 1) // 2] = 0.5
    for b, c in enumerate(s.fo.levels[k].coords):
        lo = c[::-1] * h - base
        Dbar[lo[0]:lo[0] + h + 1, lo[1]:lo[1] + h + 1, lo[2]:lo[2] + h + 1] += \
            np.einsum("zc,yd,xe,zyx->cde", T, T, T, Ub[k][b, 1:1 + n, 1:1 + n, 1:1 + n])
    for b, c in enumerate(s.fo.levels[k - 1].coords):
        o = c * n - base[::-1]
        e = Dbar[o[2]:o[2] + n, o[1]:o[1] + n, o[0]:o[0] + n]
        Ub[k - 1][b, 1:1 + n, 1:1 + n, 1:1 + n] += e
        Hb[k - 1][b] -= e


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

    # ---- the correction V-cycle M and its transpose
    def _split(self, v):
        n, L = self.n, self.fo.max_level
        out, off = {}, 0
        for k in range(1, L + 1):
            m = self.sizes[k - 1]
            out[k] = v[off:off + m].reshape(-1, n, n, n)
            off += m
        return out, v[off:].reshape(-1, n, n, n)

    def correction_cycle(self, r):
        """e = M r: one V-cycle of Alg. 1 from u = 0 on K e = r.

        Leaf rows of r are the right-hand side of the leaf blocks of levels
        >= 1 (level-0 leaves get 0); the covered level-0 rows (conv - inj) /
        h0^2 enter as the offset -h0^2 r_c of the injection into level 0.
        e is read from the leaf interiors of levels >= 1 and from the level-0
        right-hand side on covered blocks (the source s of the composite
        system).
        """
        s, fo, n = self.s, self.fo, self.n
        L = fo.max_level
        for group in (s.U, s.F, s.R, s.H):
            for A in group:
                A[...] = 0.0
        rk, rc = self._split(r)
        for k in range(1, L + 1):
            s.F[k][self.leaf_sel[k]] = rk[k]
        s.off0 = -fo.h0 ** 2 * rc
        s.vcycle()
        s.off0 = None
        xs = [s.U[k][self.leaf_sel[k], 1:1 + n, 1:1 + n, 1:1 + n].reshape(-1) for k in range(1, L + 1)]
        xs.append(s.F[0][self.cov0].reshape(-1))
        return np.concatenate(xs)

    def correction_cycle_T(self, xbar):
        """M^T xbar: the operations of ``correction_cycle`` transposed, in reverse order."""
        s, fo, n = self.s, self.fo, self.n
        L = fo.max_level
        Ub = [np.zeros_like(A) for A in s.U]
        Fb = [np.zeros_like(A) for A in s.F]
        Rb = [np.zeros_like(A) for A in s.R]
        Hb = [np.zeros_like(A) for A in s.H]
        off0b = np.zeros((len(self.cov0), n, n, n))
        xk, sb = self._split(xbar)
        for k in range(1, L + 1):
            Ub[k][self.leaf_sel[k], 1:1 + n, 1:1 + n, 1:1 + n] = xk[k]
        Fb[0][self.cov0] = sb
        for k in range(L, 0, -1):
            for _ in range(s.nu2):
                smooth_T(s, Ub, Fb, k)
                ghost_fill_T(s, Ub, k)
            prolong_correct_T(s, Ub, Hb, k)
        coarse_solve_T(s, Ub, Fb)
        for k in range(1, L + 1):
            restrict_T(s, Ub, Fb, Rb, Hb, k, off0b)
            residual_T(s, Ub, Fb, Rb, k)
            ghost_fill_T(s, Ub, k)
            for _ in range(s.nu1):
                smooth_T(s, Ub, Fb, k)
                ghost_fill_T(s, Ub, k)
        out = [Fb[k][self.leaf_sel[k]].reshape(-1) for k in range(1, L + 1)]
        out.append((-fo.h0 ** 2 * off0b).reshape(-1))
        return np.concatenate(out)

    def gradient_ir(self, w_leaf, tol=1e-12, max_iter=40):
        """Gradient with K^T lambda = E_x^T w solved by lambda += M^T (E_x^T w - K^T lambda).

        Stops when max|E_x^T w - K^T lambda| / max|E_x^T w| < tol; the
        relative residual of every iteration is left in ``self.history``.
        """
        g, fsb_e = self.E_T(w_leaf)
        gn = float(np.abs(g).max()) or 1.0
        lam = np.zeros_like(g)
        self.history = []
        for _ in range(max_iter):
            rho = g - self.K_T(lam)
            rel = float(np.abs(rho).max()) / gn
            self.history.append(rel)
            if rel < tol:
                break
            lam = lam + self.correction_cycle_T(rho)
        self.lam = lam
        _, fsb_c = self.res_T(lam)
        fsb = [a + b for a, b in zip(fsb_e, fsb_c)]
        return self.B_T(fsb)

    # ---- the gradient
    def gradient(self, w_leaf, rtol=1e-13, precondition=True):
        xw, fsb_e = self.E_T(w_leaf)
        A = LinearOperator((self.nx, self.nx), matvec=self.K_T, dtype=float)
        lam, info = gmres(A, xw, rtol=rtol, atol=0.0, restart=400, maxiter=50)
        self.info = info
        _, fsb_c = self.res_T(lam)
        fsb = [a + b for a, b in zip(fsb_e, fsb_c)]
        return self.B_T(fsb)
