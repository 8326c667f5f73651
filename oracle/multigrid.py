"""Adaptive FAS multigrid V-cycle of Alg. 1 (amg_vcycle), plain FP64 numpy.

Fields live per level as arrays ``[block][z][y][x]``; ``U`` carries one
ghost layer (all LHS stencils have radius one, Sec. 3.2), the raw source f
carries two (R^6 has width two).  Operations follow Alg. 1 in order; the
readings of the points the paper leaves open are:

* ghosting (Sec. 2.1): a halo region whose level-k neighbour block exists is
  copied from it; otherwise it is interpolated from level k-1 with the
  tensor-product Lagrange interpolant of I = M + 2 points (identity along
  axes where the ghost node coincides with a coarse node).  The level-(k-1)
  data it reads holds, on nodes covered by level k, the injection of the
  current level-k values (the coarse representation of the fine blocks).
  Outside the domain, u keeps the exterior values of the last level-0 solve
  and f is 0.
* smoothing (Sec. 3.1, one Gauss-Seidel iteration): within each block the
  nodes are visited in 8 colours c = (i&1) + 2(j&1) + 4(k&1), c = 0..7, with
  the ghost layer frozen during the sweep; blocks are independent.
* full weighting near the edge of Omega_k: a coarse node whose 27-point
  stencil reaches outside Omega_k takes the injected residual.
* the correction (Alg. 1, coarse-to-fine loop) is eps = u_{k-1} - uhat_{k-1}
  (value after the coarse solve minus the stored value), added through
  trilinear interpolation; uhat is stored for the whole level k-1 when
  level k is restricted, so eps is defined on the ring next to Omega_k.
* the coarse solve (Sec. 2.2, Sec. 3.3) writes u on all level-0 nodes and a
  one-node exterior ring; it is the LGF convolution of ``lgf``.
"""
import numpy as np

from .forest import NBR26, OracleForest
from .stencils import lhs_stencil, rhs_stencil, midpoint_lagrange, full_weighting
from .lgf import lgf_table, free_space_solve


class OracleSolver:
    def __init__(self, forest: OracleForest, M, nu1=3, nu2=3, G=None):
        self.fo = forest
        self.M = int(M)
        self.nu1, self.nu2 = int(nu1), int(nu2)
        self.n = forest.n
        self.I = self.M + 2
        self.wL = lhs_stencil(self.M)
        self.wR = rhs_stencil(self.M)
        self.wI = midpoint_lagrange(self.I)
        self.G = G if G is not None else lgf_table(self.M, max(forest.n0) + 1)
        n = self.n
        nbs = [lv.nb for lv in forest.levels]
        self.U = [np.zeros((nb, n + 2, n + 2, n + 2)) for nb in nbs]
        self.F = [np.zeros((nb, n, n, n)) for nb in nbs]
        self.R = [np.zeros((nb, n, n, n)) for nb in nbs]
        self.H = [np.zeros((nb, n, n, n)) for nb in nbs]
        self.fraw = [np.zeros((nb, n + 4, n + 4, n + 4)) for nb in nbs]
        self._neighbours = [self._neighbour_table(k) for k in range(len(nbs))]
        self._kids = [self._children_table(k) for k in range(len(nbs))]
        self._prolong_cache = {}
        self.cycles_done = 0
        # optional offset added to the covered level-0 nodes when level 1 is
        # restricted to level 0 ([covered level-0 block][z][y][x]); a correction
        # solve carries there the mismatch between the level-0 field and the
        # injection of level 1.  None in a plain solve.
        self.off0 = None

    # ------------------------------------------------------------------ forest helpers
    def _neighbour_table(self, k):
        lv = self.fo.levels[k]
        out = np.empty((lv.nb, 26), np.int64)
        for j, d in enumerate(NBR26):
            for b, c in enumerate(lv.coords):
                out[b, j] = lv.find((c[0] + d[0], c[1] + d[1], c[2] + d[2]))
        return out

    def _children(self, k):
        return self._kids[k]

    def _children_table(self, k):
        """[nb_k][8] child block indices at level k+1 (-1 for leaves); child o = (o&1, o>>1&1, o>>2&1)."""
        lv = self.fo.levels[k]
        out = -np.ones((lv.nb, 8), np.int64)
        if k + 1 < len(self.fo.levels):
            nxt = self.fo.levels[k + 1]
            for b, c in enumerate(lv.coords):
                if lv.is_leaf[b]:
                    continue
                for o in range(8):
                    out[b, o] = nxt.find((2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1),
                                          2 * c[2] + ((o >> 2) & 1)))
        return out

    def _dense(self, A, k, fill, lo_pad=1, hi_pad=1):
        """Interior values of level-k blocks in one array over their bounding box.

        Returns (D, base) with D[z, y, x] = node (base + (z, y, x)) in level-k
        node indices, and ``fill`` where no level-k block holds the node.
        """
        n = self.n
        lv = self.fo.levels[k]
        c = lv.coords
        lo = (c.min(0) - lo_pad) * n
        hi = (c.max(0) + 1 + hi_pad) * n
        D = np.full((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), fill)
        for b in range(lv.nb):
            o = c[b] * n - lo
            D[o[2]:o[2] + n, o[1]:o[1] + n, o[0]:o[0] + n] = A[b]
        return D, lo[::-1]

    # ------------------------------------------------------------------ ghosting (Sec. 2.1)
    def _prolong_matrix(self, g):
        """1-D Lagrange prolongation from a coarse patch of n/2 + 9 nodes to n + 2g fine nodes.

        Patch index 0 is coarse node (b n / 2 - 4); fine index t is fine node
        b n + t - g.  Even fine nodes coincide with a coarse node; odd ones are
        midpoints, interpolated from the I nearest coarse nodes.
        """
        if g in self._prolong_cache:
            return self._prolong_cache[g]
        n, I = self.n, self.I
        C = n // 2 + 9
        P = np.zeros((n + 2 * g, C))
        for t in range(n + 2 * g):
            r = t - g + 8                  # fine offset from the patch origin, in fine nodes
            if r % 2 == 0:
                P[t, r // 2] = 1.0
            else:
                left = (r - 1) // 2
                for m in range(I):
                    P[t, left - I // 2 + 1 + m] = self.wI[m]
        self._prolong_cache[g] = P
        return P

    def _interp_from_coarse(self, fields, k, blocks, g):
        """Prolongation of level k-1 data onto the full (n+2g)^3 box of ``blocks``."""
        n = self.n
        lvc = self.fo.levels[k - 1]
        A = fields[k - 1]
        gc = (A.shape[1] - n) // 2
        C = n // 2 + 9
        coords = self.fo.levels[k].coords[blocks]
        c0 = coords * (n // 2) - 4                      # coarse node index of patch origin (x, y, z)
        q = c0[:, :, None] + np.arange(C)[None, None, :]  # [b, axis, C]
        qb, ql = q // n, q % n
        qz, qy, qx = qb[:, 2], qb[:, 1], qb[:, 0]
        blk = lvc.map[qz[:, :, None, None], qy[:, None, :, None], qx[:, None, None, :]]
        if np.any(blk < 0):
            raise AssertionError("ghost interpolation reaches a missing coarse block")
        lz, ly, lx = ql[:, 2], ql[:, 1], ql[:, 0]
        patch = A[blk, gc + lz[:, :, None, None], gc + ly[:, None, :, None], gc + lx[:, None, None, :]]
        P = self._prolong_matrix(g)
        t = np.einsum("xe,bcde->bcdx", P, patch)
        t = np.einsum("yd,bcdx->bcyx", P, t)
        t = np.einsum("zc,bcyx->bzyx", P, t)
        return t

    def inject_into_parent(self, fields, k):
        """Covered nodes of level k-1 take the values of the coincident level-k nodes (injection)."""
        n = self.n
        h = n // 2
        g = (fields[k].shape[1] - n) // 2
        gc = (fields[k - 1].shape[1] - n) // 2
        kids = self._children(k - 1)
        covered = np.nonzero(~self.fo.levels[k - 1].is_leaf)[0]
        for P in covered:
            for o in range(8):
                ox, oy, oz = (o & 1) * h, ((o >> 1) & 1) * h, ((o >> 2) & 1) * h
                fields[k - 1][P, gc + oz:gc + oz + h, gc + oy:gc + oy + h, gc + ox:gc + ox + h] = \
                    fields[k][kids[P, o], g:g + n:2, g:g + n:2, g:g + n:2]


    def ghost_fill(self, fields, k, exterior):
        """Fill the halo of every level-k block (Sec. 2.1 ghosting).

        Ghosts at a resolution jump are reconstructed from the coarse level
        as the multiresolution grid represents it: level-(k-1) nodes covered
        by level k first take the injection of the current level-k values,
        so the interpolant sees the fine block's own data on its side of the
        jump.  exterior: 'keep' leaves halo nodes outside the domain
        untouched (u: exterior ring of the last coarse solve); 'zero' writes
        0 there (f is zero outside the domain).
        """
        if k >= 1:
            self.inject_into_parent(fields, k)
        A = fields[k]
        n = self.n
        g = (A.shape[1] - n) // 2
        if g == 0:
            return
        dst = {-1: slice(0, g), 0: slice(g, g + n), 1: slice(g + n, 2 * g + n)}
        src = {-1: slice(n, n + g), 0: slice(g, g + n), 1: slice(g, 2 * g)}
        nbr = self._neighbours[k]
        need = np.zeros(A.shape[0], bool)
        for j, (dx, dy, dz) in enumerate(NBR26):
            has = nbr[:, j] >= 0
            if np.any(has):
                b = np.nonzero(has)[0]
                A[b, dst[dz], dst[dy], dst[dx]] = A[nbr[b, j], src[dz], src[dy], src[dx]]
            out = nbr[:, j] == -2
            if exterior == "zero" and np.any(out):
                A[np.nonzero(out)[0], dst[dz], dst[dy], dst[dx]] = 0.0
            need |= nbr[:, j] == -1
        if np.any(need):
            if k == 0:
                raise AssertionError("level 0 cannot interpolate")
            blocks = np.nonzero(need)[0]
            T = self._interp_from_coarse(fields, k, blocks, g)
            for j, (dx, dy, dz) in enumerate(NBR26):
                sel = np.nonzero(nbr[blocks, j] == -1)[0]
                if len(sel):
                    A[blocks[sel], dst[dz], dst[dy], dst[dx]] = T[sel][:, dst[dz], dst[dy], dst[dx]]

    # ------------------------------------------------------------------ operators
    def apply_lhs(self, k, blocks=None):
        """(L_k u) on the interior of level-k blocks, with the current halo."""
        U = self.U[k] if blocks is None else self.U[k][blocks]
        n = self.n
        acc = np.zeros((U.shape[0], n, n, n))
        for (a, b, c), w in np.ndenumerate(self.wL):
            if w != 0.0:
                acc += w * U[:, a:a + n, b:b + n, c:c + n]
        return acc / self.fo.h(k) ** 2

    def prepare_rhs(self, f_leaf):
        """f* = R^M f at every leaf node (Sec. 3.2; computed once and stored).

        f is given at leaf nodes; a non-leaf block holds f at its nodes by
        injection (point values of the same function); its ghosts follow the
        ghosting rules with f = 0 outside the domain.
        """
        fo, n = self.fo, self.n
        L = fo.max_level
        for A in self.fraw:
            A[...] = 0.0
        for i, (lev, b) in enumerate(fo.leaf_slot):
            self.fraw[lev][b, 2:2 + n, 2:2 + n, 2:2 + n] = f_leaf[i]
        for k in range(L - 1, -1, -1):
            kids = self._children(k)
            for b in np.nonzero(~fo.levels[k].is_leaf)[0]:
                for o in range(8):
                    ox, oy, oz = (o & 1) * n // 2, ((o >> 1) & 1) * n // 2, ((o >> 2) & 1) * n // 2
                    self.fraw[k][b, 2 + oz:2 + oz + n // 2, 2 + oy:2 + oy + n // 2, 2 + ox:2 + ox + n // 2] = \
                        self.fraw[k + 1][kids[b, o], 2:2 + n:2, 2:2 + n:2, 2:2 + n:2]
        for k in range(L + 1):
            self.ghost_fill(self.fraw, k, "zero")
        self.fstar_max = 0.0
        for k in range(L + 1):
            leaf = np.nonzero(fo.levels[k].is_leaf)[0]
            A = self.fraw[k][leaf]
            acc = np.zeros((len(leaf), n, n, n))
            for (a, b, c), w in np.ndenumerate(self.wR):
                if w != 0.0:
                    acc += w * A[:, a:a + n, b:b + n, c:c + n]
            self.F[k][leaf] = acc
            if len(leaf):
                self.fstar_max = max(self.fstar_max, float(np.abs(acc).max()))

    def smooth(self, k):
        """One Gauss-Seidel iteration on every level-k block (8 colours, frozen halo)."""
        U, F, n = self.U[k], self.F[k], self.n
        h2 = self.fo.h(k) ** 2
        wc = self.wL[1, 1, 1]
        offs = [(a - 1, b - 1, c - 1, w) for (a, b, c), w in np.ndenumerate(self.wL)
                if w != 0.0 and (a, b, c) != (1, 1, 1)]
        for col in range(8):
            cx, cy, cz = col & 1, (col >> 1) & 1, (col >> 2) & 1
            acc = 0.0
            for dz, dy, dx, w in offs:
                acc = acc + w * U[:, 1 + cz + dz:1 + n + dz:2, 1 + cy + dy:1 + n + dy:2,
                                  1 + cx + dx:1 + n + dx:2]
            U[:, 1 + cz:1 + n:2, 1 + cy:1 + n:2, 1 + cx:1 + n:2] = \
                (h2 * F[:, cz::2, cy::2, cx::2] - acc) / wc

    def residual(self, k):
        """r_k = f_k - L_k u_k on every level-k node (Alg. 1)."""
        self.R[k][...] = self.F[k] - self.apply_lhs(k)

    def restrict(self, k):
        """Alg. 1, fine-to-coarse loop body after the residual, from level k to k-1.

        Injection of u, full weighting of r (injection where the stencil
        leaves Omega_k), FAS right-hand side f_{k-1} = r_{k-1} + L u_{k-1} on
        Omega_k, and the stored approximation uhat_{k-1} (whole level).
        """
        fo, n = self.fo, self.n
        h = n // 2
        lvc = fo.levels[k - 1]
        kids = self._children(k - 1)
        covered = np.nonzero(~lvc.is_leaf)[0]
        D, base = self._dense(self.R[k], k, np.nan)
        W = full_weighting()
        for P in covered:
            for o in range(8):
                ox, oy, oz = (o & 1) * h, ((o >> 1) & 1) * h, ((o >> 2) & 1) * h
                self.U[k - 1][P, 1 + oz:1 + oz + h, 1 + oy:1 + oy + h, 1 + ox:1 + ox + h] = \
                    self.U[k][kids[P, o], 1:1 + n:2, 1:1 + n:2, 1:1 + n:2]
            if k == 1 and self.off0 is not None:
                j = int(np.searchsorted(covered, P))
                self.U[0][P, 1:1 + n, 1:1 + n, 1:1 + n] += self.off0[j]
            B = lvc.coords[P]
            lo = 2 * B[::-1] * n - 1 - base            # fine window [2Bn-1, 2Bn+2n-1], (z, y, x)
            win = D[lo[0]:lo[0] + 2 * n + 1, lo[1]:lo[1] + 2 * n + 1, lo[2]:lo[2] + 2 * n + 1]
            fw = np.zeros((n, n, n))
            for (a, b, c), w in np.ndenumerate(W):
                fw += w * win[a:a + 2 * n:2, b:b + 2 * n:2, c:c + 2 * n:2]
            inj = win[1:1 + 2 * n:2, 1:1 + 2 * n:2, 1:1 + 2 * n:2]
            self.F[k - 1][P] = np.where(np.isnan(fw), inj, fw)
        self.ghost_fill(self.U, k - 1, "keep")
        if len(covered):
            self.F[k - 1][covered] += self.apply_lhs(k - 1, covered)
        self.H[k - 1][...] = self.U[k - 1][:, 1:1 + n, 1:1 + n, 1:1 + n]

    def coarse_solve(self):
        """u_0 = solve(u_0, f_0): free-space LGF convolution on level 0 (Sec. 2.2, 3.3)."""
        fo, n = self.fo, self.n
        D, base = self._dense(self.F[0], 0, 0.0, 0, 0)
        u = free_space_solve(D, self.G, fo.h0)
        for b, c in enumerate(fo.levels[0].coords):
            z, y, x = c[2] * n, c[1] * n, c[0] * n
            self.U[0][b] = u[z:z + n + 2, y:y + n + 2, x:x + n + 2]

    def prolong_correct(self, k):
        """u_k += I^k_{k-1} (u_{k-1} - uhat_{k-1}), trilinear (Alg. 1, Sec. 3.1)."""
        n = self.n
        h = n // 2
        E = self.U[k - 1][:, 1:1 + n, 1:1 + n, 1:1 + n] - self.H[k - 1]
        D, base = self._dense(E, k - 1, np.nan)
        T = np.zeros((n, h + 1))
        for i in range(n):
            if i % 2 == 0:
                T[i, i // 2] = 1.0
            else:
                T[i, (i - 1) // 2] = 0.5
                T[i, (i + 1) // 2] = 0.5
        for b, c in enumerate(self.fo.levels[k].coords):
            lo = c[::-1] * h - base
            win = D[lo[0]:lo[0] + h + 1, lo[1]:lo[1] + h + 1, lo[2]:lo[2] + h + 1]
            if np.any(np.isnan(win)):
                raise AssertionError("correction needs a missing coarse node")
            fine = np.einsum("zc,yd,xe,cde->zyx", T, T, T, win)
            self.U[k][b, 1:1 + n, 1:1 + n, 1:1 + n] += fine

    # ------------------------------------------------------------------ Alg. 1
    def vcycle(self):
        L = self.fo.max_level
        for k in range(L, 0, -1):
            for _ in range(self.nu1):
                self.ghost_fill(self.U, k, "keep")
                self.smooth(k)
            self.ghost_fill(self.U, k, "keep")
            self.residual(k)
            self.restrict(k)
        self.coarse_solve()
        for k in range(1, L + 1):
            self.prolong_correct(k)
            for _ in range(self.nu2):
                self.ghost_fill(self.U, k, "keep")
                self.smooth(k)
        self.cycles_done += 1

    def leaf_residual_max(self):
        """max |f* - L u| over leaf nodes of all levels, after ghosting every level."""
        out = 0.0
        for k in range(self.fo.max_level, -1, -1):
            self.ghost_fill(self.U, k, "keep")
            leaf = np.nonzero(self.fo.levels[k].is_leaf)[0]
            if len(leaf):
                r = self.F[k][leaf] - self.apply_lhs(k, leaf)
                out = max(out, float(np.abs(r).max()))
        return out

    def leaf_u(self):
        n = self.n
        return np.stack([self.U[l][b, 1:1 + n, 1:1 + n, 1:1 + n] for l, b in self.fo.leaf_slot])

    def solve(self, f_leaf, tol=1e-10, max_cycles=30, history=None, stop="residual"):
        """Cycles from u = 0 until the stop rule falls under tol.

        stop="residual": max|f* - L u| / max|f*| over leaf nodes (Sec. 3.1).
        stop="cauchy": the increment of the iterates, max|u^n - u^{n+1}| /
        max|u^{n+1}| over leaf nodes (Sec. 3, the criterion the paper uses
        for problems whose residual does not reach zero); u^0 = 0, and a
        zero iterate divides by 1.
        """
        for A in self.U:
            A[...] = 0.0
        self.cycles_done = 0
        self.prepare_rhs(f_leaf)
        scale = self.fstar_max if self.fstar_max > 0 else 1.0
        rel = np.inf
        prev = self.leaf_u()
        for _ in range(max_cycles):
            self.vcycle()
            if stop == "cauchy":
                cur = self.leaf_u()
                top = float(np.abs(cur).max())
                rel = float(np.abs(prev - cur).max()) / (top if top > 0 else 1.0)
                prev = cur
            else:
                rel = self.leaf_residual_max() / scale
            if history is not None:
                history.append(rel)
            if rel < tol:
                break
        return self.leaf_u(), rel
