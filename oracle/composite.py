"""Independent route to the converged composite solution (no multigrid).

At convergence of Alg. 1 every leaf node of level k >= 1 satisfies
L_k u = f* with its ghosts from the ghosting rules, and the uniform level 0
is the free-space field u_0 = h0^2 G * f_0 whose source f_0 is f* on level-0
leaves and unknown (s) on level-0 nodes covered by level 1, where u_0 must
equal the injection of u_1.  Covered nodes of levels >= 1 hold the injection
of the finer level.  This module writes that square linear system

    unknowns  x = (u at leaf nodes of levels >= 1, s at covered level-0 nodes)
    equations f* - L_k u = 0 at those leaves,
              (h0^2 G * f_0)(X) - u_1(2X) = 0 at covered level-0 nodes,

and solves it with restarted GMRES, reusing only the oracle's stencils,
ghosting and LGF convolution (not its smoother or grid transfers), so the
multigrid fixed point can be checked against it.
"""
import numpy as np
from scipy.sparse.linalg import LinearOperator, gmres

from .lgf import free_space_solve


class CompositeSystem:
    def __init__(self, solver, f_leaf):
        self.s = solver
        fo = solver.fo
        self.fo = fo
        solver.prepare_rhs(f_leaf)
        n = fo.n
        self.n = n
        self.leaf_sel = [np.nonzero(lv.is_leaf)[0] for lv in fo.levels]
        self.cov0 = np.nonzero(~fo.levels[0].is_leaf)[0]
        self.sizes = [len(self.leaf_sel[k]) * n ** 3 for k in range(1, fo.max_level + 1)]
        self.n_s = len(self.cov0) * n ** 3
        self.size = sum(self.sizes) + self.n_s

    def _unpack(self, x):
        s, n = self.s, self.n
        off = 0
        for k in range(1, self.fo.max_level + 1):
            m = self.sizes[k - 1]
            s.U[k][self.leaf_sel[k], 1:1 + n, 1:1 + n, 1:1 + n] = x[off:off + m].reshape(-1, n, n, n)
            off += m
        return x[off:].reshape(-1, n, n, n)

    def residual(self, x):
        s, fo, n = self.s, self.fo, self.n
        for A in s.U:
            A[...] = 0.0
        sv = self._unpack(x)
        # covered nodes of levels >= 1: injection of the finer level, finest first
        for k in range(fo.max_level, 1, -1):
            s.inject_into_parent(s.U, k)
        # level 0: free-space field of f0
        F0 = s.F[0].copy()
        F0[self.cov0] = sv
        D, _ = s._dense(F0, 0, 0.0, 0, 0)
        u0 = free_space_solve(D, s.G, fo.h0)
        for b, c in enumerate(fo.levels[0].coords):
            z, y, x0 = c[2] * n, c[1] * n, c[0] * n
            s.U[0][b] = u0[z:z + n + 2, y:y + n + 2, x0:x0 + n + 2]
        conv_cov = s.U[0][self.cov0, 1:1 + n, 1:1 + n, 1:1 + n].copy()
        out = []
        for k in range(fo.max_level, 0, -1):
            s.ghost_fill(s.U, k, "keep")      # also injects level k into covered level k-1
        for k in range(1, fo.max_level + 1):
            leaf = self.leaf_sel[k]
            r = s.F[k][leaf] - s.apply_lhs(k, leaf)
            out.append(r.reshape(-1))
        inj = s.U[0][self.cov0, 1:1 + n, 1:1 + n, 1:1 + n]   # = injection of u_1 after ghosting level 1
        out.append(((conv_cov - inj) / fo.h0 ** 2).reshape(-1))
        return np.concatenate(out)

    def solve(self, rtol=1e-13, restart=300, maxiter=40):
        r0 = self.residual(np.zeros(self.size))
        A = LinearOperator((self.size, self.size), matvec=lambda v: r0 - self.residual(v), dtype=float)
        x, info = gmres(A, r0, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
        self.info = info
        self.final_residual = float(np.abs(self.residual(x)).max())
        return x

    def leaf_values(self, x):
        """Solution at every input leaf, in input order (level-0 leaves from the convolution)."""
        s, fo, n = self.s, self.fo, self.n
        self.residual(x)
        return np.stack([s.U[l][b, 1:1 + n, 1:1 + n, 1:1 + n] for l, b in fo.leaf_slot])
