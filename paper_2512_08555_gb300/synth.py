"""Seeded synthetic inputs: block forests and source fields.

This module holds no arithmetic of the solver. It only builds forest
descriptions (which blocks exist at which level) and samples analytic source
functions at node positions. Both the CUDA path and the CPU oracle receive
the arrays it produces; neither is imported by the other.

Geometry conventions (shared by every consumer of these arrays):

* Level 0 is a grid of ``nb0 = (nbx, nby, nbz)`` cubic blocks of ``n`` nodes
  per edge, node spacing ``h0``, lower corner ``origin``.
* A block at level ``k`` with integer block coordinates ``(bx, by, bz)``
  holds the nodes ``origin + (b * n + i) * h_k`` for ``i = 0 .. n-1`` on each
  axis, ``h_k = h0 / 2**k`` (vertex-centred, half-open).  Coarse node ``X``
  coincides with fine node ``2X``, which is what injection needs
  (Section 3.1 of the paper: restriction of u by injection).
* Field arrays of one block are ``[z][y][x]`` with x fastest.
* A forest is given by its leaves; parents are implied.

Random draws use ``numpy.random.default_rng(seed)`` (PCG64) in the order
documented on each generator.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Forest", "uniform_forest", "adaptive_forest", "sample_leaves",
    "gaussian_blobs", "c4_bumps", "vortex_ring", "gaussian_weight",
    "config1", "config2", "config3", "oracle_sample_forest", "batched_scalar_problem",
]


@dataclass
class Forest:
    """Leaf description of a 2:1 balanced block forest."""
    nb0: tuple
    n: int
    origin: np.ndarray
    h0: float
    leaf_level: np.ndarray          # int32 [n_leaves]
    leaf_ijk: np.ndarray            # int32 [n_leaves, 3] block coords (x, y, z) at its level
    meta: dict = field(default_factory=dict)

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_level.shape[0])

    @property
    def max_level(self) -> int:
        return int(self.leaf_level.max()) if self.n_leaves else 0

    @property
    def leaf_nodes(self) -> int:
        return self.n_leaves * self.n ** 3

    def leaf_positions(self, i: int):
        """Node coordinates (x, y, z 1-D arrays) of leaf ``i``."""
        lev = int(self.leaf_level[i])
        h = self.h0 / (1 << lev)
        out = []
        for a in range(3):
            g = int(self.leaf_ijk[i, a]) * self.n + np.arange(self.n)
            out.append(self.origin[a] + g * h)
        return out


def uniform_forest(nb0, n, origin, h0) -> Forest:
    """All level-0 blocks are leaves (single uniform level)."""
    nbx, nby, nbz = nb0
    ijk = np.array([(x, y, z) for z in range(nbz) for y in range(nby) for x in range(nbx)],
                   dtype=np.int32).reshape(-1, 3)
    return Forest(tuple(nb0), int(n), np.asarray(origin, float), float(h0),
                  np.zeros(len(ijk), np.int32), ijk)


def _nbrs26():
    return [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dx, dy, dz) != (0, 0, 0)]


def adaptive_forest(nb0, n, origin, h0, max_level, want_refine, keep_boundary=True) -> Forest:
    """Refine blocks where ``want_refine(level, coords_array) -> bool array``.

    Constraints kept by construction:
    * level-0 blocks touching the domain boundary are never refined
      (unbounded-boundary blocks stay at the coarsest level, Section 3.3);
    * 2:1 balance across faces, edges and corners: every block at level
      k >= 1 has all 26 neighbour positions covered by blocks of level k-1
      or finer.  Balance is reached by refining coarse neighbours where that
      is allowed and by withdrawing the refinement that needs a forbidden one.
    """
    nb0 = tuple(int(v) for v in nb0)
    D = _nbrs26()
    ref = [set() for _ in range(max_level + 1)]      # refined blocks per level
    forb = [set() for _ in range(max_level + 1)]

    def in_dom(k, c):
        return all(0 <= c[a] < nb0[a] << k for a in range(3))

    def boundary0(c):
        return any(c[a] == 0 or c[a] == nb0[a] - 1 for a in range(3))

    # 1. criterion-driven refinement, top down
    exists = [{(x, y, z) for z in range(nb0[2]) for y in range(nb0[1]) for x in range(nb0[0])}]
    for k in range(max_level):
        cand = sorted(exists[k])
        if not cand:
            exists.append(set())
            continue
        arr = np.array(cand, dtype=np.int64)
        want = np.asarray(want_refine(k, arr), bool)
        for c, w in zip(cand, want):
            if not w:
                continue
            if k == 0 and keep_boundary and boundary0(c):
                forb[0].add(c)
                continue
            ref[k].add(c)
        nxt = set()
        for c in ref[k]:
            for o in range(8):
                nxt.add((2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + ((o >> 2) & 1)))
        exists.append(nxt)
    if keep_boundary:
        for z in range(nb0[2]):
            for y in range(nb0[1]):
                for x in range(nb0[0]):
                    if boundary0((x, y, z)):
                        forb[0].add((x, y, z))

    # 2. balance: add coarse neighbours (ripple) / withdraw what cannot be balanced
    changed = True
    while changed:
        changed = False
        for k in range(max_level - 1, 0, -1):
            for c in list(ref[k]):
                for d in D:
                    nc = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
                    if not in_dom(k, nc):
                        continue
                    p = (nc[0] >> 1, nc[1] >> 1, nc[2] >> 1)
                    if p not in ref[k - 1] and p not in forb[k - 1]:
                        ref[k - 1].add(p)
                        changed = True
        for k in range(1, max_level):
            for c in list(ref[k]):
                p = (c[0] >> 1, c[1] >> 1, c[2] >> 1)
                ok = p in ref[k - 1]
                if ok:
                    for d in D:
                        nc = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
                        if not in_dom(k, nc):
                            ok = False
                            break
                        if (nc[0] >> 1, nc[1] >> 1, nc[2] >> 1) not in ref[k - 1]:
                            ok = False
                            break
                if not ok:
                    ref[k].discard(c)
                    forb[k].add(c)
                    changed = True
        for c in list(ref[0]):
            if c in forb[0]:
                ref[0].discard(c)
                changed = True

    # 3. leaves = existing blocks that are not refined
    leaves = []
    cur = {(x, y, z) for z in range(nb0[2]) for y in range(nb0[1]) for x in range(nb0[0])}
    for k in range(max_level + 1):
        nxt = set()
        for c in sorted(cur, key=lambda t: (t[2], t[1], t[0])):
            if k < max_level and c in ref[k]:
                for o in range(8):
                    nxt.add((2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + ((o >> 2) & 1)))
            else:
                leaves.append((k, c))
        cur = nxt
    lev = np.array([l for l, _ in leaves], np.int32)
    ijk = np.array([c for _, c in leaves], np.int32).reshape(-1, 3)
    return Forest(nb0, int(n), np.asarray(origin, float), float(h0), lev, ijk)


def sample_leaves(forest: Forest, fn) -> np.ndarray:
    """Evaluate ``fn(x, y, z)`` (broadcasting) at every leaf node.

    Returns float64 ``[n_leaves, n, n, n]`` in ``[z][y][x]`` order.
    """
    n = forest.n
    out = np.empty((forest.n_leaves, n, n, n))
    for lev in np.unique(forest.leaf_level):
        sel = np.nonzero(forest.leaf_level == lev)[0]
        h = forest.h0 / (1 << int(lev))
        i = np.arange(n)
        X = forest.origin[0] + (forest.leaf_ijk[sel, 0][:, None] * n + i) * h
        Y = forest.origin[1] + (forest.leaf_ijk[sel, 1][:, None] * n + i) * h
        Z = forest.origin[2] + (forest.leaf_ijk[sel, 2][:, None] * n + i) * h
        out[sel] = fn(X[:, None, None, :], Y[:, None, :, None], Z[:, :, None, None])
    return out


# ----------------------------------------------------------------------------
# analytic sources

class gaussian_blobs:
    """Sum of Gaussian blobs ``A exp(-|x-c|^2 / (2 sigma^2))``.

    Draw order from ``default_rng(seed)``: sigma[k] ~ U[s_lo, s_hi] (k blobs),
    centres ~ U[c_lo, c_hi]^3 (k x 3), amplitudes ~ N(0, 1) (k).
    """

    def __init__(self, seed=0, k=3, s_lo=0.05, s_hi=0.1, c_lo=0.3, c_hi=0.7):
        rng = np.random.default_rng(seed)
        self.sigma = rng.uniform(s_lo, s_hi, k)
        self.centre = rng.uniform(c_lo, c_hi, (k, 3))
        self.amp = rng.normal(0.0, 1.0, k)

    def __call__(self, x, y, z):
        out = 0.0
        for s, c, a in zip(self.sigma, self.centre, self.amp):
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            out = out + a * np.exp(-r2 / (2 * s * s))
        return out


class c4_bumps:
    """Sum of compact bumps ``A (1 - r^2/R^2)^5`` for r < R, else 0.

    Draw order from ``default_rng(seed)``: R ~ U[0.1, 0.3] (k), centres
    ~ U[-0.5+R, 0.5-R]^3 per bump (k x 3, so each support lies in
    [-0.5, 0.5]^3), amplitudes ~ N(0, 1) (k).
    """

    def __init__(self, seed=0, k=8, r_lo=0.1, r_hi=0.3, box=0.5):
        rng = np.random.default_rng(seed)
        self.radius = rng.uniform(r_lo, r_hi, k)
        lo = -box + self.radius
        hi = box - self.radius
        self.centre = rng.uniform(lo[:, None], hi[:, None], (k, 3))
        self.amp = rng.normal(0.0, 1.0, k)

    def __call__(self, x, y, z):
        out = 0.0
        for R, c, a in zip(self.radius, self.centre, self.amp):
            r2 = ((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (R * R)
            out = out + a * np.where(r2 < 1.0, np.clip(1.0 - r2, 0.0, None) ** 5, 0.0)
        return out

    def block_may_touch(self, lo, hi):
        """Bool per box [lo, hi] (arrays [m, 3]) whether any support intersects it."""
        hit = np.zeros(lo.shape[0], bool)
        for R, c in zip(self.radius, self.centre):
            d2 = np.zeros(lo.shape[0])
            for a in range(3):
                q = np.clip(c[a], lo[:, a], hi[:, a]) - c[a]
                d2 += q * q
            hit |= d2 < R * R
        return hit

    @property
    def peak(self):
        return float(np.max(np.abs(self.amp)))


class vortex_ring:
    """Gaussian-core vortex ring vorticity, three components.

    omega = Gamma / (2 pi sigma^2) exp(-rho^2 / (2 sigma^2)) e_phi with rho the
    distance to the ring (radius ``R0``) and e_phi the azimuthal unit vector
    about the ring normal.  The normal is e_z tilted by theta ~ U[0, pi/6]
    about the horizontal axis (cos a, sin a, 0), a ~ U[0, 2 pi).
    Draw order: theta, a.
    """

    def __init__(self, seed=0, R0=0.5, sigma=0.05, gamma=1.0, centre=(0.0, 0.0, 0.0)):
        rng = np.random.default_rng(seed)
        self.theta = rng.uniform(0.0, np.pi / 6)
        self.alpha = rng.uniform(0.0, 2 * np.pi)
        self.R0, self.sigma, self.gamma = R0, sigma, gamma
        self.centre = np.asarray(centre, float)
        ax = np.array([np.cos(self.alpha), np.sin(self.alpha), 0.0])
        # Rodrigues rotation of e_z about ax by theta
        ez = np.array([0.0, 0.0, 1.0])
        c, s = np.cos(self.theta), np.sin(self.theta)
        self.normal = ez * c + np.cross(ax, ez) * s + ax * np.dot(ax, ez) * (1 - c)

    def component(self, comp):
        def f(x, y, z):
            p = [x - self.centre[0], y - self.centre[1], z - self.centre[2]]
            nrm = self.normal
            along = p[0] * nrm[0] + p[1] * nrm[1] + p[2] * nrm[2]
            q = [p[a] - along * nrm[a] for a in range(3)]      # in-plane part
            qr = np.sqrt(q[0] ** 2 + q[1] ** 2 + q[2] ** 2)
            rho2 = (qr - self.R0) ** 2 + along ** 2
            mag = self.gamma / (2 * np.pi * self.sigma ** 2) * np.exp(-rho2 / (2 * self.sigma ** 2))
            # e_phi = normal x q / |q|
            cr = [nrm[1] * q[2] - nrm[2] * q[1], nrm[2] * q[0] - nrm[0] * q[2], nrm[0] * q[1] - nrm[1] * q[0]]
            safe = np.where(qr > 0, qr, 1.0)
            return np.where(qr > 0, mag * cr[comp] / safe, 0.0)
        return f


class gaussian_weight(gaussian_blobs):
    """Loss weight w = exp(-|x - c_w|^2 / (2 sigma_w^2)), one blob of unit amplitude.

    Draw order: sigma_w ~ U[0.05, 0.1], c_w ~ U[0.3, 0.7]^3.
    """

    def __init__(self, seed=0):
        rng = np.random.default_rng(seed)
        self.sigma = rng.uniform(0.05, 0.1, 1)
        self.centre = rng.uniform(0.3, 0.7, (1, 3))
        self.amp = np.ones(1)


# ----------------------------------------------------------------------------
# the workloads

def config1(seed=0, n0=32, n=16):
    """Single uniform level on [0,1)^3, ``n0`` nodes per axis, h = 1/n0; 3 Gaussian blobs."""
    nb = n0 // n
    forest = uniform_forest((nb, nb, nb), n, (0.0, 0.0, 0.0), 1.0 / n0)
    src = gaussian_blobs(seed)
    forest.meta.update(workload=f"uniform {n0}^3 on [0,1)^3, 3 Gaussian blobs", seed=seed)
    return forest, src


def _bump_forest(seed, max_level, n=16, nb=5, half=1.0, thresh=1e-3, k=8):
    src = c4_bumps(seed, k=k)
    h0 = 2 * half / (nb * n)
    origin = (-half, -half, -half)
    fmax = src.peak

    def want(level, coords):
        h = h0 / (1 << level)
        lo = origin[0] + coords * n * h
        hi = lo + (n - 1) * h
        touch = src.block_may_touch(lo.astype(float), hi.astype(float))
        out = np.zeros(len(coords), bool)
        idx = np.nonzero(touch)[0]
        i = np.arange(n)
        for s in range(0, len(idx), 64):
            sel = idx[s:s + 64]
            X = origin[0] + (coords[sel, 0][:, None] * n + i) * h
            Y = origin[1] + (coords[sel, 1][:, None] * n + i) * h
            Z = origin[2] + (coords[sel, 2][:, None] * n + i) * h
            v = src(X[:, None, None, :], Y[:, None, :, None], Z[:, :, None, None])
            out[sel] = np.abs(v).reshape(len(sel), -1).max(axis=1) > thresh * fmax
        return out

    forest = adaptive_forest((nb, nb, nb), n, origin, h0, max_level, want)
    return forest, src


def config2(seed=0, max_level=2, n=16, nb=5):
    """Adaptive forest on [-1,1)^3, nb^3 level-0 blocks of n^3 (5^3 of 16^3: h0 = 1/40), levels 0..max_level;
    8 C4 bumps.

    A block is refined where max |f| over its nodes exceeds 1e-3 times the
    largest bump amplitude, subject to the boundary and 2:1 rules of
    :func:`adaptive_forest`.  Seed 0 at levels 0..2: 2,805,760 leaf nodes.
    """
    forest, src = _bump_forest(seed, max_level, n=n, nb=nb)
    forest.meta.update(workload=f"adaptive [-1,1)^3, {nb}^3 level-0 blocks of {n}^3, levels 0..{max_level}, "
                                f"8 C4 bumps", seed=seed)
    return forest, src


def config3(seed=0, max_level=4, n=16, nb=6):
    """The config-2 generator at 5 levels (0..4) on 6^3 level-0 blocks (h0 = 1/48).

    Seed 0 gives 97,853,440 leaf nodes (23,890 leaves); 5^3 level-0 blocks
    would give 29,528,064 and 7^3 174,325,760.
    """
    return config2(seed, max_level=max_level, n=n, nb=nb)


def oracle_sample_forest(seed=0):
    """The config-2 generator at its smallest block size: 4^3 level-0 blocks of 8^3 (h0 = 1/16), levels 0..2.

    Seed 0 gives 90,112 leaf nodes (176 leaves: 56 per level at 0 and 1, 64 at 2),
    small enough for a full oracle solve in seconds.
    """
    return config2(seed, max_level=2, n=8, nb=4)


def vortex_forest(seed=0, max_level=3, n=16, nb=6, half=1.5, thresh=1e-3):
    """Forest of the vortex-ring problem: [-1.5,1.5)^3, 6^3 level-0 blocks of 16^3, levels 0..3.

    A block is refined where max |omega| over its nodes exceeds 1e-3 times the
    core peak Gamma / (2 pi sigma^2).  With 4^3 level-0 blocks the boundary
    rule (boundary blocks stay level-0 leaves) and 2:1 balance stop the
    refinement at level 2; 6^3 blocks (h0 = 1/32) reach level 3.
    """
    ring = vortex_ring(seed)
    h0 = 2 * half / (nb * n)
    origin = (-half, -half, -half)
    peak = ring.gamma / (2 * np.pi * ring.sigma ** 2)

    def mag(x, y, z):
        p = [x - ring.centre[0], y - ring.centre[1], z - ring.centre[2]]
        nrm = ring.normal
        along = p[0] * nrm[0] + p[1] * nrm[1] + p[2] * nrm[2]
        q2 = (p[0] - along * nrm[0]) ** 2 + (p[1] - along * nrm[1]) ** 2 + (p[2] - along * nrm[2]) ** 2
        rho2 = (np.sqrt(q2) - ring.R0) ** 2 + along ** 2
        return peak * np.exp(-rho2 / (2 * ring.sigma ** 2))

    def want(level, coords):
        h = h0 / (1 << level)
        i = np.arange(n)
        out = np.zeros(len(coords), bool)
        for s in range(0, len(coords), 64):
            sel = slice(s, s + 64)
            X = origin[0] + (coords[sel, 0][:, None] * n + i) * h
            Y = origin[1] + (coords[sel, 1][:, None] * n + i) * h
            Z = origin[2] + (coords[sel, 2][:, None] * n + i) * h
            v = mag(X[:, None, None, :], Y[:, None, :, None], Z[:, :, None, None])
            out[sel] = v.reshape(v.shape[0], -1).max(axis=1) > thresh * peak
        return out

    forest = adaptive_forest((nb, nb, nb), n, origin, h0, max_level, want)
    forest.meta.update(workload=f"vortex ring on [-1.5,1.5)^3, levels 0..{max_level}, {n}^3 blocks", seed=seed)
    return forest, ring


def batched_scalar_problem(i, seed=0):
    """Problem ``i`` of the batched set: levels = 2 + (i mod 4), n = {12,14,16,18,20}[i mod 5]."""
    n = (12, 14, 16, 18, 20)[i % 5]
    max_level = 1 + (i % 4)
    return _bump_forest(seed + 1000 + i, max_level, n=n)


def config4(seed=0, n_scalar=16, scale_levels=0):
    """The batched workload: the vortex ring (3 components) plus ``n_scalar`` scalar problems.

    Returns ``[(forest, ncomp, [source per component])]``; the ring's sources
    are -omega_x, -omega_y, -omega_z (so that the solutions are the vector
    potential components).  ``scale_levels`` lowers every problem's finest
    level by that many (a smaller instance of the same mix).
    """
    out = []
    ring_forest, ring = vortex_forest(seed, max_level=max(0, 3 - scale_levels))

    def neg(fn):
        return lambda x, y, z: -fn(x, y, z)
    out.append((ring_forest, 3, [neg(ring.component(c)) for c in range(3)]))
    for i in range(n_scalar):
        n = (12, 14, 16, 18, 20)[i % 5]
        ml = max(0, 1 + (i % 4) - scale_levels)
        forest, src = _bump_forest(seed + 1000 + i, ml, n=n)
        out.append((forest, 1, [src]))
    return out


def batched_rhs(problems):
    """Concatenated right-hand side of :func:`config4` in the caller layout [forest][component][leaf][n^3]."""
    parts = []
    for forest, ncomp, srcs in problems:
        for c in range(ncomp):
            parts.append(sample_leaves(forest, srcs[c]).reshape(-1))
    return np.concatenate(parts)
