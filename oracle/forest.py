"""Block forest of the oracle (Sec. 2.1, Sec. 3).

The grid is a forest of cubic blocks of n^3 nodes.  Level k holds every block
of resolution h_k = h0 / 2^k: the leaves of that level and the parents of
finer blocks (the uniform grids Omega_k of Fig. grid_hierarchy; Omega_0
covers the whole domain).  A block at level k with coordinates b holds the
nodes b*n + i, i = 0..n-1 (level-k node indices; coarse node X coincides with
fine node 2X).

Checked on construction (a violation raises ``ValueError``):
* the leaves tile the domain without overlap;
* 2:1 balance across faces, edges and corners (Sec. 2.1): for every block at
  level k >= 1, each of its 26 neighbour positions is covered by a block of
  level k-1;
* blocks touching the unbounded boundary are level-0 leaves (Sec. 3.3);
* n is even and at least 8 (the widest ghost interpolant has 8 points).
"""
import numpy as np

NBR26 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
         if (dx, dy, dz) != (0, 0, 0)]


class Level:
    def __init__(self, k, coords, grid_shape):
        self.k = k
        order = np.lexsort((coords[:, 0], coords[:, 1], coords[:, 2])) if len(coords) else []
        self.coords = np.asarray(coords, np.int64)[order].reshape(-1, 3)   # (x, y, z)
        self.nb = len(self.coords)
        self.grid_shape = grid_shape                   # blocks per axis (x, y, z) at this level
        self.map = -np.ones(grid_shape[::-1], np.int64)   # [z, y, x] -> block index
        for i, c in enumerate(self.coords):
            self.map[c[2], c[1], c[0]] = i
        self.is_leaf = np.zeros(self.nb, bool)

    def find(self, c):
        x, y, z = c
        gx, gy, gz = self.grid_shape
        if not (0 <= x < gx and 0 <= y < gy and 0 <= z < gz):
            return -2
        return int(self.map[z, y, x])


class OracleForest:
    def __init__(self, nb0, n, origin, h0, leaf_level, leaf_ijk):
        self.nb0 = tuple(int(v) for v in nb0)
        self.n = int(n)
        self.origin = np.asarray(origin, float)
        self.h0 = float(h0)
        leaf_level = np.asarray(leaf_level, np.int64)
        leaf_ijk = np.asarray(leaf_ijk, np.int64).reshape(-1, 3)
        if self.n % 2 or self.n < 8:
            raise ValueError("block size must be even and >= 8")
        if len(leaf_level) == 0:
            raise ValueError("no leaves")
        L = int(leaf_level.max())
        self.max_level = L
        # blocks per level: leaves, then parents of finer blocks
        sets = [set() for _ in range(L + 1)]
        for lev, c in zip(leaf_level, leaf_ijk):
            key = tuple(int(v) for v in c)
            if key in sets[lev]:
                raise ValueError("duplicate leaf")
            sets[lev].add(key)
        leafsets = [set(s) for s in sets]
        for k in range(L, 0, -1):
            for c in sets[k]:
                sets[k - 1].add((c[0] >> 1, c[1] >> 1, c[2] >> 1))
        self.levels = []
        for k in range(L + 1):
            gs = tuple(v << k for v in self.nb0)
            coords = np.array(sorted(sets[k]), np.int64).reshape(-1, 3)
            for c in coords:
                if not all(0 <= c[a] < gs[a] for a in range(3)):
                    raise ValueError("block outside the domain")
            lv = Level(k, coords, gs)
            for i, c in enumerate(lv.coords):
                lv.is_leaf[i] = tuple(int(v) for v in c) in leafsets[k]
            self.levels.append(lv)
        # tiling: a leaf has no children; a non-leaf has all 8 children
        for k in range(L + 1):
            lv = self.levels[k]
            for i, c in enumerate(lv.coords):
                kids = [(2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + ((o >> 2) & 1))
                        for o in range(8)]
                if k == L:
                    found = [False] * 8
                else:
                    found = [self.levels[k + 1].find(q) >= 0 for q in kids]
                if lv.is_leaf[i] and any(found):
                    raise ValueError("overlapping leaves")
                if not lv.is_leaf[i] and not all(found):
                    raise ValueError("leaves do not tile the domain")
        if self.levels[0].nb != int(np.prod(self.nb0)):
            raise ValueError("leaves do not tile the domain")
        # unbounded boundary blocks stay at level 0 (Sec. 3.3)
        for i, c in enumerate(self.levels[0].coords):
            on_bnd = any(c[a] == 0 or c[a] == self.nb0[a] - 1 for a in range(3))
            if on_bnd and not self.levels[0].is_leaf[i]:
                raise ValueError("a block touching the unbounded boundary is refined")
        # 2:1 balance with faces, edges and corners
        for k in range(1, L + 1):
            for c in self.levels[k].coords:
                for d in NBR26:
                    q = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
                    if self.levels[k - 1].find((q[0] >> 1, q[1] >> 1, q[2] >> 1)) < 0:
                        raise ValueError("2:1 balance violated")
        # input leaf i -> (level, block index)
        self.leaf_slot = np.array([(int(l), self.levels[int(l)].find(tuple(int(v) for v in c)))
                                   for l, c in zip(leaf_level, leaf_ijk)], np.int64).reshape(-1, 2)

    def h(self, k):
        return self.h0 / (1 << k)

    @property
    def n0(self):
        """Level-0 nodes per axis (x, y, z)."""
        return tuple(v * self.n for v in self.nb0)

    @classmethod
    def from_desc(cls, desc):
        return cls(desc.nb0, desc.n, desc.origin, desc.h0, desc.leaf_level, desc.leaf_ijk)
