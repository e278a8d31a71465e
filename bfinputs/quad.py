"""Container, sizes and seeded random factors of a 2D (quadtree) butterfly
factorization (no butterfly arithmetic here).

The 2D factorization has the same form as the 1D one,
K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*, on quadtrees of
even depth L over an n x n grid of points (N = n^2) and of frequencies: a
node has four children, a leaf holds n0 = 4^e points, h = L/2 and there are
m = 4^h middle-level nodes.  A node of level l holds N / 4^l points, which
bounds the rank of every block with that many rows, so the rank of level l
is r_l = min(r, N / 4^l) for l = h..L (at the middle level and above it is
r; it drops over the last levels of a small-leaf tree).

Canonical layout (row-major numpy arrays, block index first):

* ``VL``: (4^L, n0, r_L); block b is V^L_{b,0}, the basis of column leaf b.
* ``H[l - h]``, l = h..L-1: (4^L, r_{l+1}, 4 r_l); block j''*4^{L-l-1} + i'
  is H^l_{j'',i'} (j'' a node of the column tree at level l+1, i' of the
  row tree at level L-l-1).
* ``S``: (m, m, r_h) real; S[i, j] is the diagonal of S^h_{i,j}.
* ``G[l - h]``: (4^L, r_{l+1}, 4 r_l); block i''*4^{L-l-1} + j' is G^l_{i'',j'}.
* ``UL``: (4^L, n0, r_L); block a is U^L_{a,0}.

Points are numbered in the quadtree (Morton) order, so a node's points are
contiguous and its four children are its four consecutive quarters.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .workloads import _cn, _rng


def quad_sizes(L: int, n0: int, r: int) -> dict:
    """N, n (grid side), h, m, the per-level ranks r_l (l = h..L) and the
    number of blocks per level (4^L)."""
    if L < 0 or L % 2:
        raise ValueError("the quadtree depth L must be even and >= 0")
    e = 0
    while (1 << (2 * e)) < n0:
        e += 1
    if (1 << (2 * e)) != n0:
        raise ValueError("the leaf size n0 must be a power of 4")
    h = L // 2
    N = n0 << (2 * L)
    ranks = {lv: min(r, N >> (2 * lv)) for lv in range(h, L + 1)}
    return {"N": N, "n": 1 << (L + e), "L": L, "h": h, "m": 1 << (2 * h), "n0": n0, "r": r,
            "ranks": ranks, "nblocks": 1 << (2 * L)}


@dataclass
class QuadFactors:
    L: int
    n0: int
    r: int
    VL: np.ndarray
    H: list
    S: np.ndarray
    G: list
    UL: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def sizes(self) -> dict:
        return quad_sizes(self.L, self.n0, self.r)

    @property
    def N(self) -> int:
        return self.n0 << (2 * self.L)

    @property
    def h(self) -> int:
        return self.L // 2

    @property
    def m(self) -> int:
        return 1 << (2 * self.h)

    def rank(self, level: int) -> int:
        return self.sizes["ranks"][level]

    def validate(self) -> "QuadFactors":
        s = self.sizes
        nb, rk, h, m = s["nblocks"], s["ranks"], s["h"], s["m"]
        if self.VL.shape != (nb, self.n0, rk[self.L]) or self.UL.shape != (nb, self.n0, rk[self.L]):
            raise ValueError("leaf factors must be (4^L, n0, r_L)")
        if len(self.H) != self.L - h or len(self.G) != self.L - h:
            raise ValueError("H and G must hold L/2 levels each")
        for t in range(self.L - h):
            lv = h + t
            for A in (self.H[t], self.G[t]):
                if A.shape != (nb, rk[lv + 1], 4 * rk[lv]):
                    raise ValueError(f"level {lv} transfer blocks must be (4^L, r_{lv + 1}, 4 r_{lv})")
        if self.S.shape != (m, m, rk[h]):
            raise ValueError("S must be (m, m, r_h)")
        return self

    def astype(self, cdtype) -> "QuadFactors":
        cdtype = np.dtype(cdtype)
        rdtype = np.float32 if cdtype == np.complex64 else np.float64
        return QuadFactors(self.L, self.n0, self.r, np.ascontiguousarray(self.VL, dtype=cdtype),
                           [np.ascontiguousarray(a, dtype=cdtype) for a in self.H],
                           np.ascontiguousarray(self.S, dtype=rdtype),
                           [np.ascontiguousarray(a, dtype=cdtype) for a in self.G],
                           np.ascontiguousarray(self.UL, dtype=cdtype), dict(self.meta))

    def nentries(self) -> int:
        """Complex factor entries (S counted as entries too)."""
        return int(self.VL.size + self.UL.size + self.S.size + sum(a.size for a in self.H)
                   + sum(a.size for a in self.G))


def synthetic_quad_factors(L: int, n0: int, r: int, seed: int = 0, dtype=np.complex64) -> QuadFactors:
    """Seeded random factors with the block shapes of a 2D factorization:
    i.i.d. complex normal entries with variances 1/n0 (V^L), 1/(4 r_l) (H, G)
    and 1/r_L (U^L), S uniform on [0.5, 1.5], so every factor keeps the
    expected squared norm of the vector it is applied to."""
    s = quad_sizes(L, n0, r)
    nb, h, m, rk = s["nblocks"], s["h"], s["m"], s["ranks"]
    VL = _cn(seed, (11,), (nb, n0, rk[L]), 1.0 / np.sqrt(n0), dtype)
    UL = _cn(seed, (12,), (nb, n0, rk[L]), 1.0 / np.sqrt(rk[L]), dtype)
    H = [_cn(seed, (13, t), (nb, rk[h + t + 1], 4 * rk[h + t]), 1.0 / np.sqrt(4 * rk[h + t]), dtype)
         for t in range(L - h)]
    G = [_cn(seed, (14, t), (nb, rk[h + t + 1], 4 * rk[h + t]), 1.0 / np.sqrt(4 * rk[h + t]), dtype)
         for t in range(L - h)]
    rdt = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    S = _rng(seed, 15).uniform(0.5, 1.5, size=(m, m, rk[h])).astype(rdt)
    return QuadFactors(L, n0, r, VL, H, S, G, UL, meta={"source": "synthetic", "seed": seed}).validate()


# The 2D workload: a 2D FIO (phase x.xi + sqrt(c1(x)^2 xi1^2 + c2(x)^2 xi2^2))
# on a 256 x 256 grid, quadtrees of depth 8 with one point per leaf, rank 24,
# 128 RHS.
QUAD_CONFIGS = {
    "fio2d_n65536_r24": {"L": 8, "n0": 1, "r": 24, "nrhs": 128},
    # a small case of the same level shapes (96 x 96 groups) for profiling: 128 x 128
    # grid, depth 6, four points per leaf, 256 vectors (level vectors of ~200 MB)
    "fio2d_n16384_r24": {"L": 6, "n0": 4, "r": 24, "nrhs": 256},
}
