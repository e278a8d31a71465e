"""Container for the factors of a butterfly factorization, in canonical layout.

The factorization is K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*
(Eq. Kfactors of the paper) for an N x N matrix with trees of even depth L,
h = L/2, m = 2^h middle-level nodes, leaf size n0 = N / 2^L and rank r.
Canonical layout (row-major numpy arrays, block index first):

* ``VL``: (2^L, n0, r) complex; block b is V^L_{b,0}, the leaf basis of
  column leaf b (rows: the n0 points of B^L_b).
* ``H[l - h]`` for l = h..L-1: (2^L, r, 2r) complex; block j'*2^{L-l-1} + i
  is H^l_{j',i} (j' < 2^{l+1} a node of T_Omega at level l+1, i < 2^{L-l-1}).
* ``S``: (m, m, r) real; S[i, j] is the diagonal of S^h_{i,j}, the weight of
  the middle-level block K^h_{i,j} (row node i, column node j).
* ``G[l - h]``: (2^L, r, 2r) complex; block i'*2^{L-l-1} + j is G^l_{i',j}.
* ``UL``: (2^L, n0, r) complex; block a is U^L_{a,0}.

This module only stores and validates arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def tree_sizes(L: int, n0: int, r: int) -> dict:
    """N, h, m and R = 2^L r (the length of every intermediate vector)."""
    if L < 0 or L % 2:
        raise ValueError("the tree depth L must be even and >= 0")
    h = L // 2
    return {"N": n0 << L, "L": L, "h": h, "m": 1 << h, "n0": n0, "r": r,
            "R": (1 << L) * r, "nblocks": 1 << L}


@dataclass
class ButterflyFactors:
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
    def N(self) -> int:
        return self.n0 << self.L

    @property
    def h(self) -> int:
        return self.L // 2

    @property
    def m(self) -> int:
        return 1 << self.h

    def validate(self) -> "ButterflyFactors":
        s = tree_sizes(self.L, self.n0, self.r)
        nb, n0, r, m, h = s["nblocks"], self.n0, self.r, s["m"], s["h"]
        if self.VL.shape != (nb, n0, r) or self.UL.shape != (nb, n0, r):
            raise ValueError("leaf factors must be (2^L, n0, r)")
        if len(self.H) != h or len(self.G) != h:
            raise ValueError("H and G must hold L/2 levels each")
        for A in list(self.H) + list(self.G):
            if A.shape != (nb, r, 2 * r):
                raise ValueError("H/G levels must be (2^L, r, 2r)")
        if self.S.shape != (m, m, r):
            raise ValueError("S must be (m, m, r)")
        return self

    def astype(self, cdtype) -> "ButterflyFactors":
        """Copy with complex arrays cast to ``cdtype`` (S to the matching real type)."""
        cdtype = np.dtype(cdtype)
        rdtype = np.float32 if cdtype == np.complex64 else np.float64
        return ButterflyFactors(
            self.L, self.n0, self.r,
            np.ascontiguousarray(self.VL, dtype=cdtype),
            [np.ascontiguousarray(a, dtype=cdtype) for a in self.H],
            np.ascontiguousarray(self.S, dtype=rdtype),
            [np.ascontiguousarray(a, dtype=cdtype) for a in self.G],
            np.ascontiguousarray(self.UL, dtype=cdtype),
            dict(self.meta))

    def nbytes(self) -> int:
        return int(self.VL.nbytes + self.UL.nbytes + self.S.nbytes
                   + sum(a.nbytes for a in self.H) + sum(a.nbytes for a in self.G))

    def save(self, path: str) -> None:
        arrs = {"VL": self.VL, "UL": self.UL, "S": self.S,
                "dims": np.array([self.L, self.n0, self.r])}
        for t, a in enumerate(self.H):
            arrs[f"H{t}"] = a
        for t, a in enumerate(self.G):
            arrs[f"G{t}"] = a
        np.savez(path, **arrs)

    @staticmethod
    def load(path: str) -> "ButterflyFactors":
        z = np.load(path)
        L, n0, r = (int(v) for v in z["dims"])
        h = L // 2
        return ButterflyFactors(L, n0, r, z["VL"], [z[f"H{t}"] for t in range(h)],
                                z["S"], [z[f"G{t}"] for t in range(h)], z["UL"]).validate()
