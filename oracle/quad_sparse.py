"""The 2D factors as explicit sparse matrices (oracle, test infrastructure only).

An apply path independent of the structured one in ``quad.py``: every factor
of K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^* is assembled
entry by entry from its block definition (the 1D definitions of Sec. 3.2
with four children per node) as a CSR matrix, and the chain is multiplied
out.  Vector orderings: t^{(l)} has entry ((j 4^{L-l} + i) r_l + x) for
column node j at level l, row node i at level L-l; w^{(l)} has entry
((i 4^{L-l} + j) r_l + x) for row node i at level l, column node j at level
L-l; the vectors g, u are in Morton point order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from bfinputs.quad import QuadFactors


def _csr(rows, cols, vals, shape):
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=shape)


def factor_list(F: QuadFactors) -> list:
    """[U^L, G^{L-1}, ..., G^h, M^h, (H^h)^*, ..., (H^{L-1})^*, (V^L)^*] as CSR."""
    s = F.sizes
    L, h, n0, N, rk = F.L, s["h"], F.n0, F.N, s["ranks"]
    nleaf = 1 << (2 * L)
    R = {lv: nleaf * rk[lv] for lv in range(h, L + 1)}
    # (V^L)^*: row (b, x) of t^{(L)}, column point b n0 + p.
    rows, cols, vals = [], [], []
    for b in range(nleaf):
        for p in range(n0):
            for x in range(rk[L]):
                rows.append([b * rk[L] + x]); cols.append([b * n0 + p]); vals.append([np.conj(F.VL[b, p, x])])
    Vs = _csr(rows, cols, vals, (R[L], N))
    Hs, Gs = {}, {}
    for lv in range(h, L):
        r0, r1 = rk[lv], rk[lv + 1]
        nlow = 1 << (2 * (L - lv - 1))          # nodes at level L-l-1 of the other tree
        hr, hc, hv, gr, gc, gv = [], [], [], [], [], []
        for a_node in range(1 << (2 * lv)):     # j (column tree) for H, i (row tree) for G
            for c in range(4):
                for low in range(nlow):
                    blk = (4 * a_node + c) * nlow + low
                    Hb, Gb = F.H[lv - h][blk], F.G[lv - h][blk]
                    for cp in range(4):
                        for a in range(r1):
                            for x in range(r0):
                                # (H^l)^*: t^{(l)}_{j, 4i'+c'} gets conj(H^l_{4j+c,i'}[a, c' r_l + x]) t^{(l+1)}_{4j+c,i'}[a]
                                hr.append([(a_node * 4 * nlow + 4 * low + cp) * r0 + x])
                                hc.append([((4 * a_node + c) * nlow + low) * r1 + a])
                                hv.append([np.conj(Hb[a, cp * r0 + x])])
                                # G^l: w^{(l+1)}_{4i+c,j'}[a] gets G^l_{4i+c,j'}[a, c' r_l + x] w^{(l)}_{i,4j'+c'}[x]
                                gr.append([((4 * a_node + c) * nlow + low) * r1 + a])
                                gc.append([(a_node * 4 * nlow + 4 * low + cp) * r0 + x])
                                gv.append([Gb[a, cp * r0 + x]])
        Hs[lv] = _csr(hr, hc, hv, (R[lv], R[lv + 1]))
        Gs[lv] = _csr(gr, gc, gv, (R[lv + 1], R[lv]))
    # M^h: w^{(h)}_{i,j}[x] = S[i, j, x] t^{(h)}_{j,i}[x]
    m = 1 << (2 * h)
    mr, mc, mv = [], [], []
    for i in range(m):
        for j in range(m):
            for x in range(rk[h]):
                mr.append([(i * m + j) * rk[h] + x]); mc.append([(j * m + i) * rk[h] + x]); mv.append([F.S[i, j, x]])
    Ms = _csr(mr, mc, mv, (R[h], R[h]))
    # U^L: point a n0 + p gets U^L_{a,0}[p, x] w^{(L)}_{a,0}[x]
    ur, uc, uv = [], [], []
    for a in range(nleaf):
        for p in range(n0):
            for x in range(rk[L]):
                ur.append([a * n0 + p]); uc.append([a * rk[L] + x]); uv.append([F.UL[a, p, x]])
    Us = _csr(ur, uc, uv, (N, R[L]))
    return [Us] + [Gs[lv] for lv in range(L - 1, h - 1, -1)] + [Ms] + [Hs[lv] for lv in range(h, L)] + [Vs]


def chain_apply(F: QuadFactors, g: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """The product of the assembled factors applied to g (or its adjoint)."""
    mats = factor_list(F)
    x = np.asarray(g, dtype=np.complex128)
    if adjoint:
        for A in mats:
            x = A.conj().T @ x
    else:
        for A in reversed(mats):
            x = A @ x
    return x
