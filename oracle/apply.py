"""Apply of a butterfly factorization and of its adjoint (oracle, test infrastructure only).

u = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^* g   (Eq. Kfactors, Sec. 3.2)

applied right to left, one sparse factor at a time, in FP64.  Vectors between
factors have length R = 2^L r and are held as (2^L, r, nrhs) arrays of
r-blocks.  The block indices follow the column indices of the block-diagonal
factors of Sec. 3:

* t^l = (V^l)^* g has block j*2^{L-l} + i' for column node j (level l of T_Omega)
  and row node i' (level L-l of T_X);
* w^l = G^{l-1} ... M^h ... g (the input of U^l) has block i*2^{L-l} + j for row
  node i (level l of T_X) and column node j (level L-l of T_Omega).

Steps (each cites the definition it evaluates):
  leaf V:   t^L[b] = (V^L_b)^* g[b n0 : (b+1) n0]                      (Sec. 3.2.2)
  H level:  [t^l_{j,2i}; t^l_{j,2i+1}] = [(H^l_{2j,i})^* (H^l_{2j+1,i})^*]
                                         [t^{l+1}_{2j,i}; t^{l+1}_{2j+1,i}]   (mirror of Eq. RSh2)
  M^h:      w^h_{i,j} = S^h_{i,j} t^h_{j,i}   (block (j,i) of M^h_{i,j} is S^h_{i,j}, Eq. KeqUMV)
  G level:  [w^{l+1}_{2i,j}; w^{l+1}_{2i+1,j}] = [G^l_{2i,j}; G^l_{2i+1,j}] [w^l_{i,2j}; w^l_{i,2j+1}]
                                                                            (Eq. RSh2 and G^l_i)
  leaf U:   u[a n0 : (a+1) n0] = U^L_a w^L[a]                           (Eq. RFUh)

The adjoint K^* g = V^L H^{L-1} ... H^h (M^h)^* (G^h)^* ... (G^{L-1})^* (U^L)^* g
runs the conjugate-transposed steps in the reverse order; (M^h)^* has the real
weight S^h_{i,j} at block (i, j) of M^h_{j,i}, i.e. t^h_{j,i} = S^h_{i,j} w^h_{i,j}.
"""
from __future__ import annotations

import numpy as np

from bfinputs.factors import ButterflyFactors


def _as_cols(g: np.ndarray, N: int):
    g = np.asarray(g, dtype=np.complex128)
    return g.reshape(N, -1), g.ndim == 1


def bf_apply(F: ButterflyFactors, g: np.ndarray) -> np.ndarray:
    """u = K_bf g for g of shape (N,) or (N, nrhs)."""
    L, n0, r, h, m = F.L, F.n0, F.r, F.h, F.m
    G2, squeeze = _as_cols(g, F.N)
    nr = G2.shape[1]
    nb = 1 << L
    # leaf: t^L[b, k] = sum_p conj(V^L_b[p, k]) g[b n0 + p]
    t = np.einsum("bpk,bpn->bkn", np.conj(F.VL), G2.reshape(nb, n0, nr))
    # H levels l = L-1 .. h: t^{l+1} -> t^l
    for l in range(L - 1, h - 1, -1):
        a, c = 1 << l, 1 << (L - l - 1)
        Hl = np.asarray(F.H[l - h]).reshape(a, 2, c, r, 2, r)      # [j, c, i, k, d, k']
        tin = t.reshape(a, 2, c, r, nr)                              # [j, c, i, k, n]
        t = np.einsum("jcikdl,jcikn->jidln", np.conj(Hl), tin).reshape(nb, r, nr)
    # M^h: w^h[i m + j] = S_{i,j} * t^h[j m + i]
    tm = t.reshape(m, m, r, nr)                                      # [j, i, k, n]
    w = (np.asarray(F.S)[:, :, :, None] * tm.transpose(1, 0, 2, 3)).reshape(nb, r, nr)
    # G levels l = h .. L-1: w^l -> w^{l+1}
    for l in range(h, L):
        a, c = 1 << l, 1 << (L - l - 1)
        Gl = np.asarray(F.G[l - h]).reshape(a, 2, c, r, 2, r)      # [i, c, j, k', d, k]
        win = w.reshape(a, c, 2, r, nr)                              # [i, j, d, k, n]
        w = np.einsum("icjldk,ijdkn->icjln", Gl, win).reshape(nb, r, nr)
    # leaf: u[a n0 + p] = sum_k U^L_a[p, k] w^L[a, k]
    u = np.einsum("apk,akn->apn", np.asarray(F.UL), w).reshape(F.N, nr)
    return u[:, 0] if squeeze else u


def bf_adjoint(F: ButterflyFactors, f: np.ndarray) -> np.ndarray:
    """g' = K_bf^* f for f of shape (N,) or (N, nrhs)."""
    L, n0, r, h, m = F.L, F.n0, F.r, F.h, F.m
    F2, squeeze = _as_cols(f, F.N)
    nr = F2.shape[1]
    nb = 1 << L
    # (U^L)^*: w^L[a, k] = sum_p conj(U^L_a[p, k]) f[a n0 + p]
    w = np.einsum("apk,apn->akn", np.conj(F.UL), F2.reshape(nb, n0, nr))
    # (G^l)^* for l = L-1 .. h: w^{l+1} -> w^l
    for l in range(L - 1, h - 1, -1):
        a, c = 1 << l, 1 << (L - l - 1)
        Gl = np.asarray(F.G[l - h]).reshape(a, 2, c, r, 2, r)      # [i, c, j, k', d, k]
        win = w.reshape(a, 2, c, r, nr)                              # [i, c, j, k', n]
        w = np.einsum("icjldk,icjln->ijdkn", np.conj(Gl), win).reshape(nb, r, nr)
    # (M^h)^*: t^h[j m + i] = S_{i,j} * w^h[i m + j]
    wm = w.reshape(m, m, r, nr)                                      # [i, j, k, n]
    t = (np.asarray(F.S)[:, :, :, None] * wm).transpose(1, 0, 2, 3).reshape(nb, r, nr)
    # H^l for l = h .. L-1: t^l -> t^{l+1}
    for l in range(h, L):
        a, c = 1 << l, 1 << (L - l - 1)
        Hl = np.asarray(F.H[l - h]).reshape(a, 2, c, r, 2, r)      # [j, c, i, k, d, k']
        tin = t.reshape(a, c, 2, r, nr)                              # [j, i, d, k', n]
        t = np.einsum("jcikdl,jidln->jcikn", Hl, tin).reshape(nb, r, nr)
    # V^L: g'[b n0 + p] = sum_k V^L_b[p, k] t^L[b, k]
    out = np.einsum("bpk,bkn->bpn", np.asarray(F.VL), t).reshape(F.N, nr)
    return out[:, 0] if squeeze else out
