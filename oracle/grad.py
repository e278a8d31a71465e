"""Reverse-mode gradient of the butterfly apply (oracle, test infrastructure only).

For u = K_bf g with K_bf = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*
(Eq. Kfactors, Sec. 3.2) and an upstream gradient ubar = dL/du of a real loss
L, this computes the gradient with respect to the input g and to every factor
block, in FP64, by running the chain forward (keeping the input of every
factor) and then back through the factors in reverse order.

Gradient convention (the one of PyTorch for complex tensors): for a complex
parameter z the gradient is dL/dRe z + i dL/dIm z = 2 dL/dz*; for the real
S^h it is dL/dS.  For one factor step y = A x this gives
    xbar = A^* ybar,   Abar = sum over RHS of ybar x^*,
and when the step uses a block through its conjugate transpose, y = B^* x,
    Bbar = (Abar)^* = sum over RHS of x ybar^*.
The chain is linear in each factor separately, so each factor's gradient is
one such outer product of the factor's input and the gradient at its output.

Steps (the forward steps are those of ``oracle.apply``; each backward step is
the adjoint of the forward one and the outer product above):
  leaf V:   t^L[b] = (V^L_b)^* g_b           Vbar_b = g_b tbar_b^*,  gbar_b = V_b tbar_b
  H level:  out_{j,i} = sum_c (H^l_{2j+c,i})^* in_{j,c,i}
            Hbar_{2j+c,i} = in_{j,c,i} outbar_{j,i}^*,  inbar_{j,c,i} = H_{2j+c,i} outbar_{j,i}
  M^h:      w_{i,j} = S_{i,j} t_{j,i}        Sbar_{i,j} = Re sum conj(wbar_{i,j}) t_{j,i},
                                              tbar_{j,i} = S_{i,j} wbar_{i,j}
  G level:  out_{i,c,j} = G^l_{2i+c,j} in_{i,j}
            Gbar_{2i+c,j} = outbar_{i,c,j} in_{i,j}^*,  inbar_{i,j} = sum_c G^*_{2i+c,j} outbar_{i,c,j}
  leaf U:   u_a = U^L_a w_a                   Ubar_a = ubar_a w_a^*,  wbar_a = U_a^* ubar_a
"""
from __future__ import annotations

import numpy as np

from bfinputs.factors import ButterflyFactors


def bf_apply_and_grad(F: ButterflyFactors, g: np.ndarray, ubar: np.ndarray):
    """Return (u, gbar, grads) with u = K_bf g, gbar = dL/dg and grads a
    ButterflyFactors of the factor gradients, for g and ubar of shape (N, nrhs)."""
    L, n0, r, h, m = F.L, F.n0, F.r, F.h, F.m
    nb = 1 << L
    g = np.asarray(g, dtype=np.complex128).reshape(F.N, -1)
    ubar = np.asarray(ubar, dtype=np.complex128).reshape(F.N, -1)
    nr = g.shape[1]
    VL, UL, S = np.asarray(F.VL), np.asarray(F.UL), np.asarray(F.S, dtype=np.float64)

    # ---- forward, keeping each factor's input
    gb = g.reshape(nb, n0, nr)
    t = np.einsum("bpk,bpn->bkn", np.conj(VL), gb)
    t_in = {}                                                        # input of H level l
    for l in range(L - 1, h - 1, -1):
        a, c = 1 << l, 1 << (L - l - 1)
        Hl = np.asarray(F.H[l - h]).reshape(a, 2, c, r, 2, r)      # [j, c, i, k, d, k']
        t_in[l] = t.reshape(a, 2, c, r, nr)                          # [j, c, i, k, n]
        t = np.einsum("jcikdl,jcikn->jidln", np.conj(Hl), t_in[l]).reshape(nb, r, nr)
    t_h = t.reshape(m, m, r, nr)                                     # [j, i, k, n]
    w = (S[:, :, :, None] * t_h.transpose(1, 0, 2, 3)).reshape(nb, r, nr)
    w_in = {}                                                        # input of G level l
    for l in range(h, L):
        a, c = 1 << l, 1 << (L - l - 1)
        Gl = np.asarray(F.G[l - h]).reshape(a, 2, c, r, 2, r)      # [i, c, j, k', d, k]
        w_in[l] = w.reshape(a, c, 2, r, nr)                          # [i, j, d, k, n]
        w = np.einsum("icjldk,ijdkn->icjln", Gl, w_in[l]).reshape(nb, r, nr)
    u = np.einsum("apk,akn->apn", UL, w).reshape(F.N, nr)

    # ---- backward
    ub = ubar.reshape(nb, n0, nr)
    gUL = np.einsum("apn,akn->apk", ub, np.conj(w))
    wbar = np.einsum("apk,apn->akn", np.conj(UL), ub)
    gG = [None] * h
    for l in range(L - 1, h - 1, -1):
        a, c = 1 << l, 1 << (L - l - 1)
        Gl = np.asarray(F.G[l - h]).reshape(a, 2, c, r, 2, r)
        ob = wbar.reshape(a, 2, c, r, nr)                            # [i, c, j, k', n]
        gG[l - h] = np.einsum("icjln,ijdkn->icjldk", ob, np.conj(w_in[l])).reshape(nb, r, 2 * r)
        wbar = np.einsum("icjldk,icjln->ijdkn", np.conj(Gl), ob).reshape(nb, r, nr)
    wb = wbar.reshape(m, m, r, nr)                                   # [i, j, k, n]
    gS = np.real(np.einsum("ijkn,jikn->ijk", np.conj(wb), t_h))
    tbar = (S[:, :, :, None] * wb).transpose(1, 0, 2, 3).reshape(nb, r, nr)
    gH = [None] * h
    for l in range(h, L):
        a, c = 1 << l, 1 << (L - l - 1)
        Hl = np.asarray(F.H[l - h]).reshape(a, 2, c, r, 2, r)
        ob = tbar.reshape(a, c, 2, r, nr)                            # [j, i, d, k', n]
        gH[l - h] = np.einsum("jcikn,jidln->jcikdl", t_in[l], np.conj(ob)).reshape(nb, r, 2 * r)
        tbar = np.einsum("jcikdl,jidln->jcikn", Hl, ob).reshape(nb, r, nr)
    gVL = np.einsum("bpn,bkn->bpk", gb, np.conj(tbar))
    gbar = np.einsum("bpk,bkn->bpn", VL, tbar).reshape(F.N, nr)
    grads = ButterflyFactors(L, n0, r, gVL, gH, gS, gG, gUL, meta={"source": "gradient"})
    return u, gbar, grads


def loss_and_grad(F: ButterflyFactors, g: np.ndarray, y: np.ndarray):
    """L = ||K_bf g - y||_F^2 (the differentiation workload's loss), its
    upstream gradient ubar = 2 (K_bf g - y), and (gbar, grads)."""
    from oracle.apply import bf_apply
    u = bf_apply(F, g)
    res = u - np.asarray(y, dtype=np.complex128).reshape(u.shape)
    ubar = 2.0 * res
    _, gbar, grads = bf_apply_and_grad(F, g, ubar)
    return float(np.vdot(res, res).real), ubar, gbar, grads
