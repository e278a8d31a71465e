"""Butterfly factorization from matrix-vector products (oracle, test infrastructure only).

Sec. 3.1, first case: only black-box routines for K g and K^* g are available.
Every middle-level block K^h_{i,j} (row node i, column node j, i, j < m = 2^h)
receives a rank-r approximate SVD by the randomized SVD of Sec. 2.1, and all
m^2 blocks share 2 m (r + p) products:

* C is N x m(r+p) and block diagonal with Gaussian diagonal blocks C_jj
  ((N/m) x (r+p)); rows of node i of the column slab j of Y = K C are
  K^h_{i,j} C_jj.
* R is built the same way and W = K^* R; rows of node j of the slab i of W
  are (K^h_{i,j})^* R_ii.
* Per block, Q_col = the first r columns of Q of a pivoted QR of K_ij C_jj,
  Q_row likewise from (K_ij)^* R_ii (Sec. 2.1, step 2), the middle matrix
  (step 3), its SVD, U_0 = Q_col U_M, V_0 = Q_row V_M (step 4), put in the form
  of Eq. (lowrankSVD) as in the entry-sampling construction.

The recursive factorization of U^h and V^h (Sec. 3.2) is the one of
``construct.py``.

Readings where the paper is silent:
* Step 3's middle matrix M = Q_col^* Z Q_row is formed from the two products
  already taken, with no further applies: since W_ij = Z^* R_ii, R_ii^* Z =
  W_ij^*, and R_ii^* Z ~ (R_ii^* Q_col)(Q_col^* Z), so
  M = pinv(R_ii^* Q_col) (W_ij^* Q_row).  (Forming Z Q_row directly would need
  products with vectors that depend on both i and j.)
* p = 5, the oversampling the paper states (Sec. 2.1 and Sec. 4); when a block
  has fewer than r + p columns, r + p is capped at that size.
* The Gaussian blocks are complex standard normal (``bfinputs.sketch_blocks``,
  shared with the device construction); pivoted QR is LAPACK geqp3 (SciPy).

Example 3 (Sec. 4): the composition K~ = K F K of the 1D FIO matrix K with the
Fourier transform F between the space points x_j = j/N and the frequencies
xi_k = k - N/2.  Reading: F is the quadrature of the Fourier integral with the
weight 1/N of the points, F_{kj} = exp(-2 pi i xi_k x_j) / N.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from bfinputs.factors import ButterflyFactors, tree_sizes
from bfinputs.workloads import sketch_blocks

from .construct import recursive_factorize
from .lowrank import form_usv

OVERSAMPLE = 5


def _range_basis(Z: np.ndarray, r: int) -> np.ndarray:
    """The first r columns of Q of the column-pivoted QR Z P = Q R (Sec. 2.1, step 2)."""
    Q, _, _ = sla.qr(Z, mode="economic", pivoting=True)
    return Q[:, :r]


def middle_level(apply, apply_adj, N: int, L: int, r: int, p: int = OVERSAMPLE, seed: int = 0):
    """Rank-r forms K^h_{i,j} ~ U_ij S_ij V_ij^* of all middle-level blocks from
    products with K and K^* only (Sec. 3.1, first case; Sec. 2.1).

    ``apply(X)`` and ``apply_adj(X)`` return K X and K^* X for X of shape (N, k).
    Returns (U, S, V) with U[i][j], V[i][j] of shape (N/m, r) and S of shape
    (m, m, r), plus the number of vectors applied in each direction.
    """
    h = L // 2
    m = 1 << h
    nb = N // m
    k = min(r + p, nb)
    rk = min(r, nb)
    Cb, Rb = sketch_blocks(N, L, r, p, seed)
    C = np.zeros((N, m * k), dtype=np.complex128)
    R = np.zeros((N, m * k), dtype=np.complex128)
    for j in range(m):
        C[j * nb:(j + 1) * nb, j * k:(j + 1) * k] = Cb[j]
        R[j * nb:(j + 1) * nb, j * k:(j + 1) * k] = Rb[j]
    Y = np.asarray(apply(C))          # slab j, rows of node i: K_ij C_jj
    W = np.asarray(apply_adj(R))      # slab i, rows of node j: K_ij^* R_ii
    U = [[None] * m for _ in range(m)]
    V = [[None] * m for _ in range(m)]
    S = np.zeros((m, m, r), dtype=np.float64)
    for i in range(m):
        Rii = R[i * nb:(i + 1) * nb, i * k:(i + 1) * k]
        for j in range(m):
            Yij = Y[i * nb:(i + 1) * nb, j * k:(j + 1) * k]
            Wij = W[j * nb:(j + 1) * nb, i * k:(i + 1) * k]
            Qc = _range_basis(Yij, rk)
            Qr = _range_basis(Wij, rk)
            M = np.linalg.pinv(Rii.conj().T @ Qc) @ (Wij.conj().T @ Qr)
            UM, s, VMh = np.linalg.svd(M)
            U0 = Qc @ UM
            V0 = Qr @ VMh.conj().T
            U[i][j], S[i, j], V[i][j] = form_usv(U0, s, V0, r)
    return U, S, V, m * k


def construct(apply, apply_adj, N: int, L: int, r: int, p: int = OVERSAMPLE, seed: int = 0) -> ButterflyFactors:
    """Butterfly factorization of the N x N matrix given only by ``apply`` and
    ``apply_adj`` (Sec. 3 with the middle level of Sec. 3.1's first case), FP64."""
    if N % (1 << L):
        raise ValueError("N must be a multiple of 2^L")
    n0 = N >> L
    s = tree_sizes(L, n0, r)
    h, m, nb = s["h"], s["m"], s["nblocks"]
    U, S, V, nvec = middle_level(apply, apply_adj, N, L, r, p, seed)
    VL = np.zeros((nb, n0, r), dtype=np.complex128)
    UL = np.zeros((nb, n0, r), dtype=np.complex128)
    H = [np.zeros((nb, r, 2 * r), dtype=np.complex128) for _ in range(h)]
    G = [np.zeros((nb, r, 2 * r), dtype=np.complex128) for _ in range(h)]
    stats = {"eps_rec": 0.0, "eps_mid": 0.0}
    for i in range(m):
        recursive_factorize([U[i][j] for j in range(m)], h, i, L, r, UL, G, stats)
    for j in range(m):
        recursive_factorize([V[i][j] for i in range(m)], h, j, L, r, VL, H, stats)
    meta = {"source": "construct_mv", "p": p, "seed": seed, "vectors_per_direction": nvec,
            "eps_rec": stats["eps_rec"]}
    return ButterflyFactors(L, n0, r, VL, H, S, G, UL, meta).validate()


# ---------------------------------------------------------------- Example 3

def fourier_apply(x: np.ndarray) -> np.ndarray:
    """F x with F_{kj} = exp(-2 pi i (k - N/2) j / N) / N: since
    exp(i pi j) = (-1)^j, F x = fft((-1)^j x) / N (x of shape (N,) or (N, k))."""
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[0]
    sign = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).reshape((N,) + (1,) * (x.ndim - 1))
    return np.fft.fft(sign * x, axis=0) / N


def fourier_adjoint(y: np.ndarray) -> np.ndarray:
    """F^* y = (-1)^j ifft(y)_j (numpy's ifft carries the 1/N)."""
    y = np.asarray(y, dtype=np.complex128)
    N = y.shape[0]
    sign = np.where(np.arange(N) % 2 == 0, 1.0, -1.0).reshape((N,) + (1,) * (y.ndim - 1))
    return sign * np.fft.ifft(y, axis=0)


def fourier_matrix(N: int) -> np.ndarray:
    """F written out entry by entry (small N)."""
    k = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    return np.exp(-2j * np.pi * (k - N // 2) * j / N) / N
