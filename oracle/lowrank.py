"""Rank-r approximations used by the construction (oracle, test infrastructure only).

* ``truncated_svd``       -- the optimal rank-r approximation Z ~ U0 Sigma0 V0^* (Sec. 2).
* ``form_usv``            -- Eq. (lowrankSVD): U = U0 Sigma0, S = Sigma0^{-1}, V^* = Sigma0 V0^*.
* ``form_us_v``           -- Eq. (lowrankSVD3): U = U0 Sigma0, V^* = V0^*.
* ``randomized_sampling`` -- Sec. 2.2, "Randomized sampling for low-rank
                             approximation", steps 1-7, with q = 3 and three
                             rounds of steps 2-3 (the parameters stated after
                             the algorithm and in Sec. 4).

Readings where the paper is silent:
* S = Sigma0^{-1} for a singular value that is zero or negligible
  (sigma_k <= 1e-14 sigma_1): the pseudo-inverse, S_k = 0, and column k of U
  and of V set to zero; the storage stays r wide.
* A block with fewer than r rows or columns gives rank min(r, rows, cols);
  the factors are padded with zero columns to width r.
* Random rows and columns are drawn uniformly without replacement; each draw
  takes r*q indices (all of them if the block is smaller); the additional
  rows and columns of step 6 are also r*q each.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

SIGMA_TOL = 1e-14


def truncated_svd(Z: np.ndarray, r: int):
    """Z ~ U0 diag(s) V0^*, the first min(r, rows, cols) singular triplets (Sec. 2)."""
    U, s, Vh = np.linalg.svd(Z, full_matrices=False)
    k = min(r, s.size)
    return U[:, :k], s[:k], Vh[:k, :].conj().T


def _pad_cols(A: np.ndarray, r: int) -> np.ndarray:
    if A.shape[1] == r:
        return A
    out = np.zeros((A.shape[0], r), dtype=A.dtype)
    out[:, :A.shape[1]] = A
    return out


def form_usv(U0, s, V0, r: int):
    """Eq. (lowrankSVD): Z ~ U S V^* with U = U0 Sigma0, S = Sigma0^{-1},
    V = V0 Sigma0 (so V^* = Sigma0 V0^*).  Returns (U, S, V) padded to width r;
    S is the real diagonal as a length-r vector (pseudo-inverse reading, see
    the module docstring)."""
    s = np.asarray(s, dtype=np.float64)
    keep = s > SIGMA_TOL * (s[0] if s.size else 0.0)
    sk = np.where(keep, s, 0.0)
    U = U0 * sk[None, :]
    V = V0 * sk[None, :]
    S = np.zeros(r, dtype=np.float64)
    S[:s.size] = np.where(keep, 1.0 / np.where(keep, s, 1.0), 0.0)
    return _pad_cols(U, r), S, _pad_cols(V, r)


def form_us_v(U0, s, V0, r: int):
    """Eq. (lowrankSVD3): Z ~ U V^* with U = U0 Sigma0 and V^* = V0^*.
    Returns (U, Vh) with U padded to r columns and Vh padded to r rows."""
    U = _pad_cols(U0 * np.asarray(s)[None, :], r)
    Vh = V0.conj().T
    if Vh.shape[0] < r:
        Vh = np.vstack([Vh, np.zeros((r - Vh.shape[0], Vh.shape[1]), dtype=Vh.dtype)])
    return U, Vh


def _pivots(A: np.ndarray) -> np.ndarray:
    """Column order chosen by a column-pivoted Householder QR, A P = Q R."""
    _, P = sla.qr(A, mode="r", pivoting=True)
    return np.asarray(P)


def _draw(rng: np.random.Generator, n: int, count: int) -> np.ndarray:
    return rng.choice(n, size=min(count, n), replace=False)


def randomized_sampling(entry, m: int, n: int, r: int, rng: np.random.Generator,
                        q: int = 3, rounds: int = 3):
    """Randomized sampling for a rank-r approximate SVD Z ~ U0 Sigma0 V0^*
    of an m x n matrix Z given only through ``entry(I, J) = Z[I][:, J]``
    (Sec. 2.2, steps 1-7).

    Step 1: Pi_col = Pi_row = {}.
    Step 2: I = (r*q random rows) U Pi_row; a pivoted QR of Z[I, :] picks Pi_col
            (the first r pivot columns).
    Step 3: J = (r*q random columns) U Pi_col; a pivoted LQ of Z[:, J] (the
            pivoted QR of its adjoint) picks Pi_row (the first r pivot rows).
    Step 4: steps 2-3 are repeated (``rounds`` times in all).
    Step 5: Q_col = first r columns of Q of a pivoted QR of Z[:, Pi_col];
            Q_row = first r columns of Q of a pivoted QR of Z[Pi_row, :]^*.
    Step 6: with I = Pi_row U (extra rows), J = Pi_col U (extra columns),
            M = pinv(Q_col[I, :]) Z[I, J] pinv(Q_row^*[:, J]).
    Step 7: M = U_M Sigma_M V_M^*; U0 = Q_col U_M, Sigma0 = Sigma_M,
            V0^* = V_M^* Q_row^*.

    Returns (U0 (m x k), s (k,), V0 (n x k)) with k = min(r, m, n).
    """
    k = min(r, m, n)
    all_rows = np.arange(m)
    all_cols = np.arange(n)
    pi_col = np.zeros(0, dtype=np.int64)
    pi_row = np.zeros(0, dtype=np.int64)
    for _ in range(rounds):
        I = np.union1d(_draw(rng, m, r * q), pi_row)
        pi_col = _pivots(entry(I, all_cols))[:k]
        J = np.union1d(_draw(rng, n, r * q), pi_col)
        pi_row = _pivots(entry(all_rows, J).conj().T)[:k]
    Qc, _, _ = sla.qr(entry(all_rows, np.sort(pi_col)), mode="economic", pivoting=True)
    Qr, _, _ = sla.qr(entry(np.sort(pi_row), all_cols).conj().T, mode="economic", pivoting=True)
    Q_col = Qc[:, :k]
    Q_row = Qr[:, :k]
    I = np.union1d(pi_row, _draw(rng, m, r * q))
    J = np.union1d(pi_col, _draw(rng, n, r * q))
    Q_row_h = Q_row.conj().T
    M = np.linalg.pinv(Q_col[I, :]) @ entry(I, J) @ np.linalg.pinv(Q_row_h[:, J])
    UM, sM, VMh = np.linalg.svd(M)
    U0 = Q_col @ UM[:, :k]
    V0 = Q_row @ VMh[:k, :].conj().T
    return U0, sM[:k], V0
