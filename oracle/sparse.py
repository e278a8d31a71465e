"""Brute-force path: every factor as an explicit sparse matrix (oracle, test infrastructure only).

Each factor of Eq. (Kfactors) is assembled entry by entry from the block
matrices displayed in Sec. 3 -- block-diagonal U^l / V^l (Eq. expression-UV
and its level-l analogue), the weighted permutation M^h (Eq. KeqUMV: block
(j, i) of M^h_{i,j} is S^h_{i,j}) and the block-diagonal G^l = diag(G^l_i)
whose G^l_i stacks diag_j G^l_{2i,j} over diag_j G^l_{2i+1,j}, each G^l_{i',j}
spanning columns 2j r .. (2j+2) r of G^l_i (Sec. 3.2.1); H^l likewise
(Sec. 3.2.2).  The chain is then multiplied out.  None of this shares index
code with ``oracle.apply``: it is the independent check of the paper's
block-matrix definitions against the structured apply.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from bfinputs.factors import ButterflyFactors


def _coo(rows, cols, vals, shape):
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=shape)


def leaf_matrix(blocks: np.ndarray, n0: int, r: int) -> sp.csr_matrix:
    """U^L (or V^L) = diag(U^L_0, ..., U^L_{2^L-1}), N x 2^L r, each block n0 x r."""
    nb = blocks.shape[0]
    rows, cols, vals = [], [], []
    pr, kc = np.meshgrid(np.arange(n0), np.arange(r), indexing="ij")
    for a in range(nb):
        rows.append((a * n0 + pr).ravel())
        cols.append((a * r + kc).ravel())
        vals.append(blocks[a].ravel())
    return _coo(rows, cols, vals, (nb * n0, nb * r))


def level_basis_matrix(blocks: np.ndarray) -> sp.csr_matrix:
    """U^l = diag(U^l_0, ..., U^l_{2^l-1}) with U^l_i = [U^l_{i,0} ... U^l_{i,2^{L-l}-1}]
    (Eq. expression-UV at level h; Sec. 3.2.1 at level l).  ``blocks`` has
    shape (2^l, 2^{L-l}, N/2^l, r): blocks[i, j] = U^l_{i,j}.  The same
    assembly gives V^l from the V^l_{j,i}."""
    ni, nj, nr, r = blocks.shape
    rows, cols, vals = [], [], []
    pr, kc = np.meshgrid(np.arange(nr), np.arange(r), indexing="ij")
    for i in range(ni):
        for j in range(nj):
            rows.append((i * nr + pr).ravel())
            cols.append(((i * nj + j) * r + kc).ravel())
            vals.append(np.asarray(blocks[i, j], dtype=np.complex128).ravel())
    return _coo(rows, cols, vals, (ni * nr, ni * nj * r))


def transfer_matrix(blocks: np.ndarray, level: int, L: int, r: int) -> sp.csr_matrix:
    """G^l (or H^l) = diag(G^l_0, ..., G^l_{2^l-1}), R x R (Sec. 3.2.1).

    G^l_i is (2^{L-l} r) x (2^{L-l} r): its top half holds G^l_{2i,j} in block
    row j, its bottom half holds G^l_{2i+1,j} in block row 2^{L-l-1} + j, both
    over columns 2j r .. (2j+2) r.  ``blocks[i' * 2^{L-l-1} + j]`` = G^l_{i',j}.
    """
    nj = 1 << (L - level - 1)
    size = (1 << (L - level)) * r
    R = (1 << L) * r
    rows, cols, vals = [], [], []
    kr, kc = np.meshgrid(np.arange(r), np.arange(2 * r), indexing="ij")
    for i in range(1 << level):
        off = i * size
        for half in (0, 1):
            for j in range(nj):
                blk = blocks[(2 * i + half) * nj + j]
                rows.append((off + (half * nj + j) * r + kr).ravel())
                cols.append((off + 2 * j * r + kc).ravel())
                vals.append(blk.ravel())
    return _coo(rows, cols, vals, (R, R))


def middle_matrix(S: np.ndarray, r: int) -> sp.csr_matrix:
    """M^h, (m^2 r) x (m^2 r): M^h_{i,j} (block (i, j), size m r x m r) is zero
    except its (j, i) sub-block, the diagonal S^h_{i,j} (Eq. KeqUMV)."""
    m = S.shape[0]
    rows, cols, vals = [], [], []
    k = np.arange(r)
    for i in range(m):
        for j in range(m):
            rows.append(i * m * r + j * r + k)
            cols.append(j * m * r + i * r + k)
            vals.append(S[i, j].astype(np.complex128))
    return _coo(rows, cols, vals, (m * m * r, m * m * r))


def factor_list(F: ButterflyFactors) -> list:
    """[U^L, G^{L-1}, ..., G^h, M^h, (H^h)^*, ..., (H^{L-1})^*, (V^L)^*] -- the
    L+3 factors of Eq. (Kfactors), left to right."""
    L, r, h = F.L, F.r, F.h
    out = [leaf_matrix(np.asarray(F.UL, np.complex128), F.n0, r)]
    for l in range(L - 1, h - 1, -1):
        out.append(transfer_matrix(np.asarray(F.G[l - h], np.complex128), l, L, r))
    out.append(middle_matrix(np.asarray(F.S, np.float64), r))
    for l in range(h, L):
        out.append(transfer_matrix(np.asarray(F.H[l - h], np.complex128), l, L, r).conj().T.tocsr())
    out.append(leaf_matrix(np.asarray(F.VL, np.complex128), F.n0, r).conj().T.tocsr())
    return out


def dense_product(F: ButterflyFactors) -> np.ndarray:
    """K_bf as a dense N x N matrix (tiny N only)."""
    mats = factor_list(F)
    acc = mats[-1].toarray()
    for M in reversed(mats[:-1]):
        acc = M @ acc
    return np.asarray(acc)


def chain_apply(F: ButterflyFactors, g: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """K_bf g (or K_bf^* g) by sparse matrix-vector products along the chain."""
    mats = factor_list(F)
    x = np.asarray(g, dtype=np.complex128)
    seq = mats if adjoint else list(reversed(mats))
    for M in seq:
        x = (M.conj().T @ x) if adjoint else (M @ x)
    return x
