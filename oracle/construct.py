"""Butterfly factorization by entry sampling (oracle, test infrastructure only).

Builds K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^* (Eq. Kfactors)
for the 1D kernels of ``oracle.kernel`` in FP64, in the two stages of Sec. 3:

1. Middle level (Sec. 3.1): every K^h_{i,j} = K(A^h_i, B^h_j), i, j < m = 2^h,
   is approximated by randomized sampling (Sec. 2.2, the paper's "second
   case": entries available) and written in the form of Eq. (lowrankSVD):
   K^h_{i,j} ~ U^h_{i,j} S^h_{i,j} (V^h_{j,i})^*.
2. Recursive factorization (Sec. 3.2): for l = h..L-1 and every (i, j), the
   top and bottom halves of [U^l_{i,2j}  U^l_{i,2j+1}] are replaced by their
   truncated SVDs in the form of Eq. (lowrankSVD3), giving
   U^{l+1}_{2i,j} G^l_{2i,j} and U^{l+1}_{2i+1,j} G^l_{2i+1,j} (Eq. RSh2);
   the same procedure on V^h gives V^L and the H^l (Sec. 3.2.2).

Order (Sec. 3.3, memory-saving variant): U^h_i is generated for one row node
i at a time and factorized at once; V^h_j likewise per column node j.  Each
middle block draws its random rows/columns from a generator keyed by
(seed, i, j), so the V pass sees exactly the (U, S, V) of the U pass.

Error bookkeeping (reading of "epsilon of the construction", which the paper
does not define): ``eps_rec`` = max over all recursive SVDs of
sigma_{r+1}/sigma_1 of the 2r-column stack; ``eps_mid`` = max over the middle
blocks of the relative error of U S V^* on a fresh random r*q x r*q sample of
entries.
"""
from __future__ import annotations

import numpy as np

from bfinputs.factors import ButterflyFactors, tree_sizes

from . import kernel as K
from .lowrank import form_us_v, form_usv, randomized_sampling


def middle_block(N: int, L: int, r: int, i: int, j: int, kind: str = "fio",
                 seed: int = 0, q: int = 3):
    """Rank-r approximation K^h_{i,j} ~ U S V^* of the middle-level block of
    row node A^h_i and column node B^h_j (Sec. 3.1, second case).

    Returns (U (N/m x r), S (r,), V (N/m x r), residual) where residual is the
    relative error on a fresh r*q x r*q sample of the block's entries.
    """
    m = 1 << (L // 2)
    nb = N // m
    rng = np.random.default_rng([int(seed), int(i), int(j)])
    r0, c0 = i * nb, j * nb

    def entry(I, J):
        return K.entries(r0 + np.asarray(I), c0 + np.asarray(J), N, kind)

    U0, s, V0 = randomized_sampling(entry, nb, nb, r, rng, q=q)
    U, S, V = form_usv(U0, s, V0, r)
    I = np.sort(rng.choice(nb, size=min(r * q, nb), replace=False))
    J = np.sort(rng.choice(nb, size=min(r * q, nb), replace=False))
    Z = entry(I, J)
    approx = (U[I] * S[None, :]) @ V[J].conj().T
    res = float(np.linalg.norm(Z - approx) / max(np.linalg.norm(Z), 1e-300))
    return U, S, V, res


def _svd_stack(Z: np.ndarray, r: int):
    """Truncated SVD of a (rows x 2r) stack plus sigma_{r+1}/sigma_1."""
    Uf, s, Vh = np.linalg.svd(Z, full_matrices=False)
    k = min(r, s.size)
    tail = float(s[k] / s[0]) if (s.size > k and s[0] > 0) else 0.0
    return Uf[:, :k], s[:k], Vh[:k].conj().T, tail


def recursive_factorize(blocks: list, level: int, node: int, L: int, r: int,
                        leaf_out: np.ndarray, trans_out: list, stats: dict) -> None:
    """Factor U^l_node = [U^l_{node,0} ... U^l_{node,2^{L-l}-1}] (``blocks``,
    each N/2^l x r) as U^L G^{L-1} ... G^l restricted to the subtree of
    ``node`` (Sec. 3.2.1, Eqs. RSh and RSh2).

    For each j < 2^{L-l-1} and each half c (0 = top, 1 = bottom):
        [U^{l,c}_{node,2j}  U^{l,c}_{node,2j+1}] ~ U^{l+1}_{2 node + c, j} G^l_{2 node + c, j}
    by a truncated SVD put in the form of Eq. (lowrankSVD3).  G^l_{i',j} is
    written to trans_out[l - L/2][i' * 2^{L-l-1} + j]; at l = L the leaf
    U^L_{node,0} is written to leaf_out[node].  The same routine factors V^h
    (Sec. 3.2.2) with the roles of the trees exchanged.
    """
    if level == L:
        leaf_out[node] = blocks[0]
        return
    half = blocks[0].shape[0] // 2
    nj = len(blocks) // 2
    base = level - L // 2
    for c in (0, 1):
        child = 2 * node + c
        new_blocks = []
        for j in range(nj):
            Z = np.hstack([blocks[2 * j][c * half:(c + 1) * half],
                           blocks[2 * j + 1][c * half:(c + 1) * half]])
            U0, s, V0, tail = _svd_stack(Z, r)
            stats["eps_rec"] = max(stats["eps_rec"], tail)
            Unew, Gblk = form_us_v(U0, s, V0, r)
            trans_out[base][child * nj + j] = Gblk
            new_blocks.append(Unew)
        recursive_factorize(new_blocks, level + 1, child, L, r, leaf_out, trans_out, stats)


def construct(N: int, L: int, r: int, kind: str = "fio", seed: int = 0, q: int = 3,
              cache_middle: bool | None = None) -> ButterflyFactors:
    """Butterfly factorization of the N x N matrix of ``kind`` with trees of
    even depth L and rank r (Sec. 3), in FP64.

    ``cache_middle`` keeps the V parts of the middle blocks from the U pass
    instead of recomputing them in the V pass (same values either way); by
    default it is on when they take under 1 GB.
    """
    if N % (1 << L):
        raise ValueError("N must be a multiple of 2^L")
    n0 = N >> L
    s = tree_sizes(L, n0, r)
    h, m, nb = s["h"], s["m"], s["nblocks"]
    if cache_middle is None:
        cache_middle = N * m * r * 16 < (1 << 30)
    VL = np.zeros((nb, n0, r), dtype=np.complex128)
    UL = np.zeros((nb, n0, r), dtype=np.complex128)
    H = [np.zeros((nb, r, 2 * r), dtype=np.complex128) for _ in range(h)]
    G = [np.zeros((nb, r, 2 * r), dtype=np.complex128) for _ in range(h)]
    S = np.zeros((m, m, r), dtype=np.float64)
    stats = {"eps_rec": 0.0, "eps_mid": 0.0}
    vcache = {}
    # U pass: one row node i at a time (Sec. 3.3).
    for i in range(m):
        blocks = []
        for j in range(m):
            U, Sd, V, res = middle_block(N, L, r, i, j, kind, seed, q)
            stats["eps_mid"] = max(stats["eps_mid"], res)
            S[i, j] = Sd
            blocks.append(U)
            if cache_middle:
                vcache[(i, j)] = V
        recursive_factorize(blocks, h, i, L, r, UL, G, stats)
    # V pass: one column node j at a time; V^h_j = [V^h_{j,0} ... V^h_{j,m-1}].
    for j in range(m):
        blocks = []
        for i in range(m):
            V = vcache.pop((i, j)) if cache_middle else middle_block(N, L, r, i, j, kind, seed, q)[2]
            blocks.append(V)
        recursive_factorize(blocks, h, j, L, r, VL, H, stats)
    meta = {"source": "construct", "kind": kind, "seed": seed, "q": q,
            "eps_rec": stats["eps_rec"], "eps_mid": stats["eps_mid"],
            "eps": max(stats["eps_rec"], stats["eps_mid"], 1e-13)}
    return ButterflyFactors(L, n0, r, VL, H, S, G, UL, meta).validate()


def block_singular_values(N: int, L: int, level: int, i: int, j: int,
                          kind: str = "fio") -> np.ndarray:
    """All singular values of K^l_{i,j} = K(A^l_i, B^{L-l}_j) (Sec. 3 notation),
    for checking the complementary low-rank property (Sec. 1.1) on small N."""
    nr = N >> level
    nc = N >> (L - level)
    rows = i * nr + np.arange(nr)
    cols = j * nc + np.arange(nc)
    return np.linalg.svd(K.entries(rows, cols, N, kind), compute_uv=False)
