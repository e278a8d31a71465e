"""2D butterfly factorization on quadtrees (oracle, test infrastructure only).

The paper develops the factorization in one dimension and notes that it
carries over to higher dimensions (Sec. 1.2).  This module is that carry-over
for an n x n grid, with the readings below where the paper says nothing; every
step otherwise follows the 1D construction and apply of ``construct.py`` and
``apply.py`` with four children per node instead of two.

Readings:
* Points and frequencies.  x = p / n with p in [0, n)^2, xi = k - n/2 with k in
  [0, n)^2 (the 1D points of Eq. 1D-xandxi in each coordinate).  Both are
  numbered in Morton order: index = sum_b (2 bit_b(p_1) + bit_b(p_2)) 4^b, so a
  quadtree node's points are contiguous and child c of a node holds its c-th
  quarter (c = 2 b_1 + b_2 for the node's next bits b_1 of p_1, b_2 of p_2).
* Ranks.  A node of level l holds N / 4^l points, so level l uses rank
  r_l = min(r, N / 4^l) (l = h..L): r at the middle level, smaller near small
  leaves.
* Recursive factorization (Sec. 3.2, Eq. RSh2, arity 4).  For a row node i at
  level l and a column node j' at level L-l-1, the four blocks
  [U^l_{i,4j'} ... U^l_{i,4j'+3}] (N/4^l x 4 r_l) are split by rows into the
  four children 4i+c of i; each quarter is replaced by its truncated SVD in
  the form of Eq. (lowrankSVD3): U^{l+1}_{4i+c,j'} (N/4^{l+1} x r_{l+1}) times
  G^l_{4i+c,j'} (r_{l+1} x 4 r_l).  The V side is the same on the column tree.
* Kernels.  "fio2": Phi(x, xi) = x.xi + sqrt(c_1(x)^2 xi_1^2 + c_2(x)^2 xi_2^2)
  with c_1 = (2 + sin(2 pi x_1) sin(2 pi x_2))/16 and
  c_2 = (2 + cos(2 pi x_1) cos(2 pi x_2))/16; "dft2": Phi = x.xi, whose product
  is a 2D inverse FFT (``dft2_closed_form``).  x.xi = (p.(k - n/2))/n is
  reduced modulo 1 exactly in integers; the square-root term (< 0.2 n) is
  formed in FP64.

Layout of the factors: ``bfinputs.quad.QuadFactors``.
"""
from __future__ import annotations

import numpy as np

from bfinputs.quad import QuadFactors, quad_sizes

from .lowrank import form_us_v, form_usv, randomized_sampling

KINDS = ("fio2", "dft2")


# ---------------------------------------------------------------- ordering

def morton(p1, p2, bits: int) -> np.ndarray:
    """Morton index of grid point (p1, p2), coordinates of ``bits`` bits."""
    p1 = np.asarray(p1, dtype=np.int64)
    p2 = np.asarray(p2, dtype=np.int64)
    idx = np.zeros(np.broadcast(p1, p2).shape, dtype=np.int64)
    for b in range(bits):
        idx |= (((p1 >> b) & 1) << (2 * b + 1)) | (((p2 >> b) & 1) << (2 * b))
    return idx


def demorton(idx, bits: int):
    """Grid coordinates (p1, p2) of Morton index ``idx``."""
    idx = np.asarray(idx, dtype=np.int64)
    p1 = np.zeros_like(idx)
    p2 = np.zeros_like(idx)
    for b in range(bits):
        p1 |= ((idx >> (2 * b + 1)) & 1) << b
        p2 |= ((idx >> (2 * b)) & 1) << b
    return p1, p2


def _bits(n: int) -> int:
    b = n.bit_length() - 1
    if (1 << b) != n:
        raise ValueError("the grid side must be a power of 2")
    return b


# ---------------------------------------------------------------- kernel

def phase_frac(rows, cols, n: int, kind: str = "fio2") -> np.ndarray:
    """frac(Phi(x_rows, xi_cols)) for Morton indices (broadcast)."""
    if kind not in KINDS:
        raise ValueError(f"unknown kernel kind {kind!r}")
    b = _bits(n)
    p1, p2 = demorton(rows, b)
    k1, k2 = demorton(cols, b)
    xi1, xi2 = k1 - n // 2, k2 - n // 2
    f = np.mod(p1 * xi1 + p2 * xi2, n).astype(np.float64) / n
    if kind == "fio2":
        x1 = p1.astype(np.float64) / n
        x2 = p2.astype(np.float64) / n
        c1 = (2.0 + np.sin(2 * np.pi * x1) * np.sin(2 * np.pi * x2)) / 16.0
        c2 = (2.0 + np.cos(2 * np.pi * x1) * np.cos(2 * np.pi * x2)) / 16.0
        f = f + np.sqrt((c1 * xi1) ** 2 + (c2 * xi2) ** 2)
    return f - np.floor(f)


def entries(rows, cols, n: int, kind: str = "fio2") -> np.ndarray:
    """K[rows][:, cols] (Morton indices) as complex128."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    ang = 2.0 * np.pi * phase_frac(rows[:, None], cols[None, :], n, kind)
    return np.cos(ang) + 1j * np.sin(ang)


def dense_apply(g: np.ndarray, n: int, kind: str = "fio2", rows=None, chunk_entries: int = 1 << 22) -> np.ndarray:
    """u = K g directly, O(N^2); g is (N,) or (N, nrhs) in Morton order."""
    N = n * n
    g = np.asarray(g, dtype=np.complex128)
    squeeze = g.ndim == 1
    Gm = g.reshape(N, -1)
    rows = np.arange(N) if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.empty((rows.size, Gm.shape[1]), dtype=np.complex128)
    step = max(1, chunk_entries // N)
    cols = np.arange(N)
    for s in range(0, rows.size, step):
        out[s:s + step] = entries(rows[s:s + step], cols, n, kind) @ Gm
    return out[:, 0] if squeeze else out


def dft2_closed_form(g: np.ndarray, n: int) -> np.ndarray:
    """K g for kind "dft2" by the FFT: K_{pk} = (-1)^{p_1 + p_2} e^{2 pi i p.k/n},
    so on the grid (K g)[p] = (-1)^{p_1+p_2} n^2 ifft2(g)[p]; in and out in
    Morton order."""
    b = _bits(n)
    g = np.asarray(g, dtype=np.complex128)
    k1, k2 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    grid = g[morton(k1, k2, b)]                      # grid[k1, k2] (, nrhs)
    y = n * n * np.fft.ifft2(grid, axes=(0, 1))
    sign = np.where((k1 + k2) % 2 == 0, 1.0, -1.0)
    y = y * sign.reshape(sign.shape + (1,) * (g.ndim - 1))
    out = np.empty_like(g)
    out[morton(k1, k2, b)] = y
    return out


# ---------------------------------------------------------------- construction

def middle_block(n: int, L: int, r: int, i: int, j: int, kind: str = "fio2", seed: int = 0, q: int = 3):
    """Rank-r_h approximation K^h_{i,j} ~ U S V^* (Sec. 3.1, entries given),
    plus the relative error on a fresh sample of the block."""
    N = n * n
    m = 1 << (2 * (L // 2))                          # 4^h nodes at the middle level
    nb = N // m
    rh = min(r, nb)
    rng = np.random.default_rng([int(seed), 2, int(i), int(j)])
    r0, c0 = i * nb, j * nb

    def entry(I, J):
        return entries(r0 + np.asarray(I), c0 + np.asarray(J), n, kind)

    U0, s, V0 = randomized_sampling(entry, nb, nb, rh, rng, q=q)
    U, S, V = form_usv(U0, s, V0, rh)
    I = np.sort(rng.choice(nb, size=min(rh * q, nb), replace=False))
    J = np.sort(rng.choice(nb, size=min(rh * q, nb), replace=False))
    Z = entry(I, J)
    approx = (U[I] * S[None, :]) @ V[J].conj().T
    res = float(np.linalg.norm(Z - approx) / max(np.linalg.norm(Z), 1e-300))
    return U, S, V, res


def recursive_factorize(blocks: list, level: int, node: int, L: int, ranks: dict,
                        leaf_out: np.ndarray, trans_out: list, stats: dict) -> None:
    """Factor the row node ``node``'s blocks U^level_{node, j} (j over the
    column tree's level L-level, in order) down to the leaves (Sec. 3.2.1 with
    four children).  G^l_{i'',j'} goes to trans_out[l - L/2][i'' 4^{L-l-1} + j'],
    U^L_{a,0} to leaf_out[a]."""
    if level == L:
        leaf_out[node] = blocks[0]
        return
    quarter = blocks[0].shape[0] // 4
    nj = len(blocks) // 4
    rk = ranks[level + 1]
    for c in range(4):
        child = 4 * node + c
        new_blocks = []
        for jp in range(nj):
            Z = np.hstack([blocks[4 * jp + cc][c * quarter:(c + 1) * quarter] for cc in range(4)])
            Uf, s, Vh = np.linalg.svd(Z, full_matrices=False)
            k = min(rk, s.size)
            if s.size > k and s[0] > 0:
                stats["eps_rec"] = max(stats["eps_rec"], float(s[k] / s[0]))
            Unew, Gblk = form_us_v(Uf[:, :k], s[:k], Vh[:k].conj().T, rk)
            trans_out[level - L // 2][child * nj + jp] = Gblk
            new_blocks.append(Unew)
        recursive_factorize(new_blocks, level + 1, child, L, ranks, leaf_out, trans_out, stats)


def construct(n: int, L: int, r: int, kind: str = "fio2", seed: int = 0, q: int = 3) -> QuadFactors:
    """2D butterfly factorization of the N x N (N = n^2) matrix of ``kind`` on
    quadtrees of depth L (Sec. 3 with four children per node), FP64."""
    N = n * n
    if N % (1 << (2 * L)):
        raise ValueError("N must be a multiple of 4^L")
    n0 = N >> (2 * L)
    s = quad_sizes(L, n0, r)
    h, m, nb, rk = s["h"], s["m"], s["nblocks"], s["ranks"]
    VL = np.zeros((nb, n0, rk[L]), dtype=np.complex128)
    UL = np.zeros((nb, n0, rk[L]), dtype=np.complex128)
    H = [np.zeros((nb, rk[lv + 1], 4 * rk[lv]), dtype=np.complex128) for lv in range(h, L)]
    G = [np.zeros((nb, rk[lv + 1], 4 * rk[lv]), dtype=np.complex128) for lv in range(h, L)]
    S = np.zeros((m, m, rk[h]), dtype=np.float64)
    stats = {"eps_rec": 0.0, "eps_mid": 0.0}
    vparts = {}
    for i in range(m):                               # U side, one row node at a time (Sec. 3.3)
        blocks = []
        for j in range(m):
            U, Sd, V, res = middle_block(n, L, r, i, j, kind, seed, q)
            stats["eps_mid"] = max(stats["eps_mid"], res)
            S[i, j] = Sd
            blocks.append(U)
            vparts[(i, j)] = V
        recursive_factorize(blocks, h, i, L, rk, UL, G, stats)
    for j in range(m):                               # V side: V^h_j = [V^h_{j,0} ... V^h_{j,m-1}]
        recursive_factorize([vparts.pop((i, j)) for i in range(m)], h, j, L, rk, VL, H, stats)
    meta = {"source": "construct", "kind": kind, "seed": seed, "q": q, "n": n,
            "eps_rec": stats["eps_rec"], "eps_mid": stats["eps_mid"],
            "eps": max(stats["eps_rec"], stats["eps_mid"], 1e-13)}
    return QuadFactors(L, n0, r, VL, H, S, G, UL, meta).validate()


def block_singular_values(n: int, L: int, level: int, i: int, j: int, kind: str = "fio2") -> np.ndarray:
    """Singular values of K^l_{i,j}: row node i at level l, column node j at
    level L - l (the complementary low-rank blocks of Sec. 1.1)."""
    N = n * n
    nr, nc = N >> (2 * level), N >> (2 * (L - level))
    return np.linalg.svd(entries(i * nr + np.arange(nr), j * nc + np.arange(nc), n, kind), compute_uv=False)


# ---------------------------------------------------------------- apply

def _cols(x: np.ndarray, N: int):
    x = np.asarray(x, dtype=np.complex128)
    if x.shape[0] != N:
        raise ValueError("vectors must have N rows")
    return x.reshape(N, -1), x.ndim == 1


def bf_apply(F: QuadFactors, g: np.ndarray) -> np.ndarray:
    """u = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^* g, factor by
    factor.  t^{(l)}[j, i] (column node j at level l, row node i at level L-l)
    and w^{(l)}[i, j] (row node i at level l, column node j at level L-l) are
    the r_l-vectors the factors act on."""
    s = F.sizes
    L, h, n0, rk = F.L, s["h"], F.n0, s["ranks"]
    X, squeeze = _cols(g, F.N)
    k = X.shape[1]
    # (V^L)^*: one leaf at a time.
    t = np.einsum("bpx,bpk->bxk", F.VL.conj(), X.reshape(-1, n0, k))[:, None]      # [j, 0, x, k]
    # (H^l)^*, l = L-1 .. h: [t_{j,4i'} .. t_{j,4i'+3}] = sum_c (H^l_{4j+c,i'})^* t^{(l+1)}_{4j+c,i'}
    for lv in range(L - 1, h - 1, -1):
        nj, nip = 1 << (2 * lv), 1 << (2 * (L - lv - 1))
        Hl = F.H[lv - h].reshape(nj, 4, nip, rk[lv + 1], 4 * rk[lv])
        tn = t.reshape(nj, 4, nip, rk[lv + 1], k)
        stack = np.einsum("jciab,jciak->jibk", Hl.conj(), tn)                   # [j, i', 4 r_l, k]
        t = stack.reshape(nj, nip * 4, rk[lv], k)
    # M^h: w^{(h)}_{i,j} = S^h_{i,j} t^{(h)}_{j,i}
    w = F.S[:, :, :, None] * t.transpose(1, 0, 2, 3)
    # G^l, l = h .. L-1: w^{(l+1)}_{4i+c,j'} = G^l_{4i+c,j'} [w_{i,4j'} .. w_{i,4j'+3}]
    for lv in range(h, L):
        ni, njp = 1 << (2 * lv), 1 << (2 * (L - lv - 1))
        Gl = F.G[lv - h].reshape(ni, 4, njp, rk[lv + 1], 4 * rk[lv])
        stack = w.reshape(ni, njp, 4 * rk[lv], k)
        w = np.einsum("icjab,ijbk->icjak", Gl, stack).reshape(ni * 4, njp, rk[lv + 1], k)
    u = np.einsum("apx,axk->apk", F.UL, w[:, 0]).reshape(F.N, k)
    return u[:, 0] if squeeze else u


def bf_adjoint(F: QuadFactors, f: np.ndarray) -> np.ndarray:
    """K^* f = V^L H^{L-1} ... H^h (M^h)^* (G^h)^* ... (G^{L-1})^* (U^L)^* f."""
    s = F.sizes
    L, h, n0, rk = F.L, s["h"], F.n0, s["ranks"]
    X, squeeze = _cols(f, F.N)
    k = X.shape[1]
    w = np.einsum("apx,apk->axk", F.UL.conj(), X.reshape(-1, n0, k))[:, None]       # [a, 0, x, k]
    for lv in range(L - 1, h - 1, -1):
        ni, njp = 1 << (2 * lv), 1 << (2 * (L - lv - 1))
        Gl = F.G[lv - h].reshape(ni, 4, njp, rk[lv + 1], 4 * rk[lv])
        wn = w.reshape(ni, 4, njp, rk[lv + 1], k)
        w = np.einsum("icjab,icjak->ijbk", Gl.conj(), wn).reshape(ni, njp * 4, rk[lv], k)
    t = (F.S[:, :, :, None] * w).transpose(1, 0, 2, 3)
    for lv in range(h, L):
        nj, nip = 1 << (2 * lv), 1 << (2 * (L - lv - 1))
        Hl = F.H[lv - h].reshape(nj, 4, nip, rk[lv + 1], 4 * rk[lv])
        stack = t.reshape(nj, nip, 4 * rk[lv], k)
        t = np.einsum("jciab,jibk->jciak", Hl, stack).reshape(nj * 4, nip, rk[lv + 1], k)
    g = np.einsum("bpx,bxk->bpk", F.VL, t[:, 0]).reshape(F.N, k)
    return g[:, 0] if squeeze else g
