"""Butterfly factorization from fast applies, on the device (Sec. 3.1, first
case; Sec. 2.1; Sec. 3.2).

The matrix is known only through products with K and K^* -- typically this
library's own apply of a factorization composed with other fast operators:
Example 3 (Sec. 4) factorizes K F K from two applies of K and an FFT.  All m^2
middle-level blocks K^h_{i,j} are served by 2 m (r + p) products with block-
diagonal Gaussian matrices (C: K_ij C_jj in rows of node i of slab j; R:
K_ij^* R_ii in rows of node j of slab i), which go through the black box as
batches of vectors (the tensor-core path of `bf_apply` for m (r + p) >= 32).
The per-block randomized SVDs (Sec. 2.1) and the recursive factorization of
U^h and V^h (Sec. 3.2, all 2^L stacks of a level at once) are batched FP64
decompositions on the device (torch.linalg).

Readings:
* Sec. 2.1's step 2 takes the first r columns of Q of a pivoted QR of each
  sketch; here the range basis is the sketch's r leading left singular
  vectors (batched pivoted QR is not available on the device).  Both are
  orthonormal bases of a dominant r-dimensional range of the same sketch.
* Step 3's middle matrix is formed from the products already taken:
  M = pinv(R_ii^* Q_col) (W_ij^* Q_row), since W_ij^* = R_ii^* K_ij.
* p = 5 (Sec. 2.1, Sec. 4), capped at the block size; the Gaussian blocks are
  ``bfinputs.sketch_blocks`` (seeded, drawn on the host).

Two ways to take the decompositions (``method``):
* "svd" (default): batched SVDs of the tall sketches and stacks.
* "gram": the same bases from the small Hermitian Gram matrices -- the
  leading eigenvectors V_r of Z^* Z (k x k or 2r x 2r, batched eigh) give
  U_0 Sigma_0 = Z V_r and V_0^* = V_r^* directly, and the sketch's range basis
  is Z V_r Lambda_r^{-1/2} re-orthonormalized once; only batched matrix
  products touch the tall matrices.  Forming Z^* Z squares the conditioning,
  so directions below 1e-7 of the largest singular value are dropped (the
  noise floor of FP32 products anyway): this form's accuracy bottoms out near
  1e-7 where "svd" reaches roundoff.  Batched SVDs of many tall complex
  matrices run one matrix at a time in the device libraries, small batched
  eigensolves do not, so this is the form meant for large N.
"""
from __future__ import annotations

import numpy as np

from bfinputs.factors import ButterflyFactors, tree_sizes
from bfinputs.workloads import sketch_blocks

from . import capi

OVERSAMPLE = 5
SIGMA_TOL = 1e-14
GRAM_TOL = 1e-14


def _pad_last(x, size: int):
    import torch
    if x.shape[-1] == size:
        return x
    pad = torch.zeros(x.shape[:-1] + (size - x.shape[-1],), dtype=x.dtype, device=x.device)
    return torch.cat([x, pad], dim=-1)


def _top_eig(Z, r: int):
    """Leading r eigenpairs (descending) of Z^* Z for a batch of tall Z."""
    import torch
    lam, V = torch.linalg.eigh(Z.conj().transpose(-1, -2) @ Z)
    lam = torch.flip(lam, dims=[-1])[..., :r].clamp_min(0.0)
    V = torch.flip(V, dims=[-1])[..., :r]
    return lam, V


def _range_basis(Z, r: int, method: str):
    """Orthonormal basis of the dominant r-dimensional range of each Z (Sec. 2.1, step 2)."""
    import torch
    if method == "svd":
        return torch.linalg.svd(Z, full_matrices=False)[0][..., :r]
    lam, V = _top_eig(Z, r)
    # directions below GRAM_TOL of the largest eigenvalue (singular-value ratio
    # 1e-7, the noise floor of FP32 products) are dropped: zero columns
    keep = lam > GRAM_TOL * lam[..., :1]
    scale = torch.where(keep, torch.rsqrt(torch.where(keep, lam, torch.ones_like(lam))), torch.zeros_like(lam))
    Q1 = (Z @ V) * scale[..., None, :].to(Z.dtype)
    lam2, V2 = torch.linalg.eigh(Q1.conj().transpose(-1, -2) @ Q1)          # one re-orthonormalization:
    keep2 = lam2 > 0.5                                                        # ~1 for kept, ~0 for dropped
    scale2 = torch.where(keep2, torch.rsqrt(torch.where(keep2, lam2, torch.ones_like(lam2))), torch.zeros_like(lam2))
    return Q1 @ (V2 * scale2[..., None, :].to(Z.dtype))


def _recursive(X, L: int, r: int, method: str = "svd"):
    """Sec. 3.2 on all nodes at once.  X[i, j] = U^h_{i,j} (rows of row node i,
    one entry per column node j); returns the leaf blocks U^L_{a,0} and the
    transfer blocks G^l in canonical order (block (2i + c) 2^{L-l-1} + j')."""
    import torch
    trans = []
    h = L // 2
    for _ in range(h, L):
        ni, nj, rows, _ = X.shape
        Z = torch.cat([X[:, 0::2], X[:, 1::2]], dim=-1)               # [U_{i,2j'}  U_{i,2j'+1}]
        half = rows // 2
        Z = Z.reshape(ni, nj // 2, 2, half, 2 * r)                   # top (c = 0) and bottom (c = 1) halves
        kk = min(r, half, 2 * r)
        if method == "svd":
            U0, s, Vh = torch.linalg.svd(Z, full_matrices=False)
            Unew = _pad_last(U0[..., :kk] * s[..., None, :kk], r)    # U^{l+1} = U_0 Sigma_0
            Gb = Vh[..., :kk, :]                                      # G^l = V_0^*
        else:
            _, V = _top_eig(Z, kk)
            Unew = _pad_last(Z @ V, r)                                # Z V_r = U_0 Sigma_0
            Gb = V.conj().transpose(-1, -2)
        if kk < r:
            Gb = torch.cat([Gb, torch.zeros(Gb.shape[:-2] + (r - kk, 2 * r), dtype=Gb.dtype, device=Gb.device)],
                           dim=-2)
        trans.append(Gb.permute(0, 2, 1, 3, 4).reshape(ni * 2 * (nj // 2), r, 2 * r))
        X = Unew.permute(0, 2, 1, 3, 4).reshape(ni * 2, nj // 2, half, r)
    return X[:, 0], trans


def construct_from_applies(apply, apply_adj, N: int, L: int, r: int, p: int = OVERSAMPLE, seed: int = 0,
                           device="cuda", method: str = "svd") -> ButterflyFactors:
    """Factors of the N x N matrix given by ``apply(X)`` = rows of X times K^T,
    i.e. K applied to each row of X ((nvec, N) complex tensors on ``device``,
    the layout of `bf_apply`), and ``apply_adj`` likewise for K^*.  Returns the
    factors in canonical layout (complex128 host arrays), ready for
    `bf_plan_create`.  ``method``: "svd" or "gram" (see the module docstring)."""
    import torch
    if method not in ("svd", "gram"):
        raise ValueError("method must be 'svd' or 'gram'")
    if N % (1 << L) or L % 2:
        raise ValueError("N must be a multiple of 2^L with L even")
    n0 = N >> L
    sz = tree_sizes(L, n0, r)
    h, m = sz["h"], sz["m"]
    nb = N // m
    k = min(r + p, nb)
    rk = min(r, nb)
    cdt = torch.complex128
    Cb, Rb = (torch.from_numpy(a).to(device) for a in sketch_blocks(N, L, r, p, seed))   # (m, nb, k)
    idx = torch.arange(m, device=device)
    C = torch.zeros((m, k, m, nb), dtype=cdt, device=device)
    C[idx, :, idx, :] = Cb.transpose(1, 2)                   # vector (j, c) is C_jj[:, c] on node j
    R = torch.zeros((m, k, m, nb), dtype=cdt, device=device)
    R[idx, :, idx, :] = Rb.transpose(1, 2)
    Y = apply(C.reshape(m * k, N)).to(cdt).reshape(m, k, m, nb)        # Y[j, c, i, :] = (K_ij C_jj)[:, c]
    W = apply_adj(R.reshape(m * k, N)).to(cdt).reshape(m, k, m, nb)    # W[i, c, j, :] = (K_ij^* R_ii)[:, c]
    Yb = Y.permute(2, 0, 3, 1)                                  # [i, j] = K_ij C_jj      (nb x k)
    Wb = W.permute(0, 2, 3, 1)                                  # [i, j] = K_ij^* R_ii    (nb x k)
    Qc = _range_basis(Yb, rk, method)
    Qr = _range_basis(Wb, rk, method)
    A = Rb.conj().transpose(-1, -2)[:, None] @ Qc               # R_ii^* Q_col
    M = torch.linalg.pinv(A) @ (Wb.conj().transpose(-1, -2) @ Qr)
    UM, s, VMh = torch.linalg.svd(M)
    U0 = Qc @ UM
    V0 = Qr @ VMh.conj().transpose(-1, -2)
    keep = s > SIGMA_TOL * s[..., :1]                           # Eq. lowrankSVD, pseudo-inverse for tiny sigma
    sk = torch.where(keep, s, torch.zeros_like(s))
    U = _pad_last(U0 * sk[..., None, :].to(cdt), r)             # U = U_0 Sigma_0
    V = _pad_last(V0 * sk[..., None, :].to(cdt), r)             # V = V_0 Sigma_0
    S = _pad_last(torch.where(keep, 1.0 / torch.where(keep, s, torch.ones_like(s)), torch.zeros_like(s)), r)
    UL, G = _recursive(U, L, r, method)                         # U side: X[i, j] = U_ij
    VL, H = _recursive(V.transpose(0, 1), L, r, method)         # V side: X[j, i] = V_ij
    host = lambda t: t.detach().cpu().numpy()
    meta = {"source": "construct_from_applies", "p": p, "seed": seed, "vectors_per_direction": m * k,
            "method": method}
    return ButterflyFactors(L, n0, r, host(VL), [host(t) for t in H], host(S).astype(np.float64),
                            [host(t) for t in G], host(UL), meta).validate()


def plan_black_box(plan):
    """(apply, apply_adj) of a `bf_plan` for `construct_from_applies`: rows of a
    (nvec, N) device tensor through `bf_apply` / `bf_apply_adjoint` in complex64."""
    import torch

    def run(fn, X):
        x = X.to(torch.complex64).contiguous()
        y = torch.empty_like(x)
        fn(plan, x, y)
        return y
    return (lambda X: run(capi.bf_apply, X)), (lambda X: run(capi.bf_apply_adjoint, X))


def fourier_rows(X):
    """F applied to each row: F_{kj} = exp(-2 pi i (k - N/2) j / N) / N (the
    Fourier-integral quadrature of Example 3), F x = fft((-1)^j x) / N."""
    import torch
    N = X.shape[-1]
    sign = 1.0 - 2.0 * (torch.arange(N, device=X.device) % 2)
    return torch.fft.fft(X * sign, dim=-1) / N


def fourier_adjoint_rows(Y):
    """F^* y = (-1)^j ifft(y)_j for each row."""
    import torch
    N = Y.shape[-1]
    sign = 1.0 - 2.0 * (torch.arange(N, device=Y.device) % 2)
    return torch.fft.ifft(Y, dim=-1) * sign


# --------------------------------------------------------------------------
# Analytic 1D kernels at large N: sketches by entry evaluation, chunked passes
# --------------------------------------------------------------------------
KERNEL_KINDS = ("fio", "dft")
EPS_FLOOR = 1e-7          # FP32 sketch products: the construction's noise floor


def c_fixed_point(kind: str, N: int):
    """c_j 2^64 as int64 bit patterns for K = exp(2 pi i (x xi + c(x)|xi|)):
    Example 1's c(x) = (2 + sin 2 pi x)/8 at x_j = j/N (Eq. 1D-FIO-kernal), or
    None for the Fourier matrix (c = 0).  Exact: an FP64 c in [2^-12, 1) times
    2^64 is an integer."""
    if kind == "dft":
        return None
    if kind != "fio":
        raise ValueError(f"unknown kernel kind {kind!r}")
    c = (2.0 + np.sin(2.0 * np.pi * (np.arange(N, dtype=np.float64) / N))) / 8.0
    mant, ex = np.frexp(c)                                    # c = mant 2^ex, mant in [0.5, 1)
    M = np.ldexp(mant, 53).astype(np.uint64)                  # 53-bit integer mantissa, exact
    out = M << (ex + 11).astype(np.uint64)                    # c 2^64 = M 2^(ex + 11), ex in [-2, -1]
    return out.view(np.int64)


def _eigh(A):
    """Batched Hermitian eigendecomposition (ascending); if the device solver
    reports a batch element that did not converge, the batch is solved on the
    host (LAPACK) instead."""
    import torch
    try:
        return torch.linalg.eigh(A)
    except RuntimeError:
        lam, V = torch.linalg.eigh(A.cpu())
        return lam.to(A.device), V.to(A.device)


def _gram_basis(Z, rk: int):
    """For each tall Z (batched): the k x rk coefficients T with Z T an
    orthonormal basis of Z's dominant rk-dimensional range (Sec. 2.1, step 2,
    from the Gram matrix: leading eigenvectors scaled by 1/sqrt(eigenvalue),
    one re-orthonormalization), the Gram matrix Z^* Z itself, and the
    normalized tail sqrt(lambda_{rk+1} / lambda_1) (0 if Z has <= rk columns)."""
    import torch
    Gz = Z.conj().transpose(-1, -2) @ Z
    lam, V = _eigh(Gz)
    lam = torch.flip(lam, dims=[-1]).clamp_min(0.0)
    V = torch.flip(V, dims=[-1])
    top = lam[..., :1].clamp_min(1e-300)
    tail = torch.sqrt(lam[..., rk] / top[..., 0]) if lam.shape[-1] > rk else torch.zeros_like(top[..., 0])
    lam, V = lam[..., :rk], V[..., :rk]
    keep = lam > GRAM_TOL * top
    T1 = V * torch.where(keep, torch.rsqrt(torch.where(keep, lam, torch.ones_like(lam))),
                         torch.zeros_like(lam))[..., None, :].to(Z.dtype)
    # re-orthonormalization (the second step of Cholesky QR): Q1^* Q1 = R^* R is
    # close to the identity on the kept columns; dropped columns are zero in T1
    # and get a unit diagonal so that they stay zero in T1 R^{-1}
    Q1 = Z @ T1
    G2 = Q1.conj().transpose(-1, -2) @ Q1
    G2 = G2 + torch.diag_embed((~keep).to(G2.dtype))
    Rc, info = torch.linalg.cholesky_ex(G2, upper=True)
    if bool((info != 0).any()):
        raise RuntimeError("re-orthonormalization: Gram matrix of the range basis is not positive definite")
    T = torch.linalg.solve_triangular(Rc, T1, upper=True, left=False)       # T1 R^{-1}
    return T, Gz, tail


def _recursive_gram(X, r: int):
    """Sec. 3.2 (Gram form) on a chunk of middle-level nodes: X[i, j] (rows of
    node i, one entry per node j of the other tree).  Returns the leaf blocks,
    the transfer blocks of every level (chunk-local canonical order) and the
    largest normalized tail sigma_{r+1} / sigma_1 over the level stacks."""
    import torch
    trans = []
    eps = 0.0
    while X.shape[1] > 1:
        ni, nj, rows, _ = X.shape
        Z = torch.cat([X[:, 0::2], X[:, 1::2]], dim=-1)
        half = rows // 2
        Z = Z.reshape(ni, nj // 2, 2, half, 2 * r)
        kk = min(r, half, 2 * r)
        lam, V = _eigh(Z.conj().transpose(-1, -2) @ Z)
        lam = torch.flip(lam, dims=[-1]).clamp_min(0.0)
        V = torch.flip(V, dims=[-1])[..., :kk]
        if 2 * r > kk:
            tail = torch.sqrt(lam[..., kk] / lam[..., 0].clamp_min(1e-300))
            eps = max(eps, float(tail.max()))
        Unew = _pad_last(Z @ V, r)                                    # Z V_r = U_0 Sigma_0
        Gb = V.conj().transpose(-1, -2)                               # V_0^*
        if kk < r:
            Gb = torch.cat([Gb, torch.zeros(Gb.shape[:-2] + (r - kk, 2 * r), dtype=Gb.dtype, device=Gb.device)],
                           dim=-2)
        trans.append(Gb.permute(0, 2, 1, 3, 4).reshape(ni * 2 * (nj // 2), r, 2 * r))
        X = Unew.permute(0, 2, 1, 3, 4).reshape(ni * 2, nj // 2, half, r)
    return X[:, 0], trans, eps


def construct_kernel_1d(kind: str, N: int, L: int, r: int, p: int = OVERSAMPLE, seed: int = 0, chunk: int = 16,
                        device="cuda", out_dtype=np.complex64, stream=None) -> ButterflyFactors:
    """Butterfly factorization of K(x_j, xi_k) = exp(2 pi i (x_j xi_k + c(x_j)|xi_k|))
    (``kind`` "fio": Example 1; "dft": c = 0, the Fourier matrix) from sketch
    products (Sec. 3.1, first case; Sec. 2.1; Sec. 3.2), at sizes where no
    dense K and no whole-level array fits: the products are formed by
    `bf_sketch_products` (entries generated on the GPU) and the work runs in
    two passes over chunks of ``chunk`` middle-level nodes.

    U pass, row nodes I: K_ij C_jj for i in I (rows of I, every column node j)
    and K_ij^* R_ii (every column); per block the Gram-form range bases
    Qc = Y Tc, Qr = W Tr, the middle matrix M = pinv(R_ii^* Qc)(W^* Qr) and its
    SVD U_M Sigma V_M^* (Eq. lowrankSVD); U_ij = Y (Tc U_M Sigma), the recursive
    factorization of the U side under I.  Only the k x r coefficients
    Z_ij = Tr V_M Sigma and S_ij = Sigma^{-1} are kept.  V pass, column nodes
    J: K_ij^* R_ii for j in J again (the same products, bit for bit: each
    output is one fixed-order sum), V_ij = W Z_ij -- the middle level's own
    SVD, not a second one -- and the recursive factorization of the V side.
    Memory is O(chunk N k) on the device; factors go to the host per chunk.

    Returns factors (``out_dtype`` host arrays) whose ``meta`` holds the phase
    timings and the construction's epsilon = max(eps_mid, eps_rec, EPS_FLOOR):
    eps_mid the largest normalized (r+1)-th singular value of a middle-block
    sketch, eps_rec the largest normalized tail of a recursive stack."""
    import time

    import torch
    if kind not in KERNEL_KINDS:
        raise ValueError(f"kind must be one of {KERNEL_KINDS}")
    if N & (N - 1) or N % (1 << L) or L % 2:
        raise ValueError("N must be a power of two, a multiple of 2^L, L even")
    log2N = N.bit_length() - 1
    n0 = N >> L
    h = L // 2
    m = 1 << h
    nb = N // m
    k = min(r + p, nb)
    rk = min(r, nb)
    chunk = max(1, min(chunk, m))
    cdt = torch.complex128
    t = {"sketch_s": 0.0, "middle_s": 0.0, "recursive_s": 0.0, "host_s": 0.0}
    on_gpu = torch.device(device).type == "cuda"
    sync = torch.cuda.synchronize if on_gpu else (lambda: None)
    t0 = time.perf_counter()
    Cb, Rb = sketch_blocks(N, L, r, p, seed)                     # (m, nb, k) complex128, host
    C32 = torch.from_numpy(Cb.astype(np.complex64)).to(device)
    R32 = torch.from_numpy(Rb.astype(np.complex64)).to(device)
    # the exact inputs of the sketch products, for R_ii^* K_ij = W^*: the
    # complex64-rounded blocks the products used
    R64 = R32.to(cdt)
    del Cb, Rb
    cf = c_fixed_point(kind, N)
    cfix = None if cf is None else torch.from_numpy(cf).to(device)
    t["inputs_s"] = time.perf_counter() - t0
    VL = np.empty((1 << L, n0, r), out_dtype)
    UL = np.empty((1 << L, n0, r), out_dtype)
    H = [np.empty((1 << L, r, 2 * r), out_dtype) for _ in range(h)]
    G = [np.empty((1 << L, r, 2 * r), out_dtype) for _ in range(h)]
    S = np.empty((m, m, r), np.float64)
    Zc = torch.empty((m, m, k, r), dtype=cdt, device=device)    # V_ij = W_ij Zc[i, j]
    eps_mid = eps_rec = 0.0
    cast = lambda x: x.detach().cpu().numpy().astype(out_dtype, copy=False)

    def sketch(blocks, node0, lo, hi, adjoint):
        out = torch.empty((blocks.shape[0], k, hi - lo), dtype=torch.complex64, device=device)
        capi.bf_sketch_products(log2N, nb, blocks, out, lo, hi, node0=node0, adjoint=adjoint, c_fixed=cfix,
                                stream=stream)
        return out

    # ---- U pass
    for i0 in range(0, m, chunk):
        ci = min(chunk, m - i0)
        a = time.perf_counter()
        Yf = sketch(C32, 0, i0 * nb, (i0 + ci) * nb, False)                 # (m_j, k, ci nb)
        Wf = sketch(R32[i0:i0 + ci].contiguous(), i0, 0, N, True)           # (ci, k, N)
        sync()
        b = time.perf_counter()
        Y = Yf.reshape(m, k, ci, nb).permute(2, 0, 3, 1).to(cdt)           # [i, j] = K_ij C_jj  (nb x k)
        del Yf
        W = Wf.reshape(ci, k, m, nb).permute(0, 2, 3, 1).to(cdt)           # [i, j] = K_ij^* R_ii (nb x k)
        del Wf
        Tc, _, tail_c = _gram_basis(Y, rk)
        Tr, Gw, tail_r = _gram_basis(W, rk)
        eps_mid = max(eps_mid, float(tail_c.max()), float(tail_r.max()))
        RY = R64[i0:i0 + ci, None].conj().transpose(-1, -2) @ Y            # R_ii^* K_ij C_jj   (k x k)
        A = RY @ Tc                                                          # R_ii^* Qc
        M = torch.linalg.pinv(A) @ (Gw @ Tr)                                 # pinv(R^* Qc) (W^* Qr)
        UM, s, VMh = torch.linalg.svd(M)
        keep = s > SIGMA_TOL * s[..., :1]
        sk = torch.where(keep, s, torch.zeros_like(s)).to(cdt)
        Xc = _pad_last((Tc @ UM) * sk[..., None, :], r)                      # U_ij = Y Xc
        Zc[i0:i0 + ci] = _pad_last((Tr @ VMh.conj().transpose(-1, -2)) * sk[..., None, :], r)
        Sblk = _pad_last(torch.where(keep, 1.0 / torch.where(keep, s, torch.ones_like(s)), torch.zeros_like(s)), r)
        U = Y @ Xc                                                           # (ci, m, nb, r)
        del Y, W, RY, A, M, Tc, Tr, Gw
        sync()
        c = time.perf_counter()
        ULc, Gc, e = _recursive_gram(U, r)
        eps_rec = max(eps_rec, e)
        del U
        sync()
        d = time.perf_counter()
        S[i0:i0 + ci] = Sblk.cpu().numpy()
        UL[i0 * m:(i0 + ci) * m] = cast(ULc)
        for lv, blk in enumerate(Gc):
            G[lv][i0 * m:(i0 + ci) * m] = cast(blk)
        del ULc, Gc
        t["sketch_s"] += b - a
        t["middle_s"] += c - b
        t["recursive_s"] += d - c
        t["host_s"] += time.perf_counter() - d
    # ---- V pass
    for j0 in range(0, m, chunk):
        cj = min(chunk, m - j0)
        a = time.perf_counter()
        Wv = sketch(R32, 0, j0 * nb, (j0 + cj) * nb, True)                  # (m_i, k, cj nb)
        sync()
        b = time.perf_counter()
        W = Wv.reshape(m, k, cj, nb).permute(2, 0, 3, 1).to(cdt)           # [j, i] = K_ij^* R_ii
        del Wv
        V = W @ Zc[:, j0:j0 + cj].transpose(0, 1)                            # [j, i] = V_ij (nb x r)
        del W
        sync()
        c = time.perf_counter()
        VLc, Hc, e = _recursive_gram(V, r)
        eps_rec = max(eps_rec, e)
        del V
        sync()
        d = time.perf_counter()
        VL[j0 * m:(j0 + cj) * m] = cast(VLc)
        for lv, blk in enumerate(Hc):
            H[lv][j0 * m:(j0 + cj) * m] = cast(blk)
        del VLc, Hc
        t["sketch_s"] += b - a
        t["middle_s"] += c - b
        t["recursive_s"] += d - c
        t["host_s"] += time.perf_counter() - d
    t["total_s"] = time.perf_counter() - t0
    eps = max(eps_mid, eps_rec, EPS_FLOOR)
    meta = {"source": "construct_kernel_1d", "kind": kind, "p": p, "seed": seed, "chunk": chunk,
            "eps": eps, "eps_mid": eps_mid, "eps_rec": eps_rec, "eps_floor": EPS_FLOOR, "timings": t,
            "sketch_multiply_adds": 3 * N * N * k}
    return ButterflyFactors(L, n0, r, VL, H, S, G, UL, meta).validate()
