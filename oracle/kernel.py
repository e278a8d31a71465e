"""Entry function and dense product of the 1D examples (oracle, test infrastructure only).

The matrices are K_{jk} = exp(2 pi i Phi(x_j, xi_k)) with the points of
Eq. (1D-xandxi) written 0-based: x_j = j/N and xi_k = k - N/2 for
j, k = 0..N-1 (the paper's 1-based (i-1)/N and j-1-N/2 are the same points).

* ``"fio"``: Example 1, Eq. (1D-FIO-kernal): Phi = x*xi + c(x)|xi|,
  c(x) = (2 + sin(2 pi x))/8.
* ``"dft"``: Phi = x*xi, the Fourier matrix of Sec. 1.1 up to the column shift
  xi = k - N/2, so K_{jk} = (-1)^j exp(2 pi i j k / N) and K g = (-1)^j N ifft(g)_j.

Phase reduction.  At N = 2^20 the phase reaches |Phi| ~ 2e5, and an FP64
product c(x)*|xi| carries a rounding error of ~1e-11 that differs from entry to
entry, i.e. full-rank noise far above the truncation level of a rank-16 block.
So frac(Phi) is formed without that rounding:
  x*xi = j*(k - N/2)/N  is reduced exactly in integers;
  c*|xi| = c_hi*|xi| + c_lo*|xi| with c_hi holding the top 30 fractional bits of
  c, so c_hi*|xi| (<= 49 significant bits) is exact and its fractional part is
  exact; c_lo*|xi| < 2^-12 is added with an error below 1e-19.
The remaining error is that of c(x_j) itself (one value per row: a rank-one
perturbation of the phase, which does not disturb the complementary low-rank
structure) and the final cos/sin of 2 pi * frac, about 1e-15.
"""
from __future__ import annotations

import numpy as np

KINDS = ("fio", "dft")


def c_of_x(j: np.ndarray, N: int) -> np.ndarray:
    """c(x_j) = (2 + sin(2 pi x_j))/8 with x_j = j/N (Example 1, Eq. 1D-FIO-kernal)."""
    x = np.asarray(j, dtype=np.float64) / N
    return (2.0 + np.sin(2.0 * np.pi * x)) / 8.0


def phase_frac(j, k, N: int, kind: str = "fio") -> np.ndarray:
    """frac(Phi(x_j, xi_k)) in [0, 1), broadcast over integer arrays j and k.

    Phi as in the module docstring; the reduction modulo 1 is exact up to the
    final FP64 additions (see the module docstring for the error budget).
    """
    if kind not in KINDS:
        raise ValueError(f"unknown kernel kind {kind!r}")
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    xi = k - N // 2
    # x*xi = j*xi/N: exact integer reduction modulo N.
    a = np.mod(j * xi, N)
    f = a.astype(np.float64) / N
    if kind == "fio":
        c = c_of_x(j, N)
        c_hi = np.round(c * 2.0**30) / 2.0**30
        c_lo = c - c_hi
        axi = np.abs(xi).astype(np.float64)
        p_hi = c_hi * axi                    # exact: <= 29 + 20 significant bits
        f = f + (p_hi - np.floor(p_hi)) + c_lo * axi
    return f - np.floor(f)


def entries(rows, cols, N: int, kind: str = "fio") -> np.ndarray:
    """The submatrix K[rows][:, cols] as complex128 (rows, cols: 1D integer arrays)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    f = phase_frac(rows[:, None], cols[None, :], N, kind)
    ang = 2.0 * np.pi * f
    return np.cos(ang) + 1j * np.sin(ang)


def dense_matrix(N: int, kind: str = "fio") -> np.ndarray:
    """The full N x N matrix K (small N only)."""
    idx = np.arange(N)
    return entries(idx, idx, N, kind)


def dense_apply(g: np.ndarray, N: int, kind: str = "fio", rows=None,
                chunk_entries: int = 1 << 24) -> np.ndarray:
    """u = K g evaluated directly, O(N^2) (the direct evaluation T_d of Sec. 4).

    ``g`` is (N,) or (N, nrhs).  ``rows`` selects the output rows (default:
    all); K is formed in row chunks and never held whole.
    """
    g = np.asarray(g, dtype=np.complex128)
    squeeze = g.ndim == 1
    G = g.reshape(N, -1)
    rows = np.arange(N) if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.empty((rows.size, G.shape[1]), dtype=np.complex128)
    step = max(1, chunk_entries // N)
    cols = np.arange(N)
    for s in range(0, rows.size, step):
        blk = entries(rows[s:s + step], cols, N, kind)
        out[s:s + step] = blk @ G
    return out[:, 0] if squeeze else out


def dft_closed_form(g: np.ndarray, N: int) -> np.ndarray:
    """K g for kind "dft" by the FFT: K_{jk} = (-1)^j e^{2 pi i jk/N}, so
    (K g)_j = (-1)^j * N * ifft(g)_j (Sec. 1.1, Fourier matrix)."""
    g = np.asarray(g, dtype=np.complex128)
    sign = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    y = N * np.fft.ifft(g, axis=0)
    return (sign.reshape((N,) + (1,) * (g.ndim - 1))) * y


def rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """Relative 2-norm error ||a - b|| / ||b|| over all entries (the epsilon^a
    measure of Sec. 4 when a, b are the sampled rows of u^a and u^d)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))
