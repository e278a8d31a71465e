"""Workload sizes and seeded random draws (no butterfly arithmetic here).

Workloads follow the paper's Example 1 (1D FIO, Sec. 4) and the sizes the
library is benchmarked at.  Every random array is drawn from a numpy PCG64
stream keyed by (seed, tag), so each array can be regenerated on its own.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from .factors import ButterflyFactors, tree_sizes


@dataclass(frozen=True)
class Config:
    name: str
    L: int
    n0: int
    r: int
    kind: str          # entry function of the oracle construction ("fio" or "dft")
    nrhs: tuple
    seed: int = 0

    @property
    def N(self) -> int:
        return self.n0 << self.L


CONFIGS = {
    # 1D FIO, N = 4096, depth 8 (16 points per leaf), rank 12, one RHS, seed 0.
    "fio_n4096_r12": Config("fio_n4096_r12", L=8, n0=16, r=12, kind="fio", nrhs=(1,)),
    # 1D FIO at N = 2^20, depth 16 (16 points per leaf), rank 16.
    "fio_n1m_r16": Config("fio_n1m_r16", L=16, n0=16, r=16, kind="fio", nrhs=(1, 8, 64, 256)),
    # 1D FIO at N = 2^18, depth 14, rank 16, 32 RHS.
    "fio_n256k_r16": Config("fio_n256k_r16", L=14, n0=16, r=16, kind="fio", nrhs=(32,)),
}


_CHUNK = 1 << 22   # real values per independent stream


def _rng(seed: int, *tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed)] + [int(t) for t in tag])


def _normals(n: int, fdt, seed: int, tag: tuple, scale: float) -> np.ndarray:
    """n i.i.d. N(0, scale^2) reals; chunk c comes from the stream keyed by
    (seed, *tag, c), so the values do not depend on the thread count."""
    out = np.empty(n, dtype=fdt)

    def fill(c):
        part = out[c * _CHUNK:(c + 1) * _CHUNK]
        _rng(seed, *tag, c).standard_normal(out=part, dtype=fdt)
        part *= fdt(scale)

    nchunks = (n + _CHUNK - 1) // _CHUNK
    if nchunks <= 1:
        fill(0)
    else:
        with ThreadPoolExecutor(min(nchunks, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, range(nchunks)))
    return out


def complex_normal(shape, seed: int, tag: int = 0, dtype=np.complex128) -> np.ndarray:
    """I.i.d. standard complex normal entries CN(0, 1): real and imaginary
    parts independent N(0, 1/2)."""
    return _cn(seed, (7919, tag), shape, 1.0, dtype)


def _cn(seed: int, tag: tuple, shape, scale: float, dtype) -> np.ndarray:
    n = int(np.prod(shape))
    fdt = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    x = _normals(2 * n, fdt, seed, tag, scale * np.sqrt(0.5))
    return x.view(np.dtype(dtype)).reshape(shape)


def synthetic_factors(L: int, n0: int, r: int, seed: int = 0,
                      dtype=np.complex64) -> ButterflyFactors:
    """Seeded random factors with the block shapes of a depth-L, leaf-n0,
    rank-r butterfly factorization.

    Entries are i.i.d. complex normal with variances 1/n0 (V^L), 1/(2r) (H, G)
    and 1/r (U^L), and S uniform on [0.5, 1.5]; with these scales every factor
    preserves the expected squared norm of the vector it is applied to.  The
    cost of an apply does not depend on the values, so these stand in for a
    constructed factorization wherever only the shapes matter.
    """
    s = tree_sizes(L, n0, r)
    nb, h, m = s["nblocks"], s["h"], s["m"]
    VL = _cn(seed, (1,), (nb, n0, r), 1.0 / np.sqrt(n0), dtype)
    UL = _cn(seed, (2,), (nb, n0, r), 1.0 / np.sqrt(r), dtype)
    H = [_cn(seed, (3, t), (nb, r, 2 * r), 1.0 / np.sqrt(2 * r), dtype) for t in range(h)]
    G = [_cn(seed, (4, t), (nb, r, 2 * r), 1.0 / np.sqrt(2 * r), dtype) for t in range(h)]
    rdt = np.float32 if np.dtype(dtype) == np.complex64 else np.float64
    S = _rng(seed, 5).uniform(0.5, 1.5, size=(m, m, r)).astype(rdt)
    return ButterflyFactors(L, n0, r, VL, H, S, G, UL,
                            meta={"source": "synthetic", "seed": seed}).validate()


def sketch_blocks(N: int, L: int, r: int, p: int = 5, seed: int = 0):
    """The random Gaussian blocks of a construction from products (Sec. 3.1,
    first case): C_jj and R_ii for the m = 2^{L/2} middle-level nodes, each
    (N/m) x k complex standard normal with k = min(r + p, N/m), drawn from
    streams keyed by (seed, side, node).  Returns (C, R) of shape (m, N/m, k)."""
    m = 1 << (L // 2)
    nb = N // m
    k = min(r + p, nb)
    out = []
    for side in (0, 1):
        blocks = np.empty((m, nb, k), dtype=np.complex128)
        for j in range(m):
            rng = _rng(seed, 77, side, j)
            blocks[j] = (rng.standard_normal((nb, k)) + 1j * rng.standard_normal((nb, k))) / np.sqrt(2.0)
        out.append(blocks)
    return out[0], out[1]


def sample_rows(N: int, count: int = 256, seed: int = 0) -> np.ndarray:
    """A sorted random set of ``count`` distinct rows (the set S of the
    accuracy measure epsilon^a in Sec. 4 has 256 points)."""
    return np.sort(_rng(seed, 31337).choice(N, size=min(count, N), replace=False))


@dataclass(frozen=True)
class BatchMember:
    """One operator of the batched workload: its tree shape, rank, vector
    count and the FIO parameters c(x) = (2 + a sin(2 pi x + phi)) / 8 it stands for."""
    L: int
    n0: int
    r: int
    nrhs: int
    a: float
    phi: float

    @property
    def N(self) -> int:
        return self.n0 << self.L


def batched_workload(count: int = 256, seed: int = 3, min_log2n: int = 10, max_log2n: int = 16,
                     ranks=(8, 12, 16), max_nrhs: int = 32) -> list:
    """The batched workload's operators: N log-uniform over 2^min_log2n ..
    2^max_log2n (the exponent uniform), r uniform over `ranks`, nrhs uniform
    over 1..max_nrhs, a ~ U[0.5, 1], phi ~ U[0, 2 pi).  Trees have even depth:
    leaf 16 when log2 N - 4 is even, else leaf 32 (L = log2 N - 5)."""
    rng = _rng(seed, 0xBA7C)
    out = []
    for _ in range(count):
        e = int(rng.integers(min_log2n, max_log2n + 1))
        n0 = 16 if (e - 4) % 2 == 0 else 32
        L = e - (4 if n0 == 16 else 5)
        r = int(ranks[int(rng.integers(0, len(ranks)))])
        nrhs = int(rng.integers(1, max_nrhs + 1))
        out.append(BatchMember(L, n0, r, nrhs, float(rng.uniform(0.5, 1.0)), float(rng.uniform(0, 2 * np.pi))))
    return out
