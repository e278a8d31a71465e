"""Pins of the oracle's entry function and dense product (no GPU).

Each pin checks the oracle against something other than itself: closed forms
of particular rows and columns of Example 1's kernel, the FFT for the Fourier
matrix, and a 40-digit evaluation of the phase.
"""
import mpmath
import numpy as np
import pytest

from bfinputs import complex_normal
from oracle import kernel as K


def _mp_entry(j, k, N, kind, c_value=None):
    """exp(2 pi i Phi) in 40-digit arithmetic; c(x_j) is either exact or the
    given FP64 value taken exactly."""
    mpmath.mp.dps = 40
    x = mpmath.mpf(j) / N
    xi = mpmath.mpf(k - N // 2)
    phi = x * xi
    if kind == "fio":
        c = mpmath.mpf(c_value) if c_value is not None else (2 + mpmath.sin(2 * mpmath.pi * x)) / 8
        phi += c * abs(xi)
    return complex(mpmath.expj(2 * mpmath.pi * phi))


@pytest.mark.parametrize("N", [64, 4096, 1 << 20])
@pytest.mark.parametrize("kind", ["fio", "dft"])
def test_phase_reduction_is_exact(N, kind):
    """Sec. 4 Eq. (1D-FIO-kernal) with the points of Eq. (1D-xandxi): given
    the FP64 value of c(x_j), every sampled entry agrees with a 40-digit
    evaluation to 4e-15, also at N = 2^20 where |Phi| ~ 2e5 and a plain FP64
    product c*|xi| would be off by ~1e-10 from entry to entry."""
    rng = np.random.default_rng(N)
    j = rng.integers(0, N, 40)
    k = rng.integers(0, N, 40)
    got = np.array([K.entries([a], [b], N, kind)[0, 0] for a, b in zip(j, k)])
    cv = K.c_of_x(j, N)
    ref = np.array([_mp_entry(int(a), int(b), N, kind, float(c) if kind == "fio" else None)
                    for a, b, c in zip(j, k, cv)])
    assert np.max(np.abs(got - ref)) < 4e-15


def test_c_of_x_to_a_few_ulps():
    """c(x) = (2 + sin 2 pi x)/8 of Eq. (1D-FIO-kernal) to a few units in the
    last place; its error is one value per row (a diagonal scaling of the
    phase), which keeps the complementary low-rank structure."""
    N = 1 << 20
    j = np.random.default_rng(1).integers(0, N, 200)
    mpmath.mp.dps = 40
    exact = np.array([float((2 + mpmath.sin(2 * mpmath.pi * mpmath.mpf(int(a)) / N)) / 8) for a in j])
    assert np.max(np.abs(K.c_of_x(j, N) - exact)) <= 2 * np.spacing(0.375)


def test_fio_closed_form_rows_and_column():
    """Example 1 reduces to closed forms on special rows/columns:
    xi = 0 (column N/2): Phi = 0, K = 1;  x = 0: c = 1/4, K = i^|xi|;
    x = 1/4: c = 3/8, Phi = xi/4 + 3|xi|/8."""
    N = 256
    K_ = K.dense_matrix(N, "fio")
    assert np.allclose(K_[:, N // 2], 1.0, atol=1e-14)
    xi = np.arange(N) - N // 2
    assert np.allclose(K_[0], 1j ** np.abs(xi), atol=1e-14)
    ph = xi / 4 + 3 * np.abs(xi) / 8
    assert np.allclose(K_[N // 4], np.exp(2j * np.pi * ph), atol=1e-13)


@pytest.mark.parametrize("N", [16, 256, 2048])
def test_dft_dense_equals_fft(N):
    """Fourier matrix of Sec. 1.1 with xi = k - N/2: K g = (-1)^j N ifft(g)."""
    g = complex_normal((N, 3), seed=1)
    u = K.dense_apply(g, N, "dft")
    ref = K.dft_closed_form(g, N)
    assert K.rel_err(u, ref) < 1e-12


def test_dense_rows_subset_and_chunking():
    N = 512
    g = complex_normal((N,), seed=2)
    full = K.dense_apply(g, N, "fio")
    rows = np.array([0, 5, 17, 300, 511])
    part = K.dense_apply(g, N, "fio", rows=rows, chunk_entries=N * 2)
    assert np.max(np.abs(part - full[rows])) < 1e-12
    assert np.allclose(full, K.dense_matrix(N, "fio") @ g, atol=1e-10)


def test_rel_err_definition():
    """epsilon^a of Sec. 4: sqrt(sum |a - d|^2 / sum |d|^2)."""
    d = np.array([3.0, 4.0j])
    a = d + np.array([0.3, 0.4])
    assert abs(K.rel_err(a, d) - 0.1) < 1e-15
