"""Pins of the rank-r approximations (Sec. 2) against matrices whose SVD is known."""
import numpy as np
import pytest

from oracle import lowrank as LR


def _known_svd(m, n, sig, seed):
    rng = np.random.default_rng(seed)
    k = sig.size
    A = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    B = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    Uq, _ = np.linalg.qr(A)
    Vq, _ = np.linalg.qr(B)
    return (Uq * sig) @ Vq.conj().T


def _entry_of(Z):
    return lambda I, J: Z[np.ix_(np.asarray(I), np.asarray(J))]


@pytest.mark.parametrize("m,n,r", [(200, 150, 5), (64, 64, 12), (40, 300, 8)])
def test_sampling_recovers_exact_rank(m, n, r):
    """A matrix of exact rank r is reproduced to rounding (Sec. 2.2, steps 1-7)."""
    Z = _known_svd(m, n, np.linspace(3.0, 0.5, r), seed=m + n)
    U0, s, V0 = LR.randomized_sampling(_entry_of(Z), m, n, r, np.random.default_rng(0))
    assert np.linalg.norm(Z - (U0 * s) @ V0.conj().T) / np.linalg.norm(Z) < 1e-12
    # U0, V0 orthonormal columns; s matches the true singular values
    assert np.allclose(U0.conj().T @ U0, np.eye(r), atol=1e-12)
    assert np.allclose(V0.conj().T @ V0, np.eye(r), atol=1e-12)
    assert np.allclose(s, np.linspace(3.0, 0.5, r), rtol=1e-10)


def test_sampling_error_near_optimal_on_decaying_spectrum():
    """With geometric singular values the rank-r error is within a small
    factor of the optimal sigma_{r+1} (incoherent singular vectors)."""
    sig = 0.1 ** np.arange(20)
    Z = _known_svd(256, 256, sig, seed=5)
    r = 6
    U0, s, V0 = LR.randomized_sampling(_entry_of(Z), 256, 256, r, np.random.default_rng(1))
    err = np.linalg.norm(Z - (U0 * s) @ V0.conj().T, 2)
    assert err < 10 * sig[r]
    assert err >= 0.99 * sig[r]


def test_sampling_small_block_smaller_than_rank():
    """Blocks with fewer rows/columns than r give rank min(r, m, n)."""
    Z = _known_svd(5, 30, np.array([2.0, 1.0, 0.5, 0.25, 0.125]), seed=3)
    U0, s, V0 = LR.randomized_sampling(_entry_of(Z), 5, 30, 8, np.random.default_rng(2))
    assert U0.shape == (5, 5) and s.size == 5 and V0.shape == (30, 5)
    assert np.linalg.norm(Z - (U0 * s) @ V0.conj().T) < 1e-12


def test_forms_usv_and_us_v():
    """Eq. (lowrankSVD): U S V^* = U0 Sigma0 V0^* with U, V scaled by Sigma0 and
    S = Sigma0^{-1}; Eq. (lowrankSVD3): U V^* with U = U0 Sigma0."""
    Z = _known_svd(30, 20, np.array([4.0, 2.0, 1.0]), seed=9)
    U0, s, V0 = LR.truncated_svd(Z, 3)
    U, S, V = LR.form_usv(U0, s, V0, 5)
    assert U.shape == (30, 5) and V.shape == (20, 5) and S.shape == (5,)
    assert np.allclose((U * S) @ V.conj().T, Z, atol=1e-13)
    assert np.allclose(np.linalg.norm(U, axis=0)[:3], s)          # columns carry sigma
    assert np.allclose(S[:3], 1.0 / s) and np.all(S[3:] == 0)
    Uu, Vh = LR.form_us_v(U0, s, V0, 5)
    assert Uu.shape == (30, 5) and Vh.shape == (5, 20)
    assert np.allclose(Uu @ Vh, Z, atol=1e-13)


def test_form_usv_pseudo_inverse_for_zero_sigma():
    """A zero singular value gives S_k = 0 and zero columns (no division by 0)."""
    U0 = np.eye(4, 2, dtype=complex)
    V0 = np.eye(3, 2, dtype=complex)
    U, S, V = LR.form_usv(U0, np.array([1.0, 0.0]), V0, 2)
    assert np.all(np.isfinite(S)) and S[1] == 0.0
    assert np.all(U[:, 1] == 0) and np.all(V[:, 1] == 0)
