"""Pins of the construction from matrix-vector products (Sec. 3.1, first case;
Sec. 2.1; Example 3): exactness at full rank, the Fourier quadrature against
its written-out matrix, agreement in accuracy with the entry-sampling
construction, the DFT through the FFT as the black box, the number of
products, and the composition K F K of Example 3."""
import numpy as np
import pytest

from bfinputs import complex_normal
from oracle import apply as A
from oracle import construct as CS
from oracle import construct_mv as CM
from oracle import kernel as KK
from oracle.kernel import rel_err

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _dense_box(K):
    return (lambda X: K @ X), (lambda X: K.conj().T @ X)


def test_full_rank_construction_is_exact():
    """r = N/m: every middle block is captured whole by r + p >= its size
    random products, so the factorization reproduces K to roundoff."""
    N, L, r = 64, 4, 16
    K = KK.dense_matrix(N, "fio")
    F = CM.construct(*_dense_box(K), N, L, r)
    g = complex_normal((N, 2), seed=1)
    assert rel_err(A.bf_apply(F, g), K @ g) < 1e-12
    assert rel_err(A.bf_adjoint(F, g), K.conj().T @ g) < 1e-12


def test_fourier_quadrature_apply_and_adjoint():
    N = 256
    Fm = CM.fourier_matrix(N)
    x = complex_normal((N, 3), seed=2)
    assert rel_err(CM.fourier_apply(x), Fm @ x) < 1e-13
    assert rel_err(CM.fourier_adjoint(x), Fm.conj().T @ x) < 1e-13


def test_matches_entry_sampling_accuracy_on_the_fio():
    """N = 1024, one point per leaf: for r = 4, 6, 8 the construction from
    products reaches the accuracy of the entry-sampling construction (within
    a factor 3) and improves with r, using m (r + p) products per direction."""
    N, L = 1024, 10
    K = KK.dense_matrix(N, "fio")
    g = complex_normal((N,), seed=3)
    prev = 1.0
    for r in (4, 6, 8):
        Fm = CM.construct(*_dense_box(K), N, L, r)
        Fs = CS.construct(N, L, r, "fio")
        em, es = rel_err(A.bf_apply(Fm, g), K @ g), rel_err(A.bf_apply(Fs, g), K @ g)
        assert em <= 3 * es, (r, em, es)
        assert em < prev / 10
        prev = em
        assert Fm.meta["vectors_per_direction"] == 32 * (r + CM.OVERSAMPLE)


def test_dft_through_the_fft_black_box():
    """The Fourier matrix (Sec. 1.1) given only by the FFT: K g = (-1)^j N
    ifft(g), K^* f = fft((-1)^j f)."""
    N, L = 1024, 10
    sign = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)[:, None]
    app = lambda X: KK.dft_closed_form(X, N)
    adj = lambda X: np.fft.fft(sign * X, axis=0)
    g = complex_normal((N,), seed=4)
    errs = [rel_err(A.bf_apply(CM.construct(app, adj, N, L, r), g), app(g[:, None])[:, 0]) for r in (2, 4)]
    assert errs[1] < 1e-2 and errs[1] < errs[0] / 10


def test_example3_composition_needs_higher_rank():
    """Example 3: K~ = K F K given by two applies of K and one Fourier
    quadrature.  Its factorization improves steadily with r, and at a given r
    it is far less accurate than K's own (the composition's ranks are larger,
    as the paper observes after Table 3)."""
    N, L = 256, 8
    K = KK.dense_matrix(N, "fio")
    Kt = K @ CM.fourier_matrix(N) @ K
    app = lambda X: K @ CM.fourier_apply(K @ X)
    adj = lambda X: K.conj().T @ CM.fourier_adjoint(K.conj().T @ X)
    g = complex_normal((N,), seed=7)
    assert rel_err(app(g[:, None])[:, 0], Kt @ g) < 1e-13
    et = {r: rel_err(A.bf_apply(CM.construct(app, adj, N, L, r), g), Kt @ g) for r in (4, 8, 12)}
    assert et[8] < et[4] / 5 and et[12] < et[8] / 50
    ek8 = rel_err(A.bf_apply(CM.construct(*_dense_box(K), N, L, 8), g), K @ g)
    assert et[8] > 100 * ek8
