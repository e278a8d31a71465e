"""The construction from applies (`construct_from_applies`): its batched
linear algebra checked on the host with an exact dense black box, against
the FP64 oracle of the same algorithm (`oracle.construct_mv`, which takes the
same random blocks) and the dense matrix.  The GPU run, with this library's
apply as the black box, is in test_gpu_construct.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from bfinputs import complex_normal
from oracle import apply as A
from oracle import construct_mv as CM
from oracle import kernel as KK
from oracle.kernel import rel_err
from paper_1502_01379_gb300 import construct as DC

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _box(K):
    Kt = torch.from_numpy(K)
    return (lambda X: X @ Kt.T), (lambda X: X @ Kt.conj())


def test_full_rank_is_exact():
    N, L, r = 64, 4, 16
    K = KK.dense_matrix(N, "fio")
    F = DC.construct_from_applies(*_box(K), N, L, r, device="cpu")
    g = complex_normal((N, 2), seed=1)
    assert rel_err(A.bf_apply(F, g), K @ g) < 1e-12
    assert rel_err(A.bf_adjoint(F, g), K.conj().T @ g) < 1e-12


def test_accuracy_tracks_the_oracle():
    """N = 1024, one point per leaf, r = 4, 6, 8: within a factor 3 of the
    oracle's construction from the same products (the SVD range basis is, if
    anything, the better one)."""
    N, L = 1024, 10
    K = KK.dense_matrix(N, "fio")
    g = complex_normal((N,), seed=3)
    for r in (4, 6, 8):
        Fd = DC.construct_from_applies(*_box(K), N, L, r, device="cpu")
        Fo = CM.construct(lambda X: K @ X, lambda X: K.conj().T @ X, N, L, r)
        ed, eo = rel_err(A.bf_apply(Fd, g), K @ g), rel_err(A.bf_apply(Fo, g), K @ g)
        assert ed <= 3 * eo and eo <= 3 * ed, (r, ed, eo)
        assert Fd.meta["vectors_per_direction"] == Fo.meta["vectors_per_direction"]


def test_example3_composition():
    N, L = 256, 8
    K = KK.dense_matrix(N, "fio")
    Kt = K @ CM.fourier_matrix(N) @ K
    Km = torch.from_numpy(K)
    app = lambda X: DC.fourier_rows(X @ Km.T) @ Km.T
    adj = lambda X: DC.fourier_adjoint_rows(X @ Km.conj()) @ Km.conj()
    g = complex_normal((N,), seed=7)
    x = torch.from_numpy(g)[None]
    assert rel_err(app(x)[0].numpy(), Kt @ g) < 1e-13
    assert rel_err(adj(x)[0].numpy(), Kt.conj().T @ g) < 1e-13
    e = {r: rel_err(A.bf_apply(DC.construct_from_applies(app, adj, N, L, r, device="cpu"), g), Kt @ g)
         for r in (4, 8, 12)}
    assert e[8] < e[4] / 5 and e[12] < e[8] / 50 and e[12] < 1e-4


def test_gram_form_matches_svd_form_down_to_its_floor():
    """method="gram" (small batched Hermitian eigensolves instead of tall
    SVDs): the same accuracy as "svd" wherever the factorization's error is
    above ~1e-7 (r = 4, 6, 8 at N = 1024), and a graceful floor near 1e-7
    where "svd" reaches roundoff (r = 12 here; full rank at N = 64)."""
    N, L = 1024, 10
    K = KK.dense_matrix(N, "fio")
    g = complex_normal((N,), seed=3)
    for r in (4, 6, 8):
        es = rel_err(A.bf_apply(DC.construct_from_applies(*_box(K), N, L, r, device="cpu"), g), K @ g)
        eg = rel_err(A.bf_apply(DC.construct_from_applies(*_box(K), N, L, r, device="cpu", method="gram"), g), K @ g)
        assert abs(eg - es) <= 0.05 * es, (r, es, eg)
    e12 = rel_err(A.bf_apply(DC.construct_from_applies(*_box(K), N, L, 12, device="cpu", method="gram"), g), K @ g)
    assert e12 < 1e-6
    K64 = KK.dense_matrix(64, "fio")
    g64 = complex_normal((64,), seed=1)
    F = DC.construct_from_applies(*_box(K64), 64, 4, 16, device="cpu", method="gram")
    assert rel_err(A.bf_apply(F, g64), K64 @ g64) < 1e-6
    with pytest.raises(ValueError):
        DC.construct_from_applies(*_box(K64), 64, 4, 16, device="cpu", method="qr")


# ----------------------------------------------------- construct_kernel_1d
def _dense_sketch(kind):
    """bf_sketch_products as its header states it, by dense FP64 entries of the
    oracle's kernel (host logic only; the GPU kernel is tested against the
    oracle in test_gpu_construct_n1m.py)."""
    def fake(log2N, nb, blocks, out, lo, hi, node0=0, adjoint=False, c_fixed=None, stream=None):
        N = 1 << log2N
        B = blocks.numpy().astype(np.complex128)
        o = np.arange(lo, hi)
        for b in range(B.shape[0]):
            s = np.arange((node0 + b) * nb, (node0 + b + 1) * nb)
            Kb = KK.entries(s, o, N, kind).conj().T if adjoint else KK.entries(o, s, N, kind)
            out[b] = torch.from_numpy((Kb @ B[b]).T.astype(np.complex64))
    return fake


def test_c_fixed_point_is_exact():
    from fractions import Fraction
    N = 1 << 12
    cf = DC.c_fixed_point("fio", N).view(np.uint64)
    c = KK.c_of_x(np.arange(N), N)
    for j in (0, 1, 7, N // 4, N // 2 + 3, N - 1):
        assert Fraction(float(c[j])) * 2**64 == int(cf[j])
    assert DC.c_fixed_point("dft", N) is None


@pytest.mark.parametrize("kind", ["fio", "dft"])
def test_kernel_construction_full_rank_and_against_the_product_form(monkeypatch, kind):
    """Full rank (N = 64, L = 4, r = 16 >= every block size) reproduces K to
    the Gram form's floor; at N = 1024, L = 10, r = 6 the chunked two-pass form
    (coefficients kept, V pass reusing the U pass's middle SVDs) matches the
    one-pass construction from the same products to 5 %, for chunks of 1 and
    of 8 nodes."""
    from paper_1502_01379_gb300 import capi
    monkeypatch.setattr(capi, "bf_sketch_products", _dense_sketch(kind))
    K = KK.dense_matrix(64, kind)
    g = complex_normal((64,), seed=1)
    F = DC.construct_kernel_1d(kind, 64, 4, 16, chunk=2, device="cpu")
    assert rel_err(A.bf_apply(F, g), K @ g) < 2e-6
    assert rel_err(A.bf_adjoint(F, g), K.conj().T @ g) < 2e-6
    N, L, r = 1024, 10, 6
    K = KK.dense_matrix(N, kind)
    g = complex_normal((N,), seed=3)
    Fp = DC.construct_from_applies(*_box(K), N, L, r, device="cpu", method="gram")
    ref = rel_err(A.bf_apply(Fp, g), K @ g)
    ref_adj = rel_err(A.bf_adjoint(Fp, g), K.conj().T @ g)
    for chunk in (1, 8):
        F = DC.construct_kernel_1d(kind, N, L, r, chunk=chunk, device="cpu", out_dtype=np.complex128)
        e = rel_err(A.bf_apply(F, g), K @ g)
        ea = rel_err(A.bf_adjoint(F, g), K.conj().T @ g)
        assert abs(e - ref) <= 0.05 * ref + 1e-6, (chunk, e, ref)
        assert abs(ea - ref_adj) <= 0.05 * ref_adj + 1e-6, (chunk, ea, ref_adj)
        assert F.meta["eps"] >= F.meta["eps_floor"] and max(e, ea) <= 10 * F.meta["eps"]
