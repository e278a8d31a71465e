"""Construction from fast applies on the GPU (Sec. 3.1 first case, Example 3):
this library's apply of a factorization of K is the black box; the
factorization it builds is planned and applied on the GPU and checked against
the dense product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_01379_gb300 import build as pkg_build
    pkg_build.build()
    import paper_1502_01379_gb300 as mod
    mod.load()
    torch.cuda.set_device(0)
    return mod


def _rel(a, b):
    from oracle.kernel import rel_err
    return rel_err(np.asarray(a), np.asarray(b))


def test_refactorize_fio_from_gpu_applies(bf):
    """K's factorization (oracle, r = 12, accurate to ~1e-10) applied on the
    GPU serves as the black box; the rank-8 factorization built from its
    products on the device is as accurate against the dense K as the
    oracle's own rank-8 construction allows (FP32 products add ~1e-6)."""
    from bfinputs import complex_normal
    from oracle import apply as A
    from oracle import construct as CS
    from oracle import kernel as KK
    from paper_1502_01379_gb300 import construct as DC
    N, L = 1024, 10
    K = KK.dense_matrix(N, "fio")
    plan = bf.bf_plan_create(CS.construct(N, L, 12, "fio"), nrhs_max=512)
    F8 = DC.construct_from_applies(*DC.plan_black_box(plan), N, L, 8, device="cuda")
    plan.destroy()
    g = complex_normal((N,), seed=3)
    assert _rel(A.bf_apply(F8, g), K @ g) < 3e-5


def test_example3_on_the_gpu(bf):
    """K~ = K F K from two GPU applies of K's factorization and an FFT; the
    factorization of K~ built on the device, then planned and applied on the
    GPU, against the dense K F K."""
    from bfinputs import complex_normal
    from oracle import construct as CS
    from oracle import construct_mv as CM
    from oracle import kernel as KK
    from paper_1502_01379_gb300 import construct as DC
    N, L = 256, 8
    K = KK.dense_matrix(N, "fio")
    Kt = K @ CM.fourier_matrix(N) @ K
    plan = bf.bf_plan_create(CS.construct(N, L, 12, "fio"), nrhs_max=256)
    kf, ka = DC.plan_black_box(plan)
    app = lambda X: kf(DC.fourier_rows(kf(X)))
    adj = lambda X: ka(DC.fourier_adjoint_rows(ka(X)))
    g = complex_normal((4, N), seed=7, dtype=np.complex64)
    ref = (Kt @ g.T.astype(np.complex128)).T
    errs = {}
    for r in (4, 8, 12):
        Ft = DC.construct_from_applies(app, adj, N, L, r, device="cuda")
        pt = bf.bf_plan_create(Ft, nrhs_max=4)
        x = torch.from_numpy(g).cuda()
        y = torch.empty_like(x)
        bf.bf_apply(pt, x, y)
        torch.cuda.synchronize()
        errs[r] = _rel(y.cpu().numpy(), ref)
        pt.destroy()
    plan.destroy()
    assert errs[8] < errs[4] / 5 and errs[12] < errs[8] / 20 and errs[12] < 2e-4, errs
