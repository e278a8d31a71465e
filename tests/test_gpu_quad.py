"""2D (quadtree) factorizations through the C ABI (bf_quad_*): GPU FP32
apply and adjoint against the FP64 oracle of the same factors, on every
ragged-rank shape the level kernel sees, on a constructed 2D FIO
factorization against the dense product, and at the full 256 x 256, rank-24
workload on sampled columns; argument errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_01379_gb300 import build as pkg_build
    pkg_build.build()
    from paper_1502_01379_gb300 import capi
    capi.load()
    torch.cuda.set_device(0)
    return capi


def _rel(a, b):
    from oracle.kernel import rel_err
    return rel_err(np.asarray(a), np.asarray(b))


def _gpu(capi, plan, g, adjoint=False, ld=None):
    nrhs, N = g.shape
    if ld is None:
        x = torch.from_numpy(g).cuda()
        y = torch.full_like(x, float("nan"))
        capi.bf_quad_apply(plan, x, y, adjoint=adjoint)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    xp = torch.zeros((nrhs, ld), dtype=torch.complex64, device="cuda")
    xp[:, :N] = torch.from_numpy(g).cuda()
    yp = torch.full((nrhs, ld), 7 + 7j, dtype=torch.complex64, device="cuda")
    capi.bf_quad_apply(plan, xp, yp, nrhs=nrhs, ld=ld, adjoint=adjoint)
    torch.cuda.synchronize()
    out = yp.cpu().numpy()
    assert np.all(out[:, N:] == 7 + 7j)          # nothing written past N in each column
    return out[:, :N]


SHAPES = [(2, 1, 2, 1), (2, 4, 5, 3), (2, 16, 3, 2), (4, 1, 3, 1), (4, 4, 6, 7), (4, 16, 8, 33),
          (4, 1, 32, 5), (6, 1, 24, 40), (6, 4, 12, 17), (4, 4, 24, 128)]


@pytest.mark.parametrize("L,n0,r,nrhs", SHAPES)
def test_quad_apply_and_adjoint_against_oracle(bf, L, n0, r, nrhs):
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    from oracle import quad as Q
    F = synthetic_quad_factors(L, n0, r, seed=L * 100 + r, dtype=np.complex64)
    plan = bf.bf_quad_create(F, nrhs_max=nrhs)
    assert bf.bf_quad_passes(plan) == L
    g = complex_normal((nrhs, F.N), seed=7 + r, dtype=np.complex64)
    for adjoint in (False, True):
        ref = (Q.bf_adjoint if adjoint else Q.bf_apply)(F, g.T).T
        assert _rel(_gpu(bf, plan, g, adjoint), ref) < TOL, adjoint
    plan.destroy()


def test_quad_chunks_and_leading_dimension(bf):
    """More vectors than nrhs_max run in chunks; ld > N leaves the padding alone."""
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    from oracle import quad as Q
    F = synthetic_quad_factors(4, 4, 6, seed=3, dtype=np.complex64)
    plan = bf.bf_quad_create(F, nrhs_max=4)
    g = complex_normal((11, F.N), seed=4, dtype=np.complex64)
    for adjoint in (False, True):
        ref = (Q.bf_adjoint if adjoint else Q.bf_apply)(F, g.T).T
        assert _rel(_gpu(bf, plan, g, adjoint, ld=F.N + 37), ref) < TOL
    plan.destroy()


def test_constructed_fio2_against_dense(bf):
    """A 2D FIO factorization built by the oracle (n = 32, depth 4, rank 24):
    the GPU apply equals the oracle apply of the same factors to FP32
    accuracy and the dense product to the construction's accuracy."""
    from bfinputs import complex_normal
    from oracle import quad as Q
    F = Q.construct(32, 4, 24, "fio2", seed=10)
    plan = bf.bf_quad_create(F, nrhs_max=3)
    g = complex_normal((3, F.N), seed=11, dtype=np.complex64)
    u = _gpu(bf, plan, g)
    assert _rel(u, Q.bf_apply(F, g.T.astype(np.complex128)).T) < TOL
    assert _rel(u, Q.dense_apply(g.T.astype(np.complex128), 32).T) <= 10 * F.meta["eps"]
    f = complex_normal((3, F.N), seed=12, dtype=np.complex64)
    assert _rel(_gpu(bf, plan, f, adjoint=True), Q.bf_adjoint(F, f.T.astype(np.complex128)).T) < TOL
    plan.destroy()


def test_full_size_256x256_rank24(bf):
    """The 2D workload: 256 x 256 grid, quadtrees of depth 8 (one point per
    leaf), rank 24 (level ranks 24, 24, 16, 4, 1), 128 vectors in one call:
    three sampled vectors of each direction against the FP64 oracle."""
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    from oracle import quad as Q
    F = synthetic_quad_factors(8, 1, 24, seed=24, dtype=np.complex64)
    plan = bf.bf_quad_create(F, nrhs_max=128)
    g = complex_normal((128, F.N), seed=25, dtype=np.complex64)
    cols = [0, 77, 127]
    for adjoint in (False, True):
        out = _gpu(bf, plan, g, adjoint)
        ref = (Q.bf_adjoint if adjoint else Q.bf_apply)(F, g[cols].T).T
        assert _rel(out[cols], ref) < TOL, adjoint
        assert np.isfinite(out).all()
    plan.destroy()


def test_quad_argument_errors(bf):
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    F = synthetic_quad_factors(2, 4, 3, seed=1, dtype=np.complex64)
    plan = bf.bf_quad_create(F, nrhs_max=2)
    x = torch.from_numpy(complex_normal((2, F.N), seed=2, dtype=np.complex64)).cuda()
    with pytest.raises(bf.BfError) as e:
        bf.bf_quad_apply(plan, x, x)                                  # in and out overlap
    assert e.value.status == bf.BF_ERR_INVALID
    with pytest.raises(bf.BfError) as e:
        bf.bf_quad_apply(plan, x.cpu(), torch.empty_like(x).cpu())    # host pointers
    assert e.value.status == bf.BF_ERR_INVALID
    with pytest.raises(bf.BfError) as e:
        bf.bf_quad_apply(plan, x, torch.empty_like(x), ld=F.N - 1)
    assert e.value.status == bf.BF_ERR_INVALID
    bf.bf_quad_apply(plan, x, torch.empty_like(x), nrhs=0)             # no-op
    plan.destroy()
    big = synthetic_quad_factors(2, 1, 33, seed=1, dtype=np.complex64)
    with pytest.raises(bf.BfError) as e:
        bf.bf_quad_create(big)
    assert e.value.status == bf.BF_ERR_UNSUPPORTED
    F.n0 = 2
    with pytest.raises(bf.BfError) as e:
        bf.bf_quad_create(F)
    assert e.value.status == bf.BF_ERR_INVALID


@pytest.mark.parametrize("L,n0,r,nrhs", [(6, 1, 24, 128), (4, 4, 24, 40), (4, 16, 8, 33), (6, 4, 16, 160)])
def test_quad_tensor_core_rungs(bf, L, n0, r, nrhs):
    """Chunks of 32 or more vectors run the inner levels on the tensor-core
    core (output parts and K-chunks of at most 64, planar tiles between the
    levels).  Every precision rung, forward and adjoint, against the FP64
    oracle: 3xTF32 and the BF16 three-way split within the FP32 tolerance,
    the others in their bands; and 3xTF32 against the CUDA-core path of the
    same plan (chunks below 32 vectors)."""
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    from oracle import quad as Q
    F = synthetic_quad_factors(L, n0, r, seed=500 + r, dtype=np.complex64)
    plan = bf.bf_quad_create(F, nrhs_max=nrhs)
    assert 0 < bf.bf_quad_tc_passes(plan) <= L - 2
    g = complex_normal((nrhs, F.N), seed=600 + L, dtype=np.complex64)
    cols = [0, nrhs // 2, nrhs - 1]
    for adjoint in (False, True):
        ref = (Q.bf_adjoint if adjoint else Q.bf_apply)(F, g[cols].T).T
        errs = {}
        for prec in (bf.BF_PREC_FP32, bf.BF_PREC_TF32, bf.BF_PREC_BF16X6, bf.BF_PREC_BF16X3, bf.BF_PREC_BF16):
            bf.bf_quad_set_precision(plan, prec)
            out = _gpu(bf, plan, g, adjoint)
            bf.bf_quad_check(plan)
            errs[prec] = _rel(out[cols], ref)
        assert errs[bf.BF_PREC_FP32] < TOL and errs[bf.BF_PREC_BF16X6] < TOL, errs
        assert 1e-4 < errs[bf.BF_PREC_TF32] < 1e-2, errs
        assert 1e-6 < errs[bf.BF_PREC_BF16X3] < 5e-5, errs
        assert 1e-3 < errs[bf.BF_PREC_BF16] < 3e-2, errs
        bf.bf_quad_set_precision(plan, bf.BF_PREC_FP32)
        tc = _gpu(bf, plan, g, adjoint)
        x = torch.from_numpy(g).cuda()
        y = torch.empty_like(x)
        for k0 in range(0, nrhs, 16):                       # 16 at a time: the CUDA-core levels
            bf.bf_quad_apply(plan, x[k0:k0 + 16], y[k0:k0 + 16], adjoint=adjoint)
        torch.cuda.synchronize()
        assert _rel(tc, y.cpu().numpy()) < TOL
    plan.destroy()


def test_quad_tensor_core_bounded_waits_report_timeout(bf, monkeypatch):
    """The 2D tensor-core levels under the stall hook: every wait expires, the
    launch returns, bf_quad_check reports BF_ERR_TIMEOUT (then clears it), and
    a plan made afterwards is correct."""
    from bfinputs import complex_normal
    from bfinputs.quad import synthetic_quad_factors
    from oracle import quad as Q
    F = synthetic_quad_factors(4, 4, 16, seed=33, dtype=np.complex64)
    monkeypatch.setenv("BF_INJECT_STALL", "1")
    stalled = bf.bf_quad_create(F, nrhs_max=64)
    monkeypatch.delenv("BF_INJECT_STALL")
    assert bf.bf_quad_tc_passes(stalled) > 0
    g = complex_normal((64, F.N), seed=34, dtype=np.complex64)
    _gpu(bf, stalled, g)
    with pytest.raises(bf.BfError) as err:
        bf.bf_quad_check(stalled)
    assert err.value.status == bf.BF_ERR_TIMEOUT
    bf.bf_quad_check(stalled)
    stalled.destroy()
    plan = bf.bf_quad_create(F, nrhs_max=64)
    assert _rel(_gpu(bf, plan, g), Q.bf_apply(F, g.T).T) < TOL
    bf.bf_quad_check(plan)
    plan.destroy()
