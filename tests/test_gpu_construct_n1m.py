"""Constructed factorizations at N = 2^20 on the GPU (Sec. 3.1 first case,
Sec. 2.1, Sec. 3.2; Sec. 4 Example 1; Sec. 1.1 Fourier matrix).

The sketch products K_ij C_jj, K_ij^* R_ii come from `bf_sketch_products`
(entries generated on the GPU); the construction is `construct_kernel_1d`.
For each factorization built here:
  * the GPU apply and adjoint against the FP64 C loops of the oracle on the
    same factors (relative 2-norm <= 1e-5, the FP32 parity bar);
  * the factorization against the matrix: every entry of K g and K^* f by the
    FFT closed form for the Fourier matrix, the paper's 256 sampled rows
    (epsilon^a of Sec. 4) of the direct product for the FIO: the oracle's
    FP64 apply of the factors within 10 epsilon of the construction, the GPU's
    within 10 epsilon + 1e-5.
Shapes: the benchmarked tree (L = 16, leaf 16, r = 16: middle blocks of
time-bandwidth product 16, which rank 16 cannot resolve, so epsilon is large)
and L = 18, leaf 4, r = 16 (time-bandwidth product 4: an accurate
factorization of the same N = 2^20 matrices)."""
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
    import paper_1502_01379_gb300 as mod
    mod.load()
    torch.cuda.set_device(0)
    return mod


def _rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- the products
@pytest.mark.parametrize("kind", ["fio", "dft"])
def test_sketch_products_against_oracle_entries(bf, kind):
    """Every output of a forward and an adjoint product at N = 4096 (16 nodes
    of 256, k = 21, a row range and a node subset), and sampled outputs at
    N = 2^20 (4096-term sums), against FP64 products of the oracle's entries."""
    from bfinputs import complex_normal
    from oracle import kernel as KK
    from paper_1502_01379_gb300 import capi, construct
    for log2N, nb, sample in ((12, 256, None), (20, 4096, 8)):
        N = 1 << log2N
        cf = construct.c_fixed_point(kind, N)
        cfix = None if cf is None else torch.from_numpy(cf).cuda()
        nodes, node0, k = 3, (N // nb) - 4, 21
        B = complex_normal((nodes, nb, k), seed=log2N, dtype=np.complex64)
        lo, hi = (N // 3, N // 3 + 700) if sample is None else (0, N)
        for adjoint in (False, True):
            out = torch.empty((nodes, k, hi - lo), dtype=torch.complex64, device="cuda")
            capi.bf_sketch_products(log2N, nb, torch.from_numpy(B).cuda(), out, lo, hi, node0=node0,
                                    adjoint=adjoint, c_fixed=cfix)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            rng = np.random.default_rng(log2N)
            o = np.arange(lo, hi) if sample is None else np.sort(rng.choice(N, sample, replace=False))
            for b in range(nodes):
                s = np.arange((node0 + b) * nb, (node0 + b + 1) * nb)
                Kb = KK.entries(s, o, N, kind).conj().T if adjoint else KK.entries(o, s, N, kind)
                ref = Kb @ B[b].astype(np.complex128)                      # (len(o), k)
                assert _rel(got[b][:, o - lo].T, ref) < 2e-6, (log2N, adjoint, b)


def test_sketch_products_argument_errors(bf):
    from paper_1502_01379_gb300 import capi
    B = torch.zeros((2, 16, 4), dtype=torch.complex64, device="cuda")
    out = torch.zeros((2, 4, 32), dtype=torch.complex64, device="cuda")
    lib = bf.load()
    import ctypes
    bad = [dict(log2N=0), dict(nb=24), dict(node0=3), dict(lo=40, hi=72), dict(lo=5, hi=5), dict(k=0)]
    for b in bad:
        d = dict(log2N=6, nb=16, k=4, node0=0, nodes=2, lo=0, hi=32, adjoint=0)
        d.update(b)
        desc = capi.bf_sketch_desc(d["log2N"], d["nb"], d["k"], d["node0"], d["nodes"], d["lo"], d["hi"],
                                   d["adjoint"])
        st = lib.bf_sketch_products(ctypes.byref(desc), None, ctypes.c_void_p(B.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
        assert st == bf.BF_ERR_INVALID, b
    desc = capi.bf_sketch_desc(6, 16, 33, 0, 2, 0, 32, 0)
    assert lib.bf_sketch_products(ctypes.byref(desc), None, ctypes.c_void_p(B.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), None) == bf.BF_ERR_UNSUPPORTED
    h = np.zeros((2, 16, 4), np.complex64)
    desc = capi.bf_sketch_desc(6, 16, 4, 0, 2, 0, 32, 0)
    assert lib.bf_sketch_products(ctypes.byref(desc), None, ctypes.c_void_p(h.ctypes.data),
                                  ctypes.c_void_p(out.data_ptr()), None) == bf.BF_ERR_INVALID


# ---------------------------------------------------- N = 2^20 factorizations
def _gpu_apply(bf, plan, X, adjoint=False):
    x = torch.from_numpy(X.astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    (bf.bf_apply_adjoint if adjoint else bf.bf_apply)(plan, x, y)
    torch.cuda.synchronize()
    bf.bf_plan_check(plan)
    return y.cpu().numpy()


def _constructed(kind, L, n0, r):
    from paper_1502_01379_gb300 import construct
    F = construct.construct_kernel_1d(kind, n0 << L, L, r, seed=3)
    print(f"\n{kind} N=2^20 L={L} leaf={n0} r={r}: eps {F.meta['eps']:.3e} (mid {F.meta['eps_mid']:.2e}, "
          f"rec {F.meta['eps_rec']:.2e}); timings {F.meta['timings']}")
    return F


@pytest.mark.parametrize("L,n0,r", [(16, 16, 16), (18, 4, 16)])
def test_dft_n1m_against_fft_closed_form(bf, L, n0, r):
    from bfinputs import complex_normal
    from oracle import capply
    from oracle import kernel as KK
    F = _constructed("dft", L, n0, r)
    N, eps = F.N, F.meta["eps"]
    plan = bf.bf_plan_create(F, nrhs_max=2)
    g = complex_normal((2, N), seed=11, dtype=np.complex64)
    u = _gpu_apply(bf, plan, g)
    a = _gpu_apply(bf, plan, g, adjoint=True)
    plan.destroy()
    P = capply.PreparedFactors(F)
    uc = capply.bf_apply_c(P, g[0])
    ac = capply.bf_adjoint_c(P, g[0])
    del P
    assert _rel(u[0], uc) < TOL and _rel(a[0], ac) < TOL            # GPU against the oracle, same factors
    sign = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    for j in range(2):
        Kg = KK.dft_closed_form(g[j], N)                            # (-1)^x N ifft(g)
        Kstar_g = np.fft.fft(sign * g[j].astype(np.complex128))     # K^* f = fft((-1)^x f)
        ea, eaa = _rel(u[j], Kg), _rel(a[j], Kstar_g)
        print(f"  eps^a (every entry, GPU): apply {ea:.3e}, adjoint {eaa:.3e}")
        assert ea <= 10 * eps + TOL and eaa <= 10 * eps + TOL
    eo, eoa = _rel(uc, KK.dft_closed_form(g[0], N)), _rel(ac, np.fft.fft(sign * g[0].astype(np.complex128)))
    print(f"  eps^a (every entry, FP64 oracle apply of the factors): apply {eo:.3e}, adjoint {eoa:.3e}")
    assert eo <= 10 * eps and eoa <= 10 * eps
    if L == 18:
        assert eps < 1e-5 and eo < 1e-5                              # an accurate factorization
    # 32 vectors through the multi-RHS cores on the same factors (the tensor-core
    # core at leaf 16; the CUDA-core core at leaf 4, which the tensor cores do not
    # take): every column against the single-vector path and the FFT
    plan = bf.bf_plan_create(F, nrhs_max=32)
    G32 = complex_normal((32, N), seed=13, dtype=np.complex64)
    G32[:2] = g
    U32 = _gpu_apply(bf, plan, G32)
    A32 = _gpu_apply(bf, plan, G32, adjoint=True)
    plan.destroy()
    assert _rel(U32[:2], u) < TOL and _rel(A32[:2], a) < TOL
    for j in (0, 5, 31):
        assert _rel(U32[j], KK.dft_closed_form(G32[j], N)) <= 10 * eps + TOL
        assert _rel(A32[j], np.fft.fft(sign * G32[j].astype(np.complex128))) <= 10 * eps + TOL


@pytest.mark.parametrize("L,n0,r", [(16, 16, 16), (18, 4, 16)])
def test_fio_n1m_on_the_sampled_rows(bf, L, n0, r):
    from bfinputs import complex_normal
    from bfinputs.workloads import sample_rows
    from oracle import capply
    from oracle import kernel as KK
    F = _constructed("fio", L, n0, r)
    N, eps = F.N, F.meta["eps"]
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, N), seed=12, dtype=np.complex64)
    u = _gpu_apply(bf, plan, g)[0]
    a = _gpu_apply(bf, plan, g, adjoint=True)[0]
    plan.destroy()
    P = capply.PreparedFactors(F)
    uc = capply.bf_apply_c(P, g[0])
    ac = capply.bf_adjoint_c(P, g[0])
    del P
    assert _rel(u, uc) < TOL and _rel(a, ac) < TOL
    rows = sample_rows(N, 256, seed=5)
    ud = KK.dense_apply(g[0], N, "fio", rows=rows)                  # the direct product on 256 rows
    ea, eo = _rel(u[rows], ud), _rel(uc[rows], ud)
    print(f"  eps^a on 256 rows: GPU {ea:.3e}, FP64 oracle apply {eo:.3e}; eps {eps:.3e}")
    assert eo <= 10 * eps and ea <= 10 * eps + TOL
