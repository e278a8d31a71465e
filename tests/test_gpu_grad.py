"""GPU differentiation (bf_diff_* through the C ABI, and the autograd
Function) against the FP64 oracle gradient of the same factors.

Tolerance: relative 2-norm <= 1e-5 for u, the input gradient and every
factor gradient (FP32 arithmetic; each gradient entry is a sum over the RHS
of products of FP32 vectors that each carry a few 1e-7 of error)."""
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
    from oracle.kernel import rel_err
    return rel_err(np.asarray(a), np.asarray(b))


def _dev_factors(F):
    dev = torch.device("cuda:0")
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(dev)
    return (c(F.VL), [c(a) for a in F.H], torch.from_numpy(np.ascontiguousarray(F.S, np.float32)).to(dev),
            [c(a) for a in F.G], c(F.UL))


def _run_c_abi(F, g, ubar, stride):
    """Forward and backward through the C ABI; returns u, gbar, grads (numpy)."""
    from paper_1502_01379_gb300 import capi
    dev = torch.device("cuda:0")
    nrhs = g.shape[0]
    plan = capi.bf_diff_create(F.L, F.n0, F.r, nrhs, stride=stride)
    fac = _dev_factors(F)
    gt = torch.from_numpy(g).to(dev)
    ut = torch.empty_like(gt)
    saved = torch.empty(capi.bf_diff_saved_bytes(plan, nrhs) // 8, dtype=torch.complex64, device=dev)
    capi.bf_diff_forward(plan, fac, gt, ut, saved)
    ub = torch.from_numpy(ubar).to(dev)
    gb = torch.empty_like(ub)
    grads = (torch.empty_like(fac[0]), [torch.empty_like(a) for a in fac[1]], torch.empty_like(fac[2]),
             [torch.empty_like(a) for a in fac[3]], torch.empty_like(fac[4]))
    capi.bf_diff_backward(plan, fac, ub, gb, saved, grads)
    torch.cuda.synchronize()
    out = (ut.cpu().numpy(), gb.cpu().numpy(),
           (grads[0].cpu().numpy(), [a.cpu().numpy() for a in grads[1]], grads[2].cpu().numpy(),
            [a.cpu().numpy() for a in grads[3]], grads[4].cpu().numpy()))
    k = capi.bf_diff_stride(plan)
    plan.destroy()
    return out, k


def _oracle_grads(F, g, ubar):
    from oracle import grad as GR
    return GR.bf_apply_and_grad(F.astype(np.complex128), g.T.astype(np.complex128), ubar.T.astype(np.complex128))


def _check_against_oracle(F, g, ubar, res, ref=None):
    u, gbar, grads = res
    ru, rg, rgrads = ref if ref is not None else _oracle_grads(F, g, ubar)
    assert _rel(u, ru.T) < TOL
    assert _rel(gbar, rg.T) < TOL
    VL, H, S, G, UL = grads
    assert _rel(VL, rgrads.VL) < TOL
    assert _rel(UL, rgrads.UL) < TOL
    assert _rel(S, rgrads.S) < TOL
    for t in range(F.h):
        assert _rel(H[t], rgrads.H[t]) < TOL, f"H level {F.h + t}"
        assert _rel(G[t], rgrads.G[t]) < TOL, f"G level {F.h + t}"


SHAPES = [(0, 5, 3), (2, 2, 3), (4, 3, 5), (6, 16, 12), (8, 16, 16), (4, 64, 32), (10, 2, 7)]


@pytest.mark.parametrize("L,n0,r", SHAPES)
def test_gradients_against_oracle(bf, L, n0, r):
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(L, n0, r, seed=600 + L + r, dtype=np.complex64)
    nrhs = 37   # two RHS chunks, the second ragged
    g = complex_normal((nrhs, F.N), seed=1, dtype=np.complex64)
    ubar = complex_normal((nrhs, F.N), seed=2, dtype=np.complex64)
    res, k = _run_c_abi(F, g, ubar, stride=1)
    assert k == 1
    _check_against_oracle(F, g, ubar, res)


@pytest.mark.parametrize("stride", [2, 3, 5, 100])
def test_checkpoint_strides_give_the_same_gradients(bf, stride):
    """Keeping every k-th factor input and recomputing the rest (k up to the
    whole chain: full recompute from the input) changes nothing."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(8, 4, 6, seed=77, dtype=np.complex64)
    g = complex_normal((9, F.N), seed=3, dtype=np.complex64)
    ubar = complex_normal((9, F.N), seed=4, dtype=np.complex64)
    ref, _ = _run_c_abi(F, g, ubar, stride=1)
    res, k = _run_c_abi(F, g, ubar, stride=stride)
    assert k == min(stride, F.L + 3)
    assert np.array_equal(res[0], ref[0]) and np.array_equal(res[1], ref[1])
    for a, b in zip(res[2][:1] + res[2][2:3] + res[2][4:], ref[2][:1] + ref[2][2:3] + ref[2][4:]):
        assert np.array_equal(a, b)
    _check_against_oracle(F, g, ubar, res)


def test_budget_picks_a_stride(bf):
    from paper_1502_01379_gb300 import capi
    L, n0, r, nrhs = 10, 4, 8, 16
    full = capi.bf_diff_create(L, n0, r, nrhs)
    assert capi.bf_diff_stride(full) == 1
    need = capi.bf_diff_saved_bytes(full, nrhs)
    tight = capi.bf_diff_create(L, n0, r, nrhs, saved_budget=need // 3)
    k = capi.bf_diff_stride(tight)
    assert 1 < k <= L + 3
    assert capi.bf_diff_saved_bytes(tight, nrhs) < need
    full.destroy()
    tight.destroy()


def test_autograd_function_loss(bf):
    """loss = ||BF(g) - y||^2 through torch.autograd: gradients of g and of
    every factor parameter against the oracle's."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import grad as GR
    from paper_1502_01379_gb300.autograd import ButterflyOperator
    F = synthetic_factors(6, 4, 5, seed=31, dtype=np.complex64)
    g = complex_normal((12, F.N), seed=5, dtype=np.complex64)
    y = complex_normal((12, F.N), seed=6, dtype=np.complex64)
    op = ButterflyOperator(F, nrhs_max=12)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    yt = torch.from_numpy(y).cuda()
    loss = (op(gt) - yt).abs().pow(2).sum()
    loss.backward()
    L64, _, rg, rgrads = GR.loss_and_grad(F.astype(np.complex128), g.T.astype(np.complex128),
                                          y.T.astype(np.complex128))
    assert abs(loss.item() - L64) <= 1e-5 * L64
    assert _rel(gt.grad.cpu().numpy(), rg.T) < TOL
    assert _rel(op.VL.grad.cpu().numpy(), rgrads.VL) < TOL
    assert _rel(op.UL.grad.cpu().numpy(), rgrads.UL) < TOL
    assert _rel(op.S.grad.cpu().numpy(), rgrads.S) < TOL
    for t in range(F.h):
        assert _rel(op.H[t].grad.cpu().numpy(), rgrads.H[t]) < TOL
        assert _rel(op.G[t].grad.cpu().numpy(), rgrads.G[t]) < TOL


def test_invalid_calls(bf):
    from paper_1502_01379_gb300 import capi
    with pytest.raises(capi.BfError):
        capi.bf_diff_create(3, 4, 4, 8)          # odd L
    with pytest.raises(capi.BfError):
        capi.bf_diff_create(4, 4, 33, 8)         # r above the limit
    plan = capi.bf_diff_create(4, 4, 4, 8)
    assert capi.bf_diff_saved_bytes(plan, 9) == 0   # nrhs above nrhs_max
    plan.destroy()


def test_differentiation_workload_n256k_r16(bf):
    """The differentiation workload: N = 2^18, L = 14 (leaf 16), r = 16, 32 RHS,
    loss = ||BF(g) - y||^2 with y a second operator's output plus 1e-3
    complex noise; the GPU gradients of g and of every factor (every level
    kept, and full recompute) against the FP64 oracle gradient."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import apply as A
    from oracle import grad as GR
    F = synthetic_factors(14, 16, 16, seed=0, dtype=np.complex64)
    Ft = synthetic_factors(14, 16, 16, seed=1, dtype=np.complex64)
    g = complex_normal((32, F.N), seed=7, dtype=np.complex64)
    g_true = complex_normal((F.N, 32), seed=8)
    y = A.bf_apply(Ft.astype(np.complex128), g_true) + 1e-3 * complex_normal((F.N, 32), seed=9)
    u0 = A.bf_apply(F.astype(np.complex128), g.T.astype(np.complex128))
    ubar = np.ascontiguousarray((2.0 * (u0 - y)).T, dtype=np.complex64)
    ref = _oracle_grads(F, g, ubar)
    for stride in (1, 17):
        res, k = _run_c_abi(F, g, ubar, stride=stride)
        assert k == stride
        _check_against_oracle(F, g, ubar, res, ref)
