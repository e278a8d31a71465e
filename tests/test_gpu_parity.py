"""GPU parity: the CUDA apply/adjoint (through the C ABI) against the FP64 oracle
apply of the same factors, element by element.

Tolerance: relative 2-norm error <= 1e-5 over all entries (FP32 arithmetic;
each output is a chain of L+3 sparse products, each summing at most 2r or n0
products, so the expected error is a few 1e-7).
"""
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


def _oracle(F, x, adjoint=False):
    from oracle import apply as A
    F64 = F.astype(np.complex128)
    fn = A.bf_adjoint if adjoint else A.bf_apply
    return fn(F64, np.asarray(x).T.astype(np.complex128)).T


def _rel(a, b):
    from oracle.kernel import rel_err
    return rel_err(a, b)


def _run(bf, plan, x_np, adjoint=False, ld=None):
    dev = torch.device("cuda:0")
    nrhs, N = x_np.shape
    if ld is None:
        x = torch.from_numpy(x_np).to(dev)
        y = torch.empty_like(x)
        (bf.bf_apply_adjoint if adjoint else bf.bf_apply)(plan, x, y)
        torch.cuda.synchronize()
        bf.bf_plan_check(plan)
        return y.cpu().numpy()
    xp = torch.zeros((nrhs, ld), dtype=torch.complex64, device=dev)
    xp[:, :N] = torch.from_numpy(x_np).to(dev)
    yp = torch.full((nrhs, ld), 7.0 + 7.0j, dtype=torch.complex64, device=dev)
    (bf.bf_apply_adjoint if adjoint else bf.bf_apply)(plan, xp, yp, nrhs=nrhs, ld=ld)
    torch.cuda.synchronize()
    bf.bf_plan_check(plan)
    out = yp.cpu().numpy()
    assert np.all(out[:, N:] == 7.0 + 7.0j), "padding between columns was written"
    return out[:, :N]


SHAPES = [  # (L, n0, r): degenerate L = 0, tiny trees, odd n0*r, r = 1, r = 32, n0 = 64
    (0, 5, 3), (0, 1, 1), (2, 2, 3), (2, 1, 1), (4, 3, 5), (4, 16, 32), (6, 1, 1), (6, 16, 12),
    (8, 16, 12), (8, 64, 4), (10, 16, 16), (12, 2, 7),
]


@pytest.mark.parametrize("L,n0,r", SHAPES)
def test_synthetic_shapes_apply_and_adjoint(bf, L, n0, r):
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(L, n0, r, seed=100 + L + r, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=4)
    for nrhs in (1, 3):
        g = complex_normal((nrhs, F.N), seed=nrhs, dtype=np.complex64)
        assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
        assert _rel(_run(bf, plan, g, adjoint=True), _oracle(F, g, True)) < TOL
    plan.destroy()


@pytest.mark.parametrize("L,n0,r", SHAPES)
def test_multi_rhs_path_shapes(bf, L, n0, r):
    """Batches of >= 8 vectors run the multi-pass path (groups of r-blocks in
    bit-reversed slot order, 16/32/64 RHS per CTA): ragged tiles and several
    passes over nrhs_max."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(L, n0, r, seed=300 + L + r, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=40)
    for nrhs in (8, 21, 40, 83):
        g = complex_normal((nrhs, F.N), seed=nrhs + 7, dtype=np.complex64)
        assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
        assert _rel(_run(bf, plan, g, adjoint=True), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_multi_rhs_path_ld_and_fio(bf):
    """Multi-RHS path on the oracle-constructed FIO (N = 4096, r = 12) with ld > N."""
    from bfinputs import complex_normal
    from oracle import construct
    F = construct.construct(4096, 8, 12, "fio", seed=0).astype(np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=64)
    g = complex_normal((64, F.N), seed=11, dtype=np.complex64)
    assert _rel(_run(bf, plan, g, ld=F.N + 40), _oracle(F, g)) < TOL
    assert _rel(_run(bf, plan, g, adjoint=True), _oracle(F, g, True)) < TOL
    plan.destroy()


TC_SHAPES = [(0, 16, 16), (2, 16, 16), (4, 16, 32), (6, 32, 16), (8, 16, 16), (8, 64, 16), (10, 16, 16),
             (4, 8, 16), (6, 16, 8), (2, 8, 8)]


@pytest.mark.parametrize("L,n0,r", TC_SHAPES)
@pytest.mark.parametrize("kmax", [None, 1])
def test_tensor_core_path(bf, L, n0, r, kmax, monkeypatch):
    """Batches on the tcgen05 core (dense per-group blocks, RHS tiles of 32 to
    128, 3xTF32; forced here for every batch size): groups of 1, 2 and 4
    slots, ragged RHS tiles and tile widths 32 (8 vectors), 64 (57), 96 (130:
    two tiles) and 128 (300: three), and one slot bit per pass (kmax = 1).
    Shapes whose blocks exceed 64 x 64 (n0 = 64) fall back to the CUDA-core
    core."""
    from bfinputs import complex_normal, synthetic_factors
    monkeypatch.setenv("BF_TC", "1")
    monkeypatch.setenv("BF_TC_MIN", "1")      # every batch on the tensor-core core
    if kmax is not None:
        monkeypatch.setenv("BF_TC_KMAX", str(kmax))
    F = synthetic_factors(L, n0, r, seed=500 + L + r, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=300)
    for nrhs in (8, 57, 130, 300):
        g = complex_normal((nrhs, F.N), seed=nrhs + 3, dtype=np.complex64)
        assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
        assert _rel(_run(bf, plan, g, adjoint=True), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_tensor_core_path_odd_ld(bf, monkeypatch):
    """Odd leading dimension: the tensor-core core's 16-byte row copies need an
    even one, so the call goes through aligned staging buffers."""
    from bfinputs import complex_normal, synthetic_factors
    monkeypatch.setenv("BF_TC", "1")
    monkeypatch.setenv("BF_TC_MIN", "1")
    F = synthetic_factors(8, 16, 16, seed=9, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=64)
    g = complex_normal((40, F.N), seed=2, dtype=np.complex64)
    assert _rel(_run(bf, plan, g, ld=F.N + 3), _oracle(F, g)) < TOL
    assert _rel(_run(bf, plan, g, adjoint=True, ld=F.N + 1), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_fio_n4096_r12_against_oracle(bf):
    """1D FIO of Example 1, N = 4096, L = 8 (leaf 16), r = 12, factors built by
    the oracle's entry-sampling construction in FP64, one RHS (seed 0)."""
    from bfinputs import complex_normal
    from oracle import construct
    F = construct.construct(4096, 8, 12, "fio", seed=0).astype(np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=0, dtype=np.complex64)
    assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
    assert _rel(_run(bf, plan, g, adjoint=True), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_dft_against_fft_closed_form(bf):
    """Fourier matrix (Sec. 1.1): the GPU apply of the oracle's factorization
    reproduces (-1)^j N ifft(g) within the construction's eps + FP32 rounding."""
    from bfinputs import complex_normal
    from oracle import construct
    from oracle import kernel as K
    N = 1024
    F64 = construct.construct(N, 10, 10, "dft", seed=0)
    plan = bf.bf_plan_create(F64.astype(np.complex64), nrhs_max=2)
    g = complex_normal((2, N), seed=3, dtype=np.complex64)
    u = _run(bf, plan, g)
    ref = K.dft_closed_form(g.T.astype(np.complex128), N).T
    assert _rel(u, ref) < max(TOL, 10 * F64.meta["eps"])
    plan.destroy()


def test_batches_ragged_tiles_chunks_and_ld(bf):
    """nrhs above nrhs_max (several passes), ragged RHS tiles, ld > N."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(8, 4, 6, seed=5, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=3)
    for nrhs in (1, 2, 5, 7):
        g = complex_normal((nrhs, F.N), seed=40 + nrhs, dtype=np.complex64)
        assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
        assert _rel(_run(bf, plan, g, adjoint=True, ld=F.N + 24), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_complex128_factor_input(bf):
    """Factors given in complex128 are rounded to complex64 on upload."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(6, 4, 5, seed=8, dtype=np.complex128)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=9, dtype=np.complex64)
    assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
    plan.destroy()


def test_host_buffers_pinned_and_pageable(bf):
    """bf_apply with host pointers stages through device buffers."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(6, 8, 6, seed=21, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=2)
    g = complex_normal((3, F.N), seed=22, dtype=np.complex64)
    # pageable numpy buffers
    out = np.zeros_like(g)
    bf.bf_apply(plan, g, out, nrhs=3)
    torch.cuda.synchronize()
    assert _rel(out, _oracle(F, g)) < TOL
    # pinned torch buffers
    gp = torch.from_numpy(g).pin_memory()
    op = torch.zeros_like(gp).pin_memory()
    bf.bf_apply_adjoint(plan, gp, op, nrhs=3)
    torch.cuda.synchronize()
    assert _rel(op.numpy(), _oracle(F, g, True)) < TOL
    plan.destroy()


def test_host_buffers_overlapped_groups(bf):
    """Host buffers on the single-vector path run as four node groups on side
    streams, each group's copies overlapping the other groups' kernels: host
    input with device output and the reverse, a leading dimension above N (2-D
    copies), several RHS chunks -- against the FP64 oracle; and at N = 2^20 the
    host-buffer result equals the device-buffer result bit for bit (the same
    kernels on the same data)."""
    from bfinputs import complex_normal, synthetic_factors
    dev = torch.device("cuda:0")
    F = synthetic_factors(10, 16, 8, seed=31, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=2)
    ld = F.N + 5
    g = complex_normal((3, F.N), seed=32, dtype=np.complex64)
    gh = np.zeros((3, ld), np.complex64)
    gh[:, :F.N] = g
    oh = np.full((3, ld), 9.0 + 9.0j, np.complex64)
    bf.bf_apply(plan, gh, oh, nrhs=3, ld=ld)                       # host -> host, ld > N
    torch.cuda.synchronize()
    assert _rel(oh[:, :F.N], _oracle(F, g)) < TOL
    assert np.all(oh[:, F.N:] == 9.0 + 9.0j), "padding between columns was written"
    od = torch.zeros((3, F.N), dtype=torch.complex64, device=dev)
    gp = torch.from_numpy(g).pin_memory()          # kept alive until the copies have run
    bf.bf_apply_adjoint(plan, gp, od)              # host -> device
    torch.cuda.synchronize()
    assert _rel(od.cpu().numpy(), _oracle(F, g, True)) < TOL
    op = torch.zeros((3, F.N), dtype=torch.complex64).pin_memory()
    gd = torch.from_numpy(g).to(dev)
    bf.bf_apply(plan, gd, op)                      # device -> host
    torch.cuda.synchronize()
    assert _rel(op.numpy(), _oracle(F, g)) < TOL
    bf.bf_plan_check(plan)
    plan.destroy()

    F = synthetic_factors(16, 16, 16, seed=0, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=33, dtype=np.complex64)
    for adjoint in (False, True):
        fn = bf.bf_apply_adjoint if adjoint else bf.bf_apply
        gd, yd = torch.from_numpy(g).to(dev), torch.empty((1, F.N), dtype=torch.complex64, device=dev)
        fn(plan, gd, yd)
        gp, yh = torch.from_numpy(g).pin_memory(), torch.empty((1, F.N), dtype=torch.complex64).pin_memory()
        fn(plan, gp, yh)
        torch.cuda.synchronize()
        assert np.array_equal(yh.numpy(), yd.cpu().numpy())
    bf.bf_plan_check(plan)
    plan.destroy()


@pytest.mark.parametrize("L,n0,r", [(0, 5, 3), (2, 4, 3), (4, 3, 5)])
def test_host_buffers_shallow_trees(bf, L, n0, r):
    """The host-buffer path on trees with fewer than four middle-level nodes
    (m = 1: one launch; m = 2: two groups of one node; m = 4: four of one),
    forward and adjoint, against the FP64 oracle."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(L, n0, r, seed=40 + L, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=2)
    g = complex_normal((3, F.N), seed=41 + L, dtype=np.complex64)
    for adjoint in (False, True):
        out = np.zeros_like(g)
        (bf.bf_apply_adjoint if adjoint else bf.bf_apply)(plan, g, out, nrhs=3)
        torch.cuda.synchronize()
        assert _rel(out, _oracle(F, g, adjoint)) < TOL
    bf.bf_plan_check(plan)
    plan.destroy()


def test_adjoint_identity_fp32(bf):
    """<K g, f> = <g, K^* f> for the GPU apply and adjoint (FP32)."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(10, 16, 8, seed=2, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=1, dtype=np.complex64)
    f = complex_normal((1, F.N), seed=2, dtype=np.complex64)
    Kg = _run(bf, plan, g).astype(np.complex128)
    Kf = _run(bf, plan, f, adjoint=True).astype(np.complex128)
    lhs = np.vdot(f, Kg)
    rhs = np.vdot(Kf, g)
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(Kg) * np.linalg.norm(f)
    plan.destroy()


def test_zero_rhs_and_invalid_calls(bf):
    from bfinputs import synthetic_factors
    F = synthetic_factors(4, 4, 4, seed=1, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    x = torch.zeros((2, F.N), dtype=torch.complex64, device="cuda")
    bf.bf_apply(plan, x, x[1:], nrhs=0)                     # no-op
    with pytest.raises(bf.BfError) as e:
        bf.bf_apply(plan, x, x, nrhs=1)                     # in == out
    assert e.value.status == bf.BF_ERR_INVALID
    with pytest.raises(bf.BfError) as e:
        bf.bf_apply(plan, x, x[1:], nrhs=1, ld=F.N - 1)     # ld < N
    assert e.value.status == bf.BF_ERR_INVALID
    assert bf.bf_plan_device_bytes(plan) > 0
    plan.destroy()


def test_profiling_counts_launches(bf):
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(6, 4, 4, seed=1, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    bf.bf_plan_set_profiling(plan, True)
    g = torch.from_numpy(complex_normal((1, F.N), seed=1, dtype=np.complex64)).cuda()
    y = torch.empty_like(g)
    for _ in range(3):
        bf.bf_apply(plan, g, y)
    t = bf.bf_plan_kernel_times(plan)
    assert t["down"][0] == 3 and t["up"][0] == 3 and t["down"][1] > 0 and t["up"][1] > 0
    plan.destroy()


@pytest.mark.slow
def test_full_size_n1m_r16_against_c_oracle(bf):
    """N = 2^20, L = 16 (leaf 16), r = 16 -- the benchmarked shape -- in the
    launch configuration the benchmark times (one RHS), every output entry
    against the FP64 C loops of the oracle on the same factors."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import capply
    F = synthetic_factors(16, 16, 16, seed=0, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=0, dtype=np.complex64)
    P = capply.PreparedFactors(F)
    u = _run(bf, plan, g)
    assert _rel(u[0], capply.bf_apply_c(P, g[0])) < TOL
    a = _run(bf, plan, g, adjoint=True)
    assert _rel(a[0], capply.bf_adjoint_c(P, g[0])) < TOL
    plan.destroy()


def test_full_size_n1m_r16_tensor_core_batch(bf):
    """N = 2^20, L = 16, r = 16 with 128 RHS -- the batch the benchmark's
    tensor-core line times -- on the tcgen05 core: four sampled RHS columns
    of the apply and of the adjoint against the FP64 C loops of the oracle,
    and, for every column, the adjoint identity <K g, f> = <g, K^* f>."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import capply
    F = synthetic_factors(16, 16, 16, seed=0, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=128)
    g = complex_normal((128, F.N), seed=5, dtype=np.complex64)
    f = complex_normal((128, F.N), seed=6, dtype=np.complex64)
    u = _run(bf, plan, g)
    a = _run(bf, plan, f, adjoint=True)
    P = capply.PreparedFactors(F)
    for j in (0, 1, 64, 127):
        assert _rel(u[j], capply.bf_apply_c(P, g[j])) < TOL
        assert _rel(a[j], capply.bf_adjoint_c(P, f[j])) < TOL
    lhs = np.einsum("ij,ij->i", u.astype(np.complex128), np.conj(f.astype(np.complex128)))
    rhs = np.einsum("ij,ij->i", g.astype(np.complex128), np.conj(a.astype(np.complex128)))
    scale = np.linalg.norm(u, axis=1) * np.linalg.norm(f, axis=1)
    assert np.max(np.abs(lhs - rhs) / scale) < TOL
    # 32 vectors (the benchmark sweep's 32-RHS point): one 32-wide tile
    u32 = _run(bf, plan, g[:32])
    a32 = _run(bf, plan, f[:32], adjoint=True)
    for j in (0, 31):
        assert _rel(u32[j], capply.bf_apply_c(P, g[j])) < TOL
        assert _rel(a32[j], capply.bf_adjoint_c(P, f[j])) < TOL
    plan.destroy()


@pytest.mark.parametrize("adjoint,nrhs", [(False, 128), (True, 128), (False, 40)])
def test_precision_ladder_tensor_core(bf, adjoint, nrhs):
    """The tensor-core core's five rungs at N = 2^16, L = 12, r = 16, 128 RHS,
    forward and adjoint, against the FP64 C oracle on sampled columns.  The
    FP32-level rungs (3xTF32, the default, and the BF16 three-way split) are
    within the FP32 tolerance.  The others sit where their operands' mantissas
    put them, well above the FP32 bar and well below 1: plain TF32 (11 bits,
    ~1e-3), the BF16 hi/lo split (16 bits, ~1e-5) and plain BF16 (8 bits,
    ~6e-3).  The order of the rungs pins that each one really forms the
    products it claims.  40 vectors run as one 64-wide tile."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import capply
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(12, 16, 16, seed=4, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=128)
    g = complex_normal((nrhs, F.N), seed=8, dtype=np.complex64)
    P = capply.PreparedFactors(F)
    fn = capply.bf_adjoint_c if adjoint else capply.bf_apply_c
    cols = (0, nrhs * 3 // 5, nrhs - 1)
    ref = [fn(P, g[j]) for j in cols]
    errs = {}
    for prec in (capi.BF_PREC_FP32, capi.BF_PREC_TF32, capi.BF_PREC_BF16X6, capi.BF_PREC_BF16X3, capi.BF_PREC_BF16):
        capi.bf_plan_set_precision(plan, prec)
        u = _run(bf, plan, g, adjoint=adjoint)
        errs[prec] = max(_rel(u[j], r) for j, r in zip(cols, ref))
    assert errs[capi.BF_PREC_FP32] < TOL
    assert errs[capi.BF_PREC_BF16X6] < TOL
    assert 1e-4 < errs[capi.BF_PREC_TF32] < 1e-2
    assert 2e-6 < errs[capi.BF_PREC_BF16X3] < 5e-5
    assert 1e-3 < errs[capi.BF_PREC_BF16] < 3e-2
    assert errs[capi.BF_PREC_BF16X6] < errs[capi.BF_PREC_BF16X3] < errs[capi.BF_PREC_TF32] < errs[capi.BF_PREC_BF16]
    with pytest.raises(capi.BfError):
        capi.bf_plan_set_precision(plan, 7)
    plan.destroy()


def test_bounded_wait_expiry_reports_timeout_and_context_survives(bf, monkeypatch):
    """Failure detection without a GPU fault: with the stall hook the fused
    kernels' producer issues no copies, every consumer wait runs into its
    bound (about 2 s), the launch ends with the error word set, and
    bf_plan_check reports BF_ERR_TIMEOUT.  The context stays usable: a plan
    created afterwards computes the right result."""
    from bfinputs import complex_normal, synthetic_factors
    monkeypatch.setenv("BF_INJECT_STALL", "1")
    F = synthetic_factors(6, 4, 5, seed=3, dtype=np.complex64)
    stalled = bf.bf_plan_create(F, nrhs_max=1)
    monkeypatch.delenv("BF_INJECT_STALL")
    g = complex_normal((1, F.N), seed=4, dtype=np.complex64)
    x = torch.from_numpy(g).cuda()
    y = torch.empty_like(x)
    bf.bf_apply(stalled, x, y)
    torch.cuda.synchronize()
    with pytest.raises(bf.BfError) as err:
        bf.bf_plan_check(stalled)
    assert err.value.status == bf.BF_ERR_TIMEOUT
    bf.bf_plan_check(stalled)          # the error word was cleared
    stalled.destroy()
    plan = bf.bf_plan_create(F, nrhs_max=1)
    assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
    plan.destroy()


def test_workspace_allocation_failure_is_reported(bf):
    """A workspace the GPU cannot hold is refused with BF_ERR_NOMEM, the
    partial plan is released, and the next plan works."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(8, 16, 16, seed=5, dtype=np.complex64)
    with pytest.raises(bf.BfError) as err:
        bf.bf_plan_create(F, nrhs_max=1 << 26)      # 2^8 r x 2^26 vectors x 8 B = 2 TB of workspace
    assert err.value.status == bf.BF_ERR_NOMEM
    g = complex_normal((3, F.N), seed=6, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=3)
    assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
    plan.destroy()


def test_bf16_rungs_keep_split_blocks_only_while_set(bf):
    """A BF16 rung splits the tensor-core blocks once into BF16 parts (2, 4
    or 6 bytes per real entry beside the FP32 blocks' 4); switching back to
    a TF32 rung releases them, and every switch reproduces the rung's result
    bit for bit."""
    from bfinputs import complex_normal, synthetic_factors
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(8, 16, 16, seed=12, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=64)
    g = complex_normal((64, F.N), seed=13, dtype=np.complex64)
    base = bf.bf_plan_device_bytes(plan)
    out = {}
    extra = {}
    for prec in (capi.BF_PREC_BF16, capi.BF_PREC_BF16X3, capi.BF_PREC_BF16X6):
        capi.bf_plan_set_precision(plan, prec)
        extra[prec] = bf.bf_plan_device_bytes(plan) - base
        out[prec] = _run(bf, plan, g)
    assert extra[capi.BF_PREC_BF16] > 0
    assert extra[capi.BF_PREC_BF16X3] == 2 * extra[capi.BF_PREC_BF16]
    assert extra[capi.BF_PREC_BF16X6] == 3 * extra[capi.BF_PREC_BF16]
    capi.bf_plan_set_precision(plan, capi.BF_PREC_FP32)
    assert bf.bf_plan_device_bytes(plan) == base
    for prec in (capi.BF_PREC_BF16X3, capi.BF_PREC_BF16):
        capi.bf_plan_set_precision(plan, prec)
        assert np.array_equal(_run(bf, plan, g), out[prec])
    plan.destroy()


def test_tensor_core_bounded_waits_report_timeout(bf, monkeypatch):
    """Failure detection on the tensor-core core, without a GPU fault: with the
    stall hook its producer issues no copies, every wait of the other warps
    runs into its bound, the launch ends with the error word set (tensor
    memory released), bf_plan_check reports BF_ERR_TIMEOUT, and a plan made
    afterwards computes the right result on the same context."""
    from bfinputs import complex_normal, synthetic_factors
    F = synthetic_factors(4, 16, 16, seed=31, dtype=np.complex64)
    monkeypatch.setenv("BF_INJECT_STALL", "1")
    stalled = bf.bf_plan_create(F, nrhs_max=128)
    monkeypatch.delenv("BF_INJECT_STALL")
    g = complex_normal((128, F.N), seed=32, dtype=np.complex64)
    x = torch.from_numpy(g).cuda()
    y = torch.empty_like(x)
    bf.bf_apply(stalled, x, y)
    torch.cuda.synchronize()
    with pytest.raises(bf.BfError) as err:
        bf.bf_plan_check(stalled)
    assert err.value.status == bf.BF_ERR_TIMEOUT
    stalled.destroy()
    plan = bf.bf_plan_create(F, nrhs_max=128)
    assert _rel(_run(bf, plan, g), _oracle(F, g)) < TOL
    plan.destroy()


def test_plan_from_factor_file_matches_plan_from_arrays(bf, tmp_path):
    """A factorization stored with bf_factor_file_save and planned with
    bf_plan_create_from_file applies bit for bit like the plan made from the
    arrays, in complex64 and complex128 files (complex128 input is rounded on
    the device side exactly as bf_plan_create rounds it)."""
    from bfinputs import complex_normal, synthetic_factors
    from paper_1502_01379_gb300 import capi
    for dtype in (np.complex64, np.complex128):
        F = synthetic_factors(8, 16, 16, seed=21, dtype=dtype)
        path = str(tmp_path / "f.bfly")
        capi.bf_factor_file_save(F, path, dtype=dtype)
        p1 = bf.bf_plan_create(F, nrhs_max=40)
        p2 = capi.bf_plan_create_from_file(path, nrhs_max=40)
        for n in (1, 40):
            g = complex_normal((n, F.N), seed=n, dtype=np.complex64)
            for adjoint in (False, True):
                a = _run(bf, p1, g, adjoint=adjoint)
                b = _run(bf, p2, g, adjoint=adjoint)
                assert np.array_equal(a, b)
                assert _rel(b, _oracle(F, g, adjoint)) < TOL
        p1.destroy()
        p2.destroy()


def test_largest_node_segment_leaf64_r32_n1m(bf):
    """The compiled limits at once: L = 14, leaf 64, rank 32 (N = 2^20), a
    middle-level node segment of m max(leaf, r) = 8192 entries (the largest a
    plan takes; its ring slots shrink to fit shared memory).  Every output
    entry of the apply and the adjoint, one vector on the fused kernels and
    9 vectors on the multi-RHS core, against the FP64 C loops of the oracle."""
    from bfinputs import complex_normal, synthetic_factors
    from oracle import capply
    F = synthetic_factors(14, 64, 32, seed=41, dtype=np.complex64)
    assert F.m * max(F.n0, F.r) == 8192
    P = capply.PreparedFactors(F)
    for nrhs in (1, 9):
        plan = bf.bf_plan_create(F, nrhs_max=nrhs)
        g = complex_normal((nrhs, F.N), seed=nrhs, dtype=np.complex64)
        u = _run(bf, plan, g)
        a = _run(bf, plan, g, adjoint=True)
        plan.destroy()
        for j in sorted({0, nrhs - 1}):
            assert _rel(u[j], capply.bf_apply_c(P, g[j])) < TOL
            assert _rel(a[j], capply.bf_adjoint_c(P, g[j])) < TOL
