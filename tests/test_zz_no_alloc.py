"""bf_apply_static_scratch: the apply/adjoint for callers that cannot allocate
device memory when they run the operator (their GPU memory belongs to another
allocator, or an allocation's implicit synchronization is not acceptable in
their loop).  It keeps the intermediate vector in the library's fixed 16 MiB
device array (2^21 complex64 entries) instead of a workspace, so it must give
the FP64 oracle's result, call after call, although every call reuses that one
array; batches whose level-h vectors do not fit the array at once run in
several passes over it.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5
SCRATCH_ENTRIES = 1 << 21


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


# (L, n0, r, nrhs, extra ld): the second shape has 2^L r = 2^20 entries per
# vector at level h, so the array holds two vectors and nrhs = 3 takes two
# passes over it, the second one partial; its columns sit ld = N + 24 apart.
@pytest.mark.parametrize("L,n0,r,nrhs,pad", [(6, 4, 5, 2, 0), (12, 16, 16, 3, 8), (16, 16, 16, 3, 24)])
def test_static_scratch_matches_the_oracle_twice(bf, L, n0, r, nrhs, pad):
    from bfinputs import complex_normal, synthetic_factors
    from oracle import capply
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(L, n0, r, seed=77 + L, dtype=np.complex64)
    passes = -(-nrhs // (SCRATCH_ENTRIES // ((1 << L) * r)))
    if L == 16:
        assert passes == 2
    P = capply.PreparedFactors(F)
    plan = bf.bf_plan_create(F, nrhs_max=nrhs)
    ld = F.N + pad
    for call in range(2):                       # two calls in a row share the array
        g = complex_normal((nrhs, F.N), seed=call + 5 + L, dtype=np.complex64)
        x = torch.zeros((nrhs, ld), dtype=torch.complex64, device="cuda")
        x[:, :F.N] = torch.from_numpy(g).cuda()
        for adjoint in (False, True):
            out = torch.full((nrhs, ld), 3.0 + 3.0j, dtype=torch.complex64, device="cuda")
            capi.bf_apply_static_scratch(plan, x, out, nrhs=nrhs, ld=ld, adjoint=adjoint)
            torch.cuda.synchronize()
            y = out.cpu().numpy()
            assert np.all(y[:, F.N:] == 3.0 + 3.0j), "padding between columns was written"
            oracle = capply.bf_adjoint_c if adjoint else capply.bf_apply_c
            for j in range(nrhs):
                assert _rel(y[j, :F.N], oracle(P, g[j])) < TOL, (call, adjoint, j)
    bf.bf_plan_check(plan)
    plan.destroy()


def test_static_scratch_rejects_host_pointers(bf):
    from bfinputs import synthetic_factors
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(4, 4, 4, seed=1, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = np.zeros((1, F.N), np.complex64)
    y = np.zeros_like(g)
    lib = bf.load()
    import ctypes
    st = lib.bf_apply_static_scratch(ctypes.c_void_p(plan.handle), ctypes.c_void_p(g.ctypes.data),
                                     ctypes.c_void_p(y.ctypes.data), 1, F.N, 0, None)
    assert st == bf.BF_ERR_INVALID
    with pytest.raises(bf.BfError):             # the wrapper refuses them before the call
        capi.bf_apply_static_scratch(plan, g, y)
    plan.destroy()


def test_static_scratch_refuses_a_plan_of_another_device(bf):
    """A plan's factors live on the device it was created on; a call made
    with another device current would pair that device's scratch array with
    them, so the library refuses it."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two devices")
    from bfinputs import synthetic_factors
    from paper_1502_01379_gb300 import capi
    import ctypes
    F = synthetic_factors(4, 4, 4, seed=1, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    x = torch.zeros((1, F.N), dtype=torch.complex64, device="cuda:0")
    y = torch.empty_like(x)
    with torch.cuda.device(1):
        st = bf.load().bf_apply_static_scratch(ctypes.c_void_p(plan.handle), ctypes.c_void_p(x.data_ptr()),
                                               ctypes.c_void_p(y.data_ptr()), 1, F.N, 0, None)
    assert st == bf.BF_ERR_INVALID
    capi.bf_apply_static_scratch(plan, x, y)
    torch.cuda.synchronize()
    plan.destroy()
