"""bf_apply_static_scratch: the apply/adjoint for callers that cannot allocate
device memory when they run the operator (their GPU memory belongs to another
allocator, or an allocation's implicit synchronization is not acceptable in
their loop).  It keeps the intermediate vector in the library's fixed 16 MiB
device array instead of a workspace, so it must give the same results as
bf_apply / bf_apply_adjoint, call after call, although every call reuses that
one array.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
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


@pytest.mark.parametrize("L,n0,r,nrhs", [(12, 16, 16, 3), (6, 4, 5, 2)])
def test_static_scratch_matches_workspace_apply_twice(bf, L, n0, r, nrhs):
    from bfinputs import complex_normal, synthetic_factors
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(L, n0, r, seed=77 + L, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=nrhs)
    for call in range(2):                       # two calls in a row share the array
        g = torch.from_numpy(complex_normal((nrhs, F.N), seed=call + 5, dtype=np.complex64)).cuda()
        for adjoint in (False, True):
            ref = torch.empty_like(g)
            out = torch.full_like(g, 3.0 + 3.0j)
            (bf.bf_apply_adjoint if adjoint else bf.bf_apply)(plan, g, ref)
            capi.bf_apply_static_scratch(plan, g, out, adjoint=adjoint)
            torch.cuda.synchronize()
            assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL
    bf.bf_plan_check(plan)
    plan.destroy()


def test_static_scratch_rejects_host_pointers(bf):
    from bfinputs import synthetic_factors
    from paper_1502_01379_gb300 import capi
    F = synthetic_factors(4, 4, 4, seed=1, dtype=np.complex64)
    plan = bf.bf_plan_create(F, nrhs_max=1)
    g = np.zeros((1, F.N), np.complex64)
    y = np.zeros_like(g)
    with pytest.raises(bf.BfError) as e:
        capi.bf_apply_static_scratch(plan, g, y)
    assert e.value.status == bf.BF_ERR_INVALID
    plan.destroy()
