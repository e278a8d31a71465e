"""The bounds-checked build (libbfly_checked.so, BF_CHECKED): the single-vector
and batched kernels test every global index against the extent their
launch's arguments define.  On valid calls no check may fire and the results
are the FP64 oracle's; a check that fires skips the access and is reported by
bf_plan_check as BF_ERR_INVALID instead of faulting.  The library is loaded
in a fresh process (the binding holds one library per process)."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_1502_01379_gb300 import build, capi
capi.load(build.build(checked=True))
from bfinputs import complex_normal, synthetic_factors
from oracle import apply as A
from oracle.kernel import rel_err
torch.cuda.set_device(0)

def oracle(F, g, adjoint):
    fn = A.bf_adjoint if adjoint else A.bf_apply
    return fn(F.astype(np.complex128), g.T.astype(np.complex128)).T

if MODE == "clean":
    for (L, n0, r, nrhs, pad) in [(0, 5, 3, 2, 0), (4, 3, 5, 3, 7), (8, 16, 16, 5, 0), (10, 2, 7, 2, 3)]:
        F = synthetic_factors(L, n0, r, seed=L + 1, dtype=np.complex64)
        plan = capi.bf_plan_create(F, nrhs_max=nrhs)
        g = complex_normal((nrhs, F.N), seed=L, dtype=np.complex64)
        ld = F.N + pad
        x = torch.zeros((nrhs, ld), dtype=torch.complex64, device="cuda"); x[:, :F.N] = torch.from_numpy(g).cuda()
        for adjoint in (False, True):
            y = torch.zeros_like(x)
            (capi.bf_apply_adjoint if adjoint else capi.bf_apply)(plan, x, y, nrhs=nrhs, ld=ld)
            torch.cuda.synchronize(); capi.bf_plan_check(plan)
            assert rel_err(y.cpu().numpy()[:, :F.N], oracle(F, g, adjoint)) < 1e-5
            yh = np.zeros((nrhs, F.N), np.complex64)          # host buffers: the staging path
            (capi.bf_apply_adjoint if adjoint else capi.bf_apply)(plan, g, yh)
            torch.cuda.synchronize(); capi.bf_plan_check(plan)
            assert rel_err(yh, oracle(F, g, adjoint)) < 1e-5
            ys = torch.zeros_like(x)
            capi.bf_apply_static_scratch(plan, x, ys, nrhs=nrhs, ld=ld, adjoint=adjoint)
            torch.cuda.synchronize(); capi.bf_plan_check(plan)
            assert rel_err(ys.cpu().numpy()[:, :F.N], oracle(F, g, adjoint)) < 1e-5
        plan.destroy()
    Fs = [synthetic_factors(L, n0, r, seed=30 + L, dtype=np.complex64) for (L, n0, r) in [(2, 4, 3), (6, 16, 8), (8, 32, 8)]]
    gs = [complex_normal((k, F.N), seed=40 + k, dtype=np.complex64) for k, F in zip((1, 6, 9), Fs)]
    ins = [torch.from_numpy(g).cuda() for g in gs]; outs = [torch.empty_like(x) for x in ins]
    for T in (1, 4, 8):
        b = capi.bf_batch_create(Fs, ins, outs, [g.shape[0] for g in gs], T=T)
        for adjoint in (False, True):
            capi.bf_batch_apply(b, adjoint, capi.BF_BATCH_GRAPH)
            torch.cuda.synchronize(); capi.bf_batch_check(b)
            for F, g, o in zip(Fs, gs, outs):
                assert rel_err(o.cpu().numpy(), oracle(F, g, adjoint)) < 1e-5
        b.destroy()
    print("CHECKED-CLEAN-OK")
else:
    F = synthetic_factors(6, 4, 5, seed=3, dtype=np.complex64)
    plan = capi.bf_plan_create(F, nrhs_max=1)
    g = complex_normal((1, F.N), seed=2, dtype=np.complex64)
    x = torch.from_numpy(g).cuda()
    y = torch.full_like(x, 5.0 + 5.0j)
    capi.bf_apply(plan, x, y)
    torch.cuda.synchronize()
    try:
        capi.bf_plan_check(plan)
        raise SystemExit("the check did not fire")
    except capi.BfError as e:
        assert e.status == capi.BF_ERR_INVALID, e.status
    out = y.cpu().numpy()[0]
    assert out[-1] == 5.0 + 5.0j, "the store outside the stated extent was not skipped"
    assert rel_err(out[:-1], oracle(F, g, False)[0][:-1]) < 1e-5
    capi.bf_plan_check(plan)                                  # cleared
    print("CHECKED-FIRES-OK")
'''


def _run(mode, env_extra=None):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **(env_extra or {}))
    code = f"ROOT = {root!r}\nMODE = {mode!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    return r.returncode, r.stdout + r.stderr


def test_checked_build_valid_calls_fire_no_check():
    rc, out = _run("clean")
    assert rc == 0 and "CHECKED-CLEAN-OK" in out, out[-3000:]


def test_checked_build_reports_an_access_outside_the_stated_extent():
    rc, out = _run("fires", {"BF_CHECKED_SHRINK_OUT": "1"})
    assert rc == 0 and "CHECKED-FIRES-OK" in out, out[-3000:]
