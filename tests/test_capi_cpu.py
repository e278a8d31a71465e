"""The C-ABI library builds, loads and exports every entry point of
include/bfly.h; argument checks that precede any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1502_01379_gb300 as bf
from paper_1502_01379_gb300 import build as pkg_build
from paper_1502_01379_gb300 import capi


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return bf.load()


def _declared(repo_root):
    text = open(os.path.join(repo_root, "include", "bfly.h")).read()
    return sorted(set(re.findall(r"^\s*(?:bf_status|size_t|int|const char \*)\s*(bf_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi(repo_root):
    names = _declared(repo_root)
    for n in ("bf_plan_create", "bf_apply", "bf_apply_adjoint", "bf_plan_destroy", "bf_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib, repo_root):
    for name in _declared(repo_root):
        assert hasattr(lib, name), name
    assert set(capi.EXPORTS) <= set(_declared(repo_root))


def test_status_strings(lib):
    for s in range(6):
        assert bf.bf_status_string(s).startswith("BF_")


class _F:
    def __init__(self, L, n0, r):
        h, m, nb = L // 2, 1 << (L // 2), 1 << L
        self.L, self.n0, self.r = L, n0, r
        self.VL = np.zeros((nb, n0, r), np.complex64)
        self.UL = np.zeros((nb, n0, r), np.complex64)
        self.H = [np.zeros((nb, r, 2 * r), np.complex64) for _ in range(h)]
        self.G = [np.zeros((nb, r, 2 * r), np.complex64) for _ in range(h)]
        self.S = np.zeros((m, m, r), np.float32)


def _create(lib, L, n0, r, nrhs_max=1, dtype=capi.BF_C64, null_vl=False):
    F = _F(min(max(L, 0) // 2 * 2, 4), max(n0, 1), max(r, 1))
    nptr = max(1, L // 2)
    h_arr = (ctypes.c_void_p * nptr)(*([F.VL.ctypes.data] * nptr))
    g_arr = (ctypes.c_void_p * nptr)(*([F.UL.ctypes.data] * nptr))
    f = capi.bf_factors(dtype, None if null_vl else F.VL.ctypes.data, ctypes.cast(h_arr, ctypes.POINTER(ctypes.c_void_p)),
                        F.S.ctypes.data, ctypes.cast(g_arr, ctypes.POINTER(ctypes.c_void_p)), F.UL.ctypes.data)
    d = capi.bf_desc(L, n0, r, nrhs_max)
    h = ctypes.c_void_p(1234)
    st = lib.bf_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.byref(f), None)
    return st, h.value


@pytest.mark.parametrize("args,expect", [
    (dict(L=3, n0=4, r=2), capi.BF_ERR_INVALID),          # L odd
    (dict(L=-2, n0=4, r=2), capi.BF_ERR_INVALID),
    (dict(L=4, n0=0, r=2), capi.BF_ERR_INVALID),
    (dict(L=4, n0=4, r=0), capi.BF_ERR_INVALID),
    (dict(L=4, n0=4, r=2, nrhs_max=0), capi.BF_ERR_INVALID),
    (dict(L=4, n0=4, r=2, dtype=7), capi.BF_ERR_INVALID),
    (dict(L=4, n0=4, r=2, null_vl=True), capi.BF_ERR_INVALID),
    (dict(L=4, n0=4, r=33), capi.BF_ERR_UNSUPPORTED),      # r above 32
    (dict(L=4, n0=65, r=2), capi.BF_ERR_UNSUPPORTED),      # leaf above 64
    (dict(L=26, n0=1, r=1), capi.BF_ERR_UNSUPPORTED),      # depth above 24
])
def test_plan_create_rejects_before_any_cuda_call(lib, args, expect):
    st, h = _create(lib, **args)
    assert st == expect
    assert h is None


def test_null_arguments(lib):
    assert lib.bf_plan_create(None, None, None, None) == capi.BF_ERR_INVALID
    h = ctypes.c_void_p(99)
    assert lib.bf_plan_create(ctypes.byref(h), None, None, None) == capi.BF_ERR_INVALID
    assert h.value is None
    assert lib.bf_apply(None, None, None, 1, 16, None) == capi.BF_ERR_INVALID
    assert lib.bf_apply_adjoint(None, None, None, 1, 16, None) == capi.BF_ERR_INVALID
    assert lib.bf_plan_destroy(None) == capi.BF_OK
    assert lib.bf_plan_device_bytes(None) == 0
    assert lib.bf_plan_check(None, None) == capi.BF_ERR_INVALID
    assert lib.bf_plan_set_profiling(None, 1) == capi.BF_ERR_INVALID
