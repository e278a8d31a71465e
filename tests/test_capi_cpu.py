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
    return sorted(set(re.findall(r"^\s*(?:bf_status|size_t|unsigned int|int|const char \*)\s*(bf_\w+)\s*\(", text, re.M)))


def test_header_declares_the_abi(repo_root):
    names = _declared(repo_root)
    for n in ("bf_plan_create", "bf_apply", "bf_apply_adjoint", "bf_plan_destroy", "bf_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib, repo_root):
    for name in _declared(repo_root):
        assert hasattr(lib, name), name
    assert set(capi.EXPORTS) <= set(_declared(repo_root))


def test_status_strings(lib):
    for s in range(7):
        assert bf.bf_status_string(s).startswith("BF_")
    assert "factor file" in bf.bf_status_string(capi.BF_ERR_CORRUPT)


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


# ---------------------------------------------------- wrapper-side buffer checks
# The kernels read (nrhs-1)*ld + N complex64 entries through a bare pointer;
# the Python wrapper is the only place that can see the buffers' sizes, dtypes
# and devices, so it must reject bad ones before any call reaches the library.
def _fake_plan(N=64):
    return capi.Plan(0, N, 4, N >> 4, 2, 1, device=0)


@pytest.mark.parametrize("case", ["x_c128", "y_short", "nrhs_too_big", "y_float", "ld_small", "nrhs_negative"])
def test_wrapper_rejects_bad_vectors_before_the_call(lib, case):
    torch = pytest.importorskip("torch")
    P = _fake_plan()
    x = np.zeros((2, P.N), np.complex64)
    y = np.zeros((2, P.N), np.complex64)
    kw = {}
    if case == "x_c128":
        x = x.astype(np.complex128)
    elif case == "y_short":
        y = y[:1]
    elif case == "nrhs_too_big":
        kw = dict(nrhs=3)
    elif case == "y_float":
        x, y = torch.from_numpy(x), torch.zeros(2 * P.N, dtype=torch.float32)
    elif case == "ld_small":
        kw = dict(nrhs=1, ld=P.N - 1)
    elif case == "nrhs_negative":
        kw = dict(nrhs=-1)
    for fn in (capi.bf_apply, capi.bf_apply_adjoint):
        with pytest.raises(capi.BfArgumentError) as e:
            fn(P, x, y, **kw)
        assert e.value.status == capi.BF_ERR_INVALID
        assert isinstance(e.value, ValueError)


def test_wrapper_rejects_host_buffers_where_device_ones_are_required(lib):
    torch = pytest.importorskip("torch")
    P = _fake_plan()
    x = torch.zeros((1, P.N), dtype=torch.complex64)
    for call in (lambda: capi.bf_apply_static_scratch(P, x, torch.empty_like(x)),
                 lambda: capi.bf_quad_apply(P, x, torch.empty_like(x)),
                 lambda: capi.bf_quad_apply(P, x.numpy(), np.empty_like(x.numpy()))):
        with pytest.raises(capi.BfArgumentError):
            call()


def test_wrapper_passes_well_formed_buffers_to_the_library(lib):
    """Correct buffers get past the wrapper; the library itself then rejects
    the null plan handle (status BF_ERR_INVALID, not a wrapper error)."""
    P = _fake_plan()
    x = np.zeros((3, P.N + 5), np.complex64)
    y = np.zeros((3, P.N + 5), np.complex64)
    with pytest.raises(capi.BfError) as e:
        capi.bf_apply(P, x, y, nrhs=3, ld=P.N + 5, stream=0)
    assert not isinstance(e.value, capi.BfArgumentError)
    assert e.value.status == capi.BF_ERR_INVALID



# ------------------------------------------------------------------ factor files
def test_crc32_check_value_and_zlib_agree(lib):
    """The CRC-32 of ISO-HDLC: check value 0xCBF43926 for "123456789" (its
    published definition), and the library agrees with zlib on odd lengths
    (the eight-bytes-per-step loop and the byte tail)."""
    import zlib
    assert capi.bf_crc32(b"123456789") == 0xCBF43926
    rng = np.random.default_rng(0)
    for n in (0, 1, 7, 8, 9, 63, 1000):
        b = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert capi.bf_crc32(b) == zlib.crc32(b)
        assert capi.bf_crc32(b[n // 2:], capi.bf_crc32(b[:n // 2])) == zlib.crc32(b)


@pytest.mark.parametrize("L,n0,r,dtype", [(4, 4, 3, np.complex64), (0, 5, 3, np.complex64), (6, 2, 5, np.complex128)])
def test_factor_file_round_trip_and_corruption(lib, tmp_path, L, n0, r, dtype):
    """A saved factor file verifies and reports its shape; a flipped byte in
    the payload or the header, a truncated or extended file, a wrong magic or
    an inconsistent size field give BF_ERR_CORRUPT, another version
    BF_ERR_UNSUPPORTED -- all before any CUDA call (no GPU here)."""
    import struct
    import zlib
    from bfinputs import synthetic_factors
    F = synthetic_factors(L, n0, r, seed=5, dtype=dtype)
    path = str(tmp_path / "f.bfly")
    nbytes = capi.bf_factor_file_save(F, path, dtype=dtype)
    assert os.path.getsize(path) == nbytes
    assert capi.bf_factor_file_check(path) == (L, n0, r, capi.BF_C64 if dtype == np.complex64 else capi.BF_C128)
    good = open(path, "rb").read()
    # the payload holds exactly the arrays in canonical order
    pay = good[64:]
    cdt = np.dtype(dtype)
    assert np.array_equal(np.frombuffer(pay[:F.VL.size * cdt.itemsize], cdt).reshape(F.VL.shape), F.VL.astype(cdt))
    assert np.array_equal(np.frombuffer(pay[-F.UL.size * cdt.itemsize:], cdt).reshape(F.UL.shape), F.UL.astype(cdt))

    def check(blob):
        bad = str(tmp_path / "bad.bfly")
        open(bad, "wb").write(blob)
        with pytest.raises(capi.BfError) as e:
            capi.bf_factor_file_check(bad)
        h = ctypes.c_void_p(7)
        st = lib.bf_plan_create_from_file(ctypes.byref(h), os.fsencode(bad), 1, None)
        assert st == e.value.status and h.value is None
        return e.value.status

    def rehead(blob, **kw):
        fields = list(struct.unpack("<IIiiiIQI", blob[8:44]))
        for k, v in kw.items():
            fields[["version", "dtype", "L", "leaf", "r", "zero", "size", "crc"].index(k)] = v
        head = blob[:8] + struct.pack("<IIiiiIQI", *fields)
        return head + struct.pack("<I", zlib.crc32(head)) + blob[48:]

    flip = lambda b, i: b[:i] + bytes([b[i] ^ 0x10]) + b[i + 1:]
    assert check(flip(good, 64 + len(pay) // 2)) == capi.BF_ERR_CORRUPT        # payload byte
    assert check(flip(good, len(good) - 1)) == capi.BF_ERR_CORRUPT              # last payload byte
    assert check(flip(good, 18)) == capi.BF_ERR_CORRUPT                         # header byte (L)
    assert check(good[:-8]) == capi.BF_ERR_CORRUPT                              # truncated
    assert check(good + b"\0" * 8) == capi.BF_ERR_CORRUPT                       # trailing bytes
    assert check(good[:40]) == capi.BF_ERR_CORRUPT                              # header cut
    assert check(b"XFLYFAC\0" + good[8:]) == capi.BF_ERR_CORRUPT                # magic
    assert check(rehead(good, size=len(pay) + 8)) == capi.BF_ERR_CORRUPT        # size field vs shape
    assert check(rehead(good, r=33)) == capi.BF_ERR_CORRUPT                     # shape beyond limits
    assert check(rehead(good, dtype=7)) == capi.BF_ERR_CORRUPT
    assert check(rehead(good, version=2)) == capi.BF_ERR_UNSUPPORTED
    assert lib.bf_factor_file_check(os.fsencode(str(tmp_path / "missing")), None, None) == capi.BF_ERR_INVALID
