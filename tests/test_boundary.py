"""Host-side checks of the C ABI: the library loads, exports every symbol the
header declares, and validates arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    syms = []
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", name)).read()
            syms += re.findall(r"^[a-z_ ]*?\*?\s*\b(obfft_[a-z_0-9]+)\s*\(", txt, re.M)
    return sorted(set(syms))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_23698_gb300 import _lib
    from paper_2606_23698_gb300 import build as B
    B.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    syms = header_symbols()
    assert "obfft_plan_create" in syms and "obfft_exec" in syms and "obfft_destroy" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    from paper_2606_23698_gb300 import _lib
    assert set(_lib.EXPORTS) == set(header_symbols())


def test_argument_validation(lib):
    h = ctypes.c_void_p()
    assert lib.obfft_plan_create(ctypes.byref(h), 0, 4, 4, 1, 1) == 1
    assert lib.obfft_plan_create(None, 4, 4, 4, 1, 1) == 1
    assert lib.obfft_plan_create(ctypes.byref(h), 4, 4, 4, 1, 7) == 1       # bad mode
    assert lib.obfft_plan_create(ctypes.byref(h), 4, 4, 134, 1, 1) == 2     # 134 = 2 * 67
    assert lib.obfft_plan_create(ctypes.byref(h), 4, 4, 8192, 1, 1) == 2    # > 64 * 64
    assert b"factor" in lib.obfft_last_error()
    assert lib.obfft_exec(None, None, None, -1, None) == 1
    assert lib.obfft_destroy(None) == 0
    assert lib.obfft_exec_many(None, None, None, -1, None) == 1


def test_host_constants_match_oracle(lib):
    """The library's own constant generator agrees with the oracle's big-integer
    definitions bit for bit (quantised twiddles, CRT slices, lift weights, M)."""
    from oracle import constants as C
    re_, im_ = ctypes.c_int64(), ctypes.c_int64()
    for N in (8, 12, 16, 24, 32, 64, 96, 128, 192, 384, 1024, 4096):
        step = max(1, N // 97)
        for m in range(0, N, step):
            for d in (-1, 1):
                assert lib.obfft_host_twiddle(m, N, d, ctypes.byref(re_), ctypes.byref(im_)) == 0
                assert (re_.value, im_.value) == C.quantised_twiddle(m, N, d), (m, N, d)
    mods = (ctypes.c_uint32 * 12)()
    us = (ctypes.c_uint8 * 180)()
    ws = (ctypes.c_uint8 * 72)()
    M4 = (ctypes.c_uint32 * 4)()
    assert lib.obfft_host_crt_constants(mods, us, ws, M4) == 0
    assert list(mods) == list(C.MODULI)
    assert [list(us[15 * k:15 * k + 15]) for k in range(12)] == C.U_SLICES
    assert [list(ws[6 * k:6 * k + 6]) for k in range(12)] == C.W_SLICES
    assert sum(int(M4[i]) << (32 * i) for i in range(4)) == C.M


def test_host_constants_fp32_variant_match_oracle(lib):
    """FP32-precision variant: RNE(2^23 omega), the six moduli, their u_k / w_k
    slices and M from the library agree with the oracle's definitions."""
    from oracle import constants as C
    re_, im_ = ctypes.c_int64(), ctypes.c_int64()
    for N in (8, 12, 16, 32, 96, 1024):
        for m in range(0, N, max(1, N // 61)):
            for d in (-1, 1):
                assert lib.obfft_host_twiddle32(m, N, d, ctypes.byref(re_), ctypes.byref(im_)) == 0
                assert (re_.value, im_.value) == C.quantised_twiddle(m, N, d, C.SIGMA_F_EXP_FP32), (m, N, d)
    mods = (ctypes.c_uint32 * 6)()
    us = (ctypes.c_uint8 * 48)()
    ws = (ctypes.c_uint8 * 18)()
    M = ctypes.c_uint64()
    assert lib.obfft_host_crt_constants32(mods, us, ws, ctypes.byref(M)) == 0
    assert list(mods) == list(C.MODULI_FP32)
    assert [list(us[8 * k:8 * k + 8]) for k in range(6)] == C.U_SLICES_FP32
    assert [list(ws[3 * k:3 * k + 3]) for k in range(6)] == C.W_SLICES_FP32
    assert M.value == C.M_FP32
    assert lib.obfft_host_crt_constants32(None, us, ws, ctypes.byref(M)) == 1


def test_huge_axis_lengths_rejected_quickly(lib):
    """Axis lengths far above 64 x 64 (a large prime, one near 1e9, and one whose
    square overflows int64) are rejected before any split search or any GPU
    call, by both plan creation and the no-allocation entry point."""
    import time
    h = ctypes.c_void_p()
    t0 = time.perf_counter()
    for n in ((1 << 61) - 1, 999999937, 4097, 65 * 64):
        for mode in (0, 1, 2):
            assert lib.obfft_plan_create(ctypes.byref(h), n, 1, 1, 1, mode) == 2
        # fake, aligned, distinct pointers: rejected before any use of them
        assert lib.obfft_exec_fp64_noalloc(ctypes.c_void_p(256), ctypes.c_void_p(512), 2, n, 2, -1, None) == 2
        assert b"factor" in lib.obfft_last_error()
    # three axes whose product wraps around int64 but each factors: the grid
    # is still refused as too large, not accepted through the wrapped product
    assert lib.obfft_exec_fp64_noalloc(ctypes.c_void_p(256), ctypes.c_void_p(512), 4096, 4096, 4096, -1, None) == 2
    assert b"exceeds" in lib.obfft_last_error()
    assert time.perf_counter() - t0 < 1.0
    dims = (ctypes.c_int64 * 6)(8, 8, 8, 8, (1 << 61) - 1, 8)
    assert lib.obfft_plan_create_many(ctypes.byref(h), 2, dims, 0) == 2
