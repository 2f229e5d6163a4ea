"""ctypes binding of libobfft.so: the C ABI of include/obfft.h, same names,
argument marshalling only (every step of the transform runs in the library's
CUDA kernels).  Loading fails loudly when the library is missing: there is no
CPU fallback."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libobfft.so")

OBFFT_OK = 0
OBFFT_ERR_ARG = 1
OBFFT_ERR_UNSUPPORTED_SIZE = 2
OBFFT_ERR_ALLOC = 3
OBFFT_ERR_CUDA = 4
OBFFT_ERR_TIMEOUT = 5
OBFFT_ERR_INTERNAL = 6
STATUS_NAMES = {0: "OBFFT_OK", 1: "OBFFT_ERR_ARG", 2: "OBFFT_ERR_UNSUPPORTED_SIZE",
                3: "OBFFT_ERR_ALLOC", 4: "OBFFT_ERR_CUDA", 5: "OBFFT_ERR_TIMEOUT",
                6: "OBFFT_ERR_INTERNAL"}

OBFFT_MODE_FP8 = 0
OBFFT_MODE_INT8 = 1
OBFFT_MODE_FP64_NATIVE = 2
OBFFT_MODE_FP16 = 3
OBFFT_MODE_FP32 = 4
OBFFT_MODE_FP32_NATIVE = 5
MODES = {"fp8": OBFFT_MODE_FP8, "int8": OBFFT_MODE_INT8, "fp64": OBFFT_MODE_FP64_NATIVE,
         "fp16": OBFFT_MODE_FP16, "fp32": OBFFT_MODE_FP32, "fp32native": OBFFT_MODE_FP32_NATIVE}
# modes whose data are complex64 (the FP32-precision variant and its comparator)
COMPLEX64_MODES = (OBFFT_MODE_FP32, OBFFT_MODE_FP32_NATIVE)

# every symbol include/obfft.h declares
EXPORTS = ("obfft_plan_create", "obfft_exec", "obfft_destroy", "obfft_plan_get_splits",
           "obfft_plan_create_many", "obfft_exec_many", "obfft_exec_stage", "obfft_last_error",
           "obfft_version", "obfft_host_twiddle", "obfft_host_crt_constants",
           "obfft_exec_fp64_noalloc", "obfft_plan_status", "obfft_selftest_bounded_wait",
           "obfft_exec_host", "obfft_host_twiddle32", "obfft_host_crt_constants32",
           "obfft_ablation_phase_b", "obfft_ablation_residues", "obfft_exec_axes", "obfft_transpose_blocks",
           "obfft_debug_layout", "obfft_exec_debug", "obfft_plan_get_tuning")

_lib = None


class ObfftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libobfft.so not built ({path}); run __graft_entry__.build() or "
                          "python paper_2606_23698_gb300/build.py")
    L = ctypes.CDLL(path)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.obfft_plan_create.argtypes = [ctypes.POINTER(vp), i64, i64, i64, i64, i32]
    L.obfft_plan_create_many.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), i32]
    L.obfft_exec.argtypes = [vp, vp, vp, i32, vp]
    L.obfft_exec_host.argtypes = [vp, vp, vp, i32, vp]
    L.obfft_exec_many.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp]
    L.obfft_exec_stage.argtypes = [vp, i32, i32, vp, vp, i32, vp]
    L.obfft_exec_axes.argtypes = [vp, i32, i32, vp, vp, i32, vp]
    L.obfft_transpose_blocks.argtypes = [vp, vp, i64, i64, i64, vp]
    L.obfft_plan_get_tuning.argtypes = [vp, i32, i32] + [ctypes.POINTER(i32)] * 4
    L.obfft_plan_get_tuning.restype = i32
    L.obfft_debug_layout.argtypes = [i32, i32, i32, i64, ctypes.POINTER(i64)]
    L.obfft_debug_layout.restype = i32
    L.obfft_exec_debug.argtypes = [vp, i32, i32, vp, vp, i32, i64, i64, vp, vp]
    L.obfft_exec_debug.restype = i32
    L.obfft_destroy.argtypes = [vp]
    L.obfft_plan_get_splits.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    for f in ("obfft_plan_create", "obfft_plan_create_many", "obfft_exec", "obfft_exec_host", "obfft_exec_many",
              "obfft_exec_stage", "obfft_destroy", "obfft_plan_get_splits", "obfft_exec_axes",
              "obfft_transpose_blocks"):
        getattr(L, f).restype = i32
    L.obfft_last_error.restype = ctypes.c_char_p
    L.obfft_last_error.argtypes = []
    L.obfft_version.restype = ctypes.c_char_p
    L.obfft_version.argtypes = []
    L.obfft_host_twiddle.argtypes = [i64, i64, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.obfft_host_twiddle.restype = i32
    L.obfft_host_crt_constants.argtypes = [vp, vp, vp, vp]
    L.obfft_host_crt_constants.restype = i32
    L.obfft_host_twiddle32.argtypes = [i64, i64, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.obfft_host_twiddle32.restype = i32
    L.obfft_host_crt_constants32.argtypes = [vp, vp, vp, vp]
    L.obfft_host_crt_constants32.restype = i32
    L.obfft_plan_status.argtypes = [vp, vp]
    L.obfft_plan_status.restype = i32
    L.obfft_selftest_bounded_wait.argtypes = [vp, vp]
    L.obfft_selftest_bounded_wait.restype = i32
    L.obfft_exec_fp64_noalloc.argtypes = [vp, vp, i64, i64, i64, i32, vp]
    L.obfft_exec_fp64_noalloc.restype = i32
    L.obfft_ablation_phase_b.argtypes = [i32, i64, i64, i32, vp, vp, vp, vp, vp]
    L.obfft_ablation_phase_b.restype = i32
    L.obfft_ablation_residues.argtypes = [i32, i64, i64, i32, vp, vp, vp, vp]
    L.obfft_ablation_residues.restype = i32
    _lib = L
    return L


def check(status: int) -> None:
    if status != OBFFT_OK:
        raise ObfftError(status, load().obfft_last_error().decode())


# ---- thin same-name wrappers (argument marshalling only) --------------------
def obfft_plan_create(n0: int, n1: int, n2: int, batch: int = 1, mode: int = OBFFT_MODE_FP8) -> int:
    h = ctypes.c_void_p()
    check(load().obfft_plan_create(ctypes.byref(h), n0, n1, n2, batch, mode))
    return h.value


def obfft_plan_create_many(dims, mode: int = OBFFT_MODE_FP8) -> int:
    flat = [int(v) for d in dims for v in d]
    arr = (ctypes.c_int64 * len(flat))(*flat)
    h = ctypes.c_void_p()
    check(load().obfft_plan_create_many(ctypes.byref(h), len(dims), arr, mode))
    return h.value


def obfft_exec(plan: int, in_ptr: int, out_ptr: int, dir: int, stream: int = 0) -> None:
    check(load().obfft_exec(plan, in_ptr, out_ptr, dir, stream))


def obfft_exec_host(plan: int, in_ptr: int, out_ptr: int, dir: int, stream: int = 0) -> None:
    check(load().obfft_exec_host(plan, in_ptr, out_ptr, dir, stream))


def obfft_exec_many(plan: int, in_ptrs, out_ptrs, dir: int, stream: int = 0) -> None:
    n = len(in_ptrs)
    ins = (ctypes.c_void_p * n)(*in_ptrs)
    outs = (ctypes.c_void_p * n)(*out_ptrs)
    check(load().obfft_exec_many(plan, ins, outs, dir, stream))


def obfft_exec_stage(plan: int, axis: int, stage: int, in_ptr: int, out_ptr: int, dir: int,
                     stream: int = 0) -> None:
    check(load().obfft_exec_stage(plan, axis, stage, in_ptr, out_ptr, dir, stream))


def obfft_exec_axes(plan: int, first_axis: int, last_axis: int, in_ptr: int, out_ptr: int, dir: int,
                    stream: int = 0) -> None:
    check(load().obfft_exec_axes(plan, first_axis, last_axis, in_ptr, out_ptr, dir, stream))


def obfft_transpose_blocks(src_ptr: int, dst_ptr: int, nblocks: int, rows: int, row_bytes: int,
                           stream: int = 0) -> None:
    check(load().obfft_transpose_blocks(src_ptr, dst_ptr, nblocks, rows, row_bytes, stream))


def obfft_plan_get_tuning(plan: int, grid: int, axis: int):
    """(p, q, lines per TMEM lane of stage 1, of stage 2) the plan runs with."""
    v = [ctypes.c_int() for _ in range(4)]
    check(load().obfft_plan_get_tuning(plan, grid, axis, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def obfft_debug_layout(mode: int, K: int, Kout: int, ncols: int):
    """Byte offsets of the seven dump sections and the total size (offsets[7])."""
    off = (ctypes.c_int64 * 8)()
    check(load().obfft_debug_layout(mode, K, Kout, ncols, off))
    return list(off)


def obfft_exec_debug(plan: int, axis: int, stage: int, in_ptr: int, out_ptr: int, dir: int, col0: int,
                     ncols: int, dump_ptr: int, stream: int = 0) -> None:
    check(load().obfft_exec_debug(plan, axis, stage, in_ptr, out_ptr, dir, col0, ncols, dump_ptr, stream))


def obfft_destroy(plan: int) -> None:
    check(load().obfft_destroy(plan))


def obfft_plan_get_splits(plan: int, grid: int, axis: int):
    p, q = ctypes.c_int(), ctypes.c_int()
    check(load().obfft_plan_get_splits(plan, grid, axis, ctypes.byref(p), ctypes.byref(q)))
    return p.value, q.value


def obfft_exec_fp64_noalloc(in_ptr: int, out_ptr: int, n0: int, n1: int, n2: int, dir: int,
                            stream: int = 0) -> None:
    """Native-FP64 3-D transform that allocates nothing (scratch reserved at load)."""
    check(load().obfft_exec_fp64_noalloc(in_ptr, out_ptr, n0, n1, n2, dir, stream))


def obfft_plan_status(plan: int, stream: int = 0) -> None:
    """Raise ObfftError(OBFFT_ERR_TIMEOUT) if a device-side bounded wait gave up."""
    check(load().obfft_plan_status(plan, stream))


def obfft_selftest_bounded_wait(plan: int, stream: int = 0) -> None:
    check(load().obfft_selftest_bounded_wait(plan, stream))


def obfft_host_twiddle32(m: int, N: int, dir: int):
    """RNE(2^23 exp(dir 2 pi i m / N)) of the FP32-precision plans (host only)."""
    re, im = ctypes.c_int64(), ctypes.c_int64()
    check(load().obfft_host_twiddle32(m, N, dir, ctypes.byref(re), ctypes.byref(im)))
    return re.value, im.value


def obfft_host_crt_constants32():
    """(moduli[6], u_slices[6][8], w_slices[6][3], M) of the FP32-precision variant (host only)."""
    mod = (ctypes.c_uint32 * 6)()
    us = (ctypes.c_uint8 * 48)()
    ws = (ctypes.c_uint8 * 18)()
    M = ctypes.c_uint64()
    check(load().obfft_host_crt_constants32(mod, us, ws, ctypes.byref(M)))
    return list(mod), [list(us[8 * k:8 * k + 8]) for k in range(6)], \
        [list(ws[3 * k:3 * k + 3]) for k in range(6)], M.value


def obfft_ablation_phase_b(variant: int, n_unique: int, n_total: int, acc_ptr: int, et_ptr: int,
                           out_ptr: int | None, checksum_ptr: int, stream: int = 0, reps: int = 1) -> None:
    """Phase B of n_total x reps scalar outputs in one accumulator layout (device pointers)."""
    check(load().obfft_ablation_phase_b(variant, n_unique, n_total, reps, acc_ptr, et_ptr, out_ptr, checksum_ptr,
                                        stream))


def obfft_ablation_residues(variant: int, n_unique: int, n_total: int, xt_ptr: int, res_ptr: int | None,
                            checksum_ptr: int, stream: int = 0, reps: int = 1) -> None:
    """Residues of n_total x reps deconstructed integers in one instruction form (device pointers)."""
    check(load().obfft_ablation_residues(variant, n_unique, n_total, reps, xt_ptr, res_ptr, checksum_ptr, stream))


def obfft_last_error() -> str:
    return load().obfft_last_error().decode()


def obfft_version() -> str:
    return load().obfft_version().decode()
