"""ctypes binding of libg3gemm.so (include/g3gemm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own.  Pointers are passed as integers (device addresses, e.g.
``tensor.data_ptr()``) and streams as ``cudaStream_t`` integers (e.g.
``torch.cuda.current_stream().cuda_stream``).  If the shared library is
missing the import of any entry point raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libg3gemm.so")

G3_F32, G3_F32_3XBF16, G3_BF16, G3_FP8_E4M3, G3_INT8, G3_FP16, G3_TF32, G3_F32_3XTF32, G3_F64, G3_INT16 = range(10)
G3_SPLIT_STREAM_K = -1   # g3_gemm_args.split_k: a stream-K tail
G3_GROUPED_SPLIT_IN_KERNEL = 1   # g3_grouped_plan_create_ex: FP32-accurate split inside the kernel
DTYPES = {"f32": G3_F32, "3xbf16": G3_F32_3XBF16, "bf16": G3_BF16, "fp8": G3_FP8_E4M3, "int8": G3_INT8,
          "fp16": G3_FP16, "tf32": G3_TF32, "3xtf32": G3_F32_3XTF32, "f64": G3_F64, "int16": G3_INT16}

G3_OK, G3_ERR_ARG, G3_ERR_UNSUPPORTED, G3_ERR_CUDA, G3_ERR_NOMEM, G3_ERR_TIMEOUT, G3_ERR_NOT_INIT = (
    0, -1, -2, -3, -4, -5, -6)

# Every symbol include/g3gemm.h declares (checked against the header by the tests).
EXPORTED = (
    "g3_gemm", "g3_gemm_host", "g3_conv2d", "g3_set_stream", "g3_gemm_args_init", "g3_gemm_ex", "g3_gemm_workspace_size",
    "g3_convert_bf16", "g3_convert_tf32", "g3_split_bf16", "g3_split3_bf16", "g3_split_tf32", "g3_quantize_fp8",
    "g3_grouped_plan_create", "g3_grouped_plan_create_ex", "g3_grouped_plan_execute", "g3_grouped_plan_destroy", "g3_gemm_grouped",
    "g3_grouped_plan_describe", "g3_autotune_grouped",
    "g3_get_last_device_status", "g3_status_string", "g3_family_size", "g3_family_describe",
    "g3_plan_query", "g3_launch_count", "g3_debug_device_allocations", "g3_stream_traffic", "g3_kernel_timing", "g3_kernel_time_ms",
    "g3_debug_withhold_next", "g3_gemm_3xbf16_noalloc",
    "g3_autotune", "g3_tune_cache_save", "g3_tune_cache_load", "g3_tune_cache_clear",
)


class G3Error(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: status {status}" if what else f"status {status}")


class g3_gemm_args(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64),
                ("dtype", ctypes.c_int),
                ("scale_a", ctypes.c_void_p), ("scale_b", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("config", ctypes.c_int), ("split_k", ctypes.c_int), ("raster", ctypes.c_int),
                ("trans_a", ctypes.c_int), ("trans_b", ctypes.c_int)]


class g3_gemm_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("scale_a", ctypes.c_float), ("scale_b", ctypes.c_float)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (built by ``build()``); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libg3gemm.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        i64, dbl, i32, vp, sz = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
        sig = {
            "g3_gemm": ([i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32], i32),
            "g3_gemm_host": ([i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, i32, vp], i32),
            "g3_conv2d": ([i64] * 13 + [dbl, vp, vp, dbl, vp, i32, vp], i32),
            "g3_set_stream": ([vp], i32),
            "g3_gemm_args_init": ([ctypes.POINTER(g3_gemm_args)], None),
            "g3_gemm_ex": ([ctypes.POINTER(g3_gemm_args), vp], i32),
            "g3_gemm_workspace_size": ([ctypes.POINTER(g3_gemm_args), ctypes.POINTER(sz)], i32),
            "g3_convert_bf16": ([vp, i64, i64, i64, vp, i64, vp], i32),
            "g3_split_bf16": ([vp, i64, i64, i64, vp, vp, i64, vp], i32),
            "g3_split3_bf16": ([vp, i64, i64, i64, vp, vp, vp, i64, vp], i32),
            "g3_convert_tf32": ([vp, i64, i64, i64, vp, i64, vp], i32),
            "g3_split_tf32": ([vp, i64, i64, i64, vp, vp, i64, vp], i32),
            "g3_quantize_fp8": ([vp, i64, i64, i64, vp, i64, vp, vp], i32),
            "g3_grouped_plan_create": ([i32, ctypes.POINTER(g3_gemm_desc), i32, ctypes.POINTER(vp)], i32),
            "g3_grouped_plan_create_ex": ([i32, ctypes.POINTER(g3_gemm_desc), i32, i32, ctypes.POINTER(vp)], i32),
            "g3_grouped_plan_execute": ([vp, vp], i32),
            "g3_grouped_plan_destroy": ([vp], i32),
            "g3_gemm_grouped": ([i32, ctypes.POINTER(g3_gemm_desc), i32, vp], i32),
            "g3_grouped_plan_describe": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
            "g3_autotune_grouped": ([i64, i64, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl)], i32),
            "g3_get_last_device_status": ([ctypes.POINTER(i32)], i32),
            "g3_status_string": ([i32], ctypes.c_char_p),
            "g3_family_size": ([], i32),
            "g3_family_describe": ([i32, ctypes.c_char_p, sz], i32),
            "g3_plan_query": ([i64, i64, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32)], i32),
            "g3_launch_count": ([], ctypes.c_uint64),
            "g3_debug_device_allocations": ([], ctypes.c_int64),
            "g3_stream_traffic": ([vp, i64, vp, i64, vp], i32),
            "g3_kernel_timing": ([i32], i32),
            "g3_kernel_time_ms": ([ctypes.POINTER(dbl), ctypes.POINTER(i32), i32], i32),
            "g3_debug_withhold_next": ([i64], i32),
            "g3_gemm_3xbf16_noalloc": ([i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp], i32),
            "g3_autotune": ([i64, i64, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                             ctypes.POINTER(dbl)], i32),
            "g3_tune_cache_save": ([ctypes.c_char_p], i32),
            "g3_tune_cache_load": ([ctypes.c_char_p], i32),
            "g3_tune_cache_clear": ([], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def check(status: int, what: str = "") -> int:
    if status != G3_OK:
        raise G3Error(status, what)
    return status


# ---- entry points, same names as the C ABI ---------------------------------

def g3_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype) -> int:
    return load().g3_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype)


def g3_conv2d(N, H, W, C, K, R, S, stride_h, stride_w, pad_h, pad_w, dil_h, dil_w, alpha, x, w, beta, y, dtype,
              stream=None) -> int:
    return load().g3_conv2d(N, H, W, C, K, R, S, stride_h, stride_w, pad_h, pad_w, dil_h, dil_w, alpha, x, w, beta,
                            y, dtype, stream)


def g3_gemm_host(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype, stream=None) -> int:
    return load().g3_gemm_host(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, dtype, stream)


def g3_set_stream(stream) -> int:
    return load().g3_set_stream(stream)


def g3_gemm_args_init() -> g3_gemm_args:
    a = g3_gemm_args()
    load().g3_gemm_args_init(ctypes.byref(a))
    return a


def g3_gemm_ex(args: g3_gemm_args, stream=None) -> int:
    return load().g3_gemm_ex(ctypes.byref(args), stream)


def g3_gemm_workspace_size(args: g3_gemm_args):
    out = ctypes.c_size_t(0)
    st = load().g3_gemm_workspace_size(ctypes.byref(args), ctypes.byref(out))
    return st, out.value


def g3_convert_bf16(x, rows, cols, ldx, y, ldy, stream=None) -> int:
    return load().g3_convert_bf16(x, rows, cols, ldx, y, ldy, stream)


def g3_split_bf16(x, rows, cols, ldx, hi, lo, ldy, stream=None) -> int:
    return load().g3_split_bf16(x, rows, cols, ldx, hi, lo, ldy, stream)


def g3_convert_tf32(x, rows, cols, ldx, y, ldy, stream=None) -> int:
    return load().g3_convert_tf32(x, rows, cols, ldx, y, ldy, stream)


def g3_split_tf32(x, rows, cols, ldx, hi, lo, ldy, stream=None) -> int:
    return load().g3_split_tf32(x, rows, cols, ldx, hi, lo, ldy, stream)


def g3_split3_bf16(x, rows, cols, ldx, hi, mid, lo, ldy, stream=None) -> int:
    return load().g3_split3_bf16(x, rows, cols, ldx, hi, mid, lo, ldy, stream)


def g3_quantize_fp8(x, rows, cols, ldx, q, ldq, scale, stream=None) -> int:
    return load().g3_quantize_fp8(x, rows, cols, ldx, q, ldq, scale, stream)


def g3_grouped_plan_create(descs, dtype, flags=None):
    """flags None: g3_grouped_plan_create; else g3_grouped_plan_create_ex with those flags."""
    arr = (g3_gemm_desc * len(descs))(*descs)
    plan = ctypes.c_void_p(None)
    if flags is None:
        st = load().g3_grouped_plan_create(len(descs), arr, dtype, ctypes.byref(plan))
    else:
        st = load().g3_grouped_plan_create_ex(len(descs), arr, dtype, flags, ctypes.byref(plan))
    return st, plan


def g3_grouped_plan_execute(plan, stream=None) -> int:
    return load().g3_grouped_plan_execute(plan, stream)


def g3_grouped_plan_destroy(plan) -> int:
    return load().g3_grouped_plan_destroy(plan)


def g3_grouped_plan_describe(plan, index):
    bm, kind = ctypes.c_int(0), ctypes.c_int(0)
    st = load().g3_grouped_plan_describe(plan, index, ctypes.byref(bm), ctypes.byref(kind))
    return st, bm.value, kind.value


def g3_autotune_grouped(m, n, k, dtype):
    bm, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    st = load().g3_autotune_grouped(m, n, k, dtype, ctypes.byref(bm), ctypes.byref(ms))
    return st, bm.value, ms.value


def g3_gemm_grouped(descs, dtype, stream=None) -> int:
    arr = (g3_gemm_desc * len(descs))(*descs)
    return load().g3_gemm_grouped(len(descs), arr, dtype, stream)


def g3_get_last_device_status():
    code = ctypes.c_int(0)
    st = load().g3_get_last_device_status(ctypes.byref(code))
    return st, code.value


def g3_status_string(status: int) -> str:
    return load().g3_status_string(status).decode()


def g3_family_size() -> int:
    return load().g3_family_size()


def g3_family_describe(index: int) -> str:
    buf = ctypes.create_string_buffer(256)
    check(load().g3_family_describe(index, buf, 256), "g3_family_describe")
    return buf.value.decode()


def g3_plan_query(m, n, k, dtype):
    c, s, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    st = load().g3_plan_query(m, n, k, dtype, ctypes.byref(c), ctypes.byref(s), ctypes.byref(r))
    return st, c.value, s.value, r.value


def g3_launch_count() -> int:
    return int(load().g3_launch_count())


def g3_debug_device_allocations() -> int:
    return int(load().g3_debug_device_allocations())


def g3_stream_traffic(in_ptr, in_bytes, out_ptr, out_bytes, stream=None) -> int:
    return load().g3_stream_traffic(in_ptr, in_bytes, out_ptr, out_bytes, stream)


def g3_kernel_timing(enable: bool) -> int:
    return load().g3_kernel_timing(1 if enable else 0)


def g3_kernel_time_ms(reset: bool = True):
    ms, n = ctypes.c_double(0.0), ctypes.c_int(0)
    load().g3_kernel_time_ms(ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0)
    return ms.value, n.value


def g3_autotune(m, n, k, dtype):
    c, s, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    st = load().g3_autotune(m, n, k, dtype, ctypes.byref(c), ctypes.byref(s), ctypes.byref(ms))
    return st, c.value, s.value, ms.value


def g3_tune_cache_save(path: str) -> int:
    return load().g3_tune_cache_save(path.encode())


def g3_tune_cache_load(path: str) -> int:
    return load().g3_tune_cache_load(path.encode())


def g3_tune_cache_clear() -> int:
    return load().g3_tune_cache_clear()


def g3_debug_withhold_next(timeout_ms: int) -> int:
    return load().g3_debug_withhold_next(timeout_ms)


def g3_gemm_3xbf16_noalloc(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None) -> int:
    """FP32-accurate GEMM whose scratch is a fixed array inside the library:
    for callers that may not allocate device memory (see include/g3gemm.h)."""
    return load().g3_gemm_3xbf16_noalloc(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream)
