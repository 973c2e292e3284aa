"""CPU oracle for the blocked GEMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import this package.  The GPU library neither imports nor
links it, and this package imports nothing from the GPU library.

The arithmetic lives in ``oracle.c`` (plain C, binary64 / int64); this module
only compiles it with gcc, loads it with ctypes and marshals numpy arrays.
What each function computes, and the passage of the paper it follows, is in
``oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, OpenMP, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
            vp = ctypes.c_void_p
            lib.oracle_gemm_rows_f64.argtypes = [i64, vp, i64, i64, dbl, vp, i64, vp, i64,
                                                 dbl, vp, i64, vp, i64, i32]
            lib.oracle_entry_f64.argtypes = [i64, dbl, vp, vp, i64, i64, dbl, dbl]
            lib.oracle_entry_f64.restype = dbl
            lib.oracle_absprod_rows_f64.argtypes = [i64, vp, i64, i64, dbl, vp, i64, vp, i64,
                                                    vp, i64, i32]
            lib.oracle_gemm_rows_i8_i64.argtypes = [i64, vp, i64, i64, i64, vp, i64, vp, i64,
                                                    i64, vp, i64, vp, i64, i32]
            lib.oracle_round_bf16.argtypes = [ctypes.c_float]
            lib.oracle_round_bf16.restype = ctypes.c_float
            lib.oracle_round_bf16_array.argtypes = [vp, vp, i64]
            lib.oracle_conv2d_nhwc_f64.argtypes = [i64] * 13 + [dbl, vp, vp, dbl, vp, vp, i32]
            lib.oracle_round_tf32.argtypes = [ctypes.c_float]
            lib.oracle_round_tf32.restype = ctypes.c_float
            lib.oracle_round_tf32_array.argtypes = [vp, vp, i64]
            lib.oracle_e4m3_decode.argtypes = [ctypes.c_uint8]
            lib.oracle_e4m3_decode.restype = ctypes.c_float
            lib.oracle_e4m3_encode.argtypes = [ctypes.c_float]
            lib.oracle_e4m3_encode.restype = ctypes.c_uint8
            lib.oracle_fp8_quantize.argtypes = [vp, i64, i64, i64, vp]
            lib.oracle_fp8_quantize.restype = ctypes.c_float
            lib.oracle_split_bf16.argtypes = [ctypes.c_float, vp, vp]
            lib.oracle_gemm_rows_3xbf16_f64.argtypes = [i64, vp, i64, i64, dbl, vp, i64, vp,
                                                        i64, dbl, vp, i64, vp, i64, i32]
            lib.oracle_gemm_rows_6xbf16_f64.argtypes = [i64, vp, i64, i64, dbl, vp, i64, vp,
                                                        i64, dbl, vp, i64, vp, i64, i32]
            lib.oracle_split3_bf16.argtypes = [ctypes.c_float, vp, vp, vp]
            lib.oracle_split_tf32.argtypes = [ctypes.c_float, vp, vp]
            lib.oracle_gemm_rows_i16_i64.argtypes = [i64, vp, i64, i64, i64, vp, i64, vp, i64,
                                                     i64, vp, i64, vp, i64, i32]
            lib.oracle_gemm_rows_3xtf32_f64.argtypes = [i64, vp, i64, i64, dbl, vp, i64, vp,
                                                        i64, dbl, vp, i64, vp, i64, i32]
            lib.oracle_max_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _rows_arg(rows, m):
    if rows is None:
        return None, m
    r = _c(rows, np.int64)
    if r.size and (r.min() < 0 or r.max() >= m):
        raise IndexError("row index out of range")
    return r, r.size


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gemm(A, B, C=None, alpha=1.0, beta=0.0, rows=None, nthreads=0):
    """beta*C + alpha*A@B in binary64 (Section 3.1 / 5.1), for all rows or the
    given row indices.  A (m,k), B (k,n), C (m,n) are converted to float64
    (exact for float32 / bfloat16 / fp8 values)."""
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    Cin = _c(C, np.float64) if (C is not None and beta != 0.0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.float64)
    _load().oracle_gemm_rows_f64(nr, _ptr(r), n, k, float(alpha), _ptr(A), max(k, 1),
                                 _ptr(B), max(n, 1), float(beta), _ptr(Cin), max(n, 1),
                                 _ptr(out), max(n, 1), int(nthreads))
    return out


def entry(A, B, i, j, C=None, alpha=1.0, beta=0.0):
    """One entry C(i,j) as a dot product, same summation order as gemm()."""
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    k = A.shape[1]
    n = B.shape[1]
    cin = float(C[i, j]) if (C is not None and beta != 0.0) else 0.0
    row = np.ascontiguousarray(A[i])
    return _load().oracle_entry_f64(k, float(alpha), _ptr(row), _ptr(B), max(n, 1), int(j),
                                    float(beta), cin)


def absprod(A, B, alpha=1.0, rows=None, nthreads=0):
    """Error-metric denominator |alpha| * |A| @ |B| in binary64."""
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    m, k = A.shape
    n = B.shape[1]
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.float64)
    _load().oracle_absprod_rows_f64(nr, _ptr(r), n, k, float(alpha), _ptr(A), max(k, 1),
                                    _ptr(B), max(n, 1), _ptr(out), max(n, 1), int(nthreads))
    return out


def gemm_i8(A, B, C=None, alpha=1, beta=0, rows=None, nthreads=0):
    """beta*C + alpha*A@B exactly in int64 for int8 A, B (int32 C)."""
    A = _c(A, np.int8)
    B = _c(B, np.int8)
    m, k = A.shape
    n = B.shape[1]
    Cin = _c(C, np.int32) if (C is not None and beta != 0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.int64)
    _load().oracle_gemm_rows_i8_i64(nr, _ptr(r), n, k, int(alpha), _ptr(A), max(k, 1), _ptr(B),
                                    max(n, 1), int(beta), _ptr(Cin), max(n, 1), _ptr(out),
                                    max(n, 1), int(nthreads))
    return out


def gemm_i16(A, B, C=None, alpha=1, beta=0, rows=None, nthreads=0):
    """beta*C + alpha*A@B exactly in int64 for int16 A, B (int64 C)."""
    A = _c(A, np.int16)
    B = _c(B, np.int16)
    m, k = A.shape
    n = B.shape[1]
    Cin = _c(C, np.int64) if (C is not None and beta != 0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.int64)
    _load().oracle_gemm_rows_i16_i64(nr, _ptr(r), n, k, int(alpha), _ptr(A), max(k, 1), _ptr(B),
                                     max(n, 1), int(beta), _ptr(Cin), max(n, 1), _ptr(out),
                                     max(n, 1), int(nthreads))
    return out


def gemm_3xbf16(A, B, C=None, alpha=1.0, beta=0.0, rows=None, nthreads=0):
    """The compensated 3-product bfloat16 split, step by step, in binary64."""
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    m, k = A.shape
    n = B.shape[1]
    Cin = _c(C, np.float64) if (C is not None and beta != 0.0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.float64)
    _load().oracle_gemm_rows_3xbf16_f64(nr, _ptr(r), n, k, float(alpha), _ptr(A), max(k, 1),
                                        _ptr(B), max(n, 1), float(beta), _ptr(Cin), max(n, 1),
                                        _ptr(out), max(n, 1), int(nthreads))
    return out


def gemm_6xbf16(A, B, C=None, alpha=1.0, beta=0.0, rows=None, nthreads=0):
    """The 6-product method on the three-part bfloat16 split, in binary64."""
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    m, k = A.shape
    n = B.shape[1]
    Cin = _c(C, np.float64) if (C is not None and beta != 0.0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.float64)
    _load().oracle_gemm_rows_6xbf16_f64(nr, _ptr(r), n, k, float(alpha), _ptr(A), max(k, 1),
                                        _ptr(B), max(n, 1), float(beta), _ptr(Cin), max(n, 1),
                                        _ptr(out), max(n, 1), int(nthreads))
    return out


def gemm_3xtf32(A, B, C=None, alpha=1.0, beta=0.0, rows=None, nthreads=0):
    """The 3-product method on the two-part TF32 split, in binary64."""
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    m, k = A.shape
    n = B.shape[1]
    Cin = _c(C, np.float64) if (C is not None and beta != 0.0) else None
    r, nr = _rows_arg(rows, m)
    out = np.empty((nr, n), np.float64)
    _load().oracle_gemm_rows_3xtf32_f64(nr, _ptr(r), n, k, float(alpha), _ptr(A), max(k, 1),
                                        _ptr(B), max(n, 1), float(beta), _ptr(Cin), max(n, 1),
                                        _ptr(out), max(n, 1), int(nthreads))
    return out


def split_tf32(x):
    """(hi, lo) float32 arrays with hi = tf32(x), lo = tf32(x - hi)."""
    lib = _load()
    x = _c(x, np.float32)
    hi, lo = np.empty_like(x), np.empty_like(x)
    h, l = ctypes.c_float(), ctypes.c_float()
    for idx, v in enumerate(x.ravel()):
        lib.oracle_split_tf32(float(v), ctypes.byref(h), ctypes.byref(l))
        hi.flat[idx], lo.flat[idx] = h.value, l.value
    return hi, lo


def split3_bf16(x):
    """(hi, mid, lo) float32 arrays of the three-part bfloat16 split."""
    lib = _load()
    x = _c(x, np.float32)
    out = [np.empty_like(x) for _ in range(3)]
    h, m, l = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    for idx, v in enumerate(x.ravel()):
        lib.oracle_split3_bf16(float(v), ctypes.byref(h), ctypes.byref(m), ctypes.byref(l))
        out[0].flat[idx], out[1].flat[idx], out[2].flat[idx] = h.value, m.value, l.value
    return tuple(out)


def round_bf16(x):
    """bfloat16 round-to-nearest-even of float32 values, returned as float32."""
    x = _c(x, np.float32)
    y = np.empty_like(x)
    _load().oracle_round_bf16_array(_ptr(x), _ptr(y), x.size)
    return y


def conv_out_size(H, R, stride, pad, dil=1):
    return (H + 2 * pad - dil * (R - 1) - 1) // stride + 1


def conv2d_nhwc(x, w, stride=(1, 1), pad=(0, 0), dil=(1, 1), y=None, alpha=1.0, beta=0.0, nthreads=0):
    """beta*y + alpha*conv2d(x, w) in binary64 (Section 8.1's convolution layers):
    x is N x H x W x C, w is R x S x C x K; returns N x P x Q x K."""
    x = _c(x, np.float64)
    w = _c(w, np.float64)
    N, H, W, C = x.shape
    R, S, C2, K = w.shape
    assert C == C2
    P = conv_out_size(H, R, stride[0], pad[0], dil[0])
    Q = conv_out_size(W, S, stride[1], pad[1], dil[1])
    yin = _c(y, np.float64) if (y is not None and beta != 0.0) else None
    out = np.empty((N, P, Q, K), np.float64)
    _load().oracle_conv2d_nhwc_f64(N, H, W, C, K, R, S, stride[0], stride[1], pad[0], pad[1], dil[0], dil[1],
                                   float(alpha), _ptr(x), _ptr(w), float(beta), _ptr(yin), _ptr(out), int(nthreads))
    return out


def round_tf32(x):
    """TF32 round-to-nearest-even of float32 values, returned as float32."""
    x = _c(x, np.float32)
    y = np.empty_like(x)
    _load().oracle_round_tf32_array(_ptr(x), _ptr(y), x.size)
    return y


def split_bf16(x):
    """(hi, lo) float32 arrays with hi = bf16(x), lo = bf16(x - hi)."""
    x = _c(x, np.float32)
    hi = round_bf16(x)
    lo = round_bf16((x - hi).astype(np.float32))
    return hi, lo


_E4M3_TABLE = None


def e4m3_decode(codes):
    """Values of E4M3 codes: each of the 256 codes is decoded once by the C
    definition (oracle_e4m3_decode) and the codes are looked up in that table."""
    global _E4M3_TABLE
    if _E4M3_TABLE is None:
        lib = _load()
        _E4M3_TABLE = np.array([lib.oracle_e4m3_decode(c) for c in range(256)], np.float32)
    codes = _c(codes, np.uint8)
    return _E4M3_TABLE[codes]


def e4m3_encode(x):
    lib = _load()
    x = _c(x, np.float32)
    return np.array([lib.oracle_e4m3_encode(float(v)) for v in x.ravel()],
                    np.uint8).reshape(x.shape)


def fp8_quantize(x):
    """(codes uint8 (rows, cols), scale float) with per-tensor amax/448 scaling."""
    x = _c(x, np.float32)
    rows, cols = x.shape
    q = np.empty((rows, cols), np.uint8)
    s = _load().oracle_fp8_quantize(_ptr(x), rows, cols, max(cols, 1), _ptr(q))
    return q, float(np.float32(s))
