"""Torch-tensor front end of the C ABI: shapes, strides, devices and streams in,
status codes out.  PyTorch supplies device memory and streams only; every step
of the computation runs in libg3gemm.so.
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_F64, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_INT16,
                   G3_TF32, check)

_ELEM = {G3_F32: (torch.float32, torch.float32), G3_F32_3XBF16: (torch.float32, torch.float32),
         G3_BF16: (torch.bfloat16, torch.float32), G3_FP8_E4M3: (torch.uint8, torch.float32),
         G3_INT8: (torch.int8, torch.int32), G3_FP16: (torch.float16, torch.float32),
         G3_TF32: (torch.float32, torch.float32), G3_F32_3XTF32: (torch.float32, torch.float32),
         G3_F64: (torch.float64, torch.float64), G3_INT16: (torch.int16, torch.int64)}


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _ld(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.shape[1] > 1 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    return max(t.stride(0), t.shape[1], 1)


def _ptr(t):
    return t.data_ptr() if t is not None else None


def gemm_args(A, B, C, alpha=1.0, beta=0.0, dtype=G3_F32, scale_a=None, scale_b=None, config=-1,
              split_k=0, raster=0, workspace=None, trans_a=False, trans_b=False):
    """trans_a / trans_b: A is given as k x m / B as n x k (op = transpose)."""
    m, k = (A.shape[1], A.shape[0]) if trans_a else tuple(A.shape)
    k2, n = (B.shape[1], B.shape[0]) if trans_b else tuple(B.shape)
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError(f"shape mismatch: A {tuple(A.shape)} B {tuple(B.shape)} C {tuple(C.shape)}")
    in_t, out_t = _ELEM[dtype]
    for t, want, name in ((A, in_t, "A"), (B, in_t, "B"), (C, out_t, "C")):
        if t.dtype != want and not (dtype == G3_FP8_E4M3 and t.dtype == torch.float8_e4m3fn and name != "C"):
            raise TypeError(f"{name} must be {want} for dtype {dtype}, got {t.dtype}")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    a = _lib.g3_gemm_args_init()
    a.m, a.n, a.k = m, n, k
    a.alpha, a.beta = float(alpha), float(beta)
    a.A, a.lda = _ptr(A), _ld(A, "A")
    a.B, a.ldb = _ptr(B), _ld(B, "B")
    a.C, a.ldc = _ptr(C), _ld(C, "C")
    a.dtype = dtype
    a.scale_a, a.scale_b = _ptr(scale_a), _ptr(scale_b)
    if workspace is not None:
        a.workspace, a.workspace_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    a.config, a.split_k, a.raster = config, split_k, raster
    a.trans_a, a.trans_b = int(bool(trans_a)), int(bool(trans_b))
    return a


def gemm(A, B, C, alpha=1.0, beta=0.0, dtype=G3_F32, stream=None, **kw):
    """C := beta*C + alpha*A@B in place through g3_gemm_ex; returns C.

    Keyword options (the g3_gemm_args fields): scale_a / scale_b (one-element
    float32 device tensors, FP8), config (a family member, -1 = planner),
    split_k (0 = planner; >= 1 forced; G3_SPLIT_STREAM_K; for G3_F32 the size
    of the thread-block cluster that shares out k), raster, workspace (a
    caller-owned uint8 device tensor), trans_a / trans_b (A given as k x m,
    B as n x k)."""
    a = gemm_args(A, B, C, alpha, beta, dtype, **kw)
    check(_lib.g3_gemm_ex(a, _stream(stream)), "g3_gemm_ex")
    return C


def gemm_host(A, B, C, alpha=1.0, beta=0.0, dtype=G3_F32, stream=None):
    """C := beta*C + alpha*A@B with CPU tensors (pin them for overlap) through
    g3_gemm_host; asynchronous on `stream` -- synchronise it before reading C."""
    m, k = A.shape
    k2, n = B.shape
    if k2 != k or tuple(C.shape) != (m, n):
        raise ValueError(f"shape mismatch: A {tuple(A.shape)} B {tuple(B.shape)} C {tuple(C.shape)}")
    in_t, out_t = _ELEM[dtype]
    for t, want, name in ((A, in_t, "A"), (B, in_t, "B"), (C, out_t, "C")):
        if t.dtype != want:
            raise TypeError(f"{name} must be {want} for dtype {dtype}, got {t.dtype}")
        if t.is_cuda:
            raise ValueError(f"{name} must be a CPU tensor")
    check(_lib.g3_gemm_host(m, n, k, float(alpha), A.data_ptr(), _ld(A, "A"), B.data_ptr(), _ld(B, "B"),
                            float(beta), C.data_ptr(), _ld(C, "C"), dtype, _stream(stream)), "g3_gemm_host")
    return C


def convert_bf16(x: torch.Tensor, stream=None) -> torch.Tensor:
    y = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    check(_lib.g3_convert_bf16(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), y.data_ptr(),
                               max(x.shape[1], 1), _stream(stream)), "g3_convert_bf16")
    return y


def conv2d(x, w, y=None, stride=(1, 1), pad=(0, 0), dil=(1, 1), alpha=1.0, beta=0.0, stream=None):
    """Implicit-GEMM convolution through g3_conv2d: x N x H x W x C and w
    R x S x C x K (both bf16 or both fp16, contiguous, on the GPU); returns y,
    N x P x Q x K float32 (given, or new when y is None)."""
    if x.dim() != 4 or w.dim() != 4 or x.dtype != w.dtype or not x.is_contiguous() or not w.is_contiguous():
        raise ValueError("x must be N x H x W x C and w R x S x C x K, contiguous, same dtype")
    dt = {torch.bfloat16: G3_BF16, torch.float16: G3_FP16}.get(x.dtype)
    if dt is None:
        raise TypeError("conv2d takes bfloat16 or float16 tensors")
    N, H, W, C = x.shape
    R, S, C2, K = w.shape
    if C2 != C:
        raise ValueError("channel mismatch")
    P = (H + 2 * pad[0] - dil[0] * (R - 1) - 1) // stride[0] + 1
    Q = (W + 2 * pad[1] - dil[1] * (S - 1) - 1) // stride[1] + 1
    if y is None:
        y = torch.zeros(N, P, Q, K, dtype=torch.float32, device=x.device)
    check(_lib.g3_conv2d(N, H, W, C, K, R, S, stride[0], stride[1], pad[0], pad[1], dil[0], dil[1], float(alpha),
                         x.data_ptr(), w.data_ptr(), float(beta), y.data_ptr(), dt, _stream(stream)), "g3_conv2d")
    return y


def convert_tf32(x: torch.Tensor, stream=None) -> torch.Tensor:
    y = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    check(_lib.g3_convert_tf32(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), y.data_ptr(),
                               max(x.shape[1], 1), _stream(stream)), "g3_convert_tf32")
    return y


def split_bf16(x: torch.Tensor, stream=None):
    hi = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    lo = torch.empty_like(hi)
    check(_lib.g3_split_bf16(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), hi.data_ptr(),
                             lo.data_ptr(), max(x.shape[1], 1), _stream(stream)), "g3_split_bf16")
    return hi, lo


def split_tf32(x: torch.Tensor, stream=None):
    """(hi, lo) float32 tensors of the two-part TF32 split, shaped like x."""
    hi = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    lo = torch.empty_like(hi)
    check(_lib.g3_split_tf32(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), hi.data_ptr(), lo.data_ptr(),
                             max(x.shape[1], 1), _stream(stream)), "g3_split_tf32")
    return hi, lo


def split3_bf16(x: torch.Tensor, stream=None):
    """(hi, mid, lo) bfloat16 planes of the three-part split, shaped like x."""
    hi = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    mid = torch.empty_like(hi)
    lo = torch.empty_like(hi)
    check(_lib.g3_split3_bf16(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), hi.data_ptr(), mid.data_ptr(),
                              lo.data_ptr(), max(x.shape[1], 1), _stream(stream)), "g3_split3_bf16")
    return hi, mid, lo


def quantize_fp8(x: torch.Tensor, stream=None):
    """(codes uint8 like x, scale float32 tensor of one element)."""
    q = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    s = torch.empty(1, dtype=torch.float32, device=x.device)
    check(_lib.g3_quantize_fp8(x.data_ptr(), x.shape[0], x.shape[1], _ld(x, "x"), q.data_ptr(),
                               max(x.shape[1], 1), s.data_ptr(), _stream(stream)), "g3_quantize_fp8")
    return q, s


def device_status():
    st, code = _lib.g3_get_last_device_status()
    return st, code


class GroupedPlan:
    """A g3_grouped_plan over (A, B, C, alpha, beta) tuples of torch tensors
    -- (A, B, C, alpha, beta, scale_a, scale_b) for G3_FP8_E4M3, the scales
    as Python floats or one-element tensors (read once here).  The tensors
    must stay alive while the plan exists.  split_in_kernel=True: an
    FP32-accurate plan splits inside the grouped kernels
    (G3_GROUPED_SPLIT_IN_KERNEL) instead of in a pre-pass."""

    def __init__(self, problems, dtype, split_in_kernel=False):
        in_t = _ELEM[dtype][0]
        descs = []
        self._keep = []
        for prob in problems:
            A, B, C, alpha, beta = prob[:5]
            sa, sb = (prob[5], prob[6]) if len(prob) > 5 else (1.0, 1.0)
            m, k = A.shape
            n = B.shape[1]
            ok_in = (A.dtype == in_t or (dtype == G3_FP8_E4M3 and A.dtype == torch.float8_e4m3fn)) and \
                    (B.dtype == in_t or (dtype == G3_FP8_E4M3 and B.dtype == torch.float8_e4m3fn))
            if not ok_in or C.dtype != torch.float32:
                raise TypeError("operand dtypes do not match the plan's dtype")
            d = _lib.g3_gemm_desc()
            d.m, d.n, d.k = m, n, k
            d.lda, d.ldb, d.ldc = _ld(A, "A"), _ld(B, "B"), _ld(C, "C")
            d.alpha, d.beta = float(alpha), float(beta)
            d.A, d.B, d.C = _ptr(A), _ptr(B), _ptr(C)
            d.scale_a = float(sa.item()) if torch.is_tensor(sa) else float(sa)
            d.scale_b = float(sb.item()) if torch.is_tensor(sb) else float(sb)
            descs.append(d)
            self._keep.append((A, B, C))
        st, plan = _lib.g3_grouped_plan_create(descs, dtype, _lib.G3_GROUPED_SPLIT_IN_KERNEL if split_in_kernel else None)
        check(st, "g3_grouped_plan_create")
        self.plan = plan

    def execute(self, stream=None):
        check(_lib.g3_grouped_plan_execute(self.plan, _stream(stream)), "g3_grouped_plan_execute")

    def close(self):
        if self.plan is not None:
            _lib.g3_grouped_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
