"""Transposed operands (trans_a / trans_b, BLAS transa / transb): every dtype
and every combination against the oracle fed the logical op(A), op(B)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded, rel_err
from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32,
                                    synth, torch_api)

pytestmark = pytest.mark.gpu
COMBOS = [(True, False), (False, True), (True, True)]


def stored(x, trans, pad):
    """The device tensor holding x (or its transpose), rows padded by `pad` elements."""
    y = np.ascontiguousarray(x.T if trans else x)
    full = torch.zeros(y.shape[0], y.shape[1] + pad, dtype=torch.from_numpy(y).dtype)
    full[:, : y.shape[1]] = torch.from_numpy(y)
    return full.cuda()[:, : y.shape[1]]


@pytest.mark.parametrize("ta,tb", COMBOS)
@pytest.mark.parametrize("dtype,tol", [(G3_F32, 2e-6), (G3_F32_3XBF16, 2e-6), (G3_F32_3XTF32, 2e-6)])
def test_trans_fp32(ta, tb, dtype, tol):
    p = synth.uniform_problem(130, 200, 300, seed=50, alpha=1.5, beta=0.5)
    A, B = stored(p.A, ta, 3), stored(p.B, tb, 5)
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=dtype, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    e = rel_err(C.cpu().numpy(), oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha),
                p.beta * p.C.astype(np.float64))
    assert e <= tol, e


@pytest.mark.parametrize("ta,tb", COMBOS)
@pytest.mark.parametrize("kind", ["bf16", "fp16"])
def test_trans_16bit(ta, tb, kind):
    p = synth.uniform_problem(257, 300, 520, seed=51)
    if kind == "bf16":
        Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
        A = stored(Aq, ta, 2).to(torch.bfloat16)
        B = stored(Bq, tb, 6).to(torch.bfloat16)
        dt = G3_BF16
    else:
        Aq, Bq = p.A.astype(np.float16).astype(np.float32), p.B.astype(np.float16).astype(np.float32)
        A, B = stored(Aq, ta, 2).half(), stored(Bq, tb, 6).half()
        dt = G3_FP16
    C = torch.empty(p.m, p.n, device="cuda")
    torch_api.gemm(A, B, C, 1.0, 0.0, dtype=dt, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    e = rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq), oracle.absprod(Aq, Bq, 1.0))
    assert e <= 1e-5, e


@pytest.mark.parametrize("ta,tb", COMBOS)
def test_trans_tf32(ta, tb):
    # TF32 stages B K-major: a transposed B is made row-major, then written
    # transposed again by the rounding pre-pass
    p = synth.uniform_problem(140, 264, 200, seed=54, beta=0.5)
    A, B = stored(p.A, ta, 1), stored(p.B, tb, 3)
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(A, B, C, 1.0, 0.5, dtype=G3_TF32, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    Aq, Bq = oracle.round_tf32(p.A), oracle.round_tf32(p.B)
    e = rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq, p.C, 1.0, 0.5), oracle.absprod(Aq, Bq, 1.0),
                0.5 * p.C.astype(np.float64))
    assert e <= 1e-5, e


@pytest.mark.parametrize("ta,tb", COMBOS)
def test_trans_int8_bit_exact(ta, tb):
    p = synth.int8_problem(200, 150, 1100, seed=52, beta=1)
    A, B = stored(p.A, ta, 16), stored(p.B, tb, 0)
    C = torch.from_numpy(p.C.copy()).cuda()
    torch_api.gemm(A, B, C, 1, 1, dtype=G3_INT8, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, 1))


@pytest.mark.parametrize("ta,tb", COMBOS)
def test_trans_fp8(ta, tb):
    p = synth.normal_problem(130, 260, 256, seed=53)
    qa, sa = oracle.fp8_quantize(p.A)
    qb, sb = oracle.fp8_quantize(p.B)
    A, B = stored(qa, ta, 16), stored(qb, tb, 32)
    C = torch.empty(p.m, p.n, device="cuda")
    dsa = torch.tensor([sa], dtype=torch.float32, device="cuda")
    dsb = torch.tensor([sb], dtype=torch.float32, device="cuda")
    torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=dsa, scale_b=dsb, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    Ad = oracle.e4m3_decode(qa).astype(np.float64) * sa
    Bd = oracle.e4m3_decode(qb).astype(np.float64) * sb
    e = rel_err(C.cpu().numpy(), oracle.gemm(Ad, Bd), oracle.absprod(Ad, Bd, 1.0))
    assert e <= 1e-4, e
