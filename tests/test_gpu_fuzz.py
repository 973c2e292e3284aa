"""Randomised parity sweep: seeded draws of dtype, shape (ragged in every
dimension, from one element to several tiles), forced family member or the
planner's choice, split-K, transposed operands and alpha/beta, each checked
against the oracle with that dtype's kernel tolerance (bit-exact for INT8)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded, rel_err
from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32,
                                    gen_family, synth, torch_api)

pytestmark = pytest.mark.gpu
FAMILY = gen_family.enumerate_family()
MODE_OF = {G3_BF16: ("bf16",), G3_FP16: ("f16",), G3_TF32: ("tf32",), G3_FP8_E4M3: ("fp8",),
           G3_INT8: ("int8emu",), G3_F32_3XBF16: ("3xbf16", "6xbf16"), G3_F32_3XTF32: ("3xtf32",), G3_F32: ()}


def draw(rng):
    dtype = int(rng.choice([G3_F32, G3_F32_3XBF16, G3_BF16, G3_FP16, G3_TF32, G3_FP8_E4M3, G3_INT8, G3_F32_3XTF32]))
    m, n, k = (int(x) for x in np.exp(rng.uniform(0, np.log(1100), 3)).astype(int) + 1)
    members = [f["index"] for f in FAMILY if f["mode"] in MODE_OF[dtype]]
    if dtype == G3_F32_3XBF16:   # the member must be of the mode the library picks at this depth
        want = "6xbf16" if k <= 512 else "3xbf16"
        members = [f["index"] for f in FAMILY if f["mode"] == want]
    config = int(rng.choice(members)) if members and rng.random() < 0.7 else -1
    split = int(rng.choice([0, 1, 2, 3])) if dtype != G3_FP8_E4M3 else 0
    ta, tb = bool(rng.random() < 0.25), bool(rng.random() < 0.25)
    if dtype == G3_INT8:
        alpha, beta = 1, int(rng.choice([0, 1]))
    else:
        alpha, beta = float(rng.choice([1.0, -0.75])), float(rng.choice([0.0, 0.5]))
    return dtype, m, n, k, config, split, ta, tb, alpha, beta


def dev_operand(x, trans, dtype):
    y = np.ascontiguousarray(x.T if trans else x)
    t = torch.from_numpy(y).cuda()
    if dtype == G3_BF16:
        return t.to(torch.bfloat16)
    if dtype == G3_FP16:
        return t.half()
    return t


@pytest.mark.parametrize("seed", range(160))
def test_random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    dtype, m, n, k, config, split, ta, tb, alpha, beta = draw(rng)
    case = (dtype, m, n, k, config, split, ta, tb, alpha, beta)
    if dtype == G3_INT8:
        p = synth.int8_problem(m, n, k, seed=seed, beta=beta)
        full, C = guarded(m, n, p.C, dtype=torch.int32)
        torch_api.gemm(dev_operand(p.A, ta, dtype), dev_operand(p.B, tb, dtype), C, 1, beta, dtype=G3_INT8,
                       config=config, split_k=split, trans_a=ta, trans_b=tb)
        torch.cuda.synchronize()
        check_guard(full, m, n)
        assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta)), case
        return
    p = synth.uniform_problem(m, n, k, seed=seed, alpha=alpha, beta=beta)
    scales = {}
    if dtype == G3_FP8_E4M3:
        qa, sa = oracle.fp8_quantize(p.A)
        qb, sb = oracle.fp8_quantize(p.B)
        A, B = dev_operand(qa, ta, dtype), dev_operand(qb, tb, dtype)
        scales = dict(scale_a=torch.tensor([sa], device="cuda"), scale_b=torch.tensor([sb], device="cuda"))
        Aq = oracle.e4m3_decode(qa).astype(np.float64) * sa
        Bq = oracle.e4m3_decode(qb).astype(np.float64) * sb
        tol = 1e-4
    else:
        if dtype == G3_BF16:
            Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
        elif dtype == G3_FP16:
            Aq, Bq = p.A.astype(np.float16).astype(np.float32), p.B.astype(np.float16).astype(np.float32)
        elif dtype == G3_TF32:
            Aq, Bq = oracle.round_tf32(p.A), oracle.round_tf32(p.B)
        else:
            Aq, Bq = p.A, p.B
        A, B = dev_operand(Aq if dtype in (G3_BF16, G3_FP16) else p.A, ta, dtype), \
            dev_operand(Bq if dtype in (G3_BF16, G3_FP16) else p.B, tb, dtype)
        tol = 2e-6 if dtype in (G3_F32, G3_F32_3XBF16, G3_F32_3XTF32) else 1e-5
    full, C = guarded(m, n, p.C)
    torch_api.gemm(A, B, C, alpha, beta, dtype=dtype, config=config, split_k=split, trans_a=ta, trans_b=tb,
                   **scales)
    torch.cuda.synchronize()
    check_guard(full, m, n)
    bc = None if p.C is None else beta * p.C.astype(np.float64)
    ref = oracle.gemm(Aq, Bq, p.C, alpha, beta)
    e = rel_err(C.cpu().numpy(), ref, oracle.absprod(Aq, Bq, alpha), bc)
    assert e <= tol, (case, e)
