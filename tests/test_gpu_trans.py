"""Transposed operands (trans_a / trans_b, BLAS transa / transb): every dtype
and every combination against the oracle fed the logical op(A), op(B).  The
first tests mostly pad rows to lengths TMA cannot address, so they run
through the row-major copy; the in-place path has its own tests below."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded, rel_err
from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32,
                                    _lib, gen_family, synth, torch_api)

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


# ---------------------------------------------------------------- in place
# BF16, FP16 and FP8 read a transposed operand in place when TMA can address
# it (16-byte aligned base and row stride): B stored n x k is staged K-major,
# A stored k x m MN-major.  Only the staging differs from the row-major path
# on the same member, so the results must match it bit for bit, with the same
# number of launches (no transpose copy).  FP8 members with 64 rows of A per
# CTA cannot stage A MN-major (half a 128-byte swizzle row) and copy it.
_FAM = gen_family.enumerate_family()
_MEMBERS = [(f["mode"], f["index"]) for f in _FAM if f["mode"] in ("bf16", "f16", "fp8")]
_DT = {"bf16": (G3_BF16, torch.bfloat16, 2), "f16": (G3_FP16, torch.float16, 2), "fp8": (G3_FP8_E4M3, None, 1)}


def aligned(x, trans, es):
    """x (or its transpose) on the device, rows 16 bytes longer than the next
    16-byte multiple, so the row stride is aligned but not the row length."""
    y = x.t() if trans else x
    r, c = y.shape
    ld = -(-c * es // 16) * 16 // es + 16 // es
    full = torch.zeros(r, ld, dtype=y.dtype, device="cuda")
    full[:, :c] = y
    return full[:, :c]


def operands(mode, m, n, k, seed):
    dt, tdt, es = _DT[mode]
    if mode == "fp8":
        p = synth.normal_problem(m, n, k, seed=seed)
        A = torch.from_numpy(oracle.fp8_quantize(p.A)[0]).cuda()
        B = torch.from_numpy(oracle.fp8_quantize(p.B)[0]).cuda()
    else:
        p = synth.uniform_problem(m, n, k, seed=seed)
        A = torch.from_numpy(p.A).cuda().to(tdt)
        B = torch.from_numpy(p.B).cuda().to(tdt)
    return dt, es, A, B


def both_paths(mode, ta, tb, m, n, k, seed, config=-1, split_k=0, beta=0.5):
    """(C from the transposed storage, C from row-major storage, launches of each)."""
    dt, es, A, B = operands(mode, m, n, k, seed)
    C0 = torch.from_numpy(synth.uniform_problem(m, n, 1, seed=seed + 1, beta=1.0).C).cuda()
    out = []
    for t_a, t_b in ((ta, tb), (False, False)):
        Ad, Bd = aligned(A, t_a, es), aligned(B, t_b, es)
        C = C0.clone()
        torch.cuda.synchronize()
        l0 = _lib.g3_launch_count()
        torch_api.gemm(Ad, Bd, C, 0.75, beta, dtype=dt, config=config, split_k=split_k, trans_a=t_a, trans_b=t_b)
        launches = _lib.g3_launch_count() - l0
        torch.cuda.synchronize()
        out.append((C.cpu().numpy(), launches))
    return out[0][0], out[1][0], out[0][1], out[1][1], (A, B)


@pytest.mark.parametrize("ta,tb", COMBOS)
@pytest.mark.parametrize("mode,config", _MEMBERS)
def test_trans_in_place_every_member_bit_identical(mode, config, ta, tb):
    # ragged in m, n and k: 257 = 4*64 + 1 rows, 300 columns (pairs: 256 + 44),
    # 520 = 8 * 64 + 8 (BF16/F16) or 4 * 128 + 8 (FP8) of k
    got, want, l_t, l_r, _ = both_paths(mode, ta, tb, 257, 300, 520, seed=61 + config, config=config, split_k=1)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    f = _FAM[config]
    copies = mode == "fp8" and ta and f["bm"] // f["cg"] < 128
    assert l_t == l_r + (int(ta) + int(tb) if copies else 0), (l_t, l_r)


@pytest.mark.parametrize("ta,tb", COMBOS)
@pytest.mark.parametrize("mode", ["bf16", "f16", "fp8"])
def test_trans_in_place_planner_split_k_and_stream_k(mode, ta, tb):
    # the planner's member, a forced three-way split-K and a stream-K tail:
    # each bit-identical to row-major storage on the same plan
    for split in (0, 3, _lib.G3_SPLIT_STREAM_K):
        got, want, l_t, l_r, _ = both_paths(mode, ta, tb, 200, 300, 3000, seed=70, split_k=split, beta=0.0)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), split
        if mode != "fp8":
            assert l_t == l_r, (split, l_t, l_r)


@pytest.mark.parametrize("ta,tb", COMBOS)
def test_trans_in_place_against_the_oracle(ta, tb):
    # the in-place path on its own, against the binary64 oracle of the
    # bfloat16-rounded operands (BF16 member with bm = 256 in a CTA pair)
    m, n, k = 390, 520, 777
    got, _, _, _, (A, B) = both_paths("bf16", ta, tb, m, n, k, seed=80, config=40, split_k=1, beta=0.0)
    Aq = A.float().cpu().numpy()
    Bq = B.float().cpu().numpy()
    e = rel_err(got, 0.75 * oracle.gemm(Aq, Bq), oracle.absprod(Aq, Bq, 0.75))
    assert e <= 1e-5, e
