"""Parity of the tensor-core (tcgen05) path with the oracle.

Two checks per quantised precision (the inputs are quantised from FP32
masters by the library's own pre-pass kernels, which are themselves checked
bit for bit against the oracle's format conversions):
  kernel check  oracle fed the exact quantised values; differences are FP32
                accumulation only (tolerance 1e-5, 1e-4 for FP8)
  gate          oracle fed the FP32 masters; the stated end-to-end tolerance
                (BF16 8e-3, FP8 6e-2, FP32-accurate split 2e-6, INT8 exact)
The FP32-accurate dtype runs the two-part split (3 products) for k > 512 and
the three-part split (6 products) for k <= 512; its kernel check uses the
oracle of the method the library applies at that depth.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, dev, gate as gate_check, guarded, rel_err
from paper_2310_20347_gb300 import (G3_BF16, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32, _lib,
                                    gen_family, synth, torch_api)

pytestmark = pytest.mark.gpu

FAMILY = gen_family.enumerate_family()
SHAPES = [(300, 520, 700), (129, 257, 65), (1, 1, 1), (17, 33, 5), (64, 1000, 147), (1000, 64, 1200),
          (256, 128, 64), (513, 300, 129)]


def members(mode, cg=None):
    return [f["index"] for f in FAMILY if f["mode"] == mode and (cg is None or f["cg"] == cg)]


def first_member(mode, bm, cg):
    return next(f["index"] for f in FAMILY if f["mode"] == mode and f["bm"] == bm and f["cg"] == cg)


# ---------------------------------------------------------------- BF16
def bf16_run(p, config=-1, split_k=0, beta=None):
    A32, B32 = dev(p.A), dev(p.B)
    Ab, Bb = torch_api.convert_bf16(A32), torch_api.convert_bf16(B32)
    beta = p.beta if beta is None else beta
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(Ab, Bb, C, p.alpha, beta, dtype=G3_BF16, config=config, split_k=split_k)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    return Ab, Bb, C.cpu().numpy()


def bf16_check(p, **kw):
    Ab, Bb, got = bf16_run(p, **kw)
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    # the library's conversion kernel equals the oracle's rounding, bit for bit
    assert np.array_equal(Ab.float().cpu().numpy().view(np.uint32), Aq.view(np.uint32))
    assert np.array_equal(Bb.float().cpu().numpy().view(np.uint32), Bq.view(np.uint32))
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    ref_k = oracle.gemm(Aq, Bq, p.C, p.alpha, p.beta)
    e_k = rel_err(got, ref_k, oracle.absprod(Aq, Bq, p.alpha), bc)
    ref_g = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    e_g = rel_err(got, ref_g, oracle.absprod(p.A, p.B, p.alpha), bc)
    assert e_k <= 1e-5, ("kernel", e_k)
    assert e_g <= 8e-3, ("gate", e_g)
    return e_k, e_g


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_shapes(shape):
    m, n, k = shape
    bf16_check(synth.normal_problem(m, n, k, seed=m + n + k, alpha=1.0, beta=0.0))
    bf16_check(synth.uniform_problem(m, n, k, seed=1, alpha=-0.75, beta=0.5))


@pytest.mark.parametrize("config", members("bf16"))
def test_bf16_every_member(config):
    bf16_check(synth.uniform_problem(300, 520, 700, seed=2, alpha=1.25, beta=-0.5), config=config)


# CTA pairs: 256-column tiles, each CTA staging half of A's rows.  Shapes put
# the second CTA's columns or rows partly or wholly outside C, and cover C
# written through TMA stores (beta = 0) and read-modify-write (beta != 0).
PAIR_SHAPES = [(300, 520, 700), (129, 257, 65), (40, 300, 200), (600, 129, 1000), (1, 1, 1), (256, 256, 64)]


@pytest.mark.parametrize("shape", PAIR_SHAPES)
@pytest.mark.parametrize("config", members("bf16", cg=2))
def test_bf16_pair_ragged(config, shape):
    m, n, k = shape
    for beta in (0.0, 0.5):
        bf16_check(synth.uniform_problem(m, n, k, seed=30, alpha=1.5, beta=beta), config=config)


@pytest.mark.parametrize("config", members("bf16", cg=2)[:1] + members("3xbf16", cg=2)[:1])
def test_pair_split_k(config):
    p = synth.uniform_problem(200, 300, 3000, seed=31, alpha=0.5, beta=1.0)
    if FAMILY[config]["mode"] == "bf16":
        bf16_check(p, config=config, split_k=3)
    else:
        x3_check(p, config=config, split_k=3)


@pytest.mark.parametrize("split", [2, 3, 7])
def test_bf16_split_k(split):
    bf16_check(synth.uniform_problem(96, 200, 3000, seed=3, alpha=0.5, beta=1.0), split_k=split)


def test_bf16_integer_inputs_bit_exact():
    p = synth.small_int_problem(300, 260, 900, seed=4, alpha=1.0, beta=1.0)
    _, _, got = bf16_run(p)
    assert np.array_equal(got.astype(np.float64), oracle.gemm(p.A, p.B, p.C, 1.0, 1.0))


def test_bf16_unaligned_operands_are_packed():
    # lda = k = 147 bf16 is a 294-byte row: not TMA-addressable, so the library
    # re-packs A into an aligned workspace (the paper's packing, Section 5.3)
    p = synth.normal_problem(64, 3136, 147, seed=5)
    bf16_check(p)
    p = synth.normal_problem(100, 49, 77, seed=6)
    bf16_check(p)


def test_bf16_beta_zero_overwrites_nan():
    p = synth.uniform_problem(200, 140, 96, seed=7)
    Ab, Bb = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    full, C = guarded(p.m, p.n, np.full((p.m, p.n), np.nan, np.float32))
    torch_api.gemm(Ab, Bb, C, 1.0, 0.0, dtype=G3_BF16)
    assert torch.isfinite(C).all()


def test_bf16_deterministic():
    p = synth.uniform_problem(700, 900, 1500, seed=8)
    a = bf16_run(p)[2]
    b = bf16_run(p)[2]
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- 3xBF16
def x3_run(p, config=-1, split_k=0):
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=G3_F32_3XBF16, config=config, split_k=split_k)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    return C.cpu().numpy()


def x3_method(p):
    # the split the library applies at this depth (k <= 512: three parts)
    f = oracle.gemm_6xbf16 if p.A.shape[1] <= 512 else oracle.gemm_3xbf16
    return f(p.A, p.B, p.C, p.alpha, p.beta)


def x3_check(p, gate=2e-6, **kw):
    got = x3_run(p, **kw)
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    D = oracle.absprod(p.A, p.B, p.alpha)
    e_k = rel_err(got, x3_method(p), D, bc)
    ref_g = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    e_g = rel_err(got, ref_g, D, bc)
    assert e_k <= 1e-5, ("kernel", e_k)
    if gate is not None:
        gate_check(got, ref_g, D, bc, p.A.shape[1], gate)
    return e_k, e_g


def test_3xbf16_split_matches_oracle():
    p = synth.uniform_problem(257, 129, 1, seed=9)
    hi, lo = torch_api.split_bf16(dev(p.A))
    ohi, olo = oracle.split_bf16(p.A)
    assert np.array_equal(hi.float().cpu().numpy().view(np.uint32), ohi.view(np.uint32))
    assert np.array_equal(lo.float().cpu().numpy().view(np.uint32), olo.view(np.uint32))


@pytest.mark.parametrize("rows,cols,ldx", [(37, 1037, 1040), (5, 2048, 2048), (3, 7, 8), (64, 1000, 1003)])
def test_3xbf16_split_vectorised_and_tail(rows, cols, ldx):
    # 16-byte-aligned rows take the 8-wide path, the last cols % 8 the scalar tail
    r = np.random.default_rng(19)
    full = (r.standard_normal((rows, ldx)) * 10.0 ** r.integers(-20, 20, (rows, ldx))).astype(np.float32)
    x = torch.from_numpy(full).cuda()[:, :cols]
    hi, lo = torch_api.split_bf16(x)
    ohi, olo = oracle.split_bf16(full[:, :cols])
    assert np.array_equal(hi.float().cpu().numpy().view(np.uint32), ohi.view(np.uint32))
    assert np.array_equal(lo.float().cpu().numpy().view(np.uint32), olo.view(np.uint32))


@pytest.mark.parametrize("rows,cols,ldx", [(257, 129, 129), (37, 1037, 1040), (3, 7, 8)])
def test_6xbf16_split3_matches_oracle(rows, cols, ldx):
    r = np.random.default_rng(20)
    full = (r.standard_normal((rows, ldx)) * 10.0 ** r.integers(-20, 20, (rows, ldx))).astype(np.float32)
    x = torch.from_numpy(full).cuda()[:, :cols]
    got = torch_api.split3_bf16(x)
    want = oracle.split3_bf16(full[:, :cols])
    for g, w in zip(got, want):
        assert np.array_equal(g.float().cpu().numpy().view(np.uint32), w.view(np.uint32))


@pytest.mark.parametrize("shape", [(300, 520, 16), (129, 257, 512), (1000, 64, 200), (17, 33, 1), (64, 700, 64)])
def test_6xbf16_small_k_gate(shape):
    # k <= 512: the three-part split holds the 2e-6 gate where the two-part
    # split's own error is above it (2.9e-6 at k = 64, 5.7e-6 at k = 16)
    m, n, k = shape
    e_k, e_g = x3_check(synth.uniform_problem(m, n, k, seed=21, beta=0.5))
    print(f"6xbf16 {shape}: kernel {e_k:.3e} gate {e_g:.3e}")


@pytest.mark.parametrize("config", members("6xbf16"))
def test_6xbf16_every_member(config):
    x3_check(synth.uniform_problem(300, 520, 300, seed=22, beta=0.5), config=config)


def test_6xbf16_split_k():
    x3_check(synth.uniform_problem(64, 100, 512, seed=23, beta=0.5), split_k=4)


@pytest.mark.parametrize("shape", SHAPES)
def test_3xbf16_shapes(shape):
    m, n, k = shape
    x3_check(synth.uniform_problem(m, n, k, seed=10, alpha=1.0, beta=0.5))


@pytest.mark.parametrize("config", members("3xbf16"))
def test_3xbf16_every_member(config):
    x3_check(synth.uniform_problem(300, 520, 1100, seed=11, beta=0.5), gate=2e-6, config=config)


def test_3xbf16_square_gate():
    # the square-sweep configuration at its smallest size, fully checked
    e_k, e_g = x3_check(synth.uniform_problem(1024, 1024, 1024, seed=0, beta=0.5), gate=2e-6)
    print(f"3xbf16 1024^3 kernel {e_k:.3e} gate {e_g:.3e}")


@pytest.mark.parametrize("config", [-1] + members("3xbf16")[:2])
def test_3xbf16_deep_k_gate(config):
    # k = 16384 as in the largest square: the tensor core truncates each FP32
    # accumulation, so depth is where the accuracy of the mode is decided
    e_k, e_g = x3_check(synth.uniform_problem(200, 300, 16384, seed=18, beta=0.5), gate=2e-6, config=config)
    print(f"3xbf16 k=16384 config {config}: kernel {e_k:.3e} gate {e_g:.3e}")


def test_3xbf16_split_k():
    x3_check(synth.uniform_problem(64, 100, 4096, seed=12, beta=0.5), gate=2e-6, split_k=5)


def test_3xbf16_integer_inputs_bit_exact():
    p = synth.small_int_problem(250, 330, 1000, seed=13, alpha=1.0, beta=2.0)
    got = x3_run(p)
    assert np.array_equal(got.astype(np.float64), oracle.gemm(p.A, p.B, p.C, 1.0, 2.0))


# ---------------------------------------------------------------- FP16
def f16_check(p, config=-1, split_k=0):
    A16, B16 = p.A.astype(np.float16), p.B.astype(np.float16)   # IEEE round to nearest even
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(torch.from_numpy(A16).cuda(), torch.from_numpy(B16).cuda(), C, p.alpha, p.beta, dtype=G3_FP16,
                   config=config, split_k=split_k)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    got = C.cpu().numpy()
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    Aq, Bq = A16.astype(np.float64), B16.astype(np.float64)
    e_k = rel_err(got, oracle.gemm(Aq, Bq, p.C, p.alpha, p.beta), oracle.absprod(Aq, Bq, p.alpha), bc)
    e_g = rel_err(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha), bc)
    assert e_k <= 1e-5, ("kernel", e_k)
    assert e_g <= 2e-3, ("gate", e_g)   # two roundings to binary16 (2^-11 each)
    return e_k, e_g


@pytest.mark.parametrize("shape", SHAPES)
def test_fp16_shapes(shape):
    m, n, k = shape
    f16_check(synth.uniform_problem(m, n, k, seed=26, alpha=0.75, beta=0.5))


@pytest.mark.parametrize("config", members("f16"))
def test_fp16_every_member(config):
    f16_check(synth.uniform_problem(300, 520, 700, seed=27, alpha=1.0, beta=0.0), config=config)


def test_fp16_split_k():
    f16_check(synth.uniform_problem(96, 200, 3000, seed=28, beta=1.0), split_k=3)


# ---------------------------------------------------------------- TF32
def test_tf32_conversion_matches_oracle():
    r = np.random.default_rng(29)
    bits = r.integers(0, 1 << 32, 300000, dtype=np.uint64).astype(np.uint32)
    bits[:4096] = (bits[:4096] & 0xFFFFE000) | 0x1000          # exact ties
    bits[4096:8192] &= 0x80001FFF                              # subnormals
    bits[8192:8200] = [0x7F7FF000, 0xFF7FF000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0, 0x80000000]
    x = bits.view(np.float32).reshape(300, 1000)
    got = torch_api.convert_tf32(torch.from_numpy(x.copy()).cuda()).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), oracle.round_tf32(x).view(np.uint32))


def tf32_check(p, config=-1, split_k=0):
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(dev(p.A), dev(p.B), C, p.alpha, p.beta, dtype=G3_TF32, config=config, split_k=split_k)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    got = C.cpu().numpy()
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    Aq, Bq = oracle.round_tf32(p.A), oracle.round_tf32(p.B)
    e_k = rel_err(got, oracle.gemm(Aq, Bq, p.C, p.alpha, p.beta), oracle.absprod(Aq, Bq, p.alpha), bc)
    e_g = rel_err(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha), bc)
    assert e_k <= 1e-5, ("kernel", e_k)
    assert e_g <= 2e-3, ("gate", e_g)   # two roundings to TF32 (2^-11 each)
    return e_k, e_g


@pytest.mark.parametrize("shape", SHAPES)
def test_tf32_shapes(shape):
    m, n, k = shape
    tf32_check(synth.uniform_problem(m, n, k, seed=31, alpha=-0.5, beta=0.5))


@pytest.mark.parametrize("config", members("tf32"))
def test_tf32_every_member(config):
    tf32_check(synth.uniform_problem(300, 520, 700, seed=32, beta=0.0), config=config)


def test_tf32_split_k_and_integers_exact():
    tf32_check(synth.uniform_problem(96, 200, 3000, seed=33, beta=1.0), split_k=3)
    p = synth.small_int_problem(200, 150, 600, seed=34, alpha=1.0, beta=1.0)
    C = dev(p.C)
    torch_api.gemm(dev(p.A), dev(p.B), C, 1.0, 1.0, dtype=G3_TF32)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), oracle.gemm(p.A, p.B, p.C, 1.0, 1.0))


# ---------------------------------------------------------------- FP8
def fp8_check(p, config=-1):
    A, B = dev(p.A), dev(p.B)
    qa, sa = torch_api.quantize_fp8(A)
    qb, sb = torch_api.quantize_fp8(B)
    oqa, osa = oracle.fp8_quantize(p.A)
    oqb, osb = oracle.fp8_quantize(p.B)
    assert np.array_equal(qa.cpu().numpy(), oqa) and np.array_equal(qb.cpu().numpy(), oqb)
    assert sa.item() == osa and sb.item() == osb
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(qa, qb, C, p.alpha, p.beta, dtype=G3_FP8_E4M3, scale_a=sa, scale_b=sb, config=config)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    got = C.cpu().numpy()
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    Ad = oracle.e4m3_decode(oqa).astype(np.float64) * osa
    Bd = oracle.e4m3_decode(oqb).astype(np.float64) * osb
    e_k = rel_err(got, oracle.gemm(Ad, Bd, p.C, p.alpha, p.beta), oracle.absprod(Ad, Bd, p.alpha), bc)
    e_g = rel_err(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha), bc)
    assert e_k <= 1e-4, ("kernel", e_k)
    if p.k >= 64:
        assert e_g <= 6e-2, ("gate", e_g)
    else:
        # a handful of products: one factor pair's E4M3 rounding (each at most
        # 2^-4 relative for normal values) is not averaged out
        assert e_g <= 2 * 2.0 ** -4 + 2.0 ** -8, ("format bound", e_g)
    return e_k, e_g


@pytest.mark.parametrize("shape", [(300, 520, 700), (129, 257, 65), (64, 1000, 256), (17, 33, 5)])
def test_fp8_shapes(shape):
    m, n, k = shape
    fp8_check(synth.normal_problem(m, n, k, seed=14, alpha=1.0, beta=0.0))


@pytest.mark.parametrize("config", members("fp8"))
def test_fp8_every_member(config):
    fp8_check(synth.normal_problem(300, 520, 700, seed=15, alpha=0.5, beta=0.5), config=config)


# ---------------------------------------------------------------- INT8
def int8_run(p, beta=0):
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(p.m, p.n, p.C if p.C is not None else None, dtype=torch.int32)
    torch_api.gemm(A, B, C, 1, beta, dtype=G3_INT8)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    return C.cpu().numpy()


@pytest.mark.parametrize("shape,beta", [((300, 520, 700), 0), ((129, 257, 2500), 1), ((64, 1000, 147), 0),
                                        ((33, 17, 1025), 1)])
def test_int8_bit_exact(shape, beta):
    m, n, k = shape
    p = synth.int8_problem(m, n, k, seed=16, beta=beta)
    got = int8_run(p, beta)
    assert np.array_equal(got.astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta))


@pytest.mark.parametrize("config", members("int8emu"))
def test_int8_every_member(config):
    # ragged m (several 256-row tiles and a tail), k across two 1024 chunks + a tail
    p = synth.int8_problem(600, 300, 2200, seed=20, beta=1)
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(p.m, p.n, p.C, dtype=torch.int32)
    torch_api.gemm(A, B, C, 1, 1, dtype=G3_INT8, config=config)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, 1))


@pytest.mark.parametrize("shape,beta,split", [((600, 300, 2200), 0, 0), ((257, 520, 3000), 1, 0),
                                              ((300, 129, 4100), 0, 3), ((1, 1, 1), 0, 0), ((513, 260, 1024), 1, 2)])
@pytest.mark.parametrize("config", [f["index"] for f in FAMILY if f["mode"] == "int8emu" and f["bm"] == 256])
def test_int8_bm256(config, shape, beta, split):
    # bm = 256 members: sixteen epilogue warps with 64 int32 running sums each,
    # two chunk accumulators in TMEM taken in turn: chunks of 1024 products,
    # ragged rows and columns, C written (beta = 0) or added in place
    # (beta = 1), and int32 split-K partials
    m, n, k = shape
    p = synth.int8_problem(m, n, k, seed=25, beta=beta)
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(m, n, p.C, dtype=torch.int32)
    torch_api.gemm(A, B, C, 1, beta, dtype=G3_INT8, config=config, split_k=split)
    torch.cuda.synchronize()
    check_guard(full, m, n)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta))


@pytest.mark.parametrize("config", [f["index"] for f in FAMILY if f["mode"] == "int8emu" and f["bm"] == 256])
def test_int8_bm256_worst_case_chunks(config):
    # all -128 at k = 4100: every chunk accumulator reaches 1024 * 2^14 = 2^24
    # (the largest sum FP32 holds exactly), five chunks alternate between the
    # two accumulators; every entry is 4100 * 2^14
    A = np.full((300, 4100), -128, np.int8)
    B = np.full((4100, 260), -128, np.int8)
    full, C = guarded(300, 260, None, dtype=torch.int32)
    torch_api.gemm(dev(A), dev(B), C, 1, 0, dtype=G3_INT8, config=config)
    torch.cuda.synchronize()
    check_guard(full, 300, 260)
    assert np.all(C.cpu().numpy() == 4100 * (1 << 14))


def test_int8_worst_case_magnitude():
    # all -128 at k = 8192: every entry is 8192 * 2^14 = 2^27 exactly
    A = np.full((40, 8192), -128, np.int8)
    B = np.full((8192, 24), -128, np.int8)
    p = synth.Problem(40, 24, 8192, 1.0, 0.0, A, B, None)
    got = int8_run(p)
    assert np.all(got == (1 << 27))
    B2 = np.full((8192, 24), 127, np.int8)
    p2 = synth.Problem(40, 24, 8192, 1.0, 0.0, A, B2, None)
    assert np.all(int8_run(p2) == -128 * 127 * 8192)


# ---------------------------------------------------------------- failure detection
def test_watchdog_pair_member_reports_timeout_without_hanging():
    # a CTA pair: the leader's MMA wait runs out first; the other CTA's waits
    # run out on their own bounded timers and both meet at the closing barrier
    assert torch_api.device_status()[0] == 0
    p = synth.uniform_problem(512, 512, 1024, seed=24)
    Ab, Bb = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    C = torch.zeros(p.m, p.n, device="cuda")
    cfg = first_member("bf16", 256, 2)
    assert _lib.g3_debug_withhold_next(200) == 0
    torch_api.gemm(Ab, Bb, C, 1.0, 0.0, dtype=G3_BF16, config=cfg)
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    bf16_check(p, config=cfg)
    assert torch_api.device_status()[0] == 0


def test_watchdog_reports_timeout_without_hanging():
    st, code = torch_api.device_status()
    assert st == 0
    p = synth.uniform_problem(256, 256, 512, seed=17)
    Ab, Bb = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    C = torch.zeros(p.m, p.n, device="cuda")
    assert _lib.g3_debug_withhold_next(200) == 0
    torch_api.gemm(Ab, Bb, C, 1.0, 0.0, dtype=G3_BF16, config=first_member("bf16", 128, 1))
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    # the context is still usable and the next call is correct
    bf16_check(p)
    assert torch_api.device_status()[0] == 0


# ---------------------------------------------------------------- 3xTF32
def test_tf32_split_matches_oracle():
    r = np.random.default_rng(73)
    bits = r.integers(0, 1 << 32, 40000, dtype=np.uint64).astype(np.uint32)
    bits[:2048] = (bits[:2048] & 0xFFFFE000) | 0x1000          # ties of the first rounding
    bits[2048:4096] &= 0x80001FFF                              # subnormals
    bits[4096:4100] = [0, 0x80000000, 0x3F800000, 0x7F7FFFFF]
    x = bits.view(np.float32)
    x = np.where(np.isfinite(x), x, np.float32(1.5)).astype(np.float32).reshape(200, 200)
    hi, lo = torch_api.split_tf32(torch.from_numpy(x.copy()).cuda())
    ohi, olo = oracle.split_tf32(x)
    assert np.array_equal(hi.cpu().numpy().view(np.uint32), ohi.view(np.uint32))
    assert np.array_equal(lo.cpu().numpy().view(np.uint32), olo.view(np.uint32))


def x3t_check(p, config=-1, split_k=0):
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(dev(p.A), dev(p.B), C, p.alpha, p.beta, dtype=G3_F32_3XTF32, config=config, split_k=split_k)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    got = C.cpu().numpy()
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    D = oracle.absprod(p.A, p.B, p.alpha)
    e_k = rel_err(got, oracle.gemm_3xtf32(p.A, p.B, p.C, p.alpha, p.beta), D, bc)
    ref_g = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    e_g = rel_err(got, ref_g, D, bc)
    # the method itself stays within 3 * 2^-22 of the exact product; the
    # kernel adds FP32 accumulation (main and correction sums kept apart)
    assert e_k <= 2e-6, ("kernel", e_k)
    gate_check(got, ref_g, D, bc, p.A.shape[1], 2e-6)
    return e_k, e_g


@pytest.mark.parametrize("shape", SHAPES)
def test_3xtf32_shapes(shape):
    m, n, k = shape
    x3t_check(synth.uniform_problem(m, n, k, seed=74, alpha=-0.75, beta=0.5))


@pytest.mark.parametrize("config", members("3xtf32"))
def test_3xtf32_every_member(config):
    x3t_check(synth.uniform_problem(300, 520, 700, seed=75, alpha=1.25, beta=0.0), config=config)
    x3t_check(synth.uniform_problem(600, 700, 130, seed=76, beta=-1.0), config=config)


def test_3xtf32_split_k_and_integers_exact():
    x3t_check(synth.uniform_problem(96, 200, 3000, seed=77, beta=1.0), split_k=3)
    p = synth.small_int_problem(250, 330, 1000, seed=78, alpha=1.0, beta=2.0)
    C = dev(p.C)
    torch_api.gemm(dev(p.A), dev(p.B), C, 1.0, 2.0, dtype=G3_F32_3XTF32)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy().astype(np.float64), oracle.gemm(p.A, p.B, p.C, 1.0, 2.0))


def test_3xtf32_deep_k_within_gate():
    # k = 32768: the planner keeps at most 8192 of k per FP32 accumulator
    # (split-K), which holds the accumulation error inside the 2e-6 gate
    st, cfg, sk, _ = _lib.g3_plan_query(160, 200, 32768, G3_F32_3XTF32)
    assert sk >= 4
    x3t_check(synth.uniform_problem(160, 200, 32768, seed=79, beta=0.5))


def test_3xbf16_deep_k_within_gate():
    # k = 65536: the planner keeps at most 32768 of k per FP32 accumulator
    st, cfg, sk, _ = _lib.g3_plan_query(128, 160, 65536, G3_F32_3XBF16)
    assert sk >= 2
    x3_check(synth.uniform_problem(128, 160, 65536, seed=80, beta=0.5))


@pytest.mark.parametrize("split", [2, 3, 5])
def test_split_k_partial_planes_ragged_rows(split):
    # split-K partial tiles leave through TMA stores into their split's plane
    # (a 3-D map: n x m x splits, rows padded to 128-byte lines); with m = 200
    # the second tile row (rows 128..255) is clipped at row 200 of its own
    # plane and must not spill into the next split's plane; n = 300 is not a
    # multiple of 32 (padded rows)
    bf16_check(synth.uniform_problem(200, 300, 3000, seed=40 + split, alpha=0.75, beta=0.0), split_k=split)
    bf16_check(synth.uniform_problem(200, 300, 3000, seed=50 + split, alpha=0.75, beta=-0.5), split_k=split)


@pytest.mark.parametrize("shape,beta,split", [((300, 129, 4100), 0, 3), ((257, 520, 3000), 1, 2),
                                              ((200, 300, 2048), 0, 5)])
@pytest.mark.parametrize("config", [f["index"] for f in FAMILY if f["mode"] == "int8emu" and f["bm"] == 128])
def test_int8_bm128_split_k(config, shape, beta, split):
    # int32 split-K partials of the bm = 128 members (TMA stores into an
    # int32 3-D map), summed in int32 by the reduction: bit-exact
    m, n, k = shape
    p = synth.int8_problem(m, n, k, seed=26, beta=beta)
    full, C = guarded(m, n, p.C, dtype=torch.int32)
    torch_api.gemm(dev(p.A), dev(p.B), C, 1, beta, dtype=G3_INT8, config=config, split_k=split)
    torch.cuda.synchronize()
    check_guard(full, m, n)
    assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta))
