"""Parity of the stream-K tail (split_k = G3_SPLIT_STREAM_K) with the oracle.

The tiles that do not fill the last wave of the persistent grid are cut along
k into one equal piece per CTA (or CTA pair); segments leave partial tiles
that a fix-up kernel adds in stream order and scales.  Shapes are chosen so
that the walk has whole waves plus a tail (or only a tail), with ragged rows,
columns and k, pieces that cross tile boundaries, pieces shorter than one tile
and streams with no work at all (k of a single k-block).  The library's launch
counter shows whether the fix-up ran: one more launch than the same call
without a split."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, dev, guarded, rel_err
from paper_2310_20347_gb300 import (G3_BF16, G3_F32_3XBF16, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_SPLIT_STREAM_K,
                                    G3_TF32, _lib, gen_family, synth, torch_api)

pytestmark = pytest.mark.gpu
SK = G3_SPLIT_STREAM_K
FAMILY = gen_family.enumerate_family()


def members(mode, cg=None, bm=None):
    return [f["index"] for f in FAMILY if f["mode"] == mode and (cg is None or f["cg"] == cg)
            and (bm is None or f["bm"] == bm)]


def launches_of(fn):
    before = _lib.g3_launch_count()
    fn()
    torch.cuda.synchronize()
    return _lib.g3_launch_count() - before


def run(A, B, C, alpha, beta, dtype, config, split_k, **kw):
    """The call with split_k, and the launches it took minus those of the same
    call without a split (into a scratch copy of C)."""
    scratch = C.clone()
    base = launches_of(lambda: torch_api.gemm(A, B, scratch, alpha, beta, dtype=dtype, config=config, split_k=1,
                                              **kw))
    n = launches_of(lambda: torch_api.gemm(A, B, C, alpha, beta, dtype=dtype, config=config, split_k=split_k, **kw))
    return n - base


# Shapes: 1883 x 1925 makes 15 x 16 tiles of 128 x 128 (one wave of 152 plus a
# tail of 88), 30 x 16 of 64 rows (three waves plus 24), 8 x 16 of 256 rows and
# 8 x 8 pair tiles (a tail only); 2600 x 2700 makes 11 x 11 pair tiles (one
# wave of pairs plus a tail on a GPU with fewer than 121 pair slots).
SINGLE = (1883, 1925, 1000)
PAIR = (2600, 2700, 600)


def shape_for(config):
    return PAIR if FAMILY[config]["cg"] == 2 else SINGLE


@pytest.mark.parametrize("config", members("bf16"))
def test_bf16_stream_k_every_member(config):
    m, n, k = shape_for(config)
    p = synth.uniform_problem(m, n, k, seed=60 + config, alpha=-0.75, beta=0.5)
    A, B = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    full, C = guarded(m, n, p.C)
    extra = run(A, B, C, p.alpha, p.beta, G3_BF16, config, SK)
    check_guard(full, m, n)
    assert extra == 1, "the stream-K fix-up did not run"
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    e = rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq, p.C, p.alpha, p.beta), oracle.absprod(Aq, Bq, p.alpha),
                p.beta * p.C.astype(np.float64))
    assert e <= 1e-5, e


@pytest.mark.parametrize("k", [40, 64, 200])
def test_bf16_stream_k_short_k(k):
    # num_kb of 1 .. 4: pieces shorter than one k-block leave streams empty,
    # tiles are covered by many streams
    m, n, _ = SINGLE
    p = synth.uniform_problem(m, n, k, seed=61, alpha=1.5, beta=0.0)
    A, B = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    full, C = guarded(m, n, None)
    C.fill_(float("nan"))   # beta = 0: C is never read, NaN must be overwritten
    cfg = members("bf16", cg=1, bm=64)[0]
    assert run(A, B, C, p.alpha, 0.0, G3_BF16, cfg, SK) == 1
    check_guard(full, m, n)
    got = C.cpu().numpy()
    assert not np.isnan(got).any()
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    assert rel_err(got, oracle.gemm(Aq, Bq, None, p.alpha, 0.0), oracle.absprod(Aq, Bq, p.alpha)) <= 1e-5


@pytest.mark.parametrize("k", [300, 1500])   # three-part split (6 products) / two-part (3 products)
@pytest.mark.parametrize("cg", [1, 2])
def test_fp32_accurate_stream_k(k, cg):
    m, n, _ = PAIR if cg == 2 else SINGLE
    mode = "6xbf16" if k <= 512 else "3xbf16"
    cfg = members(mode, cg=cg)[0]
    p = synth.uniform_problem(m, n, k, seed=62, alpha=1.0, beta=0.5)
    full, C = guarded(m, n, p.C)
    assert run(dev(p.A), dev(p.B), C, 1.0, 0.5, G3_F32_3XBF16, cfg, SK) == 1
    check_guard(full, m, n)
    got = C.cpu().numpy()
    bc = 0.5 * p.C.astype(np.float64)
    D = oracle.absprod(p.A, p.B, 1.0)
    method = oracle.gemm_6xbf16 if k <= 512 else oracle.gemm_3xbf16
    assert rel_err(got, method(p.A, p.B, p.C, 1.0, 0.5), D, bc) <= 1e-5
    assert rel_err(got, oracle.gemm(p.A, p.B, p.C, 1.0, 0.5), D, bc) <= 2e-6


def test_fp16_and_tf32_stream_k():
    m, n, k = SINGLE
    p = synth.uniform_problem(m, n, k, seed=63, alpha=0.5, beta=-1.0)
    bc = -1.0 * p.C.astype(np.float64)
    A16, B16 = p.A.astype(np.float16), p.B.astype(np.float16)
    full, C = guarded(m, n, p.C)
    assert run(torch.from_numpy(A16).cuda(), torch.from_numpy(B16).cuda(), C, 0.5, -1.0, G3_FP16,
               members("f16", cg=1, bm=128)[0], SK) == 1
    check_guard(full, m, n)
    Aq, Bq = A16.astype(np.float64), B16.astype(np.float64)
    assert rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq, p.C, 0.5, -1.0), oracle.absprod(Aq, Bq, 0.5), bc) <= 1e-5
    full, C = guarded(m, n, p.C)
    assert run(dev(p.A), dev(p.B), C, 0.5, -1.0, G3_TF32, members("tf32", cg=2)[0], SK) == 1
    check_guard(full, m, n)
    Aq, Bq = oracle.round_tf32(p.A), oracle.round_tf32(p.B)
    assert rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq, p.C, 0.5, -1.0), oracle.absprod(Aq, Bq, 0.5), bc) <= 1e-5


@pytest.mark.parametrize("cg", [1, 2])
def test_fp8_stream_k_applies_device_scales(cg):
    # the fix-up multiplies by alpha * scale_a * scale_b read from the device
    m, n, k = PAIR if cg == 2 else SINGLE
    p = synth.normal_problem(m, n, k, seed=64, alpha=0.75, beta=0.0)
    qa, sa = torch_api.quantize_fp8(dev(p.A))
    qb, sb = torch_api.quantize_fp8(dev(p.B))
    full, C = guarded(m, n, None)
    assert run(qa, qb, C, 0.75, 0.0, G3_FP8_E4M3, members("fp8", cg=cg)[0], SK, scale_a=sa, scale_b=sb) == 1
    check_guard(full, m, n)
    oqa, osa = oracle.fp8_quantize(p.A)
    oqb, osb = oracle.fp8_quantize(p.B)
    Ad = oracle.e4m3_decode(oqa).astype(np.float64) * osa
    Bd = oracle.e4m3_decode(oqb).astype(np.float64) * osb
    assert rel_err(C.cpu().numpy(), oracle.gemm(Ad, Bd, None, 0.75, 0.0), oracle.absprod(Ad, Bd, 0.75)) <= 1e-4


@pytest.mark.parametrize("beta", [0, 1])
@pytest.mark.parametrize("config", members("int8emu"))
def test_int8_stream_k_bit_exact(config, beta):
    # the exact-integer members keep their int32 sums in registers and take no
    # stream-K tail: a forced request computes the plain walk, still exact
    m, n, _ = shape_for(config)
    p = synth.int8_problem(m, n, 1100, seed=65, beta=beta)   # k: one 1024-product chunk and a tail
    full, C = guarded(m, n, p.C, dtype=torch.int32)
    extra = run(dev(p.A), dev(p.B), C, 1, beta, G3_INT8, config, SK)
    check_guard(full, m, n)
    assert extra == 0
    assert np.array_equal(C.cpu().numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta))


def test_stream_k_without_tail_is_a_plain_walk():
    # 19 x 8 = 152 tiles of 64 x 128 fill one wave of a 152-SM GPU exactly:
    # nothing is left for a tail and no fix-up runs (other SM counts: a tail)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    p = synth.uniform_problem(64 * 19, 128 * 8, 700, seed=66, beta=0.5)
    A, B = torch_api.convert_bf16(dev(p.A)), torch_api.convert_bf16(dev(p.B))
    C = dev(p.C)
    extra = run(A, B, C, 1.0, 0.5, G3_BF16, members("bf16", cg=1, bm=64)[0], SK)
    assert extra == (0 if 152 % sms == 0 else 1)
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    assert rel_err(C.cpu().numpy(), oracle.gemm(Aq, Bq, p.C, 1.0, 0.5), oracle.absprod(Aq, Bq, 1.0),
                   0.5 * p.C.astype(np.float64)) <= 1e-5


def test_stream_k_deterministic_and_graph_capturable():
    m, n, k = SINGLE
    p = synth.uniform_problem(m, n, k, seed=67, beta=0.0)
    A, B = dev(p.A), dev(p.B)
    cfg = members("3xbf16", cg=1, bm=128)[0]
    outs = []
    for _ in range(2):
        C = torch.empty(m, n, device="cuda")
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_F32_3XBF16, config=cfg, split_k=SK)
        torch.cuda.synchronize()
        outs.append(C.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    # captured into a CUDA graph (workspace grown by the eager calls above)
    Cg = torch.empty(m, n, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            torch_api.gemm(A, B, Cg, 1.0, 0.0, dtype=G3_F32_3XBF16, config=cfg, split_k=SK, stream=s)
    Cg.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(Cg.cpu().numpy(), outs[0])
