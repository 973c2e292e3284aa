"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times (the planner's member and split), checked on
sampled rows of C that the oracle computes in binary64 (int64 for INT8):

  FP32-accurate 16384^3 (alpha 1, beta 0.5, uniform [-1, 1], seed 0)  gate 2e-6
  the square sweep 2048 / 4096 / 8192 (same recipe), FP32-accurate and the
  FP32 SIMT kernel                                                       gate 2e-6
  the 3xTF32 FP32-accurate mode on the same inputs at 8192^3             gate 2e-6
  BF16 / FP16 / TF32 / FP8 / INT8 8192^3          8e-3 / 2e-3 / 2e-3 / 6e-2 / bit-exact
  BF16 / FP8 8192^3 with both operands stored transposed (read in place)
                                                   bit-identical to row-major
  the 20 im2col layer shapes (batch 16) in BF16    kernel check 1e-5, gate 8e-3
  the three batch-1 im2col examples in BF16         kernel check 1e-5, gate 8e-3
  the 20 im2col layer shapes in INT8               bit-exact (first, middle, last row)
  the 20 im2col layer shapes in FP8 (per-tensor scales)  kernel check 1e-4,
                                                   gate 6e-2; the two k = 64
                                                   layers (L2, L4) on every row
  the 1000-problem grouped batches (BF16 and FP32-accurate), every 25th
  problem checked in full

The FP32 gates hold on the stated metric, max |C - C_ref| / (|alpha||A||B|),
with beta = 0.5 (k >= 2048 here); the metric with |beta C| added to the
denominator is computed beside it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32,
                                    synth, torch_api)

pytestmark = pytest.mark.gpu


def sampled_errs(got_rows, rows, A, B, C, alpha, beta):
    """(strict, with_beta) over the sampled rows: max |C - C_ref| divided by
    |alpha| |A||B|, and by |alpha| |A||B| + |beta C|."""
    ref = oracle.gemm(A[rows], B, None if C is None else C[rows], alpha, beta)
    D = oracle.absprod(A[rows], B, alpha)
    diff = np.abs(got_rows - ref)
    strict = float(np.max(diff / np.maximum(D, 1e-300)))
    if C is None or beta == 0.0:
        return strict, strict
    Db = D + np.abs(beta * C[rows].astype(np.float64))
    return strict, float(np.max(diff / np.maximum(Db, 1e-300)))


def sampled_err(got_rows, rows, A, B, C, alpha, beta):
    """The stated metric, max |C - C_ref| / (|alpha| |A||B|), over the sampled rows."""
    return sampled_errs(got_rows, rows, A, B, C, alpha, beta)[0]


def test_fp32_accurate_16384_cubed():
    n = 16384
    p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
    A, B, C = (torch.from_numpy(x).cuda() for x in (p.A, p.B, p.C))
    torch_api.gemm(A, B, C, 1.0, 0.5, dtype=G3_F32_3XBF16)
    rows = np.array([0, 1, 5461, 8192, 12345, n - 1])
    got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del A, B, C
    e, e_b = sampled_errs(got, rows, p.A, p.B, p.C, 1.0, 0.5)
    print(f"16384^3 FP32-accurate sampled error {e:.3e} (with |beta C|: {e_b:.3e})")
    assert e <= 2e-6


@pytest.mark.parametrize("n", [2048, 4096, 8192])
def test_square_sweep_fp32_accurate_and_simt(n):
    # the square sweep's recipe (uniform [-1, 1], seed 0, alpha 1, beta 0.5):
    # the FP32-accurate mode and the plain FP32 SIMT kernel, each within the
    # 2e-6 gate on the stated metric on sampled rows
    p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
    A, B = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
    rows = np.array([0, 1, n // 3, n // 2, n - 1])
    sel = torch.from_numpy(rows).cuda()
    for dtype, name in ((G3_F32_3XBF16, "3xbf16"), (G3_F32, "simt")):
        C = torch.from_numpy(p.C).cuda()
        torch_api.gemm(A, B, C, 1.0, 0.5, dtype=dtype)
        got = C[sel].double().cpu().numpy()
        e, e_b = sampled_errs(got, rows, p.A, p.B, p.C, 1.0, 0.5)
        print(f"{n}^3 {name} sampled error {e:.3e} (with |beta C|: {e_b:.3e})")
        assert e <= 2e-6, (name, e)


def test_3xtf32_8192_cubed():
    n = 8192
    p = synth.uniform_problem(n, n, n, seed=0, alpha=1.0, beta=0.5)
    A, B, C = (torch.from_numpy(x).cuda() for x in (p.A, p.B, p.C))
    torch_api.gemm(A, B, C, 1.0, 0.5, dtype=G3_F32_3XTF32)
    rows = np.array([0, 1, 4097, n - 1])
    got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del A, B, C
    e, e_b = sampled_errs(got, rows, p.A, p.B, p.C, 1.0, 0.5)
    print(f"8192^3 3xTF32 sampled error {e:.3e} (with |beta C|: {e_b:.3e})")
    assert e <= 2e-6


@pytest.mark.parametrize("kind", ["bf16", "fp16", "tf32", "fp8", "int8"])
def test_dtype_8192_cubed(kind):
    n = 8192
    rows = np.array([0, 77, n // 2, n - 1])
    sel = torch.from_numpy(rows).cuda()
    if kind == "int8":
        p = synth.int8_problem(n, n, n, seed=0)
        A, B = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
        C = torch.empty(n, n, dtype=torch.int32, device="cuda")
        torch_api.gemm(A, B, C, 1, 0, dtype=G3_INT8)
        got = C[sel].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle.gemm_i8(p.A[rows], p.B))
        return
    p = synth.normal_problem(n, n, n, seed=0)
    A32, B32 = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
    C = torch.empty(n, n, device="cuda")
    if kind == "bf16":
        A, B = torch_api.convert_bf16(A32), torch_api.convert_bf16(B32)
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_BF16)
        tol = 8e-3
    elif kind == "fp16":
        torch_api.gemm(A32.half(), B32.half(), C, 1.0, 0.0, dtype=G3_FP16)
        tol = 2e-3
    elif kind == "tf32":
        torch_api.gemm(A32, B32, C, 1.0, 0.0, dtype=G3_TF32)
        tol = 2e-3
    else:
        (A, sa), (B, sb) = torch_api.quantize_fp8(A32), torch_api.quantize_fp8(B32)
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=sa, scale_b=sb)
        tol = 6e-2
    e = sampled_err(C[sel].double().cpu().numpy(), rows, p.A, p.B, None, 1.0, 0.0)
    print(f"{kind} 8192^3 sampled error {e:.3e}")
    assert e <= tol


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_dtype_8192_cubed_transposed_in_place(kind):
    # A stored k x m and B stored n x k, read in place by the planner's member
    # for 8192^3: every element equal to the same plan on row-major storage
    n = 8192
    p = synth.normal_problem(n, n, n, seed=0)
    A32, B32 = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
    if kind == "bf16":
        A, B, dt, kw = torch_api.convert_bf16(A32), torch_api.convert_bf16(B32), G3_BF16, {}
    else:
        (A, sa), (B, sb) = torch_api.quantize_fp8(A32), torch_api.quantize_fp8(B32)
        dt, kw = G3_FP8_E4M3, {"scale_a": sa, "scale_b": sb}
    del A32, B32
    C_r = torch.empty(n, n, device="cuda")
    torch_api.gemm(A, B, C_r, 1.0, 0.0, dtype=dt, **kw)
    At, Bt = A.t().contiguous(), B.t().contiguous()
    C_t = torch.empty(n, n, device="cuda")
    torch_api.gemm(At, Bt, C_t, 1.0, 0.0, dtype=dt, trans_a=True, trans_b=True, **kw)
    torch.cuda.synchronize()
    assert torch.equal(C_t.view(torch.int32), C_r.view(torch.int32))


def test_im2col_layers_bf16():
    worst_k = worst_g = 0.0
    for li, (name, m, n, k) in enumerate(synth.im2col_shapes(16)):
        p = synth.normal_problem(m, n, k, seed=li + 1)
        A, B = torch_api.convert_bf16(torch.from_numpy(p.A).cuda()), torch_api.convert_bf16(torch.from_numpy(p.B).cuda())
        C = torch.empty(m, n, device="cuda")
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_BF16)
        rows = np.unique(np.array([0, m // 3, m - 1]))
        got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
        e_k = sampled_err(got, rows, Aq, Bq, None, 1.0, 0.0)
        e_g = sampled_err(got, rows, p.A, p.B, None, 1.0, 0.0)
        assert e_k <= 1e-5, (name, e_k)
        assert e_g <= 8e-3, (name, e_g)
        worst_k, worst_g = max(worst_k, e_k), max(worst_g, e_g)
    print(f"im2col 20 layers: kernel {worst_k:.3e} gate {worst_g:.3e}")


def test_im2col_batch1_examples_bf16():
    # the three batch-1 examples of the convolution workload: 64 x 12544 x 147
    # (unaligned k: A is re-packed), 256 x 3136 x 576 and 2048 x 49 x 1024
    # (unaligned n: B and C rows of 49 elements); every row checked
    for li, (m, n, k) in enumerate(synth.IM2COL_BATCH1_EXAMPLES):
        p = synth.normal_problem(m, n, k, seed=100 + li)
        A, B = torch_api.convert_bf16(torch.from_numpy(p.A).cuda()), torch_api.convert_bf16(torch.from_numpy(p.B).cuda())
        C = torch.empty(m, n, device="cuda")
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_BF16)
        got = C.double().cpu().numpy()
        rows = np.arange(m)
        Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
        e_k = sampled_err(got, rows, Aq, Bq, None, 1.0, 0.0)
        e_g = sampled_err(got, rows, p.A, p.B, None, 1.0, 0.0)
        print(f"batch-1 {m}x{n}x{k}: kernel {e_k:.3e} gate {e_g:.3e}")
        assert e_k <= 1e-5, ((m, n, k), e_k)
        assert e_g <= 8e-3, ((m, n, k), e_g)


def test_im2col_layers_int8_bit_exact():
    # INT8 (exact on the BF16 tensor path) on the 20 layer shapes at batch 16,
    # uniform integers in [-128, 127], alpha 1, beta 0: the first, middle and
    # last row of every layer equal the int64 oracle exactly
    for li, (name, m, n, k) in enumerate(synth.im2col_shapes(16)):
        p = synth.int8_problem(m, n, k, seed=li + 1)
        A, B = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
        C = torch.empty(m, n, dtype=torch.int32, device="cuda")
        torch_api.gemm(A, B, C, 1, 0, dtype=G3_INT8)
        rows = np.unique(np.array([0, m // 2, m - 1]))
        got = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle.gemm_i8(p.A[rows], p.B)), name


def test_im2col_layers_fp8():
    # FP8 E4M3 with per-tensor scales on the 20 layer shapes at batch 16
    # (A ~ N(0,1)/sqrt(k), B ~ N(0,1)): the library's quantisation equals the
    # oracle's (codes and scales bit for bit), the kernel check against the
    # decoded values times the scales holds to 1e-4, and the gate against the
    # FP32 masters to 6e-2.  The k = 64 layers (L2: 64 x 50176, L4: 256 x 50176),
    # where one product's rounding is least averaged out, are checked on every
    # row; the others on the first, middle and last row.
    worst_k = worst_g = 0.0
    for li, (name, m, n, k) in enumerate(synth.im2col_shapes(16)):
        p = synth.normal_problem(m, n, k, seed=li + 1)
        (A, sa), (B, sb) = (torch_api.quantize_fp8(torch.from_numpy(x).cuda()) for x in (p.A, p.B))
        oqa, osa = oracle.fp8_quantize(p.A)
        oqb, osb = oracle.fp8_quantize(p.B)
        assert float(sa.item()) == float(osa) and float(sb.item()) == float(osb), name
        assert np.array_equal(A.view(torch.uint8).cpu().numpy(), oqa), name
        assert np.array_equal(B.view(torch.uint8).cpu().numpy(), oqb), name
        C = torch.empty(m, n, device="cuda")
        torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_FP8_E4M3, scale_a=sa, scale_b=sb)
        rows = np.arange(m) if k == 64 else np.unique(np.array([0, m // 2, m - 1]))
        got = C[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        Ad = oracle.e4m3_decode(oqa).astype(np.float64) * float(osa)
        Bd = oracle.e4m3_decode(oqb).astype(np.float64) * float(osb)
        e_k = sampled_err(got, rows, Ad, Bd, None, 1.0, 0.0)
        e_g = sampled_err(got, rows, p.A, p.B, None, 1.0, 0.0)
        assert e_k <= 1e-4, (name, e_k)
        assert e_g <= 6e-2, (name, e_g)
        worst_k, worst_g = max(worst_k, e_k), max(worst_g, e_g)
    print(f"im2col 20 layers FP8: kernel {worst_k:.3e} gate {worst_g:.3e}")


def test_resnet50_layers_implicit_gemm():
    # the 19 Table 1 layers with C % 64 == 0 as implicit-GEMM convolutions at
    # batch 16; image 0 of each output is checked against the direct oracle
    worst = 0.0
    for geo in synth.RESNET50_CONV:
        if geo["C"] % 64:
            continue
        r = np.random.default_rng(geo["layer"])
        H, C, K, R, st, pd = geo["H"], geo["C"], geo["K"], geo["R"], geo["stride"], geo["pad"]
        x = oracle.round_bf16(r.standard_normal((16, H, H, C)).astype(np.float32))
        w = oracle.round_bf16((r.standard_normal((R, R, C, K)) / np.sqrt(R * R * C)).astype(np.float32))
        y = torch_api.conv2d(torch.from_numpy(x).cuda().to(torch.bfloat16), torch.from_numpy(w).cuda().to(torch.bfloat16),
                             stride=(st, st), pad=(pd, pd))
        got = y[0].cpu().numpy()
        want = oracle.conv2d_nhwc(x[:1], w, (st, st), (pd, pd))[0]
        D = oracle.conv2d_nhwc(np.abs(x[:1]), np.abs(w), (st, st), (pd, pd))[0]
        e = float(np.max(np.abs(got - want) / np.maximum(D, 1e-300)))
        assert e <= 1e-5, (geo, e)
        worst = max(worst, e)
    print(f"ResNet-50 implicit-GEMM layers: worst error {worst:.3e}")


@pytest.mark.parametrize("dtype", [G3_BF16, G3_F32_3XBF16])
def test_grouped_1000(dtype):
    shapes = synth.grouped_shapes(1000, seed=0)
    probs, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        p = synth.uniform_problem(m, n, k, seed=i)
        A32, B32 = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.B).cuda()
        if dtype == G3_BF16:
            A, B = torch_api.convert_bf16(A32), torch_api.convert_bf16(B32)
        else:
            A, B = A32, B32
        C = torch.full((m, n), float("nan"), device="cuda")
        probs.append((A, B, C, 1.0, 0.0))
        host.append(p)
    plan = torch_api.GroupedPlan(probs, dtype)
    plan.execute()
    torch.cuda.synchronize()
    worst = 0.0
    for i in range(0, 1000, 25):
        p, C = host[i], probs[i][2].double().cpu().numpy()
        if dtype == G3_BF16:
            Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
            e = float(np.max(np.abs(C - oracle.gemm(Aq, Bq)) / np.maximum(oracle.absprod(Aq, Bq, 1.0), 1e-300)))
            assert e <= 1e-5, (i, e)
        else:
            e = float(np.max(np.abs(C - oracle.gemm(p.A, p.B)) / np.maximum(oracle.absprod(p.A, p.B, 1.0), 1e-300)))
            assert e <= 2e-6, (i, e)
        worst = max(worst, e)
    plan.close()
    print(f"grouped 1000 dtype {dtype}: worst checked error {worst:.3e}")
