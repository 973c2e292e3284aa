"""Single GEMM calls captured into CUDA graphs, for every dtype: after one
eager call (which sizes the library workspace), the call is captured on a side
stream and replayed twice; every replay reproduces the eager result bit for
bit (the launches are the same kernels on the same data, and every kernel of
the path is deterministic)."""
import numpy as np
import pytest
import torch

from paper_2310_20347_gb300 import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_F64, G3_FP16, G3_FP8_E4M3,
                                    G3_INT8, G3_INT16, G3_TF32, torch_api)

pytestmark = pytest.mark.gpu


def operands(dtype, m, n, k, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    kw = {}
    if dtype == G3_INT8:
        A = torch.randint(-128, 128, (m, k), dtype=torch.int8, device="cuda", generator=g)
        B = torch.randint(-128, 128, (k, n), dtype=torch.int8, device="cuda", generator=g)
        C = torch.randint(-1000, 1000, (m, n), dtype=torch.int32, device="cuda", generator=g)
        return A, B, C, 1, 1, kw
    if dtype == G3_INT16:
        A = torch.randint(-(1 << 15), 1 << 15, (m, k), dtype=torch.int16, device="cuda", generator=g)
        B = torch.randint(-(1 << 15), 1 << 15, (k, n), dtype=torch.int16, device="cuda", generator=g)
        C = torch.randint(-1000, 1000, (m, n), dtype=torch.int64, device="cuda", generator=g)
        return A, B, C, 1, 1, kw
    t = torch.float64 if dtype == G3_F64 else torch.float32
    A = torch.randn(m, k, dtype=t, device="cuda", generator=g)
    B = torch.randn(k, n, dtype=t, device="cuda", generator=g)
    C = torch.randn(m, n, dtype=t, device="cuda", generator=g)
    if dtype == G3_BF16:
        A, B = A.bfloat16(), B.bfloat16()
    elif dtype == G3_FP16:
        A, B = A.half(), B.half()
    elif dtype == G3_FP8_E4M3:
        (A, sa), (B, sb) = torch_api.quantize_fp8(A), torch_api.quantize_fp8(B)
        kw = dict(scale_a=sa, scale_b=sb)
    return A, B, C, 0.75, 0.5, kw


@pytest.mark.parametrize("dtype", [G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_BF16, G3_FP16, G3_TF32, G3_FP8_E4M3,
                                   G3_INT8, G3_F64, G3_INT16])
@pytest.mark.parametrize("shape", [(700, 520, 300), (300, 900, 1500)])
def test_graph_replay_matches_eager(dtype, shape):
    m, n, k = shape
    A, B, C0, alpha, beta, kw = operands(dtype, m, n, k, seed=m + k + dtype)
    eager = C0.clone()
    torch_api.gemm(A, B, eager, alpha, beta, dtype=dtype, **kw)
    torch.cuda.synchronize()
    C = C0.clone()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            torch_api.gemm(A, B, C, alpha, beta, dtype=dtype, stream=s, **kw)
    for _ in range(2):
        C.copy_(C0)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(C, eager), dtype


@pytest.mark.gpu
def test_stream_traffic_yardstick_covers_its_output():
    # the streaming yardstick of the benchmark's traffic floors writes every
    # 16-byte unit of its output (filler) for several read/write proportions,
    # leaves its input and the bytes past its output untouched, and moves
    # bytes at a rate comparable to a plain device copy for a 1:1 mix
    from paper_2310_20347_gb300 import _lib
    x = torch.arange(1 << 20, dtype=torch.int32, device="cuda")
    x0 = x.clone()
    for out_units in (1, 511, 512, 513, 4096, 65536, 1 << 18, 1 << 20):
        y = torch.zeros(4 * out_units + 8, dtype=torch.int32, device="cuda")
        assert _lib.g3_stream_traffic(x.data_ptr(), x.numel() * 4, y.data_ptr(), out_units * 16) == 0
        torch.cuda.synchronize()
        head = y[:4 * out_units].view(-1, 4)
        assert bool((head[:, 2] == 0).all() and (head[:, 3] == 0).all())
        # filler (chunk + 1, thread + 1, 0, 0): every unit was written (y was zero)
        assert bool((head[:, 0] > 0).all() and (head[:, 1] > 0).all())
        assert bool((y[4 * out_units:] == 0).all())
    assert torch.equal(x, x0)
    big = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")
    big2 = torch.empty_like(big)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _lib.g3_stream_traffic(big.data_ptr(), big.numel(), big2.data_ptr(), big2.numel())
    e0.record()
    for _ in range(5):
        _lib.g3_stream_traffic(big.data_ptr(), big.numel(), big2.data_ptr(), big2.numel())
    e1.record()
    torch.cuda.synchronize()
    t_y = e0.elapsed_time(e1) / 5
    big2.copy_(big)
    e0.record()
    for _ in range(5):
        big2.copy_(big)
    e1.record()
    torch.cuda.synchronize()
    t_c = e0.elapsed_time(e1) / 5
    print(f"yardstick 1:1 {2 * big.numel() / t_y / 1e6:.0f} GB/s, torch copy {2 * big.numel() / t_c / 1e6:.0f} GB/s")
    assert t_y < 1.5 * t_c
