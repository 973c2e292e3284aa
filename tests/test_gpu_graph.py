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
def test_stream_traffic_yardstick_moves_the_data():
    # the streaming yardstick of the benchmark's traffic floors: with equal
    # sizes it copies; with twice as many bytes out, every second 16-byte unit
    # carries the next input unit (the others are filler); with half, every
    # second input unit is written
    from paper_2310_20347_gb300 import _lib
    x = torch.arange(1 << 16, dtype=torch.int32, device="cuda")
    y = torch.zeros_like(x)
    assert _lib.g3_stream_traffic(x.data_ptr(), x.numel() * 4, y.data_ptr(), y.numel() * 4) == 0
    torch.cuda.synchronize()
    assert torch.equal(x, y)
    y2 = torch.zeros(2 * x.numel(), dtype=torch.int32, device="cuda")
    assert _lib.g3_stream_traffic(x.data_ptr(), x.numel() * 4, y2.data_ptr(), y2.numel() * 4) == 0
    torch.cuda.synchronize()
    assert torch.equal(y2.view(-1, 2, 4)[:, 1, :].reshape(-1), x)
    y3 = torch.zeros(x.numel() // 2, dtype=torch.int32, device="cuda")
    assert _lib.g3_stream_traffic(x.data_ptr(), x.numel() * 4, y3.data_ptr(), y3.numel() * 4) == 0
    torch.cuda.synchronize()
    assert torch.equal(y3.view(-1, 4), x.view(-1, 2, 4)[:, 1, :])
