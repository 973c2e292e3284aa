"""g3_gemm_host: A, B, C in page-locked host memory, copies pipelined with the
row blocks of the computation.  Checked against the oracle with each dtype's
tolerance (bit-exact for INT8), single- and multi-block, strided host rows."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import rel_err
from paper_2310_20347_gb300 import G3_BF16, G3_F32, G3_F32_3XBF16, G3_F32_3XTF32, G3_FP16, G3_INT8, G3_TF32, synth, torch_api

pytestmark = pytest.mark.gpu


def pinned(x, pad=0):
    """A page-locked host tensor holding x, optionally with `pad` extra columns per row."""
    full = torch.zeros(x.shape[0], x.shape[1] + pad, dtype=x.dtype).pin_memory()
    full[:, : x.shape[1]] = x
    return full[:, : x.shape[1]]


# (2100, 300, 4500) and (4200, 260, 9000): B goes up in two and four k-slabs,
# row block 0 accumulating slab by slab on prepared bf16 planes of B
@pytest.mark.parametrize("m,n,k,dtype,pad,beta", [(300, 200, 150, G3_F32, 0, 0.5), (2500, 300, 700, G3_F32_3XBF16, 3, 0.5),
                                                  (2049, 130, 64, G3_F32_3XBF16, 0, 0.5), (700, 520, 300, G3_F32, 5, 0.5),
                                                  (2100, 300, 4500, G3_F32_3XBF16, 2, 0.5),
                                                  (4200, 260, 9000, G3_F32_3XBF16, 0, 0.0),
                                                  (2300, 200, 700, G3_F32_3XTF32, 1, 0.5)])
def test_host_fp32(m, n, k, dtype, pad, beta):
    p = synth.uniform_problem(m, n, k, seed=40, alpha=1.25, beta=beta)
    hA, hB = pinned(torch.from_numpy(p.A), pad), pinned(torch.from_numpy(p.B), pad)
    # beta = 0: C is never read (NaN must be overwritten)
    hC = pinned(torch.from_numpy(p.C) if p.C is not None else torch.full((m, n), float("nan")), pad)
    s = torch.cuda.current_stream()
    torch_api.gemm_host(hA, hB, hC, p.alpha, p.beta, dtype=dtype, stream=s)
    s.synchronize()
    D = oracle.absprod(p.A, p.B, p.alpha)
    bc = None if p.C is None else p.beta * p.C.astype(np.float64)
    e = rel_err(hC.numpy(), oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), D, bc)
    assert e <= 2e-6, e


def test_host_bf16_beta_zero_multiblock():
    p = synth.normal_problem(3000, 260, 520, seed=41)
    Ab = torch.from_numpy(oracle.round_bf16(p.A)).to(torch.bfloat16)
    Bb = torch.from_numpy(oracle.round_bf16(p.B)).to(torch.bfloat16)
    hA, hB = pinned(Ab), pinned(Bb)
    hC = pinned(torch.full((p.m, p.n), float("nan")))
    torch_api.gemm_host(hA, hB, hC, 1.0, 0.0, dtype=G3_BF16)
    torch.cuda.current_stream().synchronize()
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    e = rel_err(hC.numpy(), oracle.gemm(Aq, Bq, None, 1.0, 0.0), oracle.absprod(Aq, Bq, 1.0))
    assert e <= 1e-5, e


@pytest.mark.parametrize("dtype", [G3_FP16, G3_TF32])
def test_host_fp16_tf32_multiblock(dtype):
    p = synth.uniform_problem(2300, 200, 330, seed=45, beta=0.5)
    if dtype == G3_FP16:
        Aq, Bq = p.A.astype(np.float16), p.B.astype(np.float16)
        hA, hB = pinned(torch.from_numpy(Aq)), pinned(torch.from_numpy(Bq))
        Aq, Bq = Aq.astype(np.float64), Bq.astype(np.float64)
    else:
        hA, hB = pinned(torch.from_numpy(p.A)), pinned(torch.from_numpy(p.B))
        Aq, Bq = oracle.round_tf32(p.A), oracle.round_tf32(p.B)
    hC = pinned(torch.from_numpy(p.C))
    torch_api.gemm_host(hA, hB, hC, 1.0, 0.5, dtype=dtype)
    torch.cuda.current_stream().synchronize()
    e = rel_err(hC.numpy(), oracle.gemm(Aq, Bq, p.C, 1.0, 0.5), oracle.absprod(Aq, Bq, 1.0),
                0.5 * p.C.astype(np.float64))
    assert e <= 1e-5, e


@pytest.mark.parametrize("m,beta", [(600, 1), (2600, 0)])
def test_host_int8_bit_exact(m, beta):
    p = synth.int8_problem(m, 300, 1100, seed=42, beta=beta)
    hA, hB = pinned(torch.from_numpy(p.A)), pinned(torch.from_numpy(p.B))
    hC = pinned(torch.from_numpy(p.C) if p.C is not None else torch.zeros(m, 300, dtype=torch.int32))
    torch_api.gemm_host(hA, hB, hC, 1, beta, dtype=G3_INT8)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(hC.numpy().astype(np.int64), oracle.gemm_i8(p.A, p.B, p.C, 1, beta))


def test_host_back_to_back_calls_reuse_the_device_copies():
    # two calls queued without a host synchronisation in between
    p = synth.uniform_problem(2100, 140, 260, seed=43, beta=0.0)
    q = synth.uniform_problem(1800, 140, 260, seed=44, beta=0.0)
    hA, hB, hC = pinned(torch.from_numpy(p.A)), pinned(torch.from_numpy(p.B)), pinned(torch.zeros(p.m, p.n))
    gA, gB, gC = pinned(torch.from_numpy(q.A)), pinned(torch.from_numpy(q.B)), pinned(torch.zeros(q.m, q.n))
    torch_api.gemm_host(hA, hB, hC, 1.0, 0.0, dtype=G3_F32_3XBF16)
    torch_api.gemm_host(gA, gB, gC, 1.0, 0.0, dtype=G3_F32_3XBF16)
    torch.cuda.current_stream().synchronize()
    for prob, out in ((p, hC), (q, gC)):
        e = rel_err(out.numpy(), oracle.gemm(prob.A, prob.B, None, 1.0, 0.0), oracle.absprod(prob.A, prob.B, 1.0))
        assert e <= 2e-6, e


def _queued(problems, streams, dtype):
    """Queue one call per problem (round robin over `streams`) without any host
    synchronisation; return the results."""
    outs = []
    for i, prob in enumerate(problems):
        hA, hB = pinned(torch.from_numpy(prob.A)), pinned(torch.from_numpy(prob.B))
        hC = pinned(torch.from_numpy(prob.C) if prob.C is not None else torch.zeros(prob.m, prob.n))
        torch_api.gemm_host(hA, hB, hC, prob.alpha, prob.beta, dtype=dtype, stream=streams[i % len(streams)])
        outs.append(hC)
    torch.cuda.synchronize()
    return [o.numpy().copy() for o in outs]


@pytest.mark.parametrize("nstreams", [2, 6])
def test_host_calls_on_several_streams_overlap_and_match_one_stream(nstreams):
    # Each stream has its own device copies and block scratch, so calls on
    # different streams run concurrently (uploads of one under the compute of
    # another); six streams exceed the four buffer sets, and the fifth and
    # sixth take over the least recently used sets.  Every result must equal
    # the same call queued alone on one stream, bit for bit: FP32-accurate
    # multi-block calls with B in k-slabs (k = 4500), the plain row-block
    # pipeline (k = 700) and a one-block call.
    shapes = [(2100, 300, 4500, 0.5), (2500, 200, 700, 0.0), (600, 180, 300, 0.5), (2300, 260, 4200, 0.0)]
    probs = [synth.uniform_problem(m, n, k, seed=90 + i, alpha=1.0, beta=b)
             for i, (m, n, k, b) in enumerate(shapes * 2)][: max(4, nstreams + 1)]
    alone = [_queued([prob], [torch.cuda.current_stream()], G3_F32_3XBF16)[0] for prob in probs]
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    got = _queued(probs, streams, G3_F32_3XBF16)
    for prob, g, a in zip(probs, got, alone):
        assert np.array_equal(g.view(np.uint32), a.view(np.uint32)), (prob.m, prob.n, prob.k)
        bc = None if prob.C is None else prob.beta * prob.C.astype(np.float64)
        e = rel_err(g, oracle.gemm(prob.A, prob.B, prob.C, prob.alpha, prob.beta),
                    oracle.absprod(prob.A, prob.B, prob.alpha), bc)
        assert e <= 2e-6, e
