"""Claimed tile walk: launches of at least 16 waves of tiles take their tiles
past the first wave from a counter in claim order.  Every tile is still
computed by the same arithmetic, so the result must be bit-identical to the
static walk (G3_STATIC_WALK=1) on every member kind, with split-K, with
operands read transposed, through a caller workspace with and without room
for the counter, inside a CUDA graph, and after a watchdog abort; sampled rows
are checked against the oracle."""
import contextlib
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_util import gate, rel_err
from paper_2310_20347_gb300 import G3_BF16, G3_F32_3XBF16, G3_FP8_E4M3, G3_INT8, _lib, gen_family, synth, torch_api

pytestmark = pytest.mark.gpu
FAMILY = gen_family.enumerate_family()
ROWS = [0, 1, 5000, 12287]


def member(mode, bm, cg):
    return next(f["index"] for f in FAMILY if f["mode"] == mode and f["bm"] == bm and f["cg"] == cg and not f.get("raw8"))


@contextlib.contextmanager
def static_walk():
    os.environ["G3_STATIC_WALK"] = "1"
    try:
        yield
    finally:
        del os.environ["G3_STATIC_WALK"]


def ws_bytes(A, B, C, **kw):
    st, n = _lib.g3_gemm_workspace_size(torch_api.gemm_args(A, B, C, **kw))
    assert st == 0
    return n


def both_walks(A, B, C0, **kw):
    """C from the claimed and from the static walk (C0 as the initial C), and
    the launches each took."""
    out = []
    for forced in (False, True):
        C = C0.clone()
        with static_walk() if forced else contextlib.nullcontext():
            n0 = _lib.g3_launch_count()
            torch_api.gemm(A, B, C, **kw)
            torch.cuda.synchronize()
            out.append((C, _lib.g3_launch_count() - n0))
    assert torch_api.device_status()[0] == 0
    return out


def bf16_problem(m, n, k, seed):
    p = synth.uniform_problem(m, n, k, seed=seed)
    Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
    return p, Aq, Bq, torch.from_numpy(Aq).cuda().bfloat16(), torch.from_numpy(Bq).cuda().bfloat16()


@pytest.mark.parametrize("mode,bm,cg", [("bf16", 256, 2), ("bf16", 128, 1), ("bf16", 64, 1)])
def test_bf16_claimed_equals_static(mode, bm, cg):
    p, Aq, Bq, A, B = bf16_problem(12288, 12288, 64, seed=900 + bm + cg)
    C0 = torch.empty(p.m, p.n, device="cuda")
    kw = dict(alpha=1.0, beta=0.0, dtype=G3_BF16, config=member(mode, bm, cg))
    # the claimed walk applies (its counter needs 256 bytes of workspace)
    with static_walk():
        w_static = ws_bytes(A, B, C0, **kw)
    assert ws_bytes(A, B, C0, **kw) == w_static + 256
    (Cc, lc), (Cs, ls) = both_walks(A, B, C0, **kw)
    assert lc == ls
    assert torch.equal(Cc, Cs)
    got = Cc[ROWS].cpu().numpy()
    e = rel_err(got, oracle.gemm(Aq, Bq, rows=ROWS), oracle.absprod(Aq, Bq, 1.0, rows=ROWS))
    assert e <= 1e-5, e


def test_planner_reports_the_claimed_walk_band():
    # 16384^3 FP32-accurate: 54 waves of 256 x 256 tiles on the CTA-pair member
    # (bands of 5: 5 x 16 MiB of bf16 planes of A within 80 MiB of L2)
    st, cfg, sk, raster = _lib.g3_plan_query(16384, 16384, 16384, G3_F32_3XBF16)
    assert st == 0 and raster == 5
    with static_walk():
        assert _lib.g3_plan_query(16384, 16384, 16384, G3_F32_3XBF16) == (0, cfg, sk, 8)
    # a launch of a few waves keeps the static walk and its bands of 8
    assert _lib.g3_plan_query(2048, 2048, 2048, G3_BF16)[3] == 8


@pytest.mark.parametrize("k", [200, 700])   # three-part split (k <= 512) and the two-part split
def test_fp32_accurate_claimed_equals_static(k):
    p = synth.uniform_problem(12288, 12288, k, seed=910 + k, alpha=1.5, beta=0.5)
    A, B, C0 = (torch.from_numpy(x).cuda() for x in (p.A, p.B, p.C))
    kw = dict(alpha=p.alpha, beta=p.beta, dtype=G3_F32_3XBF16)
    (Cc, lc), (Cs, ls) = both_walks(A, B, C0, **kw)
    assert lc == ls
    assert torch.equal(Cc, Cs)
    got = Cc[ROWS].cpu().numpy()
    ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta, rows=ROWS)
    # the strict metric (|alpha||A||B| alone) as well from k = 256 on
    gate(got, ref, oracle.absprod(p.A, p.B, p.alpha, rows=ROWS), p.beta * p.C[ROWS].astype(np.float64), k, 2e-6)


def test_split_k_claimed_equals_static():
    p, Aq, Bq, A, B = bf16_problem(12288, 6144, 1024, seed=920)
    C0 = torch.from_numpy(np.random.default_rng(921).uniform(-1, 1, (12288, 6144)).astype(np.float32)).cuda()
    kw = dict(alpha=0.75, beta=-0.5, dtype=G3_BF16, config=member("bf16", 128, 1), split_k=2)
    (Cc, _), (Cs, _) = both_walks(A, B, C0, **kw)
    assert torch.equal(Cc, Cs)
    C0h = C0[ROWS].cpu().numpy()
    ref = oracle.gemm(Aq[ROWS], Bq, C0h, 0.75, -0.5)
    e = rel_err(Cc[ROWS].cpu().numpy(), ref, oracle.absprod(Aq, Bq, 0.75, rows=ROWS), -0.5 * C0h.astype(np.float64))
    assert e <= 1e-5, e


@pytest.mark.parametrize("ta,tb", [(False, True), (True, False)])
def test_transposed_in_place_claimed_equals_static(ta, tb):
    p, Aq, Bq, A, B = bf16_problem(12288, 12288, 128, seed=930)
    At = A.t().contiguous() if ta else A
    Bt = B.t().contiguous() if tb else B
    C0 = torch.empty(p.m, p.n, device="cuda")
    kw = dict(alpha=1.0, beta=0.0, dtype=G3_BF16, trans_a=ta, trans_b=tb)
    (Cc, _), (Cs, _) = both_walks(At, Bt, C0, **kw)
    assert torch.equal(Cc, Cs)
    # and the same bits as the row-major operands
    Cr = torch.empty_like(C0)
    torch_api.gemm(A, B, Cr, 1.0, 0.0, dtype=G3_BF16)
    assert torch.equal(Cc, Cr)


def test_fp8_and_int8_pairs_claimed_equals_static():
    r = np.random.default_rng(940)
    A8 = torch.from_numpy(r.integers(0, 256, (12288, 128), dtype=np.uint8)).cuda()
    B8 = torch.from_numpy(r.integers(0, 256, (128, 12288), dtype=np.uint8)).cuda()
    # finite e4m3 codes only (0x7f / 0xff are NaN)
    A8[(A8 & 0x7F) == 0x7F] = 0x3C
    B8[(B8 & 0x7F) == 0x7F] = 0x3C
    C0 = torch.empty(12288, 12288, device="cuda")
    (Cc, _), (Cs, _) = both_walks(A8, B8, C0, alpha=1.0, beta=0.0, dtype=G3_FP8_E4M3,
                                  config=member("fp8", 256, 2))
    assert torch.equal(Cc, Cs)
    Ai = torch.from_numpy(r.integers(-128, 128, (12288, 256), dtype=np.int8)).cuda()
    Bi = torch.from_numpy(r.integers(-128, 128, (256, 12288), dtype=np.int8)).cuda()
    C0 = torch.empty(12288, 12288, dtype=torch.int32, device="cuda")
    (Cc, _), (Cs, _) = both_walks(Ai, Bi, C0, alpha=1, beta=0, dtype=G3_INT8, config=member("int8emu", 256, 2))
    assert torch.equal(Cc, Cs)
    got = Cc[ROWS].cpu().numpy()
    assert np.array_equal(got, oracle.gemm_i8(Ai.cpu().numpy()[ROWS], Bi.cpu().numpy()))


def test_caller_workspace_with_and_without_room_for_the_counter():
    p, Aq, Bq, A, B = bf16_problem(12288, 12288, 64, seed=950)
    C0 = torch.empty(p.m, p.n, device="cuda")
    kw = dict(alpha=1.0, beta=0.0, dtype=G3_BF16, config=member("bf16", 128, 1))
    need = ws_bytes(A, B, C0, **kw)
    assert need >= 256
    ref = C0.clone()
    with static_walk():
        torch_api.gemm(A, B, ref, **kw)
    for size in (need, need - 1):   # room for the counter: claimed walk; one byte short: static walk
        ws = torch.empty(max(size, 1), dtype=torch.uint8, device="cuda")
        C = C0.clone()
        torch_api.gemm(A, B, C, workspace=ws, **kw)
        torch.cuda.synchronize()
        assert torch.equal(C, ref), size
    assert torch_api.device_status()[0] == 0


def test_claimed_walk_in_a_cuda_graph():
    p, Aq, Bq, A, B = bf16_problem(12288, 12288, 64, seed=960)
    ref = torch.empty(p.m, p.n, device="cuda")
    kw = dict(alpha=1.0, beta=0.0, dtype=G3_BF16, config=member("bf16", 256, 2))
    with static_walk():
        torch_api.gemm(A, B, ref, **kw)
    C = torch.zeros_like(ref)
    torch_api.gemm(A, B, C, **kw)   # the first call outside the capture (workspace, descriptors)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        torch_api.gemm(A, B, C, stream=s, **kw)
    for _ in range(3):   # the counter is zeroed again on every replay
        C.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(C, ref)
    assert torch_api.device_status()[0] == 0


@pytest.mark.parametrize("mode,bm,cg", [("bf16", 256, 2), ("bf16", 128, 1)])
def test_watchdog_on_a_claimed_walk(mode, bm, cg):
    assert torch_api.device_status()[0] == 0
    p, Aq, Bq, A, B = bf16_problem(12288, 12288, 64, seed=970)
    C = torch.zeros(p.m, p.n, device="cuda")
    kw = dict(alpha=1.0, beta=0.0, dtype=G3_BF16, config=member(mode, bm, cg))
    assert _lib.g3_debug_withhold_next(200) == 0
    torch_api.gemm(A, B, C, **kw)
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    # the context is still usable and the next claimed walk is correct
    (Cc, _), (Cs, _) = both_walks(A, B, C, **kw)
    assert torch.equal(Cc, Cs)
    e = rel_err(Cc[ROWS].cpu().numpy(), oracle.gemm(Aq, Bq, rows=ROWS), oracle.absprod(Aq, Bq, 1.0, rows=ROWS))
    assert e <= 1e-5, e
