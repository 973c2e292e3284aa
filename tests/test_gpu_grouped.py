"""Parity of the persistent grouped launch (many uneven GEMMs, one kernel)
with the oracle, problem by problem, plus CUDA-graph capture, determinism,
guard bands, degenerate problems and the watchdog."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import SENTINEL, rel_err
from paper_2310_20347_gb300 import G3_BF16, G3_F32_3XBF16, G3_FP8_E4M3, _lib, synth, torch_api

pytestmark = pytest.mark.gpu


def make_batch(count, seed, lo=1, hi=300, dtype=G3_BF16, unaligned_every=5):
    """Problems with log-uniform sizes; every `unaligned_every`-th one gets
    leading dimensions that are not 16-byte multiples; C sits in a guard band."""
    shapes = synth.grouped_shapes(count, seed=seed, lo=lo, hi=hi)
    probs, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        p = synth.uniform_problem(m, n, k, seed=seed * 1000 + i, alpha=1.0 if i % 3 else -0.5,
                                  beta=0.0 if i % 2 else 0.5)
        pad = 3 if (unaligned_every and i % unaligned_every == 0) else 0
        A32 = torch.zeros(m, k + pad, device="cuda")[:, :k]
        A32.copy_(torch.from_numpy(p.A))
        B32 = torch.zeros(k, n + pad, device="cuda")[:, :n]
        B32.copy_(torch.from_numpy(p.B))
        if dtype == G3_BF16:
            Ab = torch.zeros(m, k + pad, dtype=torch.bfloat16, device="cuda")[:, :k]
            Ab.copy_(torch_api.convert_bf16(A32.contiguous()))
            Bb = torch.zeros(k, n + pad, dtype=torch.bfloat16, device="cuda")[:, :n]
            Bb.copy_(torch_api.convert_bf16(B32.contiguous()))
            A, B = Ab, Bb
        else:
            A, B = A32, B32
        full = torch.full((m + 2, n + 7), SENTINEL, device="cuda")
        C = full[1:1 + m, 3:3 + n]
        if p.C is not None:
            C.copy_(torch.from_numpy(p.C))
        probs.append((A, B, C, p.alpha, p.beta))
        host.append((p, full))
    return probs, host


def check_batch(probs, host, dtype):
    # an FP32-accurate plan takes the three-part split for problems with
    # k <= 512 and the two-part split for deeper ones
    worst_k = worst_g = 0.0
    for (A, B, C, alpha, beta), (p, full) in zip(probs, host):
        f = full.cpu().numpy()
        mask = np.ones(f.shape, bool)
        mask[1:1 + p.m, 3:3 + p.n] = False
        assert np.all(f[mask] == np.float32(SENTINEL)), "guard band overwritten"
        got = C.cpu().numpy()
        bc = None if p.C is None else p.beta * p.C.astype(np.float64)
        if dtype == G3_BF16:
            Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
            ref_k = oracle.gemm(Aq, Bq, p.C, p.alpha, p.beta)
            D_k = oracle.absprod(Aq, Bq, p.alpha)
            gate = 8e-3
        else:
            method = oracle.gemm_6xbf16 if p.k <= 512 else oracle.gemm_3xbf16
            ref_k = method(p.A, p.B, p.C, p.alpha, p.beta)
            D_k = oracle.absprod(p.A, p.B, p.alpha)
            gate = 2e-6
        e_k = rel_err(got, ref_k, D_k, bc)
        e_g = rel_err(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha), bc)
        assert e_k <= 1e-5, (p.m, p.n, p.k, "kernel", e_k)
        assert e_g <= gate, (p.m, p.n, p.k, "gate", e_g)
        worst_k, worst_g = max(worst_k, e_k), max(worst_g, e_g)
    return worst_k, worst_g


@pytest.mark.parametrize("dtype", [G3_BF16, G3_F32_3XBF16])
def test_grouped_parity(dtype):
    probs, host = make_batch(60, seed=1, dtype=dtype)
    plan = torch_api.GroupedPlan(probs, dtype)
    plan.execute()
    torch.cuda.synchronize()
    ek, eg = check_batch(probs, host, dtype)
    print(f"grouped dtype {dtype}: kernel {ek:.3e} gate {eg:.3e}")
    plan.close()


def test_grouped_fp32_deep_k_takes_two_part_split():
    # every k > 512: the plan runs the 3-product kernel, still within 2e-6
    probs, host = make_batch(8, seed=4, lo=600, hi=1024, dtype=G3_F32_3XBF16, unaligned_every=3)
    assert all(p.k > 512 for p, _ in host)
    plan = torch_api.GroupedPlan(probs, G3_F32_3XBF16)
    plan.execute()
    torch.cuda.synchronize()
    ek, eg = check_batch(probs, host, G3_F32_3XBF16)
    print(f"grouped fp32 deep k: kernel {ek:.3e} gate {eg:.3e}")
    plan.close()


def test_grouped_large_shapes_and_tiles():
    # sizes up to 1024 as in the 1000-problem workload: several tiles per problem
    probs, host = make_batch(12, seed=2, lo=100, hi=1024, dtype=G3_BF16, unaligned_every=0)
    plan = torch_api.GroupedPlan(probs, G3_BF16)
    plan.execute()
    torch.cuda.synchronize()
    check_batch(probs, host, G3_BF16)


def test_grouped_degenerate_problems():
    dev = "cuda"
    A = torch.zeros(5, 7, dtype=torch.bfloat16, device=dev)
    B = torch.zeros(7, 9, dtype=torch.bfloat16, device=dev)
    C0 = torch.full((5, 9), 2.0, device=dev)
    C1 = torch.full((5, 9), 2.0, device=dev)
    C2 = torch.full((0, 9), 2.0, device=dev)
    Ak = torch.zeros(5, 0, dtype=torch.bfloat16, device=dev)
    Bk = torch.zeros(0, 9, dtype=torch.bfloat16, device=dev)
    probs = [(Ak, Bk, C0, 1.0, 0.5),             # k = 0: C := beta*C
             (A, B, C1, 0.0, 3.0),               # alpha = 0: C := beta*C
             (torch.zeros(0, 7, dtype=torch.bfloat16, device=dev), B, C2, 1.0, 0.0)]   # m = 0
    plan = torch_api.GroupedPlan(probs, G3_BF16)
    plan.execute()
    torch.cuda.synchronize()
    assert torch.all(C0 == 1.0) and torch.all(C1 == 6.0)
    plan.close()


def test_grouped_graph_capture_and_determinism():
    probs, host = make_batch(40, seed=3, dtype=G3_F32_3XBF16)
    # beta = 0 everywhere so that replays are idempotent
    probs = [(A, B, C, a, 0.0) for (A, B, C, a, b) in probs]
    for (p, _full) in host:
        p.beta = 0.0
    plan = torch_api.GroupedPlan(probs, G3_F32_3XBF16)
    plan.execute()
    torch.cuda.synchronize()
    first = [C.clone() for (_, _, C, _, _) in probs]
    for (_, _, C, _, _) in probs:
        C.zero_()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.execute(stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for f, (_, _, C, _, _) in zip(first, probs):
        assert torch.equal(f, C)
    check_batch(probs, host, G3_F32_3XBF16)


def test_grouped_argument_errors():
    good = _lib.g3_gemm_desc()
    good.m = good.n = good.k = 4
    good.lda = good.ldb = good.ldc = 4
    good.A = good.B = good.C = 16
    bad = _lib.g3_gemm_desc()
    bad.m, bad.n, bad.k = 4, 4, 8
    bad.lda, bad.ldb, bad.ldc = 7, 4, 4
    bad.A = bad.B = bad.C = 16
    st, plan = _lib.g3_grouped_plan_create([good, good, bad], G3_BF16)
    assert st == -102
    st, plan = _lib.g3_grouped_plan_create([good], _lib.G3_INT8)
    assert st == _lib.G3_ERR_UNSUPPORTED
    # FP8 problems need finite, positive scales
    good.scale_a = good.scale_b = 0.5
    bad_scale = _lib.g3_gemm_desc()
    bad_scale.m = bad_scale.n = bad_scale.k = 4
    bad_scale.lda = bad_scale.ldb = bad_scale.ldc = 4
    bad_scale.A = bad_scale.B = bad_scale.C = 16
    for sa in (0.0, -1.0, float("inf"), float("nan")):
        bad_scale.scale_a, bad_scale.scale_b = sa, 1.0
        st, plan = _lib.g3_grouped_plan_create([good, bad_scale], G3_FP8_E4M3)
        assert st == -101, sa


def test_grouped_watchdog():
    probs, host = make_batch(10, seed=4, lo=64, hi=256, dtype=G3_BF16, unaligned_every=0)
    plan = torch_api.GroupedPlan(probs, G3_BF16)
    assert _lib.g3_debug_withhold_next(200) == 0
    plan.execute()
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    for (A, B, C, a, b), (p, full) in zip(probs, host):
        if p.C is not None:
            C.copy_(torch.from_numpy(p.C))
    plan.execute()
    torch.cuda.synchronize()
    check_batch(probs, host, G3_BF16)
    assert torch_api.device_status()[0] == 0


def test_grouped_fp8_parity():
    # FP8 E4M3 problems with per-problem scales (host values): each problem's
    # operands quantised per tensor by the library; the result equals the
    # oracle on the decoded codes times the scales (kernel check 1e-5 of
    # |alpha| |A||B|), and the FP32 masters within the FP8 gate (6e-2 for
    # k >= 64, the format bound 2 * 2^-4 + 2^-8 below; reading R2).  Every
    # fourth problem has rows that are not 16-byte multiples (re-packed).
    shapes = synth.grouped_shapes(48, seed=7, lo=1, hi=400)
    probs, host = [], []
    for i, (m, n, k) in enumerate(shapes):
        p = synth.normal_problem(m, n, k, seed=700 + i, alpha=1.0 if i % 3 else 0.75, beta=0.0 if i % 2 else 0.5)
        (qa, sa), (qb, sb) = (torch_api.quantize_fp8(torch.from_numpy(x).cuda()) for x in (p.A, p.B))
        pad = 5 if i % 4 == 0 else 0
        A = torch.zeros(m, k + pad, dtype=torch.uint8, device="cuda")[:, :k]
        A.copy_(qa)
        B = torch.zeros(k, n + pad, dtype=torch.uint8, device="cuda")[:, :n]
        B.copy_(qb)
        full = torch.full((m + 2, n + 7), SENTINEL, device="cuda")
        C = full[1:1 + m, 3:3 + n]
        if p.C is not None:
            C.copy_(torch.from_numpy(p.C))
        probs.append((A, B, C, p.alpha, p.beta, sa, sb))
        host.append((p, full, qa.cpu().numpy(), float(sa.item()), qb.cpu().numpy(), float(sb.item())))
    plan = torch_api.GroupedPlan(probs, G3_FP8_E4M3)
    plan.execute()
    torch.cuda.synchronize()
    worst_k = worst_g = 0.0
    for (A, B, C, *_), (p, full, qa, sa, qb, sb) in zip(probs, host):
        f = full.cpu().numpy()
        mask = np.ones(f.shape, bool)
        mask[1:1 + p.m, 3:3 + p.n] = False
        assert np.all(f[mask] == np.float32(SENTINEL)), "guard band overwritten"
        got = C.cpu().numpy()
        bc = None if p.C is None else p.beta * p.C.astype(np.float64)
        Ad = oracle.e4m3_decode(qa).astype(np.float64) * sa
        Bd = oracle.e4m3_decode(qb).astype(np.float64) * sb
        e_k = rel_err(got, oracle.gemm(Ad, Bd, p.C, p.alpha, p.beta), oracle.absprod(Ad, Bd, p.alpha), bc)
        e_g = rel_err(got, oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta), oracle.absprod(p.A, p.B, p.alpha), bc)
        assert e_k <= 1e-5, (p.m, p.n, p.k, "kernel", e_k)
        assert e_g <= (6e-2 if p.k >= 64 else 2 * 2.0 ** -4 + 2.0 ** -8), (p.m, p.n, p.k, "gate", e_g)
        worst_k, worst_g = max(worst_k, e_k), max(worst_g, e_g)
    print(f"grouped fp8: kernel {worst_k:.3e} gate {worst_g:.3e}")
    plan.close()


def _bucket(x):
    b = 0
    while (1 << b) < x:
        b += 1
    return b


def test_grouped_plan_uses_tuned_tile_height(tmp_path):
    # a tuning record for the bucket of 100 x 300 x 200 BF16 problems asks for
    # 64-row tiles (the fixed rule would take 128 for m > 64): a plan created
    # after loading it takes 64 rows for the problems in that bucket only, and
    # every problem still matches the oracle
    _lib.g3_tune_cache_clear()
    rec = tmp_path / "tune.txt"
    rec.write_text(f"# grouped record\n{100 + G3_BF16} {_bucket(100)} {_bucket(300)} {_bucket(200)} 64 1 0.01\n")
    assert _lib.g3_tune_cache_load(str(rec)) == 0
    probs, host = [], []
    for i, (m, n, k) in enumerate([(100, 300, 200), (120, 260, 150), (200, 300, 200), (90, 70, 40)]):
        p = synth.uniform_problem(m, n, k, seed=900 + i, alpha=1.0, beta=0.5)
        A = torch_api.convert_bf16(torch.from_numpy(p.A).cuda())
        B = torch_api.convert_bf16(torch.from_numpy(p.B).cuda())
        full = torch.full((m + 2, n + 7), SENTINEL, device="cuda")
        C = full[1:1 + m, 3:3 + n]
        C.copy_(torch.from_numpy(p.C))
        probs.append((A, B, C, p.alpha, p.beta))
        host.append((p, full))
    plan = torch_api.GroupedPlan(probs, G3_BF16)
    heights = [_lib.g3_grouped_plan_describe(plan.plan, i)[1] for i in range(4)]
    assert heights == [64, 64, 128, 128], heights
    plan.execute()
    torch.cuda.synchronize()
    check_batch(probs, host, G3_BF16)
    plan.close()
    _lib.g3_tune_cache_clear()


@pytest.mark.parametrize("dtype", [G3_BF16, G3_F32_3XBF16, G3_FP8_E4M3])
def test_autotune_grouped_records_the_bucket(dtype):
    _lib.g3_tune_cache_clear()
    st, bm, ms = _lib.g3_autotune_grouped(150, 400, 300, dtype)
    assert st == 0 and bm in (64, 128) and ms > 0, (st, bm, ms)
    A = torch.zeros(150, 300, dtype=torch_api._ELEM[dtype][0], device="cuda")
    B = torch.zeros(300, 400, dtype=torch_api._ELEM[dtype][0], device="cuda")
    C = torch.zeros(150, 400, device="cuda")
    prob = (A, B, C, 1.0, 0.0, 1.0, 1.0) if dtype == G3_FP8_E4M3 else (A, B, C, 1.0, 0.0)
    plan = torch_api.GroupedPlan([prob], dtype)
    assert _lib.g3_grouped_plan_describe(plan.plan, 0)[1:] == (bm, 1 if dtype == G3_F32_3XBF16 else 0)
    plan.close()
    _lib.g3_tune_cache_clear()


def _outputs(probs, host):
    """Reset every C to its initial value (or to zero where beta = 0)."""
    for (A, B, C, a, b), (p, full) in zip(probs, host):
        C.copy_(torch.from_numpy(p.C) if p.C is not None else torch.zeros(p.m, p.n))


def test_grouped_split_in_kernel_matches_the_pre_split_plan():
    # On request FP32-accurate plans split inside the grouped kernels: the
    # loader-converter warps read FP32 rows of any alignment (every second
    # problem has rows that are not 16-byte multiples) and write the bf16 parts
    # the split pre-pass would write, so each problem equals the default plan's
    # result bit for bit where that plan also takes 64-row tiles (m <= 64), and
    # every problem passes the oracle checks.  k spans both sides of 512
    # (three- and two-part splits) and ragged k-blocks; the split-in-kernel
    # plan runs no preparation kernel.
    probs, host = make_batch(48, seed=7, lo=1, hi=900, dtype=G3_F32_3XBF16, unaligned_every=2)
    assert any(p.k <= 512 for p, _ in host) and any(p.k > 512 for p, _ in host)
    fused = torch_api.GroupedPlan(probs, G3_F32_3XBF16, split_in_kernel=True)
    pre = torch_api.GroupedPlan(probs, G3_F32_3XBF16)
    kinds = set()
    for i, (p, _) in enumerate(host):
        st, bm, kind = _lib.g3_grouped_plan_describe(fused.plan, i)
        assert st == 0 and bm == 64, (i, bm)
        kinds.add(kind)
    l0 = _lib.g3_launch_count()
    fused.execute()
    assert _lib.g3_launch_count() - l0 == len(kinds)
    torch.cuda.synchronize()
    got_fused = [C.cpu().numpy().copy() for (_, _, C, _, _) in probs]
    check_batch(probs, host, G3_F32_3XBF16)
    _outputs(probs, host)
    l0 = _lib.g3_launch_count()
    pre.execute()
    # the pre-split plan: one job kernel per kind (two kinds run forked on two
    # streams), then the kinds' launches
    assert _lib.g3_launch_count() - l0 == 2 * len(kinds)
    torch.cuda.synchronize()
    check_batch(probs, host, G3_F32_3XBF16)
    same = 0
    for i, ((_, _, C, _, _), (p, _)) in enumerate(zip(probs, host)):
        if _lib.g3_grouped_plan_describe(pre.plan, i)[1] == 64:
            assert np.array_equal(C.cpu().numpy().view(np.uint32), got_fused[i].view(np.uint32)), (p.m, p.n, p.k)
            same += 1
    assert same >= 10, same
    fused.close()
    pre.close()


def test_grouped_split_in_kernel_watchdog_and_flags():
    # a stage the loader-converter warps never fill: the MMA issuer's wait
    # expires, the status reports it, and the next execution is correct;
    # unknown flag bits are rejected
    probs, host = make_batch(10, seed=8, lo=64, hi=700, dtype=G3_F32_3XBF16, unaligned_every=3)
    plan = torch_api.GroupedPlan(probs, G3_F32_3XBF16, split_in_kernel=True)
    assert _lib.g3_debug_withhold_next(200) == 0
    plan.execute()
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    _outputs(probs, host)
    plan.execute()
    torch.cuda.synchronize()
    check_batch(probs, host, G3_F32_3XBF16)
    assert torch_api.device_status()[0] == 0
    plan.close()
    d = _lib.g3_gemm_desc()
    d.m = d.n = d.k = 0
    d.lda = d.ldb = d.ldc = 1
    st, _ = _lib.g3_grouped_plan_create([d], G3_F32_3XBF16, 2)
    assert st == _lib.G3_ERR_ARG
