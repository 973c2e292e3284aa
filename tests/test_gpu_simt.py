"""Parity of the FP32 SIMT kernel (the plain method) with the binary64 oracle:
max |C - C_ref| / (|alpha| |A| |B|) <= 2e-6, bit-exact on integer inputs."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, dev, gate, guarded, rel_err
from paper_2310_20347_gb300 import G3_F32, synth, torch_api

pytestmark = pytest.mark.gpu
TOL = 2e-6


def run(p, ldpad=(0, 0, 0)):
    A = dev(p.A)
    B = dev(p.B)
    if ldpad[0]:
        A = torch.zeros(p.m, p.k + ldpad[0], device="cuda")[:, :p.k].copy_(A) if p.k else A
    if ldpad[1]:
        B = torch.zeros(p.k, p.n + ldpad[1], device="cuda")[:, :p.n].copy_(B) if p.n else B
    full, C = guarded(p.m, p.n, p.C, pad_cols=max(5, ldpad[2]))
    torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=G3_F32)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n, pad_cols=max(5, ldpad[2]))
    return C.cpu().numpy()


def check(p, tol=TOL, **kw):
    got = run(p, **kw)
    ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    D = oracle.absprod(p.A, p.B, p.alpha)
    return gate(got, ref, D, None if p.C is None else p.beta * p.C.astype(np.float64), p.k, tol)[1]


def test_config_512_cube():
    # plain FP32 GEMM C := A*B, m = n = k = 512, uniform [-1, 1] from seed 0, beta = 0
    p = synth.uniform_problem(512, 512, 512, seed=0)
    e = check(p)
    print(f"simt 512^3 rel-err {e:.3e}")


EDGE = (1, 2, 3, 15, 16, 17, 63, 64, 65, 127, 128, 129, 255, 257)


@pytest.mark.parametrize("seed", range(6))
def test_edge_shapes(seed):
    r = np.random.default_rng(100 + seed)
    for _ in range(8):
        m, n, k = (int(x) for x in r.choice(EDGE, 3))
        p = synth.uniform_problem(m, n, k, seed=seed, alpha=-0.5, beta=0.5)
        check(p)


def test_integer_inputs_bit_exact():
    p = synth.small_int_problem(200, 300, 1000, seed=3, alpha=1.0, beta=2.0)
    got = run(p)
    ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    assert np.array_equal(got.astype(np.float64), ref)


def test_unaligned_leading_dimensions():
    p = synth.uniform_problem(131, 67, 301, seed=4, alpha=1.5, beta=-1.0)
    check(p, ldpad=(1, 3, 6))


def test_beta_zero_overwrites_nan():
    p = synth.uniform_problem(70, 90, 40, seed=5)
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(p.m, p.n, np.full((p.m, p.n), np.nan, np.float32))
    torch_api.gemm(A, B, C, 1.0, 0.0, dtype=G3_F32)
    assert torch.isfinite(C).all()
    check_guard(full, p.m, p.n)


def test_alpha_zero_and_k_zero():
    p = synth.uniform_problem(33, 44, 10, seed=6, beta=0.25)
    full, C = guarded(p.m, p.n, p.C)
    A = torch.full((p.m, p.k), float("nan"), device="cuda")
    B = torch.full((p.k, p.n), float("nan"), device="cuda")
    torch_api.gemm(A, B, C, 0.0, 0.25, dtype=G3_F32)
    assert np.array_equal(C.cpu().numpy(), (np.float32(0.25) * p.C))
    full2, C2 = guarded(p.m, p.n, p.C)
    torch_api.gemm(torch.empty(p.m, 0, device="cuda"), torch.empty(0, p.n, device="cuda"), C2, 1.0, 0.25,
                   dtype=G3_F32)
    assert np.array_equal(C2.cpu().numpy(), (np.float32(0.25) * p.C))


def test_deterministic():
    p = synth.uniform_problem(300, 300, 777, seed=7, beta=0.5)
    a = run(p)
    b = run(p)
    assert np.array_equal(a, b)


def test_large_grid_ragged():
    # enough 128 x 128 blocks to fill every SM (the 128 x 128 kernel), ragged
    # in m, n and k
    p = synth.uniform_problem(1667, 1500, 301, seed=8, alpha=0.75, beta=-0.5)
    check(p)


def test_tile_size_switch_bit_identical():
    # Both block sizes accumulate each element's products in k order with one
    # FMA each, so a problem just above the SM-count threshold (128 x 128
    # blocks) and its column slice just below it (64 x 64 blocks) agree
    # bit for bit on the shared columns.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rows_blocks = 8
    cols_blocks = -(-sms // rows_blocks)          # rows_blocks * cols_blocks >= sms
    m, k = rows_blocks * 128, 200
    n_big = cols_blocks * 128
    n_small = (cols_blocks - 1) * 128 - 3         # fewer blocks than SMs, ragged
    assert rows_blocks * (-(-n_small // 128)) < sms <= rows_blocks * cols_blocks
    p = synth.uniform_problem(m, n_big, k, seed=9)
    A, B = dev(p.A), dev(p.B)
    C_big = torch.empty(m, n_big, device="cuda")
    torch_api.gemm(A, B, C_big, 1.0, 0.0, dtype=G3_F32)
    Bs = B[:, :n_small].contiguous()
    C_small = torch.empty(m, n_small, device="cuda")
    torch_api.gemm(A, Bs, C_small, 1.0, 0.0, dtype=G3_F32)
    torch.cuda.synchronize()
    assert torch.equal(C_big[:, :n_small], C_small)
    ref = oracle.gemm(p.A, p.B[:, :n_small], None, 1.0, 0.0)
    D = oracle.absprod(p.A, p.B[:, :n_small], 1.0)
    assert rel_err(C_small.cpu().numpy(), ref, D, None) <= TOL


@pytest.mark.parametrize("splits", [2, 3, 4, 5, 8])
def test_cluster_split_k(splits):
    # k cut over a cluster of `splits` CTAs per 64 x 64 block (forced), ragged
    # m, n and k, beta != 0 with C, unaligned leading dimension of A
    for (m, n, k) in ((70, 130, 301), (64, 64, 16 * splits), (200, 33, 1000)):
        p = synth.uniform_problem(m, n, k, seed=splits * 7 + k, alpha=-0.75, beta=0.5)
        A, B = dev(p.A), dev(p.B)
        full, C = guarded(p.m, p.n, p.C)
        torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=G3_F32, split_k=splits)
        torch.cuda.synchronize()
        check_guard(full, p.m, p.n)
        ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
        D = oracle.absprod(p.A, p.B, p.alpha)
        assert rel_err(C.cpu().numpy(), ref, D, p.beta * p.C.astype(np.float64)) <= TOL
    p = synth.uniform_problem(131, 67, 301, seed=4, alpha=1.5, beta=-1.0)
    A = torch.zeros(p.m, p.k + 1, device="cuda")[:, :p.k].copy_(dev(p.A))
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(A, dev(p.B), C, p.alpha, p.beta, dtype=G3_F32, split_k=splits)
    torch.cuda.synchronize()
    ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    assert rel_err(C.cpu().numpy(), ref, oracle.absprod(p.A, p.B, p.alpha),
                   p.beta * p.C.astype(np.float64)) <= TOL


def test_cluster_split_more_ctas_than_k_blocks():
    # k = 20 over 8 CTAs: two CTAs hold k-blocks, six hold empty ranges and
    # contribute zero partials
    p = synth.uniform_problem(90, 70, 20, seed=11, beta=0.25)
    A, B = dev(p.A), dev(p.B)
    full, C = guarded(p.m, p.n, p.C)
    torch_api.gemm(A, B, C, 1.0, 0.25, dtype=G3_F32, split_k=8)
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    ref = oracle.gemm(p.A, p.B, p.C, 1.0, 0.25)
    assert rel_err(C.cpu().numpy(), ref, oracle.absprod(p.A, p.B, 1.0), 0.25 * p.C.astype(np.float64)) <= TOL


def test_cluster_split_deterministic_and_planned():
    # the 512^3 problem takes the planner's cluster split; repeated calls are
    # bit-identical (partials summed in a fixed order)
    from paper_2310_20347_gb300 import _lib
    st, cfg, sk, rs = _lib.g3_plan_query(512, 512, 512, G3_F32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert sk > 1 and 64 * sk <= 2 * sms
    p = synth.uniform_problem(512, 512, 512, seed=0)
    a = run(p)
    b = run(p)
    assert np.array_equal(a, b)
    C = torch.empty(512, 512, device="cuda")
    torch_api.gemm(dev(p.A), dev(p.B), C, 1.0, 0.0, dtype=G3_F32, split_k=sk)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), a)


@pytest.mark.parametrize("blocking", [2, 3])
def test_wide_blocks_parity_and_bit_identity(blocking):
    # the 128 x 256 blocks (8 x 16 micro-tiles; k-blocks of 8 or 16): ragged
    # m, n, k, beta != 0, unaligned leading dimensions, k = 1; within 2e-6 of
    # the oracle and bit-identical to the 128 x 128 blocks (every element's
    # products added in k order, one FMA each)
    for (m, n, k, pad) in ((300, 520, 700, 0), (129, 257, 65, 0), (1, 1, 1, 0), (200, 300, 1, 0),
                           (131, 517, 301, 1), (640, 1280, 1024, 0)):
        p = synth.uniform_problem(m, n, k, seed=blocking * 100 + m, alpha=-0.75, beta=0.5)
        A, B = dev(p.A), dev(p.B)
        if pad:
            A = torch.zeros(m, k + pad, device="cuda")[:, :k].copy_(A)
        outs = []
        for cfg in (0, blocking):
            full, C = guarded(m, n, p.C)
            torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=G3_F32, config=cfg)
            torch.cuda.synchronize()
            check_guard(full, m, n)
            outs.append(C.cpu().numpy())
        assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32)), (m, n, k)
        ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
        gate(outs[1], ref, oracle.absprod(p.A, p.B, p.alpha), p.beta * p.C.astype(np.float64), k, TOL)
