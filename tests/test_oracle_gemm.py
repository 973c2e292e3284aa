"""Pins for the binary64 / int64 GEMM oracle against facts fixed by mathematics,
not by the oracle itself: closed forms (identity, permutation, rank-1),
brute force on tiny sizes, a library routine (numpy's float64 / int64 matmul),
and the edge rules of the routine C := beta*C + alpha*A*B (Section 3.1)."""
import itertools

import numpy as np
import pytest

from paper_2310_20347_gb300 import synth


def rng(seed=0):
    return np.random.default_rng(seed)


def test_identity_closed_form(oracle):
    # A = I gives C = alpha*B + beta*C exactly: the sum adds zeros to one term.
    r = rng(1)
    k, n = 37, 29
    B = r.uniform(-1, 1, (k, n)).astype(np.float32)
    C = r.uniform(-1, 1, (k, n)).astype(np.float32)
    A = np.eye(k, dtype=np.float32)
    got = oracle.gemm(A, B, C, alpha=1.5, beta=-0.5)
    want = np.float64(-0.5) * C.astype(np.float64) + np.float64(1.5) * B.astype(np.float64)
    assert np.array_equal(got, want)


def test_permutation_closed_form(oracle):
    # A = P (a row permutation) gives C = alpha * B[perm] exactly.
    r = rng(2)
    k, n = 23, 17
    perm = r.permutation(k)
    A = np.zeros((k, k), np.float32)
    A[np.arange(k), perm] = 1.0
    B = r.uniform(-1, 1, (k, n)).astype(np.float32)
    got = oracle.gemm(A, B, alpha=2.0)
    assert np.array_equal(got, 2.0 * B[perm].astype(np.float64))
    # and a column permutation on the right: C = A P -> columns of A permuted
    Am = r.uniform(-1, 1, (5, k)).astype(np.float32)
    P = np.zeros((k, k), np.float32)
    P[perm, np.arange(k)] = 1.0
    got = oracle.gemm(Am, P)
    assert np.array_equal(got, Am[:, perm].astype(np.float64))


def test_rank1_closed_form(oracle):
    # A = u 1^T, B = 1 v^T  ->  C_ij = k u_i v_j (integers: exact).
    r = rng(3)
    m, n, k = 19, 13, 41
    u = r.integers(-9, 10, m).astype(np.float64)
    v = r.integers(-9, 10, n).astype(np.float64)
    A = np.repeat(u[:, None], k, axis=1)
    B = np.repeat(v[None, :], k, axis=0)
    C = r.integers(-5, 6, (m, n)).astype(np.float64)
    got = oracle.gemm(A, B, C, alpha=3.0, beta=2.0)
    assert np.array_equal(got, 3.0 * k * np.outer(u, v) + 2.0 * C)


def test_brute_force_tiny(oracle):
    # Every (m, n, k) in {1..4}^3: the hand-expanded sum of products in
    # increasing p (plain Python binary64, same order) must agree bit for bit.
    r = rng(4)
    for m, n, k in itertools.product(range(1, 5), repeat=3):
        A = r.uniform(-1, 1, (m, k))
        B = r.uniform(-1, 1, (k, n))
        C = r.uniform(-1, 1, (m, n))
        alpha, beta = 0.75, -1.25
        got = oracle.gemm(A, B, C, alpha=alpha, beta=beta)
        for i in range(m):
            for j in range(n):
                s = 0.0
                for p in range(k):
                    s = s + float(A[i, p]) * float(B[p, j])
                want = beta * float(C[i, j]) + alpha * s
                assert got[i, j] == want, (m, n, k, i, j)


def test_against_numpy_float64(oracle):
    # A library routine of the same definition: agreement to binary64 rounding.
    for seed, (m, n, k) in enumerate([(64, 48, 300), (7, 129, 65), (130, 3, 1000)]):
        p = synth.uniform_problem(m, n, k, seed=seed, alpha=-0.5, beta=0.5)
        got = oracle.gemm(p.A, p.B, p.C, alpha=p.alpha, beta=p.beta)
        A64, B64, C64 = (x.astype(np.float64) for x in (p.A, p.B, p.C))
        want = p.beta * C64 + p.alpha * (A64 @ B64)
        D = np.abs(p.alpha) * (np.abs(A64) @ np.abs(B64)) + np.abs(p.beta * C64)
        assert np.max(np.abs(got - want) / D) < 1e-12


def test_edge_rules(oracle):
    r = rng(5)
    m, n, k = 6, 5, 4
    A = r.uniform(-1, 1, (m, k))
    B = r.uniform(-1, 1, (k, n))
    C = r.uniform(-1, 1, (m, n))
    nanA = np.full((m, k), np.nan)
    nanB = np.full((k, n), np.nan)
    nanC = np.full((m, n), np.nan)
    # alpha == 0: A and B are not read
    assert np.array_equal(oracle.gemm(nanA, nanB, C, alpha=0.0, beta=0.5), 0.5 * C)
    # beta == 0: C is not read (NaN overwritten)
    got = oracle.gemm(A, B, nanC, alpha=1.0, beta=0.0)
    assert np.all(np.isfinite(got))
    # k == 0: C = beta*C
    got = oracle.gemm(np.zeros((m, 0)), np.zeros((0, n)), C, alpha=2.0, beta=3.0)
    assert np.array_equal(got, 3.0 * C)
    # m == 0 / n == 0: empty results
    assert oracle.gemm(np.zeros((0, k)), B).shape == (0, n)
    assert oracle.gemm(A, np.zeros((k, 0))).shape == (m, 0)


def test_entry_rows_and_threads_agree_exactly(oracle):
    p = synth.uniform_problem(33, 45, 200, seed=6, alpha=1.25, beta=-0.75)
    full = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta, nthreads=1)
    full4 = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta, nthreads=4)
    assert np.array_equal(full, full4)
    rows = np.array([32, 0, 7, 7, 19])
    sub = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta, rows=rows)
    assert np.array_equal(sub, full[rows])
    for i, j in [(0, 0), (32, 44), (7, 13), (19, 1)]:
        assert oracle.entry(p.A, p.B, i, j, p.C, p.alpha, p.beta) == full[i, j]


def test_absprod(oracle):
    p = synth.uniform_problem(20, 30, 50, seed=7)
    D = oracle.absprod(p.A, p.B, alpha=-2.0)
    want = 2.0 * (np.abs(p.A.astype(np.float64)) @ np.abs(p.B.astype(np.float64)))
    assert np.max(np.abs(D - want) / want) < 1e-13
    # |alpha A B| <= D elementwise (triangle inequality)
    C = oracle.gemm(p.A, p.B, alpha=-2.0)
    assert np.all(np.abs(C) <= D * (1 + 1e-15))


def test_int8_oracle(oracle):
    p = synth.int8_problem(40, 24, 300, seed=8, beta=1)
    got = oracle.gemm_i8(p.A, p.B, p.C, alpha=1, beta=1)
    want = p.C.astype(np.int64) + p.A.astype(np.int64) @ p.B.astype(np.int64)
    assert np.array_equal(got, want)
    # worst-case magnitude: all -128 at k = 8192 gives 8192 * 2^14 = 2^27 exactly
    A = np.full((2, 8192), -128, np.int8)
    B = np.full((8192, 3), -128, np.int8)
    assert np.all(oracle.gemm_i8(A, B) == 1 << 27)
    A2 = np.full((2, 8192), 127, np.int8)
    assert np.all(oracle.gemm_i8(A2, B) == -127 * 128 * 8192)


def test_int16_oracle(oracle):
    r = np.random.default_rng(81)
    A = r.integers(-(1 << 15), 1 << 15, (23, 410)).astype(np.int16)
    B = r.integers(-(1 << 15), 1 << 15, (410, 17)).astype(np.int16)
    C = r.integers(-(1 << 40), 1 << 40, (23, 17)).astype(np.int64)
    got = oracle.gemm_i16(A, B, C, alpha=1, beta=1)
    assert np.array_equal(got, C + A.astype(np.int64) @ B.astype(np.int64))
    # worst case: all -32768 at k = 8192 gives 8192 * 2^30 = 2^43 exactly (beyond int32)
    A = np.full((2, 8192), -32768, np.int16)
    B = np.full((8192, 3), -32768, np.int16)
    assert np.all(oracle.gemm_i16(A, B) == 1 << 43)
    A2 = np.full((2, 8192), 32767, np.int16)
    assert np.all(oracle.gemm_i16(A2, B) == -32767 * 32768 * 8192)
    # int8-range inputs: the same as the int8 definition
    p = synth.int8_problem(11, 13, 70, seed=82)
    assert np.array_equal(oracle.gemm_i16(p.A.astype(np.int16), p.B.astype(np.int16)), oracle.gemm_i8(p.A, p.B))


def test_int8_matches_f64_on_integer_inputs(oracle):
    # Two independent code paths of the oracle agree where both are exact.
    p = synth.int8_problem(17, 9, 64, seed=9)
    assert np.array_equal(oracle.gemm_i8(p.A, p.B).astype(np.float64),
                          oracle.gemm(p.A.astype(np.float64), p.B.astype(np.float64)))


def test_planted_transpose_is_caught(oracle):
    # A plausible mistake -- using B^T where B is meant -- changes the result on
    # a non-square, non-symmetric case; the permutation pin above would fail.
    r = rng(10)
    k = 6
    perm = r.permutation(k)
    A = np.zeros((k, k))
    A[np.arange(k), perm] = 1.0
    B = r.uniform(-1, 1, (k, k))
    wrong = oracle.gemm(A, B.T.copy())
    assert not np.array_equal(wrong, B[perm])


def test_table1_golden_matches_synth():
    rows = []
    with open(__file__.replace("test_oracle_gemm.py", "golden/resnet50_table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    assert tuple(rows) == synth.RESNET50_TABLE1
    shapes = synth.im2col_shapes(16)
    ms = sorted({s[1] for s in shapes})
    ns = sorted({s[2] for s in shapes})
    ks = sorted({s[3] for s in shapes})
    assert ms[0] == 64 and ms[-1] == 2048
    assert ns[0] == 784 and ns[-1] == 200704
    assert ks[0] == 64 and ks[-1] == 4608
