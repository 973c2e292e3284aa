"""Pins for the oracle's number formats and for the 3-product split.

bfloat16 and E4M3 rounding are checked against torch's CPU conversions (a
library routine implementing the same IEEE / OCP definitions) over every
representable pattern and every rounding tie; the split and the 3-product
oracle are checked against closed forms and the split's error bound."""
import numpy as np
import pytest
import torch

from paper_2310_20347_gb300 import synth


def _f32(bits):
    return np.asarray(bits, np.uint32).view(np.float32)


def test_bf16_all_patterns_fixed_points(oracle):
    pats = (np.arange(1 << 16, dtype=np.uint32) << 16)
    x = _f32(pats)
    y = oracle.round_bf16(x)
    finite = ~np.isnan(x)
    assert np.array_equal(y[finite].view(np.uint32), pats[finite])
    assert np.all(np.isnan(y[~finite]))


def test_bf16_against_torch_ties_and_random(oracle):
    r = np.random.default_rng(0)
    hi = r.integers(0, 1 << 16, 200000, dtype=np.uint32) << 16
    # exact ties, just below and just above ties, random low bits
    low = np.concatenate([np.full(50000, 0x8000), np.full(50000, 0x7FFF),
                          np.full(50000, 0x8001), r.integers(0, 1 << 16, 50000)]).astype(np.uint32)
    x = _f32(hi | low)
    x = x[~np.isnan(x)]
    want = torch.from_numpy(x.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    got = oracle.round_bf16(x)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    # overflow to infinity
    big = _f32([0x7F7FFFFF, 0xFF7FFFFF, 0x7F7F8000, 0x7F7F7FFF])
    assert np.array_equal(oracle.round_bf16(big),
                          np.array([np.inf, -np.inf, np.inf, _f32(0x7F7F0000)], np.float32))


def test_e4m3_decode_all_codes(oracle):
    codes = np.arange(256, dtype=np.uint8)
    got = oracle.e4m3_decode(codes)
    want = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float32).numpy()
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], want[~nan])
    # closed forms from the format definition
    assert got[0x7E] == 448.0 and got[0x01] == 2.0 ** -9 and got[0x08] == 2.0 ** -6
    assert got[0x38] == 1.0


def test_e4m3_encode_against_torch(oracle):
    vals = oracle.e4m3_decode(np.arange(0x7F, dtype=np.uint8)).astype(np.float64)
    mids = (vals[:-1] + vals[1:]) / 2            # exact ties
    r = np.random.default_rng(1)
    rand = r.uniform(-460, 460, 20000)
    small = r.uniform(-0.02, 0.02, 5000)
    x = np.concatenate([vals, -vals, mids, -mids, np.nextafter(mids, 0),
                        np.nextafter(mids, 1e9), rand, small]).astype(np.float32)
    x = x[np.abs(x) < 464]                       # torch does not saturate beyond
    got = oracle.e4m3_encode(x)
    want = torch.from_numpy(x.copy()).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(got, want)


def test_e4m3_satfinite(oracle):
    x = np.array([448, 449, 464, 480, 1e6, np.inf, -500, -np.inf], np.float32)
    got = oracle.e4m3_encode(x)
    assert list(got) == [0x7E] * 6 + [0xFE] * 2
    assert oracle.e4m3_encode(np.array([np.nan], np.float32))[0] == 0x7F


def test_fp8_quantize_scale(oracle):
    p = synth.normal_problem(31, 17, 8, seed=2)
    q, s = oracle.fp8_quantize(p.A)
    amax = np.float32(np.max(np.abs(p.A)))
    assert s == np.float32(amax / np.float32(448.0))
    # the element of largest magnitude maps to +-448
    i = np.unravel_index(np.argmax(np.abs(p.A)), p.A.shape)
    assert q[i] in (0x7E, 0xFE)
    # dequantised values are within half an E4M3 step (relative 2^-4) of x/s
    deq = oracle.e4m3_decode(q).astype(np.float64)
    t = (p.A / np.float32(s)).astype(np.float64)
    normal = np.abs(t) >= 2.0 ** -6
    assert np.all(np.abs(deq - t)[normal] <= np.abs(t)[normal] * 2.0 ** -4)
    q0, s0 = oracle.fp8_quantize(np.zeros((3, 3), np.float32))
    assert s0 == 1.0 and np.all(q0 == 0)


def test_split_error_bound(oracle):
    r = np.random.default_rng(3)
    x = np.concatenate([r.uniform(-1, 1, 100000), r.standard_normal(100000) * 1e6,
                        r.standard_normal(1000) * 1e-30]).astype(np.float32)
    hi, lo = oracle.split_bf16(x)
    assert np.all((hi.view(np.uint32) & 0xFFFF) == 0)
    assert np.all((lo.view(np.uint32) & 0xFFFF) == 0)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= np.abs(x.astype(np.float64)) * 2.0 ** -16)
    # bfloat16-exact values split with a zero low part
    ints = np.arange(-256, 257).astype(np.float32)
    h, l = oracle.split_bf16(ints)
    assert np.array_equal(h, ints) and np.all(l == 0)


def test_3xbf16_closed_form(oracle):
    # a = 1 + 2^-9 splits as (1, 2^-9); b = 1 + 2^-10 as (1, 2^-10).
    # ab = 1 + 2^-9 + 2^-10 + 2^-19; the 3-product method drops lo*lo = 2^-19.
    a = np.array([[1 + 2.0 ** -9]], np.float32)
    b = np.array([[1 + 2.0 ** -10]], np.float32)
    got = oracle.gemm_3xbf16(a, b)[0, 0]
    assert got == 1 + 2.0 ** -9 + 2.0 ** -10
    assert oracle.gemm(a, b)[0, 0] - got == 2.0 ** -19


def test_3xbf16_exact_on_bf16_inputs(oracle):
    p = synth.small_int_problem(21, 34, 57, seed=4, alpha=0.5, beta=2.0)
    assert np.array_equal(oracle.gemm_3xbf16(p.A, p.B, p.C, 0.5, 2.0),
                          oracle.gemm(p.A, p.B, p.C, 0.5, 2.0))


def test_split3_is_exact_and_bf16(oracle):
    r = np.random.default_rng(5)
    x = np.concatenate([r.uniform(-1, 1, 20000), r.standard_normal(20000) * 1e5]).astype(np.float32)
    h, m, l = oracle.split3_bf16(x)
    for plane in (h, m, l):
        assert np.all((plane.view(np.uint32) & 0xFFFF) == 0)
    # hi + mid + lo reproduces every normal binary32 value exactly
    assert np.array_equal(h.astype(np.float64) + m.astype(np.float64) + l.astype(np.float64),
                          x.astype(np.float64))
    assert np.all(np.abs(m) <= np.abs(x) * 2.0 ** -8) and np.all(np.abs(l) <= np.abs(x) * 2.0 ** -16)


def test_6xbf16_closed_form(oracle):
    # a = 1 + 2^-9 + 2^-17 splits as (1, 2^-9, 2^-17); b = 1 + 2^-10 + 2^-18 as
    # (1, 2^-10, 2^-18).  ab adds mid*lo + lo*mid = 2^-26 and lo*lo = 2^-35 to
    # the six kept products 1 + 2^-9 + 2^-10 + 2^-17 + 2^-18 + 2^-19.
    a = np.array([[1 + 2.0 ** -9 + 2.0 ** -17]], np.float32)
    b = np.array([[1 + 2.0 ** -10 + 2.0 ** -18]], np.float32)
    got = oracle.gemm_6xbf16(a, b)[0, 0]
    assert got == 1 + 2.0 ** -9 + 2.0 ** -10 + 2.0 ** -17 + 2.0 ** -18 + 2.0 ** -19
    assert oracle.gemm(a, b)[0, 0] - got == 2.0 ** -26 + 2.0 ** -35


def test_6xbf16_within_bound_at_every_k(oracle):
    # dropped products: |mid*lo| + |lo*mid| + |lo*lo| <= (2^-23 + 2^-32)|a||b|
    bound = 2.0 ** -23 + 2.0 ** -32
    for k in (1, 3, 16, 200):
        p = synth.uniform_problem(30, 40, k, seed=k)
        exact = oracle.gemm(p.A, p.B)
        approx = oracle.gemm_6xbf16(p.A, p.B)
        D = oracle.absprod(p.A, p.B)
        assert np.max(np.abs(approx - exact) / D) <= bound


def test_3xbf16_within_split_bound(oracle):
    # |ab - (ah bh + ah bl + al bh)| <= (2^-16 + 2^-16 + 2^-16 + 2^-32)|a||b|.
    bound = 3 * 2.0 ** -16 + 2.0 ** -32
    for seed, (m, n, k) in enumerate([(40, 50, 16), (20, 30, 600)]):
        p = synth.uniform_problem(m, n, k, seed=seed)
        exact = oracle.gemm(p.A, p.B)
        approx = oracle.gemm_3xbf16(p.A, p.B)
        D = oracle.absprod(p.A, p.B)
        rel = np.max(np.abs(approx - exact) / D)
        assert rel <= bound
        assert rel < 2e-5            # far below bfloat16's own 2^-8
        assert rel > 0               # it is an approximation: lo*lo is dropped


# ---------------------------------------------------------------- TF32
def test_tf32_fixed_points_every_pattern(oracle):
    # every sign / exponent / 10-bit fraction combination is a TF32 value
    sign_exp = np.arange(1 << 9, dtype=np.uint32) << 23
    frac = np.arange(1 << 10, dtype=np.uint32) << 13
    pats = (sign_exp[:, None] | frac[None, :]).ravel()
    x = _f32(pats)
    keep = ~np.isnan(x)
    assert np.array_equal(oracle.round_tf32(x[keep]).view(np.uint32), pats[keep])


def test_tf32_nearest_with_ties_to_even(oracle):
    # against the grid itself: the result lies on the TF32 grid (low 13 bits
    # zero), no grid neighbour (one step in the encoding) is nearer, and a tie
    # picks the neighbour with an even last fraction bit
    r = np.random.default_rng(1)
    hi = r.integers(0, 0xFF, 120000, dtype=np.uint32) << 23 | (r.integers(0, 1 << 10, 120000, dtype=np.uint32) << 13)
    hi |= r.integers(0, 2, 120000, dtype=np.uint32) << 31
    low = np.concatenate([np.full(30000, 0x1000), np.full(30000, 0x0FFF), np.full(30000, 0x1001),
                          r.integers(0, 1 << 13, 30000)]).astype(np.uint32)
    x = _f32(hi | low)
    y = oracle.round_tf32(x)
    yb = y.view(np.uint32)
    fin = np.isfinite(y)
    assert np.all(yb[fin] & 0x1FFF == 0)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    for step in (0x2000, -0x2000):
        nb = (yb.astype(np.int64) + step)
        ok = fin & (nb >= 0) & ((nb & 0x7F800000) != 0x7F800000) & ((nb & 0x7FFFFFFF) <= 0x7F7FE000)
        ok &= ((nb ^ yb.astype(np.int64)) & 0x80000000) == 0   # same sign
        nd = nb[ok].astype(np.uint32).view(np.float32).astype(np.float64)
        d_here, d_nb = np.abs(xd[ok] - yd[ok]), np.abs(xd[ok] - nd)
        assert np.all(d_here <= d_nb)
        tie = d_here == d_nb
        assert np.all((yb[ok][tie] >> 13) & 1 == 0)


def test_tf32_closed_forms_and_overflow(oracle):
    one = 1.0
    cases = [(one + 2.0 ** -10, one + 2.0 ** -10), (one + 2.0 ** -11, one),
             (one + 3 * 2.0 ** -11, one + 2.0 ** -9), (one + 2.0 ** -11 + 2.0 ** -20, one + 2.0 ** -10),
             (-(one + 2.0 ** -11 + 2.0 ** -20), -(one + 2.0 ** -10)), (2049.0, 2048.0), (2051.0, 2052.0)]
    for x, want in cases:
        assert oracle.round_tf32(np.array([x], np.float32))[0] == np.float32(want), x
    big = _f32([0x7F7FE000, 0x7F7FEFFF, 0x7F7FF000, 0xFF7FF000, 0x7F7FFFFF])
    got = oracle.round_tf32(big).view(np.uint32)
    assert list(got) == [0x7F7FE000, 0x7F7FE000, 0x7F800000, 0xFF800000, 0x7F800000]
    sub = _f32([0x00000FFF, 0x00001000, 0x00003000, 0x00001001])   # subnormals: spacing 2^-136
    assert list(oracle.round_tf32(sub).view(np.uint32)) == [0x0, 0x0, 0x4000, 0x2000]


# ---------------------------------------------------------------- 3xTF32
def test_split_tf32_error_bound_and_grid(oracle):
    # hi = tf32(x) keeps 11 significant bits, so x - hi is exact and lo = tf32(x - hi)
    # leaves |x - hi - lo| <= 2^-11 |x - hi| <= 2^-22 |x|
    r = np.random.default_rng(70)
    x = np.concatenate([r.uniform(-1, 1, 50000), r.standard_normal(50000) * 1e6,
                        r.standard_normal(1000) * 1e-30]).astype(np.float32)
    hi, lo = oracle.split_tf32(x)
    assert np.all((hi.view(np.uint32) & 0x1FFF) == 0) and np.all((lo.view(np.uint32) & 0x1FFF) == 0)
    assert np.array_equal(hi, oracle.round_tf32(x))
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= np.abs(x.astype(np.float64)) * 2.0 ** -22)
    # values with at most 22 significant bits split exactly
    y = (r.integers(-(1 << 21), 1 << 21, 10000) * 2.0 ** -30).astype(np.float32)
    h, l = oracle.split_tf32(y)
    assert np.array_equal(h.astype(np.float64) + l.astype(np.float64), y.astype(np.float64))


def test_3xtf32_closed_form(oracle):
    # a = 1 + 2^-12 splits as (1, 2^-12) (TF32's spacing at 1 is 2^-10);
    # b = 1 + 2^-13 as (1, 2^-13).  ab = 1 + 2^-12 + 2^-13 + 2^-25; the
    # 3-product method drops lo*lo = 2^-25.
    a = np.array([[1 + 2.0 ** -12]], np.float32)
    b = np.array([[1 + 2.0 ** -13]], np.float32)
    got = oracle.gemm_3xtf32(a, b)[0, 0]
    assert got == 1 + 2.0 ** -12 + 2.0 ** -13
    assert oracle.gemm(a, b)[0, 0] - got == 2.0 ** -25


def test_3xtf32_exact_on_tf32_inputs(oracle):
    p = synth.small_int_problem(23, 31, 45, seed=71, alpha=0.5, beta=2.0)
    assert np.array_equal(oracle.gemm_3xtf32(p.A, p.B, p.C, 0.5, 2.0), oracle.gemm(p.A, p.B, p.C, 0.5, 2.0))


def test_3xtf32_within_split_bound(oracle):
    # a = ah + al + ea with |al| <= 2^-11 |a|, |ea| <= 2^-22 |a| (likewise b):
    # |ab - (ah bh + ah bl + al bh)| <= (3 * 2^-22 + 2^-33)|a||b| to first order
    bound = 3 * 2.0 ** -22 + 2.0 ** -32
    for seed, (m, n, k) in enumerate([(40, 50, 16), (20, 30, 600)]):
        p = synth.uniform_problem(m, n, k, seed=72 + seed)
        exact = oracle.gemm(p.A, p.B)
        approx = oracle.gemm_3xtf32(p.A, p.B)
        rel = np.max(np.abs(approx - exact) / oracle.absprod(p.A, p.B))
        assert 0 < rel <= bound
        # against the two-part bfloat16 split: the 22-bit split is far closer
        assert rel < np.max(np.abs(oracle.gemm_3xbf16(p.A, p.B) - exact) / oracle.absprod(p.A, p.B)) / 8
