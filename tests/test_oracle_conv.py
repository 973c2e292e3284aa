"""Pins for the oracle's direct convolution (the layers of the paper's
Section 8.1, Table 1), each against something other than its own loops:
  * a 1 x 1, stride-1 convolution is the plain GEMM (the GEMM oracle)
  * an explicit im2col matrix built here, times the filter matrix, with
    numpy's matmul, for strided / padded / dilated 3 x 3 and 7 x 7 cases
  * all-ones input and filter: every output counts the in-image taps, a
    closed form that exposes any padding or stride slip
  * a filter that picks one tap and one channel reproduces the shifted input
  * the output sizes of the ResNet-50 layer geometries against Table 1"""
import numpy as np
import pytest

from paper_2310_20347_gb300 import synth


def im2col_reference(x, R, S, stride, pad, dil):
    N, H, W, C = x.shape
    P = (H + 2 * pad[0] - dil[0] * (R - 1) - 1) // stride[0] + 1
    Q = (W + 2 * pad[1] - dil[1] * (S - 1) - 1) // stride[1] + 1
    xp = np.zeros((N, H + 2 * pad[0], W + 2 * pad[1], C))
    xp[:, pad[0]:pad[0] + H, pad[1]:pad[1] + W, :] = x
    cols = np.empty((N, P, Q, R, S, C))
    for r in range(R):
        for s in range(S):
            hs, ws = r * dil[0], s * dil[1]
            cols[:, :, :, r, s, :] = xp[:, hs:hs + stride[0] * P:stride[0], ws:ws + stride[1] * Q:stride[1], :]
    return cols.reshape(N * P * Q, R * S * C), (N, P, Q)


def test_1x1_is_the_gemm(oracle):
    r = np.random.default_rng(0)
    x = r.standard_normal((2, 5, 7, 16))
    w = r.standard_normal((1, 1, 16, 9))
    y = oracle.conv2d_nhwc(x, w)
    ref = oracle.gemm(x.reshape(-1, 16), w.reshape(16, 9))
    assert np.allclose(y.reshape(-1, 9), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("R,S,stride,pad,dil", [(3, 3, (1, 1), (1, 1), (1, 1)), (3, 3, (2, 2), (1, 1), (1, 1)),
                                                (7, 7, (2, 2), (3, 3), (1, 1)), (3, 2, (2, 1), (0, 2), (2, 1)),
                                                (1, 1, (2, 2), (0, 0), (1, 1))])
def test_against_explicit_im2col(oracle, R, S, stride, pad, dil):
    r = np.random.default_rng(1)
    x = r.standard_normal((2, 11, 9, 6))
    w = r.standard_normal((R, S, 6, 5))
    cols, (N, P, Q) = im2col_reference(x, R, S, stride, pad, dil)
    want = (cols @ w.reshape(R * S * 6, 5)).reshape(N, P, Q, 5)
    y0 = r.standard_normal((N, P, Q, 5))
    got = oracle.conv2d_nhwc(x, w, stride, pad, dil, y=y0, alpha=0.5, beta=-2.0)
    assert np.allclose(got, 0.5 * want - 2.0 * y0, rtol=1e-12, atol=1e-12)


def test_all_ones_counts_taps(oracle):
    N, H, W, C, K, R, S = 1, 6, 5, 3, 2, 3, 3
    got = oracle.conv2d_nhwc(np.ones((N, H, W, C)), np.ones((R, S, C, K)), (2, 1), (1, 1))
    P, Q = (H + 2 - 3) // 2 + 1, W
    for p in range(P):
        for q in range(Q):
            rows = sum(1 for rr in range(R) if 0 <= 2 * p - 1 + rr < H)
            colc = sum(1 for ss in range(S) if 0 <= q - 1 + ss < W)
            assert np.all(got[0, p, q] == rows * colc * C)


def test_single_tap_filter_shifts_the_input(oracle):
    r = np.random.default_rng(2)
    x = r.standard_normal((1, 8, 8, 4))
    w = np.zeros((3, 3, 4, 4))
    for c in range(4):
        w[2, 0, c, c] = 1.0   # tap (r, s) = (2, 0): y[p][q] = x[p + 1][q - 1] with pad 1
    y = oracle.conv2d_nhwc(x, w, (1, 1), (1, 1))
    for p in range(8):
        for q in range(8):
            h, v = p + 1, q - 1
            want = x[0, h, v] if (0 <= h < 8 and 0 <= v < 8) else np.zeros(4)
            assert np.array_equal(y[0, p, q], want)


def test_resnet50_geometry_matches_table1(oracle):
    # the convolution geometry behind each Table 1 layer reproduces its GEMM shape
    for (layer, m, n, k), geo in zip(synth.RESNET50_TABLE1, synth.RESNET50_CONV):
        assert geo["layer"] == layer
        P = oracle.conv_out_size(geo["H"], geo["R"], geo["stride"], geo["pad"])
        assert m == 128 * P * P and n == geo["K"] and k == geo["C"] * geo["R"] * geo["R"], (layer, geo)
