"""Implicit-GEMM convolution (g3_conv2d) against the oracle's direct
convolution, element by element, on bfloat16-exact inputs: strided, padded,
dilated and 1 x 1 filters, ragged pixel and channel tiles, beta != 0, every
BF16 family member through the planner's forced choice, and split-K."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_20347_gb300 import G3_BF16, torch_api

pytestmark = pytest.mark.gpu

CASES = [  # N, H, W, C, K, R, S, stride, pad, dil
    (2, 12, 12, 64, 72, 3, 3, (1, 1), (1, 1), (1, 1)),
    (2, 13, 11, 64, 64, 3, 3, (2, 2), (1, 1), (1, 1)),
    (1, 9, 17, 128, 40, 1, 1, (1, 1), (0, 0), (1, 1)),
    (3, 10, 10, 64, 96, 1, 1, (2, 2), (0, 0), (1, 1)),
    (1, 15, 14, 64, 24, 3, 3, (1, 2), (2, 1), (2, 1)),
    (2, 8, 8, 192, 136, 3, 3, (1, 1), (1, 1), (1, 1)),
    (1, 23, 23, 64, 64, 7, 7, (2, 2), (3, 3), (1, 1)),
]


def run(case, beta=0.0, dtype=torch.bfloat16, seed=0):
    N, H, W, C, K, R, S, st, pd, dl = case
    r = np.random.default_rng(seed)
    x = oracle.round_bf16(r.standard_normal((N, H, W, C)).astype(np.float32))
    w = oracle.round_bf16((r.standard_normal((R, S, C, K)) / np.sqrt(R * S * C)).astype(np.float32))
    P = oracle.conv_out_size(H, R, st[0], pd[0], dl[0])
    Q = oracle.conv_out_size(W, S, st[1], pd[1], dl[1])
    y0 = r.standard_normal((N, P, Q, K)).astype(np.float32)
    y = torch.from_numpy(y0.copy()).cuda()
    torch_api.conv2d(torch.from_numpy(x).cuda().to(dtype), torch.from_numpy(w).cuda().to(dtype), y, st, pd, dl,
                     alpha=1.25, beta=beta)
    torch.cuda.synchronize()
    want = oracle.conv2d_nhwc(x, w, st, pd, dl, y=y0, alpha=1.25, beta=beta)
    D = oracle.conv2d_nhwc(np.abs(x), np.abs(w), st, pd, dl, alpha=1.25) + abs(beta) * np.abs(y0)
    return float(np.max(np.abs(y.cpu().numpy() - want) / np.maximum(D, 1e-300)))


@pytest.mark.parametrize("case", CASES)
def test_conv_matches_oracle(case):
    e = run(case)
    assert e <= 1e-5, e


@pytest.mark.parametrize("case", CASES[:3])
def test_conv_beta_and_fp16(case):
    assert run(case, beta=-0.5) <= 1e-5
    assert run(case, dtype=torch.float16, seed=1) <= 1e-5   # bf16-exact values are fp16-exact here


@pytest.mark.parametrize("case", [(4, 28, 28, 128, 256, 3, 3, (1, 1), (1, 1), (1, 1)),     # CTA-pair tiles
                                  (1, 7, 7, 512, 512, 3, 3, (1, 1), (1, 1), (1, 1)),        # few tiles, split-K
                                  (2, 14, 14, 256, 1024, 1, 1, (2, 2), (0, 0), (1, 1))])
def test_conv_planner_members(case):
    from paper_2310_20347_gb300 import _lib
    N, H, W, C, K, R, S, st, pd, dl = case
    P = oracle.conv_out_size(H, R, st[0], pd[0], dl[0])
    print(case, _lib.g3_plan_query(N * P * P, K, R * S * C, G3_BF16))
    assert run(case, beta=0.5) <= 1e-5


def test_conv_unsupported_channels():
    x = torch.zeros(1, 4, 4, 3, dtype=torch.bfloat16, device="cuda")
    w = torch.zeros(3, 3, 3, 8, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(Exception):
        torch_api.conv2d(x, w, pad=(1, 1))
