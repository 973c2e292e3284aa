"""Parity of the INT16 GEMM (G3_INT16, int16 A and B, int64 C) with the int64
oracle: bit-exact, including magnitudes beyond int32, ragged shapes, beta in
{0, 1}, transposed operands, k = 0 and the host-buffer entry point."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded
from paper_2310_20347_gb300 import G3_INT16, torch_api

pytestmark = pytest.mark.gpu


def ints(shape, seed, lo=-(1 << 15), hi=1 << 15, dtype=np.int16):
    return np.random.default_rng(seed).integers(lo, hi, shape).astype(dtype)


def stored(x, trans=False, pad=0):
    y = np.ascontiguousarray(x.T if trans else x)
    full = torch.zeros(y.shape[0], y.shape[1] + pad, dtype=torch.int16)
    full[:, : y.shape[1]] = torch.from_numpy(y)
    return full.cuda()[:, : y.shape[1]]


@pytest.mark.parametrize("shape", [(1, 1, 1), (17, 33, 5), (300, 520, 700), (129, 257, 65), (513, 300, 129),
                                   (64, 1000, 147)])
@pytest.mark.parametrize("beta", [0, 1])
def test_int16_bit_exact(shape, beta):
    m, n, k = shape
    A, B = ints((m, k), m + k), ints((k, n), n + k + 1)
    C0 = ints((m, n), 3, -(1 << 40), 1 << 40, np.int64) if beta else None
    full, C = guarded(m, n, C0, dtype=torch.int64)
    torch_api.gemm(stored(A, pad=3), stored(B, pad=5), C, 1, beta, dtype=G3_INT16)
    torch.cuda.synchronize()
    check_guard(full, m, n)
    assert np.array_equal(C.cpu().numpy(), oracle.gemm_i16(A, B, C0, 1, beta))


def test_int16_worst_case_and_transposes():
    # all -32768 at k = 4100: every entry is 4100 * 2^30, far beyond int32
    A = np.full((70, 4100), -32768, np.int16)
    B = np.full((4100, 90), -32768, np.int16)
    C = torch.zeros(70, 90, dtype=torch.int64, device="cuda")
    torch_api.gemm(stored(A), stored(B), C, 1, 0, dtype=G3_INT16)
    torch.cuda.synchronize()
    assert np.all(C.cpu().numpy() == 4100 * (1 << 30))
    A, B = ints((150, 260), 5), ints((260, 110), 6)
    for ta, tb in ((True, False), (False, True), (True, True)):
        C = torch.zeros(150, 110, dtype=torch.int64, device="cuda")
        torch_api.gemm(stored(A, ta), stored(B, tb), C, 1, 0, dtype=G3_INT16, trans_a=ta, trans_b=tb)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy(), oracle.gemm_i16(A, B)), (ta, tb)


def test_int16_k0_and_host_buffers():
    C0 = ints((40, 30), 7, -(1 << 40), 1 << 40, np.int64)
    C = torch.from_numpy(C0.copy()).cuda()
    empty_a = torch.empty(40, 0, dtype=torch.int16, device="cuda")
    empty_b = torch.empty(0, 30, dtype=torch.int16, device="cuda")
    torch_api.gemm(empty_a, empty_b, C, 1, 1, dtype=G3_INT16)   # beta = 1: unchanged
    torch_api.gemm(empty_a[:20], empty_b, C[:20], 1, 0, dtype=G3_INT16)   # beta = 0: zeros
    torch.cuda.synchronize()
    want = C0.copy()
    want[:20] = 0
    assert np.array_equal(C.cpu().numpy(), want)
    A, B = ints((2200, 300), 8), ints((300, 140), 9)
    C0 = ints((2200, 140), 10, -(1 << 40), 1 << 40, np.int64)
    hA, hB, hC = (torch.from_numpy(x.copy()).pin_memory() for x in (A, B, C0))
    torch_api.gemm_host(hA, hB, hC, 1, 1, dtype=G3_INT16)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(hC.numpy(), oracle.gemm_i16(A, B, C0, 1, 1))
