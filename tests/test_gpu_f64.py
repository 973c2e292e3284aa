"""Parity of the FP64 GEMM (G3_F64, the binary64 entry of the datatype study)
with the binary64 oracle.  Both compute every product exactly rounded and sum
in binary64, in different orders, so they differ by at most about
2 k 2^-53 of sum |alpha a b| (plus the rounding of beta*C): the tolerance is
k * 2^-52; integer inputs are bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded, rel_err
from paper_2310_20347_gb300 import G3_F64, torch_api

pytestmark = pytest.mark.gpu


def problem(m, n, k, seed, beta=0.5):
    r = np.random.default_rng(seed)
    A = r.uniform(-1, 1, (m, k))
    B = r.standard_normal((k, n))
    C = r.uniform(-1, 1, (m, n)) if beta != 0.0 else None
    return A, B, C


def stored(x, pad=0, trans=False):
    y = np.ascontiguousarray(x.T if trans else x)
    full = torch.zeros(y.shape[0], y.shape[1] + pad, dtype=torch.float64)
    full[:, : y.shape[1]] = torch.from_numpy(y)
    return full.cuda()[:, : y.shape[1]]


def check(m, n, k, seed=0, alpha=1.25, beta=0.5, pad=(0, 0), trans=(False, False)):
    A, B, C0 = problem(m, n, k, seed, beta)
    full, C = guarded(m, n, C0, dtype=torch.float64)
    torch_api.gemm(stored(A, pad[0], trans[0]), stored(B, pad[1], trans[1]), C, alpha, beta, dtype=G3_F64,
                   trans_a=trans[0], trans_b=trans[1])
    torch.cuda.synchronize()
    check_guard(full, m, n)
    got = C.cpu().numpy()
    bc = None if C0 is None else beta * C0
    e = rel_err(got, oracle.gemm(A, B, C0, alpha, beta), oracle.absprod(A, B, alpha), bc)
    assert e <= max(k, 1) * 2.0 ** -52, e
    return e


@pytest.mark.parametrize("shape", [(1, 1, 1), (17, 33, 5), (300, 520, 700), (129, 257, 65), (64, 1000, 147),
                                   (513, 300, 129), (1000, 64, 1200)])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_f64_shapes(shape, beta):
    check(*shape, seed=sum(shape), beta=beta)


def test_f64_unaligned_rows_and_transposes():
    check(130, 77, 91, seed=1, pad=(1, 3))               # odd leading dimensions: scalar loads
    for trans in ((True, False), (False, True), (True, True)):
        check(130, 200, 300, seed=2, trans=trans)


def test_f64_integers_exact_and_edge_rules():
    r = np.random.default_rng(3)
    A = r.integers(-50, 50, (200, 300)).astype(np.float64)
    B = r.integers(-50, 50, (300, 150)).astype(np.float64)
    C0 = r.integers(-50, 50, (200, 150)).astype(np.float64)
    C = torch.from_numpy(C0.copy()).cuda()
    torch_api.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 1.0, 2.0, dtype=G3_F64)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B, C0, 1.0, 2.0))
    # beta = 0 never reads C: NaN is overwritten; k = 0 scales C by beta in binary64
    C = torch.full((200, 150), float("nan"), dtype=torch.float64, device="cuda")
    torch_api.gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, 1.0, 0.0, dtype=G3_F64)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.gemm(A, B))
    C = torch.from_numpy(C0.copy()).cuda()
    beta = 1.0 / 3.0
    torch_api.gemm(torch.empty(200, 0, dtype=torch.float64, device="cuda"),
                   torch.empty(0, 150, dtype=torch.float64, device="cuda"), C, 1.0, beta, dtype=G3_F64)
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), beta * C0)


def test_f64_host_buffers():
    A, B, C0 = problem(2100, 130, 300, seed=4)
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    hC = torch.from_numpy(C0.copy()).pin_memory()
    torch_api.gemm_host(hA, hB, hC, 0.75, 0.5, dtype=G3_F64)
    torch.cuda.current_stream().synchronize()
    e = rel_err(hC.numpy(), oracle.gemm(A, B, C0, 0.75, 0.5), oracle.absprod(A, B, 0.75), 0.5 * C0)
    assert e <= 300 * 2.0 ** -52, e
