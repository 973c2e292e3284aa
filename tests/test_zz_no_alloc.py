"""The allocation-free FP32-accurate GEMM, for callers that may not allocate
device memory (a framework that owns every byte of it, a fixed memory budget,
or code that must not trigger the synchronisation cudaMalloc can cause).

It must give the same result as the allocating entry point, g3_gemm_ex with
G3_F32_3XBF16 and no split-K, on two calls in a row: the second call sees the
scratch array exactly as the first one left it.  This file is collected last
so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import rel_err
from paper_2310_20347_gb300 import G3_F32_3XBF16, _lib, synth, torch_api

TOL = 1e-6   # relative to |alpha||A||B| + |beta C|; both calls run the same kernels


def noalloc(p, C):
    A = torch.from_numpy(p.A).cuda()
    B = torch.from_numpy(p.B).cuda()
    st = _lib.g3_gemm_3xbf16_noalloc(p.m, p.n, p.k, p.alpha, A.data_ptr(), p.k, B.data_ptr(), p.n, p.beta,
                                     C.data_ptr(), p.n, torch.cuda.current_stream().cuda_stream)
    assert st == 0, _lib.g3_status_string(st)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def reference(p):
    A = torch.from_numpy(p.A).cuda()
    B = torch.from_numpy(p.B).cuda()
    C = torch.from_numpy(p.C).cuda()
    torch_api.gemm(A, B, C, p.alpha, p.beta, dtype=G3_F32_3XBF16, split_k=1)
    torch.cuda.synchronize()
    return C.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    # two different problems back to back through the same scratch array
    for p in (synth.uniform_problem(700, 900, 1300, seed=21, alpha=1.0, beta=0.5),
              synth.uniform_problem(333, 257, 2049, seed=22, alpha=-0.75, beta=0.25)):
        got = noalloc(p, torch.from_numpy(p.C).cuda())
        want = reference(p)
        D = oracle.absprod(p.A, p.B, p.alpha)
        e = rel_err(got, want.astype(np.float64), D, p.beta * p.C.astype(np.float64))
        assert e <= TOL, e
    # the result is also right against the binary64 oracle (the mode's 2e-6)
    ref = oracle.gemm(p.A, p.B, p.C, p.alpha, p.beta)
    assert rel_err(got, ref, D, p.beta * p.C.astype(np.float64)) <= 2e-6


@pytest.mark.gpu
def test_noalloc_rejects_problems_beyond_the_scratch():
    # 4 * (m*k + k*n) bytes of bfloat16 planes exceed the 64 MiB array
    p = 16
    assert _lib.g3_gemm_3xbf16_noalloc(4096, 4096, 4096, 1.0, p, 4096, p, 4096, 0.0, p, 4096,
                                       None) == _lib.G3_ERR_UNSUPPORTED
