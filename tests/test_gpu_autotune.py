"""The autotuner picks a valid member and split for a shape's bucket, and the
GEMM stays correct under the tuned choice."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import rel_err
from paper_2310_20347_gb300 import G3_BF16, G3_F32_3XBF16, _lib, gen_family, synth, torch_api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,mode", [(G3_BF16, "bf16"), (G3_F32_3XBF16, "3xbf16")])
def test_autotune_then_gemm(dtype, mode):
    _lib.g3_tune_cache_clear()
    m, n, k = 384, 1000, 2048
    st, cfg, sk, ms = _lib.g3_autotune(m, n, k, dtype)
    assert st == 0 and ms > 0 and sk >= 1
    fam = gen_family.enumerate_family()
    assert fam[cfg]["mode"] == mode
    assert _lib.g3_plan_query(m, n, k, dtype)[1:3] == (cfg, sk)
    p = synth.uniform_problem(m, n, k, seed=30, beta=0.5)
    A, B, C = (torch.from_numpy(x).cuda() for x in (p.A, p.B, p.C))
    if dtype == G3_BF16:
        A, B = torch_api.convert_bf16(A), torch_api.convert_bf16(B)
        Aq, Bq = oracle.round_bf16(p.A), oracle.round_bf16(p.B)
        ref = oracle.gemm(Aq, Bq, p.C, 1.0, 0.5)
        D = oracle.absprod(Aq, Bq)
        tol = 1e-5
    else:
        ref = oracle.gemm(p.A, p.B, p.C, 1.0, 0.5)
        D = oracle.absprod(p.A, p.B)
        tol = 2e-6
    torch_api.gemm(A, B, C, 1.0, 0.5, dtype=dtype)
    torch.cuda.synchronize()
    assert rel_err(C.cpu().numpy(), ref, D, 0.5 * p.C.astype(np.float64)) <= tol
    _lib.g3_tune_cache_clear()
