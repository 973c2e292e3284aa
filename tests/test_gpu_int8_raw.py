"""INT8 read as int8: the single-CTA INT8 members' twins (RAW8) that load the
raw int8 tiles of A and B by TMA into a ring of their own and convert them
in the kernel to the exact bfloat16 tiles the tensor core reads, replacing
the int8 -> bf16 conversion pass (rows TMA cannot address get an aligned
int8 copy).  Integer results are exact, so every case must equal the int64
oracle bit for bit, whichever member runs."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import check_guard, guarded
from paper_2310_20347_gb300 import G3_INT8, _lib, gen_family, synth, torch_api

pytestmark = pytest.mark.gpu
FAMILY = gen_family.enumerate_family()
RAW8 = [f["index"] for f in FAMILY if f["raw8"]]


def run(p, beta, A=None, B=None, **kw):
    full, C = guarded(p.m, p.n, p.C, dtype=torch.int32)
    A = torch.from_numpy(p.A).cuda() if A is None else A
    B = torch.from_numpy(p.B).cuda() if B is None else B
    l0 = _lib.g3_launch_count()
    torch_api.gemm(A, B, C, 1, beta, dtype=G3_INT8, **kw)
    launches = _lib.g3_launch_count() - l0
    torch.cuda.synchronize()
    check_guard(full, p.m, p.n)
    return C.cpu().numpy().astype(np.int64), launches


def test_raw8_members_are_the_int8_single_cta_twins():
    assert [(FAMILY[i]["mode"], FAMILY[i]["bm"], FAMILY[i]["cg"]) for i in RAW8] == [("int8emu", 128, 1),
                                                                                    ("int8emu", 64, 1)]


# convolution-shaped problems (m output channels, n pixels, k taps x channels):
# k = 147 leaves A's rows unaligned and n = 49 B's (aligned copies); the deep
# one splits k
@pytest.mark.parametrize("m,n,k,beta", [(64, 12544, 147, 0), (256, 3136, 576, 1), (2048, 49, 1024, 0),
                                        (512, 784, 4608, 0), (96, 1000, 64, 1)])
def test_planner_reads_int8_as_is_for_single_cta_shapes(m, n, k, beta):
    st, cfg, split, _ = _lib.g3_plan_query(m, n, k, G3_INT8)
    assert st == 0
    p = synth.int8_problem(m, n, k, seed=70 + m, beta=beta)
    got, launches = run(p, beta)
    rows = np.unique(np.array([0, m // 3, m - 1]))
    want = oracle.gemm_i8(p.A[rows], p.B, None if p.C is None else p.C[rows], 1, beta)
    assert np.array_equal(got[rows], want)
    if FAMILY[cfg]["raw8"]:
        # the planner's single-CTA choice runs as its RAW8 twin: no conversion
        # pass, only copies of unaligned operands and the split-K reduction
        copies = int(k % 16 != 0) + int(n % 16 != 0)
        assert launches == 1 + copies + (1 if split > 1 else 0), (launches, split, copies)
        # every split one exact accumulation chunk
        assert -(-(-(-k // 64)) // max(split, 1)) <= 16, (k, split)
    else:
        # the conversion pass stays for CTA pairs only
        assert FAMILY[cfg]["cg"] == 2, (m, n, k, cfg, split)
        assert launches == 2 + (1 if split > 1 else 0), (launches, split)


@pytest.mark.parametrize("config", RAW8)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
def test_raw8_member_equals_the_conversion_pass(config, ta, tb):
    # the same problem through a RAW8 member and through the member of the
    # same height that converts in a pre-pass (transposed operands are made
    # row-major first): identical, and equal to the oracle
    bm = FAMILY[config]["bm"]
    twin = next(f["index"] for f in FAMILY if f["mode"] == "int8emu" and f["bm"] == bm and f["cg"] == 1
                and not f["raw8"])
    p = synth.int8_problem(257, 304, 1100, seed=80 + bm, beta=1)
    outs = []
    for cfg in (config, twin):
        A = torch.from_numpy(np.ascontiguousarray(p.A.T) if ta else p.A).cuda()
        B = torch.from_numpy(np.ascontiguousarray(p.B.T) if tb else p.B).cuda()
        got, _ = run(p, 1, A=A, B=B, config=cfg, trans_a=ta, trans_b=tb)
        outs.append(got)
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], oracle.gemm_i8(p.A, p.B, p.C, 1, 1))


@pytest.mark.parametrize("config", RAW8)
@pytest.mark.parametrize("m,n,k,split", [(1, 1, 1, 0), (3, 9, 7, 0), (130, 70, 65, 0), (64, 129, 2049, 0),
                                         (200, 300, 3000, 3)])
def test_raw8_member_small_ragged_and_split(config, m, n, k, split):
    # single elements, boxes cut by the matrix edge in every dimension, k
    # across two 1024-product accumulation chunks plus a ragged block, and a
    # forced three-way split-K (int32 partials); RAW8 members split k by
    # themselves so that every split is one exact chunk (k = 2049: 3 splits)
    p = synth.int8_problem(m, n, k, seed=90 + m, beta=1)
    got, _ = run(p, 1, config=config, split_k=split)
    assert np.array_equal(got, oracle.gemm_i8(p.A, p.B, p.C, 1, 1))


def test_raw8_watchdog():
    # a raw stage that never fills: the converters' wait expires, the status
    # reports it, and the next call is exact
    p = synth.int8_problem(200, 300, 700, seed=95, beta=0)
    assert _lib.g3_debug_withhold_next(200) == 0
    run(p, 0, config=RAW8[0])
    st, code = torch_api.device_status()
    assert st == _lib.G3_ERR_TIMEOUT and code != 0
    got, _ = run(p, 0, config=RAW8[0])
    assert np.array_equal(got, oracle.gemm_i8(p.A, p.B, None, 1, 0))
    assert torch_api.device_status()[0] == 0
