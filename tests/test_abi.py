"""CPU checks of the boundary: the library builds, loads and exports every
symbol include/g3gemm.h declares; argument validation returns the documented
positional codes without touching a GPU; the generated family and the planner
(host logic) behave as specified."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_20347_gb300 import _lib, build
    build()
    return _lib


def header_symbols():
    text = open(os.path.join(ROOT, "include", "g3gemm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(g3_\w+)\s*\(", text)))


def test_exports_match_header(lib):
    declared = header_symbols()
    assert sorted(lib.EXPORTED) == declared
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared:
        assert hasattr(so, name), name


def test_library_has_no_oracle_dependency(lib):
    # the product library must not link or embed the test oracle
    data = open(lib.LIB_PATH, "rb").read()
    assert b"oracle_gemm" not in data and b"liboracle" not in data


def test_argument_errors(lib):
    L = lib
    p = 16  # any non-null "device" address: validation fails before any use
    assert L.g3_gemm(-1, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, 0) == -101
    assert L.g3_gemm(4, -1, 4, 1.0, p, 4, p, 4, 0.0, p, 4, 0) == -102
    assert L.g3_gemm(4, 4, -1, 1.0, p, 4, p, 4, 0.0, p, 4, 0) == -103
    assert L.g3_gemm(4, 4, 8, 1.0, p, 7, p, 4, 0.0, p, 4, 0) == -106
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 3, 0.0, p, 4, 0) == -108
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, p, 3, 0) == -111
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, p, 4, 10) == -112
    assert L.g3_gemm(4, 4, 8, 1.0, None, 8, p, 4, 0.0, p, 4, 0) == -105
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, None, 4, 0.0, p, 4, 0) == -107
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, None, 4, 0) == -110
    # transposed operands: lda >= m for A stored k x m, ldb >= k for B stored n x k
    a = L.g3_gemm_args_init()
    a.m, a.n, a.k, a.A, a.B, a.C, a.alpha = 6, 4, 8, p, p, p, 1.0
    a.lda, a.ldb, a.ldc, a.trans_a = 5, 4, 4, 1
    assert L.g3_gemm_workspace_size(a)[0] == -106
    a.lda, a.trans_b, a.ldb = 6, 1, 7
    assert L.g3_gemm_workspace_size(a)[0] == -108
    a.ldb, a.trans_b = 8, 2
    assert L.g3_gemm_workspace_size(a)[0] == -120
    # CUDA-core dtypes: row blocks on grid.y, at most 65535 of them
    a = L.g3_gemm_args_init()
    a.n, a.k, a.A, a.B, a.C, a.alpha, a.lda, a.ldb, a.ldc = 4, 8, p, p, p, 1.0, 8, 4, 4
    for dt, rows in ((L.G3_F32, 128), (L.G3_F64, 64), (L.G3_INT16, 64)):
        a.dtype = dt
        a.m = 65536 * rows
        assert L.g3_gemm_workspace_size(a)[0] == L.G3_ERR_UNSUPPORTED, dt
        a.k = 0                # C := beta*C alone has no such limit
        assert L.g3_gemm_workspace_size(a)[0] == 0, dt
        a.k = 8
    # host-buffer entry point: the same validation, nothing touches a device
    assert L.g3_gemm_host(-1, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, 0, None) == -101
    assert L.g3_gemm_host(4, 4, 8, 1.0, p, 7, p, 4, 0.0, p, 4, 0, None) == -106
    assert L.g3_gemm_host(4, 4, 8, 1.0, p, 8, p, 4, 0.0, None, 4, 0, None) == -110
    assert L.g3_gemm_host(0, 4, 8, 1.0, None, 8, None, 4, 0.0, None, 4, 0, None) == 0
    # operand preparation: the same positional codes
    assert L.g3_convert_bf16(p, 4, 8, 8, p, 7) == -106
    assert L.g3_split_bf16(p, 4, 8, 8, p, p, 7) == -107
    assert L.g3_split_bf16(p, 4, 8, 8, p, None, 8) == -106
    assert L.g3_split3_bf16(p, 4, 8, 7, p, p, p, 8) == -104
    assert L.g3_split3_bf16(p, 4, 8, 8, None, p, p, 8) == -105
    assert L.g3_split3_bf16(p, 4, 8, 8, p, None, p, 8) == -106
    assert L.g3_split3_bf16(p, 4, 8, 8, p, p, None, 8) == -107
    assert L.g3_split3_bf16(p, 4, 8, 8, p, p, p, 7) == -108
    assert L.g3_split3_bf16(p, 0, 8, 8, None, None, None, 8) == 0
    assert L.g3_split_tf32(p, 4, 8, 8, p, p, 7) == -107
    assert L.g3_split_tf32(p, 4, 8, 8, p, None, 8) == -106
    assert L.g3_split_tf32(p, 0, 8, 8, None, None, 8) == 0
    # allocation-free entry: k beyond one FP32 accumulator's bound (no device touched)
    assert L.g3_gemm_3xbf16_noalloc(64, 64, 40000, 1.0, p, 40000, p, 64, 0.0, p, 64, None) == L.G3_ERR_UNSUPPORTED
    # a dtype beyond the last one
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, p, 4, 10) == -112
    # INT16 accepts only alpha == 1 and beta in {0, 1}
    assert L.g3_gemm(4, 4, 8, 2.0, p, 8, p, 4, 0.0, p, 4, L.G3_INT16) == L.G3_ERR_UNSUPPORTED
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.5, p, 4, L.G3_INT16) == L.G3_ERR_UNSUPPORTED
    # INT8 accepts only alpha == 1 and beta in {0, 1}
    assert L.g3_gemm(4, 4, 8, 2.0, p, 8, p, 4, 0.0, p, 4, 4) == L.G3_ERR_UNSUPPORTED
    assert L.g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.5, p, 4, 4) == L.G3_ERR_UNSUPPORTED
    assert L.g3_gemm(4, 4, 131073, 1.0, p, 131073, p, 4, 0.0, p, 4, 4) == L.G3_ERR_UNSUPPORTED
    # m == 0 or n == 0: a no-op, even with null pointers
    assert L.g3_gemm(0, 4, 8, 1.0, None, 8, None, 4, 0.0, None, 4, 0) == 0
    assert L.g3_gemm(4, 0, 8, 1.0, None, 8, None, 1, 0.0, None, 1, 0) == 0
    assert L.g3_status_string(-5) == "device wait timed out"
    assert L.g3_debug_withhold_next(0) == -101


def test_family_matches_generator(lib):
    from paper_2310_20347_gb300 import gen_family
    members = gen_family.enumerate_family()
    assert lib.g3_family_size() == len(members)
    with open(os.path.join(ROOT, "paper_2310_20347_gb300", "family.json")) as f:
        assert json.load(f) == {"members": members, "grouped": gen_family.enumerate_grouped()}
    for m in members:
        d = lib.g3_family_describe(m["index"])
        assert f"mode={m['mode']} bm={m['bm']} bn={128 * m['cg']} stages={m['stages']}" in d, d
        assert f"bufs={m['tmem_bufs']} cg={m['cg']}" in d, d
        assert m["smem"] <= gen_family.SMEM_LIMIT and 2 * m["bm"] <= gen_family.TMEM_COLUMNS


def test_planner_choices(lib):
    from paper_2310_20347_gb300 import gen_family
    fam = gen_family.enumerate_family()
    L = lib
    # large square, FP32-accurate: the 256 x 256 CTA-pair tile (its single
    # accumulator set costs little against 256 k-blocks of main loop)
    st, cfg, sk, rs = L.g3_plan_query(16384, 16384, 16384, L.G3_F32_3XBF16)
    assert st == 0 and fam[cfg]["mode"] == "3xbf16" and fam[cfg]["bm"] == 256 and fam[cfg]["cg"] == 2 and sk == 1
    # BF16 8192^3: the 256 x 256 CTA pair with double-buffered accumulators
    st, cfg, sk, rs = L.g3_plan_query(8192, 8192, 8192, L.G3_BF16)
    assert fam[cfg]["bm"] == 256 and fam[cfg]["cg"] == 2 and fam[cfg]["tmem_bufs"] == 2
    # Cout = 64 convolution layer: a 64-row tile, no split
    st, cfg, sk, rs = L.g3_plan_query(64, 200704, 147, L.G3_BF16)
    assert fam[cfg]["bm"] == 64 and sk == 1
    # few output tiles, deep k: split-K
    st, cfg, sk, rs = L.g3_plan_query(512, 49, 4608, L.G3_BF16)
    assert sk > 1
    # INT8 runs on the exact-integer members (k chunked inside the kernel): the
    # bm = 256 CTA pair (16 epilogue warps, two chunk accumulators), no split needed
    st, cfg, sk, rs = L.g3_plan_query(8192, 8192, 8192, L.G3_INT8)
    assert fam[cfg]["mode"] == "int8emu" and fam[cfg]["bm"] == 256 and fam[cfg]["cg"] == 2 and sk == 1
    # FP32-accurate at k <= 512: the three-part split (6 products); above: two-part
    for k, mode in ((16, "6xbf16"), (512, "6xbf16"), (513, "3xbf16"), (4096, "3xbf16")):
        st, cfg, sk, rs = L.g3_plan_query(2048, 2048, k, L.G3_F32_3XBF16)
        assert st == 0 and fam[cfg]["mode"] == mode, (k, fam[cfg])
    st, cfg, sk, rs = L.g3_plan_query(128, 128, 100, L.G3_F32)
    assert cfg == -1
    # FP32 SIMT: cluster split of k only while 64 x 64 blocks leave SMs idle,
    # within two CTAs per SM and two k-blocks of 16 per CTA (152 SMs assumed
    # without a GPU)
    import torch
    if not torch.cuda.is_available():
        for (m, n, k), want in (((512, 512, 512), 4), ((128, 128, 100), 2), ((128, 128, 40), 1),
                                ((256, 256, 4096), 8), ((1024, 1024, 1024), 1), ((4096, 4096, 64), 1)):
            st, cfg, sk, rs = L.g3_plan_query(m, n, k, L.G3_F32)
            assert st == 0 and cfg == -1 and sk == want, (m, n, k, sk)
            # the autotuner does not time the CUDA-core kernels: it reports
            # the planner's choice
            assert L.g3_autotune(m, n, k, L.G3_F32) == (0, -1, want, 0.0)
            assert L.g3_autotune(m, n, k, L.G3_F64) == (0, -1, 1, 0.0)


def test_tuning_cache_overrides_planner(lib, tmp_path):
    from paper_2310_20347_gb300 import gen_family
    fam = gen_family.enumerate_family()
    L = lib
    assert L.g3_tune_cache_clear() == 0
    st, cfg0, sk0, _ = L.g3_plan_query(1000, 3000, 700, L.G3_BF16)
    _, cfg1, sk1, _ = L.g3_plan_query(1000, 3000, 1500, L.G3_BF16)   # another k bucket
    other = next(f["index"] for f in fam if f["mode"] == "bf16" and f["index"] != cfg0)
    # bucket of (1000, 3000, 700) = (10, 12, 10); dtype G3_BF16 = 2
    path = tmp_path / "tune.txt"
    path.write_text(f"# test\n2 10 12 10 {other} 3 0.5\n")
    assert L.g3_tune_cache_load(str(path)) == 0
    st, cfg, sk, _ = L.g3_plan_query(1000, 3000, 700, L.G3_BF16)
    assert (cfg, sk) == (other, 3)
    # another shape of the same bucket follows the record; another bucket does not
    assert L.g3_plan_query(600, 2100, 513, L.G3_BF16)[1:3] == (other, 3)
    assert L.g3_plan_query(1000, 3000, 1500, L.G3_BF16)[1:3] == (cfg1, sk1)
    out = tmp_path / "saved.txt"
    assert L.g3_tune_cache_save(str(out)) == 0
    assert f"2 10 12 10 {other} 3" in out.read_text()
    assert L.g3_tune_cache_clear() == 0
    assert L.g3_plan_query(1000, 3000, 700, L.G3_BF16)[1:3] == (cfg0, sk0)
    assert L.g3_tune_cache_load(str(tmp_path / "missing.txt")) == -101


def test_planner_invariants_over_random_shapes(lib):
    # host logic only: for every dtype and 300 seeded shapes the plan names a
    # member of the mode the dtype runs (the FP32-accurate mode by depth), a
    # split count within [1, k-blocks], never a stream-K tail unasked, and the
    # FP32-accurate modes keep at most 32768 (3xBF16) / 8192 (3xTF32) of k per
    # accumulator; the CUDA-core dtypes report no member.
    import numpy as np
    from paper_2310_20347_gb300 import gen_family
    fam = gen_family.enumerate_family()
    L = lib
    mode_of = {L.G3_BF16: "bf16", L.G3_FP16: "f16", L.G3_TF32: "tf32", L.G3_FP8_E4M3: "fp8",
               L.G3_INT8: "int8emu", L.G3_F32_3XTF32: "3xtf32"}
    kblock = {"bf16": 64, "f16": 64, "tf32": 32, "fp8": 128, "int8emu": 64, "3xtf32": 32, "3xbf16": 64,
              "6xbf16": 64}
    rng = np.random.default_rng(90)
    for _ in range(300):
        m, n = (int(x) for x in np.exp(rng.uniform(0, np.log(20000), 2)).astype(int) + 1)
        k = int(np.exp(rng.uniform(0, np.log(70000))) + 1)
        for dt in (L.G3_BF16, L.G3_FP16, L.G3_TF32, L.G3_FP8_E4M3, L.G3_INT8, L.G3_F32_3XTF32, L.G3_F32_3XBF16):
            st, cfg, sk, rs = L.g3_plan_query(m, n, k, dt)
            assert st == 0 and 0 <= cfg < len(fam), (m, n, k, dt)
            mode = mode_of.get(dt) or ("6xbf16" if k <= 512 else "3xbf16")
            assert fam[cfg]["mode"] == mode, (m, n, k, dt, fam[cfg])
            num_kb = -(-k // kblock[mode])
            assert sk != L.G3_SPLIT_STREAM_K and 1 <= sk <= num_kb, (m, n, k, dt, sk)
            if mode == "3xtf32":
                assert -(-num_kb // sk) <= 256, (k, sk)
            if mode == "3xbf16":
                assert -(-num_kb // sk) <= 512, (k, sk)
            assert rs >= 1
        for dt in (L.G3_F32, L.G3_F64, L.G3_INT16):
            assert L.g3_plan_query(m, n, k, dt)[1] == -1
        # FP32 SIMT: a cluster split of k (2, 4 or 8 CTAs) only while 64 x 64
        # blocks leave SMs idle, within two CTAs per SM and two k-blocks of 16
        # per CTA (152 SMs without a GPU); FP64 / INT16 never split
        import torch
        if not torch.cuda.is_available():
            sk = L.g3_plan_query(m, n, k, L.G3_F32)[2]
            tiles64 = -(-m // 64) * -(-n // 64)
            assert sk in (1, 2, 4, 8), sk
            if sk > 1:
                assert tiles64 < 152 and tiles64 * sk <= 304 and -(-k // sk) >= 32, (m, n, k, sk)
            elif tiles64 < 152 and -(-m // 128) * -(-n // 128) < 152:
                assert tiles64 * 2 > 304 or -(-k // 2) < 32, (m, n, k)
            assert L.g3_plan_query(m, n, k, L.G3_F64)[2] == 1
            assert L.g3_plan_query(m, n, k, L.G3_INT16)[2] == 1


def test_planner_thread_safe(lib):
    # host threads planning at once (ctypes drops the GIL around each call)
    # get the answers a single thread gets
    import threading

    import numpy as np
    L = lib
    rng = np.random.default_rng(7)
    dts = (L.G3_F32, L.G3_BF16, L.G3_F32_3XBF16, L.G3_INT8, L.G3_FP8_E4M3, L.G3_F32_3XTF32)
    queries = [(int(m), int(n), int(k), int(dts[i % len(dts)]))
               for i, (m, n, k) in enumerate(np.exp(rng.uniform(0, np.log(30000), (400, 3))).astype(int) + 1)]
    want = [L.g3_plan_query(*q) for q in queries]
    errors = []

    def worker(t):
        for i in range(len(queries)):
            j = (i * 7 + t) % len(queries)
            if L.g3_plan_query(*queries[j]) != want[j]:
                errors.append(queries[j])

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(8)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors[:5]


def test_stream_traffic_argument_errors(lib):
    # sizes must be non-negative multiples of 16 bytes (at most 32 GiB), and
    # pointers 16-byte aligned when their size is non-zero; checked before any
    # device work
    assert lib.g3_stream_traffic(16, 17, 16, 16) == -102
    assert lib.g3_stream_traffic(16, -16, 16, 16) == -102
    assert lib.g3_stream_traffic(16, 1 << 36, 16, 16) == -102
    assert lib.g3_stream_traffic(16, 16, 16, 24) == -104
    assert lib.g3_stream_traffic(None, 16, 16, 16) == -101
    assert lib.g3_stream_traffic(8, 16, 16, 16) == -101
    assert lib.g3_stream_traffic(16, 16, None, 16) == -103
