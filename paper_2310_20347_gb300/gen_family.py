"""Generator of the tensor-core kernel family (run at build time).

The paper's contribution is a generator that emits a whole family of blocked
GEMM routines and micro-kernels from a few parameters (Sections 5-7), plus a
search that keeps the best member per problem shape (Section 8.4).  This
script plays the generator's role for the GPU kernels: it enumerates the
parameter space

    mode     bf16 | f16 | tf32 | 3xbf16 | 6xbf16 | 3xtf32 | fp8 | int8emu   operand format of the MMA
    bm       64 | 128 | 256           output rows per tile = MMA N
    cg       1 | 2                    CTAs per MMA: one SM (tile bm x 128), or a
                                      CTA pair on two SMs (tile bm x 256, each CTA
                                      staging half of A's rows: the cluster shape)
    stages   2 .. 8                   depth of the shared-memory k-block ring

filters it with the hardware's analytical limits -- the shared-memory budget
of one CTA and the TMEM columns of an SM, the GPU counterpart of the cache
model that fixes (mc, nc, kc) in Section 8.2 -- keeps the deepest pipeline that
fits plus one shallower variant, and writes

    csrc/family_gen.inc   an X-macro list the library instantiates
    family.json           the same list for the planner's tests and tooling

Split-K and the raster band are run-time knobs of every member, and the
operand "residency" of the paper's variant names (which operand stays in which
memory level) is expressed by the raster: a band walked m-fastest keeps B's
panels hot in L2 (B3A2C0-like), the transposed walk keeps A's (A3B2C0-like).
"""
from __future__ import annotations

import json
import os

SMEM_LIMIT = 232448          # bytes of dynamic shared memory per CTA (227 KiB)
TMEM_COLUMNS = 512           # 32-bit columns per SM
BAR_BYTES = 256
ALIGN_SLACK = 1024

MODES = {            # name: (planes, element bytes)
    "bf16": (1, 2),
    "3xbf16": (2, 2),
    "fp8": (1, 1),
    "int8emu": (1, 2),   # exact int8 on the BF16 path, k accumulated in chunks of <= 1024
    "6xbf16": (3, 2),    # FP32-accurate, three-part split, 6 products: used for small k
    "f16": (1, 2),       # IEEE binary16 operands on kind::f16
    "tf32": (1, 4),      # TF32 operands (binary32 storage) on kind::tf32
    "3xtf32": (2, 4),    # FP32-accurate on a two-part TF32 split, 3 kind::tf32 products
}
MODE_ENUM = {"bf16": "TC_BF16", "3xbf16": "TC_3XBF16", "fp8": "TC_FP8", "int8emu": "TC_I8EMU",
             "6xbf16": "TC_6XBF16", "f16": "TC_F16", "tf32": "TC_TF32", "3xtf32": "TC_3XTF32"}
SPLIT_MODES = ("3xbf16", "6xbf16", "3xtf32")   # two accumulators per tile (main + corrections)
BMS = (256, 128, 64)
# int8emu keeps one int32 running sum per row of its column in registers
# (with bm = 256: sixteen epilogue warps of 64 rows each)
MAX_BM = {"int8emu": 256}
# CTA-pair members: tile heights worth pairing (a pair of bm = 64 tiles would
# stage 32-row halves of A, no better than a single bm = 128 CTA)
PAIR_BMS = (256, 128)
RAW8_BMS = (128, 64)
RAW8_STAGES = 4
# TMEM columns one CTA of a pair allocates (the pair allocates collectively:
# both CTAs receive the same address, which the kernel checks)
PAIR_TMEM_COLUMNS = 512


def stage_bytes(mode: str, bm: int, cg: int = 1) -> int:
    planes, _elem = MODES[mode]
    bt = 128 * 128           # 128 columns of B x 128 bytes of k
    a = bm * 128 // cg       # this CTA's rows of A x 128 bytes of k
    return planes * (bt + a)


C_STAGE_BYTES = 2 * 32 * 128 * 4   # epilogue staging of C for TMA stores (two 32 x 128 fp32 boxes)


def smem_bytes(mode: str, bm: int, stages: int, cg: int = 1) -> int:
    return ALIGN_SLACK + stages * stage_bytes(mode, bm, cg) + C_STAGE_BYTES + BAR_BYTES


def enumerate_family():
    members = []
    for cg in (1, 2):
        tmem = TMEM_COLUMNS if cg == 1 else PAIR_TMEM_COLUMNS
        for mode in MODES:
            for bm in (BMS if cg == 1 else PAIR_BMS):
                acc_cols = (2 if mode in SPLIT_MODES else 1) * bm  # main (+ correction) accumulators
                if acc_cols > tmem or bm > MAX_BM.get(mode, 256):
                    continue
                fits = [s for s in range(2, 9) if smem_bytes(mode, bm, s, cg) <= SMEM_LIMIT]
                if not fits:
                    continue
                chosen = [max(fits)]
                if max(fits) - 1 in fits and max(fits) > 3:
                    chosen.append(max(fits) - 1)
                bufs = min(4, tmem // acc_cols)                     # accumulator sets across tiles
                for st in chosen:
                    members.append({"mode": mode, "bm": bm, "stages": st, "cg": cg,
                                    "smem": smem_bytes(mode, bm, st, cg), "tmem_bufs": bufs, "raw8": 0})
    # INT8 members that read the int8 operands as they are: TMA fills a ring
    # of raw int8 tiles (RAW8_STAGES k-blocks of bm x 64 + 64 x 128 bytes) and
    # converter warps write the exact bfloat16 tile into the stage; single-CTA,
    # at most 128 rows; the deepest bf16 ring that fits beside the raw ring
    for bm in RAW8_BMS:
        raw = RAW8_STAGES * (bm * 64 + 64 * 128)
        fits = [s for s in range(2, 9) if smem_bytes("int8emu", bm, s, 1) + raw <= SMEM_LIMIT]
        st = max(fits)
        members.append({"mode": "int8emu", "bm": bm, "stages": st, "cg": 1,
                        "smem": smem_bytes("int8emu", bm, st, 1) + raw, "tmem_bufs": min(4, TMEM_COLUMNS // bm),
                        "raw8": 1})
    for i, m in enumerate(members):
        m["index"] = i
    return members


# Grouped launches: problems of at most 1024 x 1024 take tiles of 64 or 128
# rows (chosen per problem by the planner's size bucket), so the kernel's
# buffers are sized for bm_max = 128; one member per mode with the deepest ring.
GROUPED_MODES = ("bf16", "3xbf16", "6xbf16", "fp8")
GROUPED_BM_MAX = 128
# Grouped FP32-accurate members that split inside the kernel: loader-converter
# warps read the FP32 operands and write the bf16 parts into the stages
# themselves (no TMA loads, no split pre-pass); 64-row tiles keep a k-block's
# runs in the registers of two groups of eight warps, and there is no C
# staging (grouped launches write C with plain stores).
GROUPED_FUSED_MODES = ("3xbf16", "6xbf16")
GROUPED_FUSED_BM = 64


def smem_bytes_fused(mode: str, bm: int, stages: int) -> int:
    return ALIGN_SLACK + stages * stage_bytes(mode, bm) + BAR_BYTES


def enumerate_grouped():
    out = []
    for mode in GROUPED_MODES:
        fits = [s for s in range(2, 9) if smem_bytes(mode, GROUPED_BM_MAX, s) <= SMEM_LIMIT]
        st = max(fits)
        out.append({"index": len(out), "mode": mode, "bm_max": GROUPED_BM_MAX, "stages": st,
                    "smem": smem_bytes(mode, GROUPED_BM_MAX, st), "fused": 0})
    for mode in GROUPED_FUSED_MODES:
        fits = [s for s in range(2, 9) if smem_bytes_fused(mode, GROUPED_FUSED_BM, s) <= SMEM_LIMIT]
        st = max(fits)
        out.append({"index": len(out), "mode": mode, "bm_max": GROUPED_FUSED_BM, "stages": st,
                    "smem": smem_bytes_fused(mode, GROUPED_FUSED_BM, st), "fused": 1})
    return out


def write(out_dir: str) -> list:
    members = enumerate_family()
    grouped = enumerate_grouped()
    lines = ["// Generated by gen_family.py -- do not edit.",
             "// X(index, mode, bm, stages, cg, raw8): raw8 = 1 reads int8 operands as they are",
             "#define G3_FAMILY_LIST(X) \\"]
    for m in members:
        lines.append(f"  X({m['index']}, {MODE_ENUM[m['mode']]}, {m['bm']}, {m['stages']}, {m['cg']}, {m['raw8']}) \\")
    lines.append("")
    lines.append(f"#define G3_FAMILY_SIZE {len(members)}")
    lines.append("")
    lines.append("// X(index, mode, bm_max, stages, fused): persistent grouped kernels (fused = 1: the")
    lines.append("// FP32-accurate split inside the kernel)")
    lines.append("#define G3_GROUPED_LIST(X) \\")
    for g in grouped:
        lines.append(f"  X({g['index']}, {MODE_ENUM[g['mode']]}, {g['bm_max']}, {g['stages']}, {g['fused']}) \\")
    lines.append("")
    lines.append(f"#define G3_GROUPED_SIZE {len(grouped)}")
    text = "\n".join(lines) + "\n"
    inc = os.path.join(out_dir, "csrc", "family_gen.inc")
    old = open(inc).read() if os.path.exists(inc) else None
    if old != text:
        with open(inc, "w") as f:
            f.write(text)
    js = os.path.join(out_dir, "family.json")
    jtext = json.dumps({"members": members, "grouped": grouped}, indent=1) + "\n"
    old = open(js).read() if os.path.exists(js) else None
    if old != jtext:
        with open(js, "w") as f:
            f.write(jtext)
    return members


if __name__ == "__main__":
    for m in write(os.path.dirname(os.path.abspath(__file__))):
        print(m)
