// tc_gemm.cuh -- the tensor-core member of the blocked-GEMM family (sm_103a).
//
// C := beta*C + alpha*A*B with A (m x k) and B (k x n) row-major, computed by a
// persistent, warp-specialised kernel:
//
//   warp 0      TMA producer: streams k-blocks of A and B into a STAGES-deep ring
//               of 128-byte-swizzled shared-memory tiles (the packed buffers Ac, Bc
//               of the paper's Section 3.1 / Figure "packing": TMA writes them in
//               exactly the layout the tensor core reads, so packing costs no pass)
//   warp 1      MMA issuer: one thread issues tcgen05.mma per 32-byte k-step (16
//               BF16/FP16, 32 FP8 or 8 TF32 elements); the accumulator micro-tile
//               lives in TMEM (the "C resident" micro-kernel of Section 4.1 with
//               TMEM in place of the register file), multi-buffered across tiles
//   warps 2..5  epilogue: tcgen05.ld of the accumulator, alpha/beta, stores
//               (warps 2..17 for the exact-integer member with bm = 256)
//
// Orientation.  The MMA computes D = Bt * At, i.e. the transpose of the C tile:
// TMEM lane = column j of C (128 per tile), TMEM column = row i of C (bm per
// tile).  The MMA's A operand is the k x 128 slice of B (stored n-contiguous, so
// "MN-major"), its B operand the bm x k slice of A (k-contiguous, "K-major").
// Each epilogue thread then owns one column of C and a warp's store of one row
// is 32 consecutive floats: every global store is a full 128-byte line.
// Transposed storage (BLAS transa/transb) changes only the staging: B stored
// n x k is staged K-major, A stored k x m MN-major, each described as such to
// the tensor core, so the one-plane 8- and 16-bit modes read them in place.
//
// The blocked loops of the paper's baseline algorithm (Figure "B3A2C0") map to:
// L1/L3 (jc, ic) -> the persistent tile walk with a banded raster (a band of
// `raster` m-tiles walked m-fastest keeps that band's A panels and the current
// B panels in L2); L2 (pc) -> the k-block loop, optionally split across CTAs
// (split-K, the analogue of the C-in-cache variants of Section 7); L4/L5 (jr, ir)
// -> the 128 x bm tile of one MMA; L6 (pr) -> the k-steps of the MMA.
//
// Which tiles a CTA walks comes from a scheduler policy: SingleSched for one
// problem (TcParams, tensor maps as kernel parameters), GroupedSched for many
// independent problems in one launch (a device table of problems, six tensor
// maps per problem in global memory, and per problem its own tile height bm).
//
// CTA pairs (CG = 2, a cluster of two CTAs on neighbouring SMs).  One MMA of
// M = 256 spans both SMs: the tile is 256 columns of C x bm rows; each CTA
// stages its own 128 columns of B and HALF of the bm rows of A, so a CTA moves
// 16 KB + bm*64 B per k-block instead of 16 KB + bm*128 B for the same MMA
// work -- shared-memory fill bandwidth per SM, not the tensor core, is what
// limits the single-CTA members.  The leader (cluster rank 0) issues every MMA
// and waits for both CTAs' TMA bytes on its own barriers; its commits arrive on
// the barriers of both CTAs; each CTA's epilogue drains its own TMEM (its 128
// columns of C) and reports to the leader.
//
// Split inside the kernel (FUSED, grouped FP32-accurate launches on request):
// sixteen loader-converter warps take the TMA producer's place.  They read FP32 A and
// B from global memory (any alignment), split every element into bfloat16
// parts exactly as the split pre-pass does, and store the parts where TMA
// would have put them, so the MMA issuer and the epilogue are unchanged and
// the FP32 operands cross the memory system once instead of three times
// (read, planes written, planes read).
//
// INT8 read as int8 (RAW8 members): TMA loads the raw int8 tiles of A and B
// into a small ring of their own, and converter warps write their exact
// binary16 values into the stage in the swizzled layout (kind::f16 with the
// F16 format; every split is one chunk of at most 1024 products, whose FP32
// sum stays exact), so the operands
// cross HBM once at one byte per element instead of through a conversion pass
// that writes and re-reads two.
//
// Implicit-GEMM convolution (TcParams::conv): A is an NHWC activation tensor;
// the producer loads each k-block of A (64 channels of one filter tap for bm
// output pixels) with a TMA im2col load, so the convolution runs through the
// same pipeline without a materialised im2col matrix.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "bf16.cuh"
#include "ptx.cuh"
#include "sched.cuh"

namespace g3 {

// TC_I8EMU: int8 GEMM computed exactly on the BF16 tensor path (int8 values are
// exact in bfloat16); k is accumulated in chunks of at most 1024 products per
// TMEM accumulator, which keeps every FP32 partial sum an exact integer, and
// the epilogue adds the chunks in int32.
// TC_6XBF16: the FP32-accurate mode for small k: operands split in three
// bfloat16 parts (hi + mid + lo), six products per k-step.
// TC_3XTF32: a second FP32-accurate mode: operands split in two TF32 parts
// (hi + lo, 22 significant bits), three kind::tf32 products per k-step.
enum TcMode : int {
  TC_BF16 = 0, TC_3XBF16 = 1, TC_FP8 = 2, TC_I8EMU = 3, TC_6XBF16 = 4, TC_F16 = 5, TC_TF32 = 6, TC_3XTF32 = 7
};
enum OutMode : int { OUT_F32 = 0, OUT_I32 = 1, OUT_PARTIAL = 2 };

// Watchdog status codes (written to the device status word; see g3gemm.h).
enum : int {
  WD_PRODUCER_EMPTY = 0x101,
  WD_MMA_FULL = 0x102,
  WD_MMA_TMEM_EMPTY = 0x103,
  WD_EPI_TMEM_FULL = 0x104,
  WD_DRAIN = 0x105,
  WD_PAIR_TMEM = 0x106,   // the two CTAs of a pair did not receive the same TMEM address
  WD_TILE_QUEUE = 0x107,  // a claimed tile number (or a free entry for one) never arrived
};

struct TcParams {
  int m, n, k;
  int tiles_m, tiles_n;   // ceil(m / BM_T), ceil(n / 128)
  int splits;             // number of k-splits (1 = none)
  int kb_per_split;       // k-blocks handled by one split
  int num_kb;             // ceil(k / BK)
  int raster;             // band width, in m-tiles, of the tile walk
  float alpha, beta;
  const float* scale_a;   // FP8 per-tensor scales (device, may be null = 1)
  const float* scale_b;
  void* C;                // float (OUT_F32) or int32 (OUT_I32)
  long long ldc;
  float* partial;         // OUT_PARTIAL: [splits][m][ldp] float; stream-K: [sk_streams * sk_segs] tiles
  long long ldp;          // OUT_PARTIAL: row stride of the partial planes (elements, rows on 128-byte lines)
  int out_mode;
  unsigned long long timeout_ns;
  int* status;
  int debug_withhold;     // test hook: producer iteration whose stage never fills (-1: none)
  int kchunk;             // k-blocks per accumulation chunk (0: the whole k range of a tile)
  int c_tma;              // 1: C (beta == 0) -- or, with split-K, the partial planes -- is written through
                          // TMA stores with the tmC map (3-D for the partial planes: n x m x splits)
  // Implicit-GEMM convolution (conv = 1): A is the NHWC activation tensor read
  // through an im2col tensor map; row i of A is output pixel i = (n, p, q) and
  // k-block kb is filter tap (r, s) = divmod(kb / cblocks, S), channel block
  // kb % cblocks of 64 channels.
  int conv;
  int conv_pq, conv_q;            // P * Q and Q of the output
  int conv_sh, conv_sw, conv_ph, conv_pw, conv_dh, conv_dw;
  int conv_s, conv_cblocks;       // filter width S, C / 64
  // Stream-K tail (sk_streams > 0; see sched.cuh): the first sk_dp tiles of the
  // walk (a multiple of sk_streams) are computed whole, the last sk_tail tiles
  // in segments whose partial tiles (bm x 128*CG, FP32 or int32) go to
  // `partial`; the grid must then hold exactly sk_streams CTAs (or pairs).
  int sk_streams, sk_dp, sk_tail, sk_segs;
  // Operands read in place in their transposed storage (one-plane 8- and
  // 16-bit modes only): a_mn = 1, A stored k x m (lda >= m) and staged
  // MN-major; b_km = 1, B stored n x k (ldb >= k) and staged K-major.
  int a_mn, b_km;
  // Claimed tile walk (non-null; zeroed before the launch): the tiles past each
  // CTA's (or pair's) first are claimed from this counter in claim order
  // instead of the static every-gridDim-th walk (not with a stream-K tail).
  int* tile_ctr;
};

// One problem of a grouped launch (device table entry).
struct GroupDesc {
  int m, n, k;
  int tiles_m, tiles_n, num_kb;
  int bm;                 // rows per tile for this problem (MMA N), <= the kernel's BM_T
  int pad;
  float alpha, beta;
  float* C;
  long long ldc;
  // FP32 operands read by the loader-converter warps of the FUSED kernels
  // (row-major, leading dimensions in elements; null otherwise)
  const float* A;
  const float* B;
  long long lda, ldb;
};

// Tensor maps of one problem: A and B of each operand plane (hi, then the
// lower parts of the split modes), then C.
constexpr int kMapsPerProblem = 6;

struct GroupedParams {
  const GroupDesc* groups;
  const CUtensorMap* maps;   // kMapsPerProblem per problem: A/B of plane 0, 1, 2
  const int2* tile_info;     // per global tile: (problem, tile index within the problem)
  int total_tiles;
  unsigned long long timeout_ns;
  int* status;
  int debug_withhold;
};

template <int MODE>
struct TcTraits {
  static constexpr bool kTf32 = (MODE == TC_TF32 || MODE == TC_3XTF32);
  static constexpr int kPlanes = (MODE == TC_3XBF16 || MODE == TC_3XTF32) ? 2 : (MODE == TC_6XBF16 ? 3 : 1);
  static constexpr int kElem = (MODE == TC_FP8) ? 1 : (kTf32 ? 4 : 2);   // bytes per element
  static constexpr int kBK = 128 / kElem;                        // k per block: one 128-B row
  static constexpr int kKStep = 32 / kElem;                      // k per MMA instruction
  static constexpr int kKSteps = kBK / kKStep;                   // = 4
  static constexpr int kBoxN = 128 / kElem;                      // n per TMA box of B
  static constexpr int kNBoxes = 128 / kBoxN;                    // boxes per 128-wide n tile
  static constexpr uint32_t kBtBytes = 128 * 128;                // 128 n x 128 bytes of k
  // operand format code: 0 = E4M3 (kind::f8f6f4) or F16 (kind::f16), 1 = BF16,
  // 2 = TF32 (kind::tf32)
  static constexpr uint32_t kAFmt = (MODE == TC_FP8 || MODE == TC_F16) ? 0u : (kTf32 ? 2u : 1u);
  // Leading byte offset of the MN-major Bt operand: the distance between its
  // 128-byte-wide n groups (one TMA box each).  With a single group (FP8) the
  // field is unused; 1024 keeps every address inside the stage either way.
  static constexpr uint32_t kBtLBO = (kNBoxes > 1) ? kBK * 128 : 1024;
  // TF32 operands must be K-major on the tensor core (measured: an MN-major
  // TF32 operand reads wrong elements): B arrives transposed (n x k) from the
  // rounding pre-pass and its tile is staged like A's, 128 n-rows of 128 bytes.
  static constexpr bool kBtKMajor = kTf32;
  // One-plane 8- and 16-bit modes take either operand in either major order
  // straight from the caller's storage (the INT8 and split modes stage
  // converted row-major planes instead).
  static constexpr bool kTransOk = kPlanes == 1 && !kTf32 && MODE != TC_I8EMU;
};

template <int BM_T, int STAGES, int MODE, int CG = 1, bool FUSED = false, bool RAW8 = false>
struct TcConfig {
  using T = TcTraits<MODE>;
  static constexpr uint32_t kABytes = BM_T * 128 / CG;                 // this CTA's rows of A x 128 B
  static constexpr uint32_t kPlaneBytes = T::kBtBytes + kABytes;       // one plane of a stage
  static constexpr uint32_t kStageBytes = T::kPlanes * kPlaneBytes;
  // The tensor core adds each MMA's products to its FP32 accumulator with
  // truncation, so the FP32-accurate mode keeps the hi*hi products and the
  // hi*lo + lo*hi corrections in separate accumulators (one third of the
  // truncating updates each for the large term) and adds them, rounded to
  // nearest, in the epilogue.  Accumulator sets are multi-buffered across
  // output tiles as far as TMEM (512 columns) allows, up to kMaxBufs, so that
  // the MMA can run several short tiles ahead of the epilogue.
  static constexpr uint32_t kAccPerTile = (MODE == TC_3XBF16 || MODE == TC_6XBF16 || MODE == TC_3XTF32) ? 2 : 1;
  static constexpr uint32_t kSetCols = kAccPerTile * BM_T;
  static constexpr uint32_t kMaxBufs = 4;
  static constexpr uint32_t kNumBufs = (512 / kSetCols) < kMaxBufs ? (512 / kSetCols) : kMaxBufs;
  static constexpr uint32_t kTmemCols = kNumBufs * kSetCols;
  // Epilogue warps: one per TMEM lane quarter, each thread owning all bm rows
  // of its column -- except the exact-integer member with bm = 256, whose
  // int32 running sums (one per row of the thread's column) live in
  // registers: sixteen warps (four per lane quarter, 64 rows each) keep them
  // within the 96 registers an 18-warp CTA allows, and TMEM holds two chunk
  // accumulators, so the drain of one 1024-product chunk overlaps the MMAs of
  // the next.  (Earlier designs with the sums in TMEM beside a single chunk
  // accumulator made the MMA wait at every chunk: 0.74 of the peak against
  // 0.93 now; eight warps with 128 register sums spilled.)
  static constexpr int kEpiWarps = (MODE == TC_I8EMU && BM_T == 256) ? 16 : 4;
  static constexpr int kEpiRows = BM_T / (kEpiWarps / 4);   // rows of the tile per epilogue thread
  // Loader-converter warps of the FUSED members: two groups of eight, each
  // group filling alternate k-blocks (one group's loads are in flight while
  // the other splits and stores).  The loads in flight are bounded by the
  // registers that hold them: six runs of eight per thread here (measured:
  // 0.75 ms for the 1000-problem batch against 1.20 ms with groups of four
  // and twelve runs per thread, which spill).
  // RAW8: one group of eight converter warps (measured on the 20 im2col
  // layers: 0.302 ms against 0.338 with four and ~0.5 with two).
  static constexpr int kConvWarpsPerGroup = 8;
  static constexpr int kConvWarps = FUSED ? 2 * kConvWarpsPerGroup : (RAW8 ? kConvWarpsPerGroup : 0);
  // RAW8 members: a ring of raw int8 tiles (bm rows x 64 bytes of A, 64
  // k-rows x 128 bytes of B per k-block) between the TMA and the converters.
  static constexpr int kRawStages = RAW8 ? 4 : 0;
  static constexpr uint32_t kRawBytes = RAW8 ? (uint32_t)(BM_T * 64 + 64 * 128) : 0u;
  // Epilogue staging for TMA stores of C: two buffers of 32 rows x 128
  // columns x 4 bytes (none for the FUSED members, whose grouped launches
  // write C with plain stores).
  static constexpr uint32_t kCStageBytes = FUSED ? 0 : 2 * 32 * 128 * 4;
  static constexpr uint32_t kBarBytes = 256;
  // Entries of the claimed-tile queue (tile number + full / empty barriers);
  // the RAW8 and FUSED members always walk statically.
  static constexpr int kTileQ = (RAW8 || FUSED) ? 0 : 2;
  static constexpr uint32_t kSmemBytes = 1024 + STAGES * kStageBytes + kRawStages * kRawBytes + kCStageBytes + kBarBytes;
  static constexpr int kThreads = 64 + 32 * kEpiWarps + 32 * kConvWarps;
  static_assert(BM_T == 64 || BM_T == 128 || BM_T == 256, "MMA N must be 64, 128 or 256");
  static_assert(CG == 1 || CG == 2, "one CTA or a CTA pair");
  static_assert(kNumBufs >= 1, "TMEM budget");
  static_assert(kSmemBytes <= 232448, "shared memory budget");
  static_assert((kTmemCols & (kTmemCols - 1)) == 0 && kTmemCols >= 32 && kTmemCols <= 512, "TMEM allocation");
  static_assert(8 * (2 * STAGES + 2 * kMaxBufs + 1) + 8 + 16 * kRawStages + 20 * kTileQ <= (int)kBarBytes,
                "barrier area");
  static_assert(!RAW8 || (MODE == TC_I8EMU && CG == 1 && BM_T <= 128 && !FUSED),
                "raw int8 staging: single-CTA INT8 members of at most 128 rows");
  static_assert(!FUSED || (CG == 1 && BM_T == 64 && (MODE == TC_3XBF16 || MODE == TC_6XBF16)),
                "in-kernel split: single-CTA FP32-accurate members with 64-row tiles");
};

// One output tile: rows m0 .. m0+bm-1, columns n0 .. n0+127 of problem g, k-blocks kb0 .. kb1-1.
struct TileJob {
  int m0, n0, kb0, kb1, bm, split, g;
  int kchunk;   // k-blocks per accumulation chunk, 0 = one chunk
  int sk;       // 1: a stream-K segment (split = its partial slot); kb0 == kb1: nothing to do
};

// Where and how a tile's result is written.
struct EpiJob {
  void* C;
  long long ldc;
  int m, n;
  float alpha, beta;
  int out_mode;
  // OUT_PARTIAL: element (i, j) of C's partial result goes to partial[i * ldp + j]
  // (split-K: this split's m x n plane, ldp = n; stream-K: a bm x 128*CG slot,
  // addressed through a base shifted back by the tile's origin)
  float* partial;
  const CUtensorMap* cmap;    // non-null: store C (beta == 0) or the partial tile by TMA through this map
  long long ldp;
  int cz;                     // >= 0: cmap is 3-D (split-K partial planes) and this is the tile's plane
};

// Stream-K work item u (>= 0) of the tail: segment u / streams of stream
// u % streams as (tile row, tile column, k-blocks [kb0, kb1), slot); kb0 ==
// kb1 when that stream has no such segment.  Kept out of line: its 64-bit
// divisions would otherwise add to the register pressure of the epilogue.
static __device__ __noinline__ int4 stream_k_item(const TcParams* p, int u, int* slot) {
  const int c = u % p->sk_streams, jseg = u / p->sk_streams;
  const StreamK sk{(long long)p->sk_tail * p->num_kb, p->sk_streams, p->num_kb};
  int tt = 0, kb0 = 0, kb1 = 0;
  if (!sk.segment(c, jseg, tt, kb0, kb1)) return make_int4(0, 0, 0, 0);
  int tm, tn;
  raster_tile(p->sk_dp + tt, p->tiles_m, p->tiles_n, p->raster, tm, tn);
  *slot = c * p->sk_segs + jseg;
  return make_int4(tm, tn, kb0, kb1);
}

// Whether a member takes a stream-K tail: all but the exact-integer members,
// whose int32 running sums fill the epilogue's registers (64 or 128 per
// thread) and leave none to spare for per-tile output descriptors.
template <int BM_T, int MODE>
struct TcStreamK {
  static constexpr bool value = MODE != TC_I8EMU;
};

template <int BM_T, int CG = 1, bool kStreamK = true>
struct SingleSched {
  const TcParams* p;
  const CUtensorMap* maps[kMapsPerProblem];   // A, B of planes 0..2 (kernel parameters)
  const CUtensorMap* cmap;      // C for TMA stores, or null
  int n_off;                    // 128 * (rank in the CTA pair): this CTA's columns of a pair tile

  // Work items: tiles x splits; with a stream-K tail, the sk_dp whole tiles
  // and then sk_segs segment slots per stream (item sk_dp + j * sk_streams + c
  // is segment j of stream c, so the persistent CTA c walks exactly its own
  // stream when the grid holds sk_streams CTAs or pairs).
  __device__ __forceinline__ int total() const {
    return kStreamK && p->sk_streams > 0 ? p->sk_dp + p->sk_streams * p->sk_segs
                                         : p->tiles_m * p->tiles_n * p->splits;
  }
  // counter of the claimed walk, or null for the static walk
  __device__ __forceinline__ int* claim_ctr() const {
    return kStreamK && p->sk_streams > 0 ? nullptr : p->tile_ctr;
  }

  __device__ __forceinline__ TileJob tile(int t) const {
    int tm, tn;
    if (kStreamK && p->sk_streams > 0 && t >= p->sk_dp) {
      int slot = 0;
      const int4 w = stream_k_item(p, t - p->sk_dp, &slot);
      return TileJob{w.x * BM_T, w.y * (128 * CG) + n_off, w.z, w.w, BM_T, slot, 0, p->kchunk, 1};
    }
    const int per_split = p->tiles_m * p->tiles_n;
    const int s = t / per_split;
    raster_tile(t - s * per_split, p->tiles_m, p->tiles_n, p->raster, tm, tn);
    const int kb0 = s * p->kb_per_split;
    return TileJob{tm * BM_T, tn * (128 * CG) + n_off, kb0, min(p->num_kb, kb0 + p->kb_per_split), BM_T, s, 0,
                   p->kchunk, 0};
  }

  __device__ __forceinline__ const CUtensorMap* map(const TileJob&, int which) const { return maps[which]; }

  __device__ __forceinline__ EpiJob epi(const TileJob& j) const {
    if (kStreamK && j.sk) {   // a stream-K segment: its partial tile, (bm rows) x (128 * CG columns)
      constexpr long long ldp = 128 * CG;
      const uintptr_t slot = reinterpret_cast<uintptr_t>(p->partial + (long long)j.split * (BM_T * ldp));
      const long long origin = (long long)j.m0 * ldp + (j.n0 - n_off);   // the slot holds elements from here on
      return EpiJob{p->C, p->ldc, p->m, p->n, p->alpha, p->beta, OUT_PARTIAL,
                    reinterpret_cast<float*>(slot - (uintptr_t)origin * sizeof(float)), nullptr, ldp, -1};
    }
    const bool part = p->out_mode == OUT_PARTIAL;
    return EpiJob{p->C, p->ldc, p->m, p->n, p->alpha, p->beta, p->out_mode,
                  part ? p->partial + (long long)j.split * p->m * p->ldp : nullptr, cmap, p->ldp,
                  part ? j.split : -1};
  }

  __device__ __forceinline__ bool conv() const { return p->conv != 0; }
  __device__ __forceinline__ bool a_mn() const { return p->a_mn != 0; }
  __device__ __forceinline__ bool b_km() const { return p->b_km != 0; }
  // im2col coordinates of k-block kb for the A rows starting at output pixel `pix`
  __device__ __forceinline__ void conv_coords(int pix, int kb, int (&xyzw)[4], uint16_t (&off)[2]) const {
    const int n = pix / p->conv_pq;
    const int rem = pix - n * p->conv_pq;
    const int pp = rem / p->conv_q;
    const int qq = rem - pp * p->conv_q;
    const int rs = kb / p->conv_cblocks;
    const int cb = kb - rs * p->conv_cblocks;
    const int r = rs / p->conv_s;
    const int s = rs - r * p->conv_s;
    xyzw[0] = cb * 64;
    xyzw[1] = qq * p->conv_sw - p->conv_pw;
    xyzw[2] = pp * p->conv_sh - p->conv_ph;
    xyzw[3] = n;
    off[0] = static_cast<uint16_t>(s * p->conv_dw);
    off[1] = static_cast<uint16_t>(r * p->conv_dh);
  }
};

struct GroupedSched {
  const GroupedParams* gp;

  __device__ __forceinline__ int total() const { return gp->total_tiles; }
  __device__ __forceinline__ int* claim_ctr() const { return nullptr; }   // grouped launches walk statically

  __device__ __forceinline__ TileJob tile(int t) const {
    const int2 ti = __ldg(gp->tile_info + t);
    const int g = ti.x;
    const GroupDesc* d = gp->groups + g;
    const int tm = ti.y % d->tiles_m, tn = ti.y / d->tiles_m;
    return TileJob{tm * d->bm, tn * 128, 0, d->num_kb, d->bm, 0, g, 0, 0};
  }

  __device__ __forceinline__ const CUtensorMap* map(const TileJob& j, int which) const {
    return gp->maps + kMapsPerProblem * j.g + which;
  }

  __device__ __forceinline__ EpiJob epi(const TileJob& j) const {
    const GroupDesc* d = gp->groups + j.g;
    return EpiJob{d->C, d->ldc, d->m, d->n, d->alpha, d->beta, OUT_F32, nullptr, nullptr, 0, -1};
  }

  __device__ __forceinline__ const GroupDesc* desc(const TileJob& j) const { return gp->groups + j.g; }

  __device__ __forceinline__ bool conv() const { return false; }
  __device__ __forceinline__ bool a_mn() const { return false; }
  __device__ __forceinline__ bool b_km() const { return false; }
  __device__ __forceinline__ void conv_coords(int, int, int (&)[4], uint16_t (&)[2]) const {}
};

// Shared::cluster address of a barrier of the pair's leader (CTA pairs), or
// the local barrier's address.
template <bool kPair>
__device__ __forceinline__ uint32_t mapa_or_local(uint64_t* bar) {
  return kPair ? mapa_shared(smem_u32(bar), 0) : smem_u32(bar);
}

// Eight consecutive FP32 elements x[row][col0 .. col0+7] of a row-major
// matrix (rows x cols, leading dimension ld) into v, zeros outside it; the
// widest loads the address allows.
__device__ __forceinline__ void load_run8(const float* __restrict__ x, long long ld, int row, int rows, int col0,
                                          int cols, float (&v)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = 0.0f;
  if (row >= rows || col0 >= cols) return;
  const float* p = x + (long long)row * ld + col0;
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  if (col0 + 8 <= cols && (a & 15u) == 0) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    const float4 w = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w; v[4] = w.x; v[5] = w.y; v[6] = w.z; v[7] = w.w;
  } else if (col0 + 8 <= cols && (a & 7u) == 0) {
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const float2 u = __ldg(reinterpret_cast<const float2*>(p + e));
      v[e] = u.x;
      v[e + 1] = u.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (col0 + e < cols) v[e] = __ldg(p + e);
  }
}

// Eight int8 values (8 bytes) as IEEE binary16, exact, in one 16-byte row
// chunk at dst, two values per instruction: each byte, biased by 128, becomes
// the low mantissa byte of 1024 in a half2 (one byte permute per pair), and
// one packed subtraction of 1024 + 128 leaves the pair exactly (|x| <= 128
// needs 8 of binary16's 11 significant bits).
__device__ __forceinline__ void store_i8_as_f16(uint8_t* dst, const uint2& v) {
  const uint32_t b[2] = {v.x ^ 0x80808080u, v.y ^ 0x80808080u};
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t biased = __byte_perm(b[q >> 1], 0x64646464u, (q & 1) ? 0x4342u : 0x4140u);
    asm("sub.f16x2 %0, %1, %2;" : "=r"(w[q]) : "r"(biased), "r"(0x64806480u));
  }
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// The bfloat16 parts of eight FP32 values -- hi = bf16(x), then lo =
// bf16(x - hi) (two planes) or mid = bf16(x - hi), lo = bf16((x - hi) - mid)
// (three planes), the split pre-pass's arithmetic -- as one 16-byte row
// chunk per plane at dst, dst + plane_bytes, ...
template <int PLANES>
__device__ __forceinline__ void store_split8(uint8_t* dst, uint32_t plane_bytes, const float (&v)[8]) {
  uint32_t w[PLANES][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint16_t h[2], m[2], l[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      h[q] = bf16_bits(v[e + q]);
      const float d = v[e + q] - bf16_value(h[q]);
      m[q] = bf16_bits(d);
      l[q] = bf16_bits(d - bf16_value(m[q]));
    }
    w[0][e / 2] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    w[1][e / 2] = (uint32_t)m[0] | ((uint32_t)m[1] << 16);   // two planes: lo = bf16(x - hi); three: mid
    if constexpr (PLANES == 3) w[2][e / 2] = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
  }
#pragma unroll
  for (int p = 0; p < PLANES; ++p)
    *reinterpret_cast<uint4*>(dst + p * plane_bytes) = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

template <int BM_T, int STAGES, int MODE, int CG, class Sched, bool FUSED = false, bool RAW8 = false>
__device__ __forceinline__ void tc_gemm_body(const Sched& S, unsigned long long timeout_ns, int* status,
                                             int debug_withhold, const float* scale_a, const float* scale_b) {
  using T = TcTraits<MODE>;
  using Cfg = TcConfig<BM_T, STAGES, MODE, CG, FUSED, RAW8>;
  constexpr bool kPair = (CG == 2);
  // INT8 members sum k in exact chunks of at most 1024 products, added in
  // int32 registers by the epilogue; RAW8 members instead keep every tile's
  // k range (every split) within one chunk, so their FP32 accumulator is exact
  // as it stands and the epilogue converts it to int32 once.
  constexpr bool kIntChunked = (MODE == TC_I8EMU) && !RAW8;
  constexpr bool kIntOut = (MODE == TC_I8EMU);
  static_assert(!kIntChunked || Cfg::kEpiRows <= 128,
                "int32 running sums in registers: <= 128 rows");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* ring8 = smem + STAGES * Cfg::kStageBytes;   // RAW8: the int8 ring
  float* cstage = reinterpret_cast<float*>(ring8 + Cfg::kRawStages * Cfg::kRawBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring8 + Cfg::kRawStages * Cfg::kRawBytes + Cfg::kCStageBytes);
  uint64_t* empty = full + STAGES;
  uint64_t* tmem_full = empty + STAGES;
  uint64_t* tmem_empty = tmem_full + Cfg::kMaxBufs;
  uint64_t* drain = tmem_empty + Cfg::kMaxBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint64_t* raw_full = reinterpret_cast<uint64_t*>(tmem_slot + 2);   // RAW8 only
  uint64_t* raw_empty = raw_full + Cfg::kRawStages;
  uint64_t* tq_full = raw_empty + Cfg::kRawStages;   // claimed-tile queue
  uint64_t* tq_empty = tq_full + Cfg::kTileQ;
  volatile int* tq = reinterpret_cast<volatile int*>(tq_empty + Cfg::kTileQ);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = kPair ? cluster_ctarank() : 0u;   // 0: the pair's leader (or a lone CTA)
  const bool leader = rank == 0;
  const int first_tile = blockIdx.x / CG;                 // tiles are walked per cluster
  const int tile_stride = gridDim.x / CG;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      // FUSED: the group's warps arrive; RAW8: the converter warps
      mbar_init(&full[s], (FUSED || RAW8) ? Cfg::kConvWarpsPerGroup : 1);
      mbar_init(&empty[s], 1);
    }
    for (int r = 0; r < Cfg::kRawStages; ++r) {
      mbar_init(&raw_full[r], 1);
      mbar_init(&raw_empty[r], Cfg::kConvWarpsPerGroup);
    }
    for (int a = 0; a < (int)Cfg::kNumBufs; ++a) {
      mbar_init(&tmem_full[a], 1);
      mbar_init(&tmem_empty[a], CG * Cfg::kEpiWarps);   // the epilogue warps of every CTA of the pair
    }
    for (int q = 0; q < Cfg::kTileQ; ++q) {
      mbar_init(&tq_full[q], 1);   // the leader's producer publishes
      // read by the MMA issuer (leader) or producer (peer) and the epilogue
      // warps of every CTA of the pair; only the leader's barrier is used
      mbar_init(&tq_empty[q], CG * (1 + Cfg::kEpiWarps));
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc<CG>(tmem_slot, Cfg::kTmemCols);
    tmem_relinquish<CG>();
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (kPair) cluster_sync();   // the peer's barriers are initialised before any remote arrive
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  bool pair_ok = true;
  if constexpr (kPair) {
    // the pair's MMAs write the same TMEM address in both CTAs
    const uint32_t peer_base = ld_shared_cluster_u32(mapa_shared(smem_u32(tmem_slot), rank ^ 1u));
    pair_ok = peer_base == tmem_base;
    if (!pair_ok && threadIdx.x == 0) atomicCAS(status, 0, WD_PAIR_TMEM);
  }
  // Programmatic dependent launch: the set-up above overlaps the tail of the
  // previous kernel in the stream; wait for that kernel (and its memory) before
  // any global access, and let the next kernel start its own set-up.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  Watchdog wd{timeout_ns, status, abort_flag};
  const int total_tiles = pair_ok ? S.total() : 0;

  // Tile walk.  Static: this CTA's (pair's) first tile, then every
  // tile_stride-th work item.  Claimed (a counter from the host, zeroed
  // before the launch): the first tile as above, each further one claimed
  // from the counter by the pair leader's producer as it moves on, so the
  // tiles in flight are always the most recently claimed -- neighbours in
  // the banded raster, whose panels of A and B are then read from L2 at
  // about the same time however far the CTAs of a long launch drift apart.
  // The producer hands each claimed number to the other roles, and to the
  // peer CTA of a pair, through a kTileQ-entry queue in shared memory.
  int* const claim_ctr = Cfg::kTileQ > 0 ? S.claim_ctr() : nullptr;
  // role 0: the claimer (leader's producer); 1: one thread of a warp; 2: a whole warp
  auto next_tile = [&](int t, uint32_t& qn, int role) -> int {
    if constexpr (Cfg::kTileQ == 0) {
      return t + tile_stride;
    } else {
      if (claim_ctr == nullptr) return t + tile_stride;
      const uint32_t slot = qn % (uint32_t)Cfg::kTileQ, ph = (qn / (uint32_t)Cfg::kTileQ) & 1u;
      ++qn;
      if (role == 0) {
        if (!wait_parity<kPair>(&tq_empty[slot], ph ^ 1u, wd, WD_TILE_QUEUE)) return total_tiles;
        const int nt = tile_stride + atomicAdd(claim_ctr, 1);
        tq[slot] = nt;
        if constexpr (kPair) {
          st_shared_cluster_u32(mapa_shared(smem_u32(const_cast<int*>(&tq[slot])), 1u), (uint32_t)nt);
          mbar_arrive_cluster(mapa_shared(smem_u32(&tq_full[slot]), 1u));
        }
        mbar_arrive(&tq_full[slot]);
        return nt;
      }
      bool got = wait_parity<kPair>(&tq_full[slot], ph, wd, WD_TILE_QUEUE);
      if (role == 2) got = __all_sync(0xffffffffu, got);
      if (!got) return total_tiles;
      const int nt = tq[slot];
      if (role == 2) __syncwarp();   // every lane has read the entry before it is released
      if (role == 1 || lane == 0) {
        if constexpr (kPair) mbar_arrive_cluster(mapa_shared(smem_u32(&tq_empty[slot]), 0u));
        else mbar_arrive(&tq_empty[slot]);
      }
      return nt;
    }
  };
  // Operand layouts of this launch.  Bt (the instruction's A, 128*CG columns
  // of C) is MN-major when B is stored k x n, K-major when stored n x k (and
  // always for TF32).  The A tile (the instruction's B, bm rows of C) is
  // K-major when A is stored m x k, MN-major when stored k x m: boxes of
  // kBoxN rows of C x BK, which need this CTA's bm/CG rows to fill whole
  // 128-byte swizzle rows (the host never sets a_mn otherwise).
  constexpr int kAmnBoxes = (BM_T / CG) / T::kBoxN;
  const bool bt_km = T::kBtKMajor || (T::kTransOk && S.b_km());
  const bool a_mn = T::kTransOk && kAmnBoxes >= 1 && S.a_mn();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (RAW8 && lane == 0) {
      // raw int8 boxes: A (64 bytes of k x bm rows) and B (128 columns x 64
      // k-rows), unswizzled, into the raw ring
      uint32_t it = 0;
      bool ok = true;
      for (int t = first_tile; ok && t < total_tiles; t += tile_stride) {
        const TileJob j = S.tile(t);
        if (j.kb1 <= j.kb0) continue;
        for (int kb = j.kb0; kb < j.kb1; ++kb, ++it) {
          const uint32_t rs = it % Cfg::kRawStages, rph = (it / Cfg::kRawStages) & 1u;
          if (!wait_parity(&raw_empty[rs], rph ^ 1u, wd, WD_PRODUCER_EMPTY)) { ok = false; break; }
          if ((int)it == debug_withhold) continue;   // failure-detection test: never arrive
          mbar_arrive_expect_tx(&raw_full[rs], Cfg::kRawBytes);
          uint8_t* rb = ring8 + rs * Cfg::kRawBytes;
          tma_load_2d(rb, S.map(j, 0), kb * 64, j.m0, &raw_full[rs]);
          tma_load_2d(rb + BM_T * 64, S.map(j, 1), j.n0, kb * 64, &raw_full[rs]);
        }
      }
      // the last raw loads have landed before the CTA can retire
      const uint32_t first = it > (uint32_t)Cfg::kRawStages ? it - Cfg::kRawStages : 0u;
      for (uint32_t q = first; q < it; ++q) {
        uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(&raw_full[q % Cfg::kRawStages], (q / Cfg::kRawStages) & 1u))
          if (globaltimer_ns() - t0 > timeout_ns) { atomicCAS(status, 0, WD_DRAIN); break; }
      }
    }
    if (!FUSED && !RAW8 && lane == 0) {
      uint32_t it = 0, qn = 0;
      bool ok = true;
      for (int t = first_tile; ok && t < total_tiles; t = next_tile(t, qn, leader ? 0 : 1)) {
        const TileJob j = S.tile(t);
        if (j.kb1 <= j.kb0) continue;   // an empty stream-K slot (every role skips it)
        // bytes this CTA stages per k-block; a pair's leader counts both CTAs'
        const uint32_t stage_bytes = T::kPlanes * (T::kBtBytes + (uint32_t)j.bm * 128u / CG);
        const int a_row = j.m0 + (int)rank * (j.bm / CG);
        for (int kb = j.kb0; kb < j.kb1; ++kb, ++it) {
          const uint32_t stage = it % STAGES, ph = (it / STAGES) & 1u;
          if (!wait_parity<kPair>(&empty[stage], ph ^ 1u, wd, WD_PRODUCER_EMPTY)) { ok = false; break; }
          if ((int)it == debug_withhold) continue;   // failure-detection test: never arrive
          if (leader) mbar_arrive_expect_tx(&full[stage], CG * stage_bytes);
          const uint32_t full_c = mapa_or_local<kPair>(&full[stage]);
          uint8_t* st = smem + stage * Cfg::kStageBytes;
          const int k0 = kb * T::kBK;
#pragma unroll
          for (int pl = 0; pl < T::kPlanes; ++pl) {
            uint8_t* bt = st + pl * Cfg::kPlaneBytes;
            uint8_t* at = bt + T::kBtBytes;
            const CUtensorMap* mb = S.map(j, 2 * pl + 1);
            const CUtensorMap* ma = S.map(j, 2 * pl);
            if (bt_km) {
              // B stored n x k: one box of 128 n-rows x kBK k
              if constexpr (kPair) tma_load_2d_pair(bt, mb, k0, j.n0, full_c);
              else tma_load_2d(bt, mb, k0, j.n0, &full[stage]);
            } else if constexpr (kPair) {
#pragma unroll
              for (int h = 0; h < T::kNBoxes; ++h)
                tma_load_2d_pair(bt + h * (T::kBK * 128), mb, j.n0 + h * T::kBoxN, k0, full_c);
            } else {
#pragma unroll
              for (int h = 0; h < T::kNBoxes; ++h)
                tma_load_2d(bt + h * (T::kBK * 128), mb, j.n0 + h * T::kBoxN, k0, &full[stage]);
            }
            if (T::kElem == 2 && S.conv()) {   // implicit GEMM: im2col rows of the activations
              int xyzw[4];
              uint16_t off[2];
              S.conv_coords(a_row, kb, xyzw, off);
              if constexpr (kPair)
                tma_load_im2col_4d_pair(at, ma, xyzw[0], xyzw[1], xyzw[2], xyzw[3], off[0], off[1], full_c);
              else
                tma_load_im2col_4d(at, ma, xyzw[0], xyzw[1], xyzw[2], xyzw[3], off[0], off[1], &full[stage]);
            } else if (a_mn) {
              // A stored k x m: kAmnBoxes boxes of kBoxN rows of C x kBK k
#pragma unroll
              for (int h = 0; h < kAmnBoxes; ++h) {
                if constexpr (kPair) tma_load_2d_pair(at + h * (T::kBK * 128), ma, a_row + h * T::kBoxN, k0, full_c);
                else tma_load_2d(at + h * (T::kBK * 128), ma, a_row + h * T::kBoxN, k0, &full[stage]);
              }
            } else if constexpr (kPair) {
              tma_load_2d_pair(at, ma, k0, a_row, full_c);
            } else {
              tma_load_2d(at, ma, k0, a_row, &full[stage]);
            }
          }
        }
      }
      // Let every load already issued land before the CTA can retire (a pair's
      // loads all complete on the leader's barriers; the closing cluster
      // barrier orders the other CTA after them).
      const uint32_t first = !leader ? it : (it > (uint32_t)STAGES ? it - STAGES : 0u);
      for (uint32_t q = first; q < it; ++q) {
        uint64_t t0 = globaltimer_ns();
        while (!(kPair ? mbar_try_wait_cluster(&full[q % STAGES], (q / STAGES) & 1u)
                       : mbar_try_wait(&full[q % STAGES], (q / STAGES) & 1u)))
          if (globaltimer_ns() - t0 > timeout_ns) { atomicCAS(status, 0, WD_DRAIN); break; }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && leader) {
      uint32_t it = 0, lt = 0;   // lt counts accumulation chunks (one per tile unless k is chunked)
      bool ok = true;
      // commits of a pair arrive on the barrier of both CTAs
      auto commit = [&](uint64_t* bar) {
        if constexpr (kPair) mma_commit_pair(bar, 0x3);
        else mma_commit(bar);
      };
      uint32_t qn = 0;
      for (int t = first_tile; ok && t < total_tiles; t = next_tile(t, qn, 1)) {
        const TileJob j = S.tile(t);
        if (j.kb1 <= j.kb0) continue;
        // RAW8 stages hold binary16 (exact int8 values), the others T's format
        constexpr uint32_t kFmt = RAW8 ? 0u : T::kAFmt;
        const uint32_t idesc = make_idesc(kFmt, kFmt, /*a_mn=*/!bt_km, /*b_mn=*/a_mn, 128 * CG, j.bm);
        const int span = j.kchunk > 0 ? j.kchunk : j.kb1 - j.kb0;
        for (int c0 = j.kb0; ok && c0 < j.kb1; c0 += span, ++lt) {
        const int c1 = min(j.kb1, c0 + span);
        const uint32_t acc = lt % Cfg::kNumBufs, aph = (lt / Cfg::kNumBufs) & 1u;
        if (!wait_parity<kPair>(&tmem_empty[acc], aph ^ 1u, wd, WD_MMA_TMEM_EMPTY)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * Cfg::kSetCols;   // main accumulator
        const uint32_t d_corr = d_tmem + BM_T;                       // 3xBF16 corrections
        uint32_t accumulate = 0;
        for (int kb = c0; kb < c1; ++kb, ++it) {
          const uint32_t stage = it % STAGES, ph = (it / STAGES) & 1u;
          if (!wait_parity<kPair>(&full[stage], ph, wd, WD_MMA_FULL)) { ok = false; break; }
          tc_fence_after();
          const uint32_t st = smem_u32(smem + stage * Cfg::kStageBytes);
#pragma unroll
          for (int ks = 0; ks < T::kKSteps; ++ks) {
            // MN-major operand: a k-step is kKStep whole 128-byte rows (kKStep/8
            // atoms); LBO = distance between its 128-byte-wide boxes, SBO = 8 rows.
            // K-major operand: a k-step is 32 bytes inside the swizzled 128-byte row.
            const uint32_t bt_off = bt_km ? ks * 32 : ks * T::kKStep * 128;
            const uint32_t a_off = T::kBtBytes + (a_mn ? ks * T::kKStep * 128 : ks * 32);
            const uint64_t bt_hi = bt_km ? smem_desc_sw128(st + bt_off, 16, 1024)
                                         : smem_desc_sw128(st + bt_off, T::kBtLBO, 1024);
            const uint64_t a_hi = a_mn ? smem_desc_sw128(st + a_off, T::kBK * 128, 1024)
                                       : smem_desc_sw128(st + a_off, 16, 1024);
            if (MODE == TC_3XBF16) {
              const uint32_t lo = Cfg::kPlaneBytes;
              const uint64_t bt_lo = smem_desc_sw128(st + lo + bt_off, T::kBtLBO, 1024);
              const uint64_t a_lo = smem_desc_sw128(st + lo + a_off, 16, 1024);
              // corrections Bhi*Alo + Blo*Ahi in their own accumulator, then the
              // main term Bhi*Ahi; Blo*Alo is dropped
              mma_f16<CG>(d_corr, bt_hi, a_lo, idesc, accumulate);
              mma_f16<CG>(d_corr, bt_lo, a_hi, idesc, 1u);
              mma_f16<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            } else if (MODE == TC_6XBF16) {
              const uint32_t p1 = Cfg::kPlaneBytes, p2 = 2 * Cfg::kPlaneBytes;
              const uint64_t bt_mid = smem_desc_sw128(st + p1 + bt_off, T::kBtLBO, 1024);
              const uint64_t a_mid = smem_desc_sw128(st + p1 + a_off, 16, 1024);
              const uint64_t bt_lo = smem_desc_sw128(st + p2 + bt_off, T::kBtLBO, 1024);
              const uint64_t a_lo = smem_desc_sw128(st + p2 + a_off, 16, 1024);
              // corrections hi*mid + mid*hi + hi*lo + lo*hi + mid*mid, then hi*hi;
              // mid*lo, lo*mid and lo*lo (<= 2^-23 relative) are dropped
              mma_f16<CG>(d_corr, bt_hi, a_mid, idesc, accumulate);
              mma_f16<CG>(d_corr, bt_mid, a_hi, idesc, 1u);
              mma_f16<CG>(d_corr, bt_hi, a_lo, idesc, 1u);
              mma_f16<CG>(d_corr, bt_lo, a_hi, idesc, 1u);
              mma_f16<CG>(d_corr, bt_mid, a_mid, idesc, 1u);
              mma_f16<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            } else if (MODE == TC_3XTF32) {
              // both planes K-major (TF32): Bhi*Alo + Blo*Ahi into the
              // corrections, then Bhi*Ahi; Blo*Alo is dropped
              const uint32_t lo = Cfg::kPlaneBytes;
              const uint64_t bt_lo = smem_desc_sw128(st + lo + bt_off, 16, 1024);
              const uint64_t a_lo = smem_desc_sw128(st + lo + a_off, 16, 1024);
              mma_tf32<CG>(d_corr, bt_hi, a_lo, idesc, accumulate);
              mma_tf32<CG>(d_corr, bt_lo, a_hi, idesc, 1u);
              mma_tf32<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            } else if (MODE == TC_FP8) {
              mma_f8<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            } else if (MODE == TC_TF32) {
              mma_tf32<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            } else {
              mma_f16<CG>(d_tmem, bt_hi, a_hi, idesc, accumulate);
            }
            accumulate = 1u;
          }
          commit(&empty[stage]);   // frees the stage when these MMAs finish
        }
        if (!ok) break;
        commit(&tmem_full[acc]);   // accumulator ready for the epilogue
        }
      }
      // Make sure no MMA is in flight before TMEM is released.
      mma_commit<CG>(drain);
      uint64_t t0 = globaltimer_ns();
      while (!mbar_try_wait(drain, 0))
        if (globaltimer_ns() - t0 > timeout_ns) { atomicCAS(status, 0, WD_DRAIN); break; }
    }
  } else if (warp < 2 + Cfg::kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                  // TMEM lane quarter this warp may access
    float scale = 1.0f;
    if (MODE == TC_FP8) {
      const float sa = scale_a ? *scale_a : 1.0f;
      const float sb = scale_b ? *scale_b : 1.0f;
      scale = sa * sb;
    }
    uint32_t lt = 0;   // accumulation chunks consumed, in the MMA issuer's order
    uint32_t schunk = 0;   // 32-row chunks staged for TMA stores (selects the staging buffer)
    bool alive = true;
    uint32_t qn = 0;
    for (int t = first_tile; alive && t < total_tiles; t = next_tile(t, qn, 2)) {
      const TileJob j = S.tile(t);
      if (j.kb1 <= j.kb0) continue;
      const EpiJob e = S.epi(j);
      const float alpha = e.alpha * scale;
      const float beta = e.beta;
      const int col = j.n0 + q * 32 + lane;               // column of C owned by this thread
      const bool cok = col < e.n;
      const int rows_here = min(j.bm, e.m - j.m0);
      const int nchunks = (rows_here + 31) >> 5;
      const int span = j.kchunk > 0 ? j.kchunk : j.kb1 - j.kb0;
      const int nkc = (j.kb1 - j.kb0 + span - 1) / span;
      // Outputs that do not read C -- C with beta == 0, or a split's partial
      // tile -- leave through shared memory and TMA stores (whole 32 x 128
      // boxes, clipped to C or to the split's plane by the tensor map).
      // (staging assumes the four epilogue warps cover the same rows)
      const bool use_tma = e.cmap != nullptr && Cfg::kEpiWarps == 4 &&
                           (e.out_mode == OUT_PARTIAL || (beta == 0.0f && (e.out_mode == OUT_F32 || e.out_mode == OUT_I32)));
      const int r0 = ((warp - 2) >> 2) * Cfg::kEpiRows;   // first tile row of this thread's rows
      // stage_begin: a free staging buffer (the store issued from it two chunks
      // ago has read it); this thread's column of the 32 rows goes to
      // buf[i * 128 + q * 32 + lane]; stage_end: hand the box to the TMA unit.
      auto stage_begin = [&]() -> float* {
        if (threadIdx.x == 64) bulk_wait_group_read<1>();
        named_barrier_sync(1, 128);
        return cstage + (schunk & 1u) * (32 * 128) + q * 32 + lane;
      };
      auto stage_end = [&](int c) {
        fence_proxy_async_smem();
        named_barrier_sync(1, 128);
        if (threadIdx.x == 64) {
          if (e.cz >= 0) tma_store_3d(e.cmap, j.n0, j.m0 + c * 32, e.cz, cstage + (schunk & 1u) * (32 * 128));
          else tma_store_2d(e.cmap, j.n0, j.m0 + c * 32, cstage + (schunk & 1u) * (32 * 128));
          bulk_commit_group();
        }
        ++schunk;
      };
      // exact-integer mode: int32 running sums of this thread's column, one per
      // row r0 .. r0 + kEpiRows - 1 of the tile
      constexpr int kSums = kIntChunked ? Cfg::kEpiRows : 1;
      int isum[kSums];
#pragma unroll
      for (int i = 0; i < kSums; ++i) isum[i] = 0;
      const int rows_mine = min(Cfg::kEpiRows, rows_here - r0);            // may be <= 0
      const int nchunks_mine = rows_mine > 0 ? (rows_mine + 31) >> 5 : 0;
      for (int kc = 0; kc < nkc; ++kc, ++lt) {
      const uint32_t acc = lt % Cfg::kNumBufs, aph = (lt / Cfg::kNumBufs) & 1u;
      bool ok = wait_parity<kPair>(&tmem_full[acc], aph, wd, WD_EPI_TMEM_FULL);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        alive = false;
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem_base + (static_cast<uint32_t>(q * 32) << 16) + acc * Cfg::kSetCols;
      // Hand the accumulator set back to the MMA issuer once its last TMEM load completed.
      auto release = [&]() {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (kPair) mbar_arrive_cluster(mapa_shared(smem_u32(&tmem_empty[acc]), 0));
          else mbar_arrive(&tmem_empty[acc]);
        }
      };
      if constexpr (kIntChunked) {
        // Each chunk holds an integer-valued FP32 sum of at most 1024 products
        // of magnitude <= 2^14, hence exact; convert and add in int32.
        if constexpr (Cfg::kEpiWarps == 16) {
          // 64 sums per thread within the 96 registers of an 18-warp CTA:
          // 8-row blocks, one at a time (the other accumulator set keeps the
          // MMA busy meanwhile)
#pragma unroll
          for (int rc = 0; rc < Cfg::kEpiRows / 8; ++rc) {
            if (rc < 4 * nchunks_mine) {
              uint32_t rv[8];
              tmem_ld_32x32b_x8(tbase + r0 + rc * 8, rv);
              tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 8; ++i) isum[rc * 8 + i] += __float2int_rn(__uint_as_float(rv[i]));
            }
          }
        } else {
        // 16-row blocks, software-pipelined: block b+1 loads while b is added.
        constexpr int kBlocks = Cfg::kEpiRows / 16;   // even
        const int nb = 2 * nchunks_mine;
        uint32_t ra[16], rb[16];
        if (nb > 0) {
          tmem_ld_32x32b_x16(tbase + r0, ra);
          tmem_ld_wait();
        }
#pragma unroll
        for (int rc = 0; rc < kBlocks; rc += 2) {
          if (rc < nb) {
            const bool has_b = rc + 1 < nb;
            if (has_b) tmem_ld_32x32b_x16(tbase + r0 + (rc + 1) * 16, rb);
#pragma unroll
            for (int i = 0; i < 16; ++i) isum[rc * 16 + i] += __float2int_rn(__uint_as_float(ra[i]));
            if (has_b) {
              tmem_ld_wait();
              const bool has_a = rc + 2 < nb;
              if (has_a) tmem_ld_32x32b_x16(tbase + r0 + (rc + 2) * 16, ra);
#pragma unroll
              for (int i = 0; i < 16; ++i) isum[(rc + 1) * 16 + i] += __float2int_rn(__uint_as_float(rb[i]));
              if (has_a) tmem_ld_wait();
            }
          }
        }
        }
        release();
        if (kc == nkc - 1 && use_tma) {
#pragma unroll
          for (int rc = 0; rc < Cfg::kEpiRows / 32; ++rc) {
            if (rc < nchunks) {
              float* buf = stage_begin();
#pragma unroll
              for (int i = 0; i < 32; ++i) buf[i * 128] = __int_as_float(isum[rc * 32 + i]);
              stage_end(rc);
            }
          }
        } else if (kc == nkc - 1 && cok) {
          // One row after the other through a running pointer (the compiler
          // would otherwise keep an address per row live across the tile).
          const int i0 = j.m0 + r0;
          const bool partial = e.out_mode == OUT_PARTIAL;
          const long long ld = partial ? e.ldp : e.ldc;
          int* cp = partial ? reinterpret_cast<int*>(e.partial) + (long long)i0 * e.ldp + col
                            : static_cast<int*>(e.C) + (long long)i0 * e.ldc + col;
          const bool add_c = !partial && beta != 0.0f;
#pragma unroll
          for (int i = 0; i < Cfg::kEpiRows; ++i) {
            if (i < rows_mine) *cp = add_c ? *cp + isum[i] : isum[i];
            cp += ld;
            asm volatile("" ::: "memory");
          }
        }
      } else {
      // Rows i0 .. i0+31 of this thread's column: alpha/beta and the stores.
      auto store_chunk = [&](const uint32_t (&r)[32], int c) {
        if (use_tma) {
          float* buf = stage_begin();
          if (e.out_mode == OUT_I32) {
#pragma unroll
            for (int i = 0; i < 32; ++i) buf[i * 128] = __int_as_float(__float2int_rn(__uint_as_float(r[i])));
          } else if (e.out_mode == OUT_PARTIAL) {   // the raw sum: alpha is applied by the reduction
#pragma unroll
            for (int i = 0; i < 32; ++i)
              buf[i * 128] = kIntOut ? __int_as_float(__float2int_rn(__uint_as_float(r[i]))) : __uint_as_float(r[i]);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) buf[i * 128] = alpha * __uint_as_float(r[i]);
          }
          stage_end(c);
          return;
        }
        const int i0 = j.m0 + c * 32;
        const int iend = min(32, e.m - i0);
        if (cok) {
          if (e.out_mode == OUT_F32) {
            float* cp = static_cast<float*>(e.C) + (long long)i0 * e.ldc + col;
            if (beta != 0.0f) {
              // all 32 reads of C first (one memory round trip), then the stores
              float cv[32];
#pragma unroll
              for (int i = 0; i < 32; ++i) cv[i] = (i < iend) ? cp[i * e.ldc] : 0.0f;
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < iend) cp[i * e.ldc] = fmaf(alpha, __uint_as_float(r[i]), beta * cv[i]);
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < iend) cp[i * e.ldc] = alpha * __uint_as_float(r[i]);
            }
          } else if (e.out_mode == OUT_I32) {
            int* cp = static_cast<int*>(e.C) + (long long)i0 * e.ldc + col;
            int cv[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) cv[i] = (beta != 0.0f && i < iend) ? cp[i * e.ldc] : 0;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < iend) cp[i * e.ldc] = cv[i] + __float2int_rn(__uint_as_float(r[i]));
          } else {
            float* pp = e.partial + (long long)i0 * e.ldp + col;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (i < iend)
                pp[(long long)i * e.ldp] =
                    kIntOut ? __int_as_float(__float2int_rn(__uint_as_float(r[i]))) : __uint_as_float(r[i]);
          }
        }
      };
      if (MODE == TC_3XBF16 || MODE == TC_6XBF16 || MODE == TC_3XTF32) {
        for (int c = 0; c < nchunks; ++c) {
          uint32_t r[32], rc[32];
          tmem_ld_32x32b_x32(tbase + c * 32, r);
          tmem_ld_32x32b_x32(tbase + BM_T + c * 32, rc);
          tmem_ld_wait();
          if (c == nchunks - 1) release();
#pragma unroll
          for (int i = 0; i < 32; ++i)
            r[i] = __float_as_uint(__fadd_rn(__uint_as_float(r[i]), __uint_as_float(rc[i])));
          store_chunk(r, c);
        }
      } else if (RAW8) {
        // one 32-row chunk at a time: the RAW8 block's 448 threads get 128
        // registers each, and the pipelined form below spilled there
        // (measured on the im2col layers: 0.277 ms against 0.289)
        for (int c = 0; c < nchunks; ++c) {
          uint32_t r[32];
          tmem_ld_32x32b_x32(tbase + c * 32, r);
          tmem_ld_wait();
          if (c == nchunks - 1) release();
          store_chunk(r, c);
        }
      } else {
        // Software pipeline: the TMEM load of chunk c+1 is in flight while
        // chunk c is scaled and stored.
        uint32_t ra[32], rb[32];
        tmem_ld_32x32b_x32(tbase, ra);
        tmem_ld_wait();
        if (nchunks == 1) release();
        for (int c = 0; c < nchunks; c += 2) {
          const bool has_b = c + 1 < nchunks;
          if (has_b) tmem_ld_32x32b_x32(tbase + (c + 1) * 32, rb);
          store_chunk(ra, c);
          if (has_b) {
            tmem_ld_wait();
            if (c + 1 == nchunks - 1) release();
            const bool has_a = c + 2 < nchunks;
            if (has_a) tmem_ld_32x32b_x32(tbase + (c + 2) * 32, ra);
            store_chunk(rb, c + 1);
            if (has_a) {
              tmem_ld_wait();
              if (c + 2 == nchunks - 1) release();
            }
          }
        }
      }
      }   // float / 3xBF16 epilogue
      }   // accumulation chunks
    }
    if (threadIdx.x == 64) bulk_wait_group_all();   // every TMA store of C has completed
  } else if constexpr (RAW8) {
    // ------------------------------------------------------------ int8 converters
    // The converter warps turn each raw k-block into the stage's binary16 tile: run u of
    // eight int8 values -- A: row r = u / 8, bytes 8*(u % 8) of its 64; B:
    // k-row kk = u / 16, columns 8*(u % 16) of its 128 -- read from the raw
    // tile and stored as binary16 where TMA puts the 16-bit operands (A: row r, chunk c at
    // c ^ (r % 8); B: box of 64 columns, k-row kk, chunk at c ^ (kk % 8)).
    constexpr int kThreadsC = 32 * Cfg::kConvWarpsPerGroup;
    constexpr int kARuns = BM_T * 8, kBRuns = 64 * 16;
    static_assert(kARuns % kThreadsC == 0 && kBRuns % kThreadsC == 0, "runs per thread");
    const int ct = (warp - 2 - Cfg::kEpiWarps) * 32 + lane;
    uint32_t it = 0;
    bool ok = true;
    for (int t = first_tile; ok && t < total_tiles; t += tile_stride) {
      const TileJob j = S.tile(t);
      if (j.kb1 <= j.kb0) continue;
      for (int kb = j.kb0; kb < j.kb1; ++kb, ++it) {
        const uint32_t stage = it % STAGES, ph = (it / STAGES) & 1u;
        const uint32_t rs = it % Cfg::kRawStages, rph = (it / Cfg::kRawStages) & 1u;
        bool w_ok = wait_parity(&raw_full[rs], rph, wd, WD_MMA_FULL);
        w_ok = w_ok && wait_parity(&empty[stage], ph ^ 1u, wd, WD_PRODUCER_EMPTY);
        w_ok = __all_sync(0xffffffffu, w_ok);
        if (!w_ok) {
          ok = false;
          break;
        }
        const uint8_t* rb = ring8 + rs * Cfg::kRawBytes;
        uint8_t* st = smem + stage * Cfg::kStageBytes;
#pragma unroll
        for (int i = 0; i < kARuns / kThreadsC; ++i) {
          const int u = ct + i * kThreadsC;
          const int r = u >> 3, c = u & 7;
          store_i8_as_f16(st + T::kBtBytes + r * 128 + ((c ^ (r & 7)) << 4),
                          *reinterpret_cast<const uint2*>(rb + r * 64 + c * 8));
        }
#pragma unroll
        for (int i = 0; i < kBRuns / kThreadsC; ++i) {
          const int u = ct + i * kThreadsC;
          const int kk = u >> 4, c = u & 15;
          store_i8_as_f16(st + (c >> 3) * (T::kBK * 128) + kk * 128 + (((c & 7) ^ (kk & 7)) << 4),
                          *reinterpret_cast<const uint2*>(rb + BM_T * 64 + kk * 128 + c * 8));
        }
        // the tensor core reads the stage through the async proxy
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&full[stage]);
          mbar_arrive(&raw_empty[rs]);
        }
      }
    }
  } else if constexpr (FUSED) {
    // ------------------------------------------------------------ loader-converters
    // Group g (kConvWarpsPerGroup warps) fills the stages of the k-blocks whose
    // iteration index is g mod 2.  A k-block of a 64-row tile is 64 x 64 FP32
    // elements of A and 64 x 128 of B, i.e. 512 + 1024 runs of eight along the
    // contiguous dimension, shared out evenly over the group's threads and
    // loaded into registers before the stage is free, then split and stored --
    // A's runs in its K-major rows (row r, 16-byte chunk c at chunk position
    // c ^ (r % 8)), B's in the MN-major boxes of 64 columns (k-row kk, chunk of
    // 8 columns c at position c ^ (kk % 8)): the 128-byte swizzle TMA applies.
    constexpr int kGroupThreads = 32 * Cfg::kConvWarpsPerGroup;
    constexpr int kARuns = BM_T * (T::kBK / 8);            // 512
    constexpr int kBRuns = T::kBK * (128 / 8);             // 1024
    static_assert(kARuns % kGroupThreads == 0 && kBRuns % kGroupThreads == 0, "runs per thread");
    constexpr int kAPer = kARuns / kGroupThreads, kBPer = kBRuns / kGroupThreads;
    const int cw = warp - 2 - Cfg::kEpiWarps;
    const uint32_t grp = (uint32_t)(cw / Cfg::kConvWarpsPerGroup);
    const int gt = (cw % Cfg::kConvWarpsPerGroup) * 32 + lane;
    uint32_t it = 0;
    bool ok = true;
    for (int t = first_tile; ok && t < total_tiles; t += tile_stride) {
      const TileJob j = S.tile(t);
      if (j.kb1 <= j.kb0) continue;
      const GroupDesc* d = S.desc(j);
      const float* A = d->A;
      const float* B = d->B;
      const long long lda = d->lda, ldb = d->ldb;
      const int m = d->m, n = d->n, k = d->k;
      for (int kb = j.kb0; kb < j.kb1; ++kb, ++it) {
        if ((it & 1u) != grp) continue;
        const uint32_t stage = it % STAGES, ph = (it / STAGES) & 1u;
        const int k0 = kb * T::kBK;
        float va[kAPer][8], vb[kBPer][8];
#pragma unroll
        for (int i = 0; i < kAPer; ++i) {
          const int u = gt + i * kGroupThreads;
          load_run8(A, lda, j.m0 + (u >> 3), m, k0 + (u & 7) * 8, k, va[i]);
        }
#pragma unroll
        for (int i = 0; i < kBPer; ++i) {
          const int u = gt + i * kGroupThreads;
          load_run8(B, ldb, k0 + (u >> 4), k, j.n0 + (u & 15) * 8, n, vb[i]);
        }
        bool free_ok = wait_parity(&empty[stage], ph ^ 1u, wd, WD_PRODUCER_EMPTY);
        free_ok = __all_sync(0xffffffffu, free_ok);
        if (!free_ok) {
          ok = false;
          break;
        }
        if ((int)it == debug_withhold) continue;   // failure-detection test: the stage never fills
        uint8_t* st = smem + stage * Cfg::kStageBytes;
#pragma unroll
        for (int i = 0; i < kAPer; ++i) {
          const int u = gt + i * kGroupThreads;
          const int r = u >> 3, c = u & 7;
          store_split8<T::kPlanes>(st + T::kBtBytes + r * 128 + ((c ^ (r & 7)) << 4), Cfg::kPlaneBytes, va[i]);
        }
#pragma unroll
        for (int i = 0; i < kBPer; ++i) {
          const int u = gt + i * kGroupThreads;
          const int kk = u >> 4, c = u & 15;
          store_split8<T::kPlanes>(st + (c >> 3) * (T::kBK * 128) + kk * 128 + (((c & 7) ^ (kk & 7)) << 4),
                                   Cfg::kPlaneBytes, vb[i]);
        }
        // the tensor core reads the stage through the async proxy
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[stage]);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // a pair's leader has drained its MMAs (which write both CTAs' TMEM and read
  // both CTAs' shared memory) and both epilogues are done before either frees
  if constexpr (kPair) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc<CG>(tmem_base, Cfg::kTmemCols);
  }
}

template <int BM_T, int STAGES, int MODE, int CG>
__global__ void __launch_bounds__(TcConfig<BM_T, STAGES, MODE, CG>::kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmB1,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ TcParams p) {
  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    if (TcTraits<MODE>::kPlanes > 1) {
      tma_prefetch_desc(&tmA1);
      tma_prefetch_desc(&tmB1);
    }
    if (TcTraits<MODE>::kPlanes > 2) {
      tma_prefetch_desc(&tmA2);
      tma_prefetch_desc(&tmB2);
    }
    if (p.c_tma) tma_prefetch_desc(&tmC);
  }
  const int n_off = (CG == 2) ? 128 * (int)cluster_ctarank() : 0;
  const SingleSched<BM_T, CG, TcStreamK<BM_T, MODE>::value> S{&p, {&tmA, &tmB, &tmA1, &tmB1, &tmA2, &tmB2}, p.c_tma ? &tmC : nullptr, n_off};
  tc_gemm_body<BM_T, STAGES, MODE, CG>(S, p.timeout_ns, p.status, p.debug_withhold, p.scale_a, p.scale_b);
}

// INT8 members that read the int8 operands as they are (RAW8): tmA / tmB
// address the raw int8 matrices.
template <int BM_T, int STAGES, int MODE>
__global__ void __launch_bounds__(TcConfig<BM_T, STAGES, MODE, 1, false, true>::kThreads, 1)
    tc_gemm_raw8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmC, const __grid_constant__ TcParams p) {
  if (threadIdx.x == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    if (p.c_tma) tma_prefetch_desc(&tmC);
  }
  using Sch = SingleSched<BM_T, 1, TcStreamK<BM_T, MODE>::value>;
  const Sch S{&p, {&tmA, &tmB, &tmA, &tmB, &tmA, &tmB}, p.c_tma ? &tmC : nullptr, 0};
  tc_gemm_body<BM_T, STAGES, MODE, 1, Sch, false, true>(S, p.timeout_ns, p.status, p.debug_withhold, p.scale_a,
                                                        p.scale_b);
}

// The same with the FP32-accurate split inside the kernel (loader-converter
// warps in place of TMA loads; C by plain stores).
template <int BM_T, int STAGES, int MODE>
__global__ void __launch_bounds__(TcConfig<BM_T, STAGES, MODE, 1, true>::kThreads, 1)
    tc_grouped_fused_kernel(const __grid_constant__ GroupedParams gp) {
  const GroupedSched S{&gp};
  tc_gemm_body<BM_T, STAGES, MODE, 1, GroupedSched, true>(S, gp.timeout_ns, gp.status, gp.debug_withhold, nullptr,
                                                          nullptr);
}

// Many independent problems in one persistent launch: every CTA walks the
// global tile index of all problems; each tile finds its problem in
// gp.tile_info and uses that problem's tensor maps, tile height and epilogue.
template <int BM_T, int STAGES, int MODE>
__global__ void __launch_bounds__(TcConfig<BM_T, STAGES, MODE>::kThreads, 1)
    tc_grouped_kernel(const __grid_constant__ GroupedParams gp) {
  const GroupedSched S{&gp};
  tc_gemm_body<BM_T, STAGES, MODE, 1>(S, gp.timeout_ns, gp.status, gp.debug_withhold, nullptr, nullptr);
}

}  // namespace g3
