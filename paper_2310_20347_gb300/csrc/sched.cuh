// sched.cuh -- the tile walk of one GEMM: the banded raster and the stream-K
// tail.  Plain integer arithmetic shared by the tensor-core kernel (which
// tiles and k-block ranges each persistent CTA computes), the stream-K fix-up
// kernel (which partial results make up a tail tile) and the host planner, so
// that all three agree by construction.
#pragma once

#if defined(__CUDACC__)
#define G3_HD __host__ __device__ __forceinline__
#else
#define G3_HD inline
#endif

namespace g3 {

// Banded raster: ordinal r of the walk -> output tile (tm, tn).  The tile rows
// are cut into bands of `band` rows (the last band may be shorter); inside a
// band the walk goes down the band's rows first, then on to the next tile
// column, so the band's panels of A and the current panel of B stay in L2
// (the loop order L1/L3 of the paper's baseline algorithm, Section 3.1).
G3_HD void raster_tile(int r, int tiles_m, int tiles_n, int band, int& tm, int& tn) {
  const int b = r / (band * tiles_n);
  const int in_band = r - b * band * tiles_n;
  const int rows = band < tiles_m - b * band ? band : tiles_m - b * band;
  tm = b * band + in_band % rows;
  tn = in_band / rows;
}

// Stream-K tail.  When the tiles do not fill the last wave of the persistent
// grid, the last `tail` tiles of the walk are not handed out whole: their
// k-blocks, numbered x = t * num_kb + kb for tail tile t (0 .. tail-1) and
// k-block kb, form one range [0, iters), iters = tail * num_kb, which is cut
// into `streams` contiguous pieces of nearly equal length, one per persistent
// CTA (or CTA pair): stream c covers [begin(c), begin(c+1)) with
// begin(c) = floor(c * iters / streams).  A piece crosses tile boundaries; the
// part of it inside one tile is a segment.  Segment j of stream c lies in tail
// tile first_tile(c) + j and leaves its partial result in slot c * segs + j
// (segs = the most segments any stream has); a fix-up pass adds each tail
// tile's segments in stream order (deterministic) and applies alpha and beta.
// This is the GPU analogue of the paper's variants that keep C in a cache
// level while k is split (Sections 3.2 and 7), balanced so that every CTA does
// the same number of k-blocks.
struct StreamK {
  long long iters;   // tail * num_kb
  int streams;
  int num_kb;

  G3_HD long long begin(int c) const { return (long long)c * iters / streams; }
  // the stream whose piece holds iteration x (0 <= x < iters): the largest c
  // with begin(c) <= x, i.e. ceil((x + 1) * streams / iters) - 1
  G3_HD int stream_of(long long x) const { return (int)(((x + 1) * streams + iters - 1) / iters) - 1; }
  G3_HD int first_tile(int c) const { return (int)(begin(c) / num_kb); }
  // segments of stream c (0 for an empty piece)
  G3_HD int segments(int c) const {
    const long long b = begin(c), e = begin(c + 1);
    return e > b ? (int)((e - 1) / num_kb - b / num_kb) + 1 : 0;
  }
  // segment j of stream c: tail tile t and its k-blocks [kb0, kb1); false
  // when stream c has no segment j
  G3_HD bool segment(int c, int j, int& t, int& kb0, int& kb1) const {
    const long long b = begin(c), e = begin(c + 1);
    t = (int)(b / num_kb) + j;
    const long long t0 = (long long)t * num_kb;
    const long long s0 = b > t0 ? b : t0;
    const long long s1 = e < t0 + num_kb ? e : t0 + num_kb;
    if (s0 >= s1) return false;
    kb0 = (int)(s0 - t0);
    kb1 = (int)(s1 - t0);
    return true;
  }
};

}  // namespace g3
