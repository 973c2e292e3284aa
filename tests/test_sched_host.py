"""CPU checks of the tile walk shared by the GEMM kernel, the stream-K fix-up
kernel and the planner (csrc/sched.cuh), compiled with the host compiler:
the banded raster visits every tile once; the stream-K tail covers every
k-block of every tail tile exactly once, each stream's segments lie inside its
own piece, and the slots the fix-up adds for a tile are exactly the segments
that fall in that tile, in stream order."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_20347_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "sched.cuh"
using namespace g3;

static int fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails++ < 20) { std::printf(__VA_ARGS__); std::printf("\n"); } } } while (0)

static void raster(int tm_n, int tn_n, int band) {
  std::vector<int> seen(tm_n * tn_n, 0);
  for (int r = 0; r < tm_n * tn_n; ++r) {
    int tm, tn;
    raster_tile(r, tm_n, tn_n, band, tm, tn);
    CHECK(tm >= 0 && tm < tm_n && tn >= 0 && tn < tn_n, "raster %d %d %d: r=%d out of range", tm_n, tn_n, band, r);
    if (tm >= 0 && tm < tm_n && tn >= 0 && tn < tn_n) seen[tm * tn_n + tn]++;
  }
  for (int i = 0; i < tm_n * tn_n; ++i) CHECK(seen[i] == 1, "raster %d %d %d: tile %d seen %d", tm_n, tn_n, band, i, seen[i]);
}

static void streamk(int tail, int num_kb, int streams) {
  const StreamK sk{(long long)tail * num_kb, streams, num_kb};
  const long long I = sk.iters;
  std::vector<int> cover(I, 0);
  int segs = 0;
  for (int c = 0; c < streams; ++c) segs = segs > sk.segments(c) ? segs : sk.segments(c);
  // tile -> list of slots, in the order the kernel's streams produce them
  std::vector<std::vector<int>> by_tile(tail);
  for (int c = 0; c < streams; ++c) {
    int count = 0;
    long long next = sk.begin(c);
    for (int j = 0; j < segs; ++j) {
      int t, kb0, kb1;
      if (!sk.segment(c, j, t, kb0, kb1)) continue;
      ++count;
      CHECK(t >= 0 && t < tail && 0 <= kb0 && kb0 < kb1 && kb1 <= num_kb, "bad segment c=%d j=%d", c, j);
      const long long x0 = (long long)t * num_kb + kb0, x1 = (long long)t * num_kb + kb1;
      CHECK(x0 == next, "stream %d segment %d starts at %lld, expected %lld", c, j, x0, next);
      next = x1;
      for (long long x = x0; x < x1; ++x) cover[x]++;
      by_tile[t].push_back(c * segs + j);
    }
    CHECK(count == sk.segments(c), "stream %d: %d segments, segments() = %d", c, count, sk.segments(c));
    CHECK(next == sk.begin(c + 1), "stream %d ends at %lld, expected %lld", c, next, sk.begin(c + 1));
  }
  for (long long x = 0; x < I; ++x) CHECK(cover[x] == 1, "I=%lld S=%d: k-block %lld covered %d times", I, streams, x, cover[x]);
  for (long long x = 0; x < I; ++x) {
    const int c = sk.stream_of(x);
    CHECK(c >= 0 && c < streams && sk.begin(c) <= x && x < sk.begin(c + 1), "stream_of(%lld) = %d", x, c);
  }
  // the fix-up's view of each tile: streams stream_of(first) .. stream_of(last)
  for (int t = 0; t < tail; ++t) {
    const int c0 = sk.stream_of((long long)t * num_kb), c1 = sk.stream_of((long long)(t + 1) * num_kb - 1);
    std::vector<int> slots;
    for (int c = c0; c <= c1; ++c) {
      const int j = t - sk.first_tile(c);
      int tt, kb0, kb1;
      if (j >= 0 && sk.segment(c, j, tt, kb0, kb1)) {
        CHECK(tt == t, "fix-up tile %d: stream %d segment %d is in tile %d", t, c, j, tt);
        slots.push_back(c * segs + j);
      }
    }
    CHECK(slots == by_tile[t], "fix-up tile %d: slot lists differ (%zu vs %zu)", t, slots.size(), by_tile[t].size());
  }
}

int main() {
  for (int tm = 1; tm <= 9; ++tm)
    for (int tn = 1; tn <= 7; ++tn)
      for (int band : {1, 2, 3, 4, 8, 16}) raster(tm, tn, band);
  raster(64, 64, 8);
  const int streams_list[] = {1, 2, 3, 7, 74, 76, 148, 152};
  const int kb_list[] = {1, 2, 3, 5, 16, 17, 32, 128, 256};
  for (int S : streams_list)
    for (int kb : kb_list)
      for (int tail = 1; tail <= 2 * S + 1; tail += (tail < 8 ? 1 : 7)) streamk(tail, kb, S);
  streamk(104, 32, 152);   // 2048^3, bm = 128 tiles on 152 SMs
  streamk(36, 128, 76);    // 8192^3, 256 x 256 pair tiles on 76 pairs
  std::printf(fails ? "FAIL %d\n" : "OK\n", fails);
  return fails ? 1 : 0;
}
"""


def test_sched_walk_and_stream_k_partition(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "sched_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "sched_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout + r.stderr
