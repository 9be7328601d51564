"""The leaf kernel's k-nearest selection arithmetic, checked on the host.

The kernel finds each query's k_eff nearest candidates (order: d^2, then input
index) by counting the candidates' squared-distance bit patterns into bucket
histograms (gd_knn_select.cuh: bucket words, bit-sliced Harley-Seal counters,
the walk to the boundary bucket, refinement levels, packed keys).  A host
program built from that header runs the same per-query steps as the kernel on
seeded FP32 distance sets -- random, heavy ties, duplicates at d^2 = 0, huge
ranges, an upper bound far above the answer -- and compares the chosen set
with a full sort.  No GPU is needed.
"""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_10386_gb300", "csrc")

PROGRAM = r"""
#include "gd_knn_select.cuh"
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

using namespace gd;

static int32_t bits(float f) { int32_t b; std::memcpy(&b, &f, 4); return b; }
static float flt(int32_t b) { float f; std::memcpy(&f, &b, 4); return f; }

// One query as the kernel runs it: candidates d[0..n) (d[self] = 0 is the query
// itself), input indices idx[], upper bound theta0 of the keff-th smallest.
template <int PL>
static bool select(const std::vector<float> &d, const std::vector<uint32_t> &idx, int self, uint32_t keff,
                   float theta0, uint32_t pbits, std::vector<int> &out, int *levels, int *tie_rounds) {
  const int n = (int)d.size();
  const int n16 = (n + 15) / 16;
  std::vector<float> dd(n16 * 16, flt(0x7FFFFFFF));          // NaN padding, as in shared memory
  for (int j = 0; j < n; ++j) dd[j] = d[j];
  SelLevel L{bits(theta0), -1, kSelS0, 0u, 0};
  uint32_t c[PL];
  auto count = [&](bool general) {
    for (int p = 0; p < PL; ++p) c[p] = 0;
    for (int s = 0; s < n16; ++s) {
      uint32_t m[16];
      for (int u = 0; u < 16; ++u) {
        const int32_t db = bits(dd[16 * s + u]);
        uint32_t b = sel_bucket_bit(L.tb, db, L.S);
        m[u] = general ? (db > L.lo ? b : 0u) : b;
      }
      sel_add16<PL>(c, m);
    }
  };
  count(false);
  SelCut cut = sel_walk<PL>(c, L, keff);
  int level = 0;
  for (;;) {
    const bool single = cut.hi == cut.lo + 1;
    const bool again = !single && (cut.c_at > kSelBuf || !sel_fits(cut, pbits));
    if (!again) break;
    if (++level > kSelMaxLevels) return false;
    L = sel_refine(L, cut);
    count(true);
    cut = sel_walk<PL>(c, L, keff);
  }
  *levels = level;
  const uint32_t need = keff - cut.c_below;
  const bool ties_only = cut.c_at > kSelBuf;
  *tie_rounds = ties_only;
  const int32_t kbase = cut.lo + 1;
  const float lo_f = cut.lo >= 0 ? flt(cut.lo) : -1.0f, hi_f = flt(cut.hi);
  std::vector<uint32_t> park;
  uint32_t a = 0, np = 0;
  for (int j = 0; j < n; ++j) {                              // pass 2 (position order)
    if (j == self) continue;
    if (d[j] <= lo_f) { out.push_back(j); ++a; }
    else if (d[j] <= hi_f) {
      if (!ties_only) park.push_back(((uint32_t)(bits(d[j]) - kbase) << pbits) | (uint32_t)j);
      ++np;
    }
  }
  if (a != cut.c_below || np != cut.c_at) return false;
  if (!ties_only) {
    std::sort(park.begin(), park.end());
    const uint32_t th_off = park[need - 1] >> pbits;
    uint32_t n_lt = 0, n_eq = 0;
    for (uint32_t k : park) { n_lt += (k >> pbits) < th_off; n_eq += (k >> pbits) == th_off; }
    const uint32_t need_eq = need - n_lt;
    const uint32_t pm = (1u << pbits) - 1u;
    for (uint32_t i = 0; i < park.size(); ++i) {
      const uint32_t off = park[i] >> pbits, j = park[i] & pm;
      bool take = i < need;
      if (n_eq > need_eq && off == th_off) {
        uint32_t before = 0;
        for (uint32_t k : park) if ((k >> pbits) == th_off && idx[k & pm] < idx[j]) ++before;
        take = before < need_eq;
      }
      if (take) out.push_back((int)j);
    }
  } else {                                                   // rounds over exact ties
    uint32_t last = 0;
    for (uint32_t r = 0; r < need; ++r) {
      uint32_t bg = 0xFFFFFFFFu; int bp = -1;
      for (int j = 0; j < n; ++j)
        if (j != self && d[j] == hi_f && (r == 0 || idx[j] > last) && idx[j] < bg) { bg = idx[j]; bp = j; }
      out.push_back(bp);
      last = bg;
    }
  }
  return out.size() == keff;
}

int main() {
  std::mt19937_64 rng(11);
  long cases = 0, refined = 0, ties = 0;
  for (int t = 0; t < 60000; ++t) {
    const int kind = t % 6;
    const int n = 2 + (int)(rng() % (kind == 5 ? 2000 : 520));
    const uint32_t K = 1 + (uint32_t)(rng() % 64);
    const uint32_t keff = std::min<uint32_t>(K, (uint32_t)n - 1);
    std::vector<float> d(n);
    std::vector<uint32_t> idx(n);
    std::uniform_real_distribution<float> u(0.f, 1.f);
    for (int j = 0; j < n; ++j) {
      float v = u(rng);
      switch (kind) {
        case 0: v = v * v; break;                                   // smooth
        case 1: v = (float)(rng() % 7) * 0.25f; break;              // few distinct values: ties
        case 2: v = (rng() % 3 == 0) ? 0.0f : v; break;             // duplicates at d^2 = 0
        case 3: v = std::ldexp(v, -(int)(rng() % 100)); break;      // values spread over 100 octaves
        case 4: v = 1e-3f * v; break;                               // answer far below theta0
        default: v = std::ldexp(1.0f + (float)(rng() % 3) * 0x1p-23f, -(int)(rng() % 3)); break;
      }
      d[j] = v;
      idx[j] = (uint32_t)(rng() % 1000000);
    }
    const int self = (int)(rng() % n);
    d[self] = 0.0f;
    for (int j = 0; j < n; ++j) idx[j] = idx[j] * 4096 + (uint32_t)j;   // distinct input indices
    // theta0: max over keff others (a window), then possibly a far point in it
    float theta0 = 0.f;
    for (uint32_t r = 0, j = 0; r < keff; ++j) if ((int)j != self) { theta0 = std::max(theta0, d[j]); ++r; }
    if (kind == 4) theta0 = std::max(theta0, 50.0f);
    uint32_t pbits = 1;
    while ((1u << pbits) < (uint32_t)n) ++pbits;
    std::vector<int> got;
    int levels = 0, tr = 0;
    const bool ok = n <= 2047 ? select<11>(d, idx, self, keff, theta0, pbits, got, &levels, &tr)
                              : select<21>(d, idx, self, keff, theta0, pbits, got, &levels, &tr);
    // reference: full sort by (d^2, input index)
    std::vector<int> ord;
    for (int j = 0; j < n; ++j) if (j != self) ord.push_back(j);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] != d[y] ? d[x] < d[y] : idx[x] < idx[y]; });
    std::vector<int> want(ord.begin(), ord.begin() + keff);
    std::sort(want.begin(), want.end());
    std::sort(got.begin(), got.end());
    if (!ok || got != want) {
      std::printf("mismatch: case %d kind %d n %d keff %u ok %d\n", t, kind, n, keff, (int)ok);
      return 1;
    }
    ++cases;
    refined += levels > 0;
    ties += tr;
  }
  std::printf("cases %ld refined %ld tie_rounds %ld\n", cases, refined, ties);
  return 0;
}
"""


def test_histogram_selection_equals_full_sort(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "sel.cpp"
    exe = tmp_path / "sel"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "cases 60000" in r.stdout
    counts = dict(zip(r.stdout.split()[0::2], (int(v) for v in r.stdout.split()[1::2])))
    assert counts["refined"] > 1000 and counts["tie_rounds"] > 100      # every path exercised
