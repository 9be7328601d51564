// gd_knn_select.cuh -- exact k-nearest selection by bucket histograms of the
// squared distances' bit patterns (host-usable arithmetic of the leaf kernel's
// kNN, kept apart so that a host test can run the same steps).
//
// The selection the method needs (Sec. 3, the kNN step; tie rule: distance,
// then input index) is the set of the k_eff smallest (d^2, index) among the
// candidates.  For FP32 values d^2 >= 0 the IEEE bit pattern, read as an
// integer, orders like the value, so the selection works on integer "bits":
//
//  level:  a top `tb` (bits of an upper bound of the k_eff-th smallest d^2),
//          an exclusive bottom `lo` (-1 = none) and a bucket width 2^S; a
//          candidate with lo < db <= tb falls in bucket min((tb - db) >> S, 31)
//          (bucket 31 also takes everything below its range).  Buckets are
//          counted in bit-sliced form: plane p holds bit p of all 32 counts.
//  walk:   the bucket B where the cumulative count from the smallest distances
//          reaches k_eff; every candidate below B's range is a neighbour
//          (c_below of them), and `need` = k_eff - c_below more come from B.
//  refine: if B holds more candidates than the per-query buffer, or its range
//          does not fit a packed key, the same count runs again inside B's
//          range with 32 buckets covering it (width 2^(S-5) for an ordinary
//          bucket), until it fits or holds a single d^2 value.
//  select: B's members are parked as keys ((db - base) << pbits | position),
//          sorted, and the first `need` taken; where d^2 ties straddle the cut
//          the tied ones are ranked by input index.
#pragma once

#include <stdint.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace gd {

constexpr int kSelBuckets = 32;
constexpr int kSelS0 = 20;          // first-level bucket width: 2^20 patterns = an eighth of an octave of d^2
constexpr uint32_t kSelBuf = 16;    // parked boundary-bucket candidates per query
constexpr int kSelMaxLevels = 12;   // refinement levels before a consistency failure is reported

__host__ __device__ __forceinline__ uint32_t sel_popc(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __popc(v);
#else
  return (uint32_t)__builtin_popcount(v);
#endif
}

// 1 << s, and 0 for any s >= 32 (PTX shl clamps the shift amount)
__host__ __device__ __forceinline__ uint32_t sel_shl1(uint32_t s) {
#ifdef __CUDA_ARCH__
  uint32_t r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(s));
  return r;
#else
  return s >= 32u ? 0u : 1u << s;
#endif
}

// One-hot bucket word of a candidate (bits db) at a level with top tb and width
// 2^S: bit min((tb - db) >> S, 31) when db <= tb, 0 above the top (including the
// NaN padding, whose canonical pattern 0x7FFFFFFF is above every top).
__host__ __device__ __forceinline__ uint32_t sel_bucket_bit(int32_t tb, int32_t db, int S) {
  int32_t b = (tb - db) >> S;  // arithmetic shift: negative above the top
  b = b < 31 ? b : 31;
  return sel_shl1((uint32_t)b);
}

// carry-save adder: l = a ^ b ^ c (same weight), h = majority (next weight)
__host__ __device__ __forceinline__ void sel_csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

// Add 16 one-hot words into the bit-sliced counters c[0..P) (Harley-Seal tree:
// planes 1, 2, 4, 8 through carry-save adders, the carry of weight 16 rippled
// into the planes above).
template <int P>
__host__ __device__ __forceinline__ void sel_add16(uint32_t (&c)[P], const uint32_t *m) {
  uint32_t tA, tB, fA, fB, eA, eB, s;
  sel_csa(tA, c[0], c[0], m[0], m[1]);
  sel_csa(tB, c[0], c[0], m[2], m[3]);
  sel_csa(fA, c[1], c[1], tA, tB);
  sel_csa(tA, c[0], c[0], m[4], m[5]);
  sel_csa(tB, c[0], c[0], m[6], m[7]);
  sel_csa(fB, c[1], c[1], tA, tB);
  sel_csa(eA, c[2], c[2], fA, fB);
  sel_csa(tA, c[0], c[0], m[8], m[9]);
  sel_csa(tB, c[0], c[0], m[10], m[11]);
  sel_csa(fA, c[1], c[1], tA, tB);
  sel_csa(tA, c[0], c[0], m[12], m[13]);
  sel_csa(tB, c[0], c[0], m[14], m[15]);
  sel_csa(fB, c[1], c[1], tA, tB);
  sel_csa(eB, c[2], c[2], fA, fB);
  sel_csa(s, c[3], c[3], eA, eB);
#pragma unroll
  for (int p = 4; p < P; ++p) {
    const uint32_t t = c[p] & s;
    c[p] ^= s;
    s = t;
  }
}

// sum of the counts of the buckets selected by `mask`
template <int P>
__host__ __device__ __forceinline__ uint32_t sel_count(const uint32_t (&c)[P], uint32_t mask) {
  uint32_t n = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) n += sel_popc(c[p] & mask) << p;
  return n;
}

// State of one query's selection at the current level.
struct SelLevel {
  int32_t tb;        // top (inclusive) bits
  int32_t lo;        // exclusive bottom bits (-1: none; then the query itself, d^2 = 0, is counted)
  int32_t S;         // bucket width 2^S
  uint32_t c_base;   // neighbours below `lo` (found at earlier levels)
  int32_t slides;    // catch-all refinements taken at the first level's resolution so far
};

// Result of the walk: bucket B's range and counts.
struct SelCut {
  int32_t hi;        // inclusive top bits of bucket B
  int32_t lo;        // exclusive bottom bits of bucket B (-1: none)
  uint32_t c_below;  // candidates (the query excluded) below B's range
  uint32_t c_at;     // candidates (the query excluded) in B's range
  int32_t B;
};

// Walk the counts of a level: B = the largest bucket index (smallest distances
// first) at which the cumulative count, the query itself excluded, reaches keff.
template <int P>
__host__ __device__ __forceinline__ SelCut sel_walk(const uint32_t (&c)[P], const SelLevel &L, uint32_t keff) {
  // the query's own d^2 = 0 lies in bucket bself when the level reaches down to 0
  // (bself = -1: the level does not reach 0, the query is not counted)
  const int32_t bself = (L.lo < 0) ? ((L.tb >> L.S) < 31 ? (L.tb >> L.S) : 31) : -1;
  auto cum = [&](int32_t b) -> uint32_t {  // b in [0, 32]
    if (b >= 32) return L.c_base;
    return L.c_base + sel_count<P>(c, 0xFFFFFFFFu << b) - (b <= bself ? 1u : 0u);
  };
  int32_t lo = 0, hi = 31;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (cum(mid) >= keff) lo = mid;
    else hi = mid - 1;
  }
  SelCut r;
  r.B = lo;
  const uint32_t at_or_below = cum(lo);
  r.c_below = cum(lo + 1);
  r.c_at = at_or_below - r.c_below;
  r.hi = L.tb - (lo << L.S);
  const int32_t bot = (lo < 31) ? L.tb - ((lo + 1) << L.S) : L.lo;
  r.lo = bot > L.lo ? bot : L.lo;
  return r;
}

__host__ __device__ __forceinline__ int32_t sel_bitlen(uint32_t v) {
#ifdef __CUDA_ARCH__
  return 32 - __clz(v);
#else
  return v ? 32 - __builtin_clz(v) : 0;
#endif
}

// The level that counts inside bucket `cut`: 32 buckets whose widths cover its
// range (lo, hi].  For an ordinary bucket (2^S patterns) the width is 2^(S-5);
// the catch-all last bucket of a level that reaches down to 0 can be wider, and
// its width is then taken from the range itself.  Either way the largest offset
// in the range loses at least 5 bits per level.  The exception: the catch-all
// of a level that reaches down to 0 is first searched (up to kSelSlides times)
// by the next 31 buckets below it at the same width, with a new catch-all under
// them -- the k-th distance is then usually a few octaves below the bound, and
// the boundary bucket comes out narrow at once (split by range, the catch-all's
// buckets would each span octaves, and take a further level).
constexpr int32_t kSelSlides = 2;
__host__ __device__ __forceinline__ SelLevel sel_refine(const SelLevel &L, const SelCut &cut) {
  SelLevel n;
  n.tb = cut.hi;
  n.lo = cut.lo;
  n.c_base = cut.c_below;
  n.slides = L.slides;
  if (cut.B == kSelBuckets - 1 && L.lo < 0 && L.slides < kSelSlides) {
    n.S = L.S;
    n.slides = L.slides + 1;
  } else {
    const int32_t nb = sel_bitlen((uint32_t)(cut.hi - cut.lo - 1));  // bits of the largest offset
    n.S = nb > 5 ? nb - 5 : 0;
  }
  return n;
}

// Does bucket B's range fit a packed key with `pbits` position bits?
__host__ __device__ __forceinline__ bool sel_fits(const SelCut &cut, uint32_t pbits) {
  const uint32_t range = (uint32_t)(cut.hi - (cut.lo + 1));  // largest offset in the range
  return pbits >= 32u ? range == 0u : (uint64_t)range < (1ull << (32u - pbits));
}

}  // namespace gd
