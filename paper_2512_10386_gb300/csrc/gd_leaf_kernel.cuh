// gd_leaf_kernel.cuh -- device code of the fused per-leaf kernel, shared by the
// two translation units that instantiate it (gd_leaf.cu: the plain path;
// gd_leaf_rec.cu: the instantiation that also writes debug / training tensors).
// Split so the two sets of instantiations compile in parallel.
#pragma once

#include <type_traits>

#include "gd_common.cuh"
#include "gd_f32x2.cuh"
#include "gd_knn_select.cuh"

namespace gd {

constexpr int kLeafThreads = 128;
constexpr int kLeafWarps = kLeafThreads / 32;
constexpr unsigned long long kEmpty = ~0ull;
constexpr unsigned long long kInvalid = ~0ull - 1ull;
// P_1 is followed by kPad NaN points: the kNN passes read whole steps of 4, 16
// or 32 candidates past the last one without a bounds test (a NaN distance falls
// in no bucket, and the chunk masks drop positions past P_1).
constexpr uint32_t kPad = 32;
// largest leaf of the shared-memory path: bit-sliced counts of the kNN hold < 2^11
constexpr uint32_t kLeafSmemMax = 2048;

__host__ __device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~size_t(15); }
// smallest power of two >= x (x <= 2^31; larger x gives 2^31)
__host__ __device__ __forceinline__ uint32_t pow2ceil(uint32_t x) {
  uint32_t p = 1;
  while (p < x && p < 0x80000000u) p <<= 1;
  return p;
}

// Per-leaf working arrays: shared memory (small leaves) or global spill (large).
// P_1 is kept as structure of arrays (X, Y, Z, W), so that four consecutive
// candidates come in one 16-byte load per coordinate and pair up for the
// packed two-lane FP32 arithmetic of the distance passes.
struct LeafMem {
  float *X, *Y, *Z;          // [cap + kPad] P_1 coordinates, then NaN padding
  uint32_t *W;               // [cap + kPad] input index of each P_1 point
  float4 *raw;               // [cap] raw points of a shared-memory leaf (the bulk copy lands here)
  unsigned long long *hkey;  // [hcap] voxel hash keys
  uint32_t *hcnt;            // [hcap] voxel occupancy
  unsigned long long *sbuf;  // [scap] sort buffer
  uint32_t *pend;            // [kSelBuf][kLeafThreads] parked boundary-bucket keys (shared memory, both paths)
  float *r2, *wa;            // [cap] per P_1 position: r_K^2, (alpha/2) ell; wa also holds voxel hash slots
  float *F;                  // [cap] score; shares r2's storage (F_i is written after r2_i's last read)
  uint8_t *flag;             // [cap] 0 removed by density gate, 1 scored, 2 kept
  uint32_t *spos;            // [cap] leaf offset of each P_1 point (cross-leaf mode)
  uint32_t *cmask;           // [cap] the chunks of a query's bitmap row that hold neighbours (shares spos:
                             // the cross-leaf mode, which reads spos later, runs no kNN in this kernel)
  void *nbr;                 // neighbours: bitmaps (shared-memory path, see bitmap_words) or [KMAX][cap] u32 (global)
  uint32_t nbr_bytes;        // bytes of the region that holds nbr
  uint32_t hcap, scap, cap;
};

// bits of a position in a leaf of `cap` points (the position field of a parked kNN key)
__host__ __device__ __forceinline__ uint32_t nb_bits(uint32_t cap) {
  uint32_t b = 1;
  while ((1u << b) < cap) ++b;
  return b;
}
// Neighbour table of the shared-memory path: a bitmap of neighbour positions,
// word (c, q) at index c * n1 + q holding bit b for position 32c + b among query
// q's neighbours (chunk-major: a warp's 32 queries touch 32 consecutive words).
// The kNN records a whole chunk of 32 candidates with one store, the score walks
// the neighbours in position order.  The table lives in region A (after the
// voxel hash is done with it) when it fits there, else in the leaf's part of
// the global spill area (L2-resident), through the same generic pointer.
__host__ __device__ __forceinline__ uint32_t bitmap_words(uint32_t n1) { return ((n1 + 31u) / 32u) * n1; }

// Layout of the per-leaf arrays.  Region A holds the voxel hash table, later
// (the lifetimes do not overlap) the neighbour table.  Region R holds a
// shared-memory leaf's raw points (voxel gate), then the parked kNN keys, then
// the sort buffer of the order statistics.
template <typename IdxT>
__host__ __device__ __forceinline__ size_t carve(unsigned char *base, uint32_t cap, int kmax, LeafMem *m) {
  constexpr bool kSmem = sizeof(IdxT) == 2;
  const uint32_t hcap = pow2ceil(2 * cap), scap = pow2ceil(cap);
  const size_t hash_end = al16((size_t)hcap * 8) + al16((size_t)hcap * 4);
  const size_t nbr_bytes = kSmem ? hash_end : al16((size_t)cap * kmax * sizeof(IdxT));
  size_t o = al16(hash_end > nbr_bytes ? hash_end : nbr_bytes);
  size_t rbytes = (size_t)scap * 8;
  if (kSmem) {
    const size_t raw = (size_t)cap * 16, park = (size_t)kSelBuf * kLeafThreads * 4;
    if (raw > rbytes) rbytes = raw;
    if (park > rbytes) rbytes = park;
  }
  if (m) {
    m->hkey = (unsigned long long *)base;
    m->hcnt = (uint32_t *)(base + al16((size_t)hcap * 8));
    m->nbr = (void *)base;
    m->nbr_bytes = (uint32_t)o;
    m->hcap = hcap;
    m->scap = scap;
    m->cap = cap;
  }
  auto take = [&](size_t bytes) { size_t r = o; o = al16(o + bytes); return r; };
  const size_t rr = take(rbytes);
  const size_t soa = (size_t)(cap + kPad) * 4;
  const size_t x = take(soa), y = take(soa), z = take(soa), w = take(soa);
  const size_t r2 = take((size_t)cap * 4), wa = take((size_t)cap * 4), fl = take((size_t)cap);
  const size_t sp = take((size_t)cap * 4);
  if (m) {
    m->raw = kSmem ? (float4 *)(base + rr) : nullptr;
    m->sbuf = (unsigned long long *)(base + rr);
    m->pend = kSmem ? (uint32_t *)(base + rr) : nullptr;  // the spill path parks in the CTA's shared memory
    m->X = (float *)(base + x);
    m->Y = (float *)(base + y);
    m->Z = (float *)(base + z);
    m->W = (uint32_t *)(base + w);
    m->r2 = (float *)(base + r2);
    m->wa = (float *)(base + wa);
    m->F = m->r2;
    m->flag = (uint8_t *)(base + fl);
    m->spos = (uint32_t *)(base + sp);
    m->cmask = m->spos;
  }
  return o;
}

struct LeafShared {
  uint32_t leaf;
  uint32_t n1, keff, m, keep_n, run;
  uint32_t nless, ntied;  // Top-lambda cut: P_2 keys below / equal to the keep_n-th
  uint32_t crank;  // Eq. 14 cut rank c, from the top of the ascending r^2 order
  uint32_t qblk;   // next 32-query block of the kNN
  float lo[3], h, delta, r2ref, Lref;
  float lshift;  // cross-leaf mode: ell_j = log2(rho_j) - lshift for a neighbour j of any leaf
  double rho_med;
  uint32_t wsum[kLeafWarps];
  uint32_t red[kLeafWarps][6];
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Eq. 11 cube root: u = m 2^e (frexp), y0 = 2^floor(e/3), ten Newton steps
// y <- y - (y*y*y - u) / (3*(y*y)), every operation rounded in FP64.  The step
// is a fixed function of y, so once it reaches a fixed point, or a 2-cycle, the
// tenth iterate is known and the remaining steps are skipped (same bits as all
// ten; FP64 issue is slow on this part).
__device__ __forceinline__ double cbrt_spec(double u) {
  int e = 0;
  (void)frexp(u, &e);
  const int k = (e >= 0) ? e / 3 : -((-e + 2) / 3);
  double y = ldexp(1.0, k), prev = 0.0;  // y = y_i, prev = y_(i-1)
#pragma unroll 1
  for (int it = 0; it < 10; ++it) {
    const double y2 = __dmul_rn(y, y);
    const double y3 = __dmul_rn(y2, y);
    const double yn = __dsub_rn(y, __ddiv_rn(__dsub_rn(y3, u), __dmul_rn(3.0, y2)));  // y_(it+1)
    if (yn == y) return y;                                  // fixed point: y_10 = y_it
    if (it > 0 && yn == prev) return (it & 1) ? yn : y;     // y_(it-1), y_it alternate: y_10
    prev = y;
    y = yn;
  }
  return y;
}

__device__ __forceinline__ uint32_t vox_index(float x, float lo, float h) {
  const float f = floorf(__fdiv_rn(__fsub_rn(x, lo), h));
  return (f < 2097151.0f) ? (uint32_t)f : kQMax;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ uint32_t hash_insert(unsigned long long *hk, uint32_t hcap, unsigned long long key,
                                                Counters *ctr) {
  const uint32_t mask = hcap - 1;
  uint32_t s = (uint32_t)mix64(key) & mask;
  for (uint32_t probe = 0; probe < hcap; ++probe) {
    const unsigned long long prev = atomicCAS(hk + s, kEmpty, key);
    if (prev == kEmpty || prev == key) return s;
    s = (s + 1) & mask;
  }
  atomicOr(&ctr->status, kStInternal);
  return s;
}

// Ascending bitonic sort of a[0..n) (n a power of two) by the whole block, one
// compare-exchange stage per barrier: the general form, for any n.
template <typename T>
__device__ void bitonic_sort_smem(T *a, uint32_t n) {
  for (uint32_t k = 2; k <= n; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const T x = a[i], y = a[l];
          const bool asc = (i & k) == 0;
          if ((x > y) == asc) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// The same network on N = blockDim.x * E elements held in registers: thread t owns
// elements t*E .. t*E+E-1 (a padded with `pad` from n up to N).  A stage whose
// partner distance j is below E stays in the thread, below 32*E it is a warp
// shuffle, and only the stages with j >= 32*E go through shared memory (3 of
// the 45 stages at N = 512 with 128 threads), so the sort needs a handful of
// barriers instead of one per stage.  Writes the sorted N elements back to a
// (a must hold N).
template <typename T, int E>
__device__ __forceinline__ void bitonic_sort_regs(T *a, uint32_t n, T pad) {
  const uint32_t N = blockDim.x * E;
  const uint32_t t = threadIdx.x;
  T v[E];
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const uint32_t e = t * E + k;
    v[k] = (e < n) ? a[e] : pad;
  }
  __syncthreads();
#pragma unroll 1
  for (uint32_t size = 2; size <= N; size <<= 1) {
#pragma unroll 1
    for (uint32_t j = size >> 1; j > 0; j >>= 1) {
      if (j < (uint32_t)E) {  // partners inside the thread (register indices fixed per jj)
#pragma unroll
        for (int jj = 1; jj < E; jj <<= 1) {
          if ((uint32_t)jj != j) continue;
#pragma unroll
          for (int k = 0; k < E; ++k) {
            const int l = k ^ jj;
            if (l > k) {
              const bool asc = ((t * E + k) & size) == 0;
              const T x = v[k], y = v[l];
              const T lo = x < y ? x : y, hi = x < y ? y : x;
              v[k] = asc ? lo : hi;
              v[l] = asc ? hi : lo;
            }
          }
        }
      } else if (j < 32u * E) {
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const uint32_t e = t * E + k;
          const T y = __shfl_xor_sync(0xFFFFFFFFu, v[k], j / E);
          const bool take_min = ((e & j) == 0) == ((e & size) == 0);
          v[k] = take_min ? (v[k] < y ? v[k] : y) : (v[k] < y ? y : v[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < E; ++k) a[t * E + k] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const uint32_t e = t * E + k;
          const T y = a[e ^ j];
          const bool take_min = ((e & j) == 0) == ((e & size) == 0);
          v[k] = take_min ? (v[k] < y ? v[k] : y) : (v[k] < y ? y : v[k]);
        }
        __syncthreads();
      }
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k) a[t * E + k] = v[k];
  __syncthreads();
}

// The same network on N = 32 * E elements by the first warp alone (small leaves:
// no block-wide stage, no barrier until the sorted keys are written back).
template <typename T, int E>
__device__ __forceinline__ void warp_sort_regs(T *a, uint32_t n, T pad) {
  if (threadIdx.x < 32) {
    const uint32_t t = threadIdx.x;
    T v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint32_t e = t * E + k;
      v[k] = (e < n) ? a[e] : pad;
    }
#pragma unroll 1
    for (uint32_t size = 2; size <= 32u * E; size <<= 1) {
#pragma unroll 1
      for (uint32_t j = size >> 1; j > 0; j >>= 1) {
        if (j < (uint32_t)E) {
#pragma unroll
          for (int jj = 1; jj < E; jj <<= 1) {
            if ((uint32_t)jj != j) continue;
#pragma unroll
            for (int k = 0; k < E; ++k) {
              const int l = k ^ jj;
              if (l > k) {
                const bool asc = ((t * E + k) & size) == 0;
                const T x = v[k], y = v[l];
                const T lo = x < y ? x : y, hi = x < y ? y : x;
                v[k] = asc ? lo : hi;
                v[l] = asc ? hi : lo;
              }
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < E; ++k) {
            const uint32_t e = t * E + k;
            const T y = __shfl_xor_sync(0xFFFFFFFFu, v[k], j / E);
            const bool take_min = ((e & j) == 0) == ((e & size) == 0);
            v[k] = take_min ? (v[k] < y ? v[k] : y) : (v[k] < y ? y : v[k]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < E; ++k) a[t * E + k] = v[k];
  }
  __syncthreads();
}

// ascending sort of a[0..n), n a power of two; entries n.. up to the next
// multiple of blockDim.x (at most 512) may be overwritten with `pad`.  Not inlined:
// the unrolled networks would otherwise raise the whole kernel's register count.
template <typename T>
__device__ __noinline__ void block_sort(T *a, uint32_t n, T pad) {
  const uint32_t nt = blockDim.x;
  // small leaves of 128-thread CTAs: one warp sorts, no block-wide stage (with
  // 64-thread CTAs the block sort of 64 keys keeps both warps busy and stays faster)
  if (n <= 32 && nt >= 128) warp_sort_regs<T, 1>(a, n, pad);
  else if (n <= 64 && nt >= 128) warp_sort_regs<T, 2>(a, n, pad);
  else if (n <= nt) bitonic_sort_regs<T, 1>(a, n, pad);
  else if (n <= 2 * nt) bitonic_sort_regs<T, 2>(a, n, pad);
  else if (n <= 4 * nt) bitonic_sort_regs<T, 4>(a, n, pad);
  else if (n <= 8 * nt && n <= 512) bitonic_sort_regs<T, 8>(a, n, pad);
  else bitonic_sort_smem<T>(a, n);
}

// the SFU's exp2 and reciprocal (PTX ex2.approx.ftz.f32, rcp.approx.ftz.f32: about
// 2 ulp and 1 ulp; a subnormal argument or result is taken as 0: a score term that
// small lies below what FP32 resolves in a sum anyway)
__device__ __forceinline__ float ex2_hw(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_hw(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// squared distance with the fixed FP32 operation order of the method's reading:
// dx = x_j - x_i;  d^2 = fma(dz, dz, fma(dy, dy, dx*dx))
__device__ __forceinline__ float sqdist(float xi, float yi, float zi, float xj, float yj, float zj) {
  const float dx = __fsub_rn(xj, xi), dy = __fsub_rn(yj, yi), dz = __fsub_rn(zj, zi);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// d^2 from the query (packed broadcast QX = (x_i, x_i), ...) to the four
// candidates j .. j+3 (j a multiple of 4): three 16-byte loads, six packed
// subtractions and six packed multiply / fused multiply-adds
__device__ __forceinline__ void sqdist4(const float *__restrict__ X, const float *__restrict__ Y,
                                        const float *__restrict__ Z, uint32_t j, f32x2 QX, f32x2 QY, f32x2 QZ,
                                        float (&d)[4]) {
  const float4 x = *reinterpret_cast<const float4 *>(X + j);
  const float4 y = *reinterpret_cast<const float4 *>(Y + j);
  const float4 z = *reinterpret_cast<const float4 *>(Z + j);
  const f32x2 dx0 = sub2(pk2(x.x, x.y), QX), dx1 = sub2(pk2(x.z, x.w), QX);
  const f32x2 dy0 = sub2(pk2(y.x, y.y), QY), dy1 = sub2(pk2(y.z, y.w), QY);
  const f32x2 dz0 = sub2(pk2(z.x, z.y), QZ), dz1 = sub2(pk2(z.z, z.w), QZ);
  f32x2 s0 = mul2(dx0, dx0), s1 = mul2(dx1, dx1);
  s0 = fma2(dy0, dy0, s0);
  s1 = fma2(dy1, dy1, s1);
  s0 = fma2(dz0, dz0, s0);
  s1 = fma2(dz1, dz1, s1);
  upk2(s0, d[0], d[1]);
  upk2(s1, d[2], d[3]);
}

// ---------------------------------------------------------------------------
// register sorting network (all indices compile-time)
// ---------------------------------------------------------------------------
// ascending sort network: Batcher's odd-even merge sort (19 comparators for 8
// values, 63 for 16, 191 for 32, against 24, 80 and 240 for a bitonic sort).
// The comparator list is built at compile time, so every register index is a
// constant.
template <int N>
struct OddEvenNet {
  static constexpr int count() {
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k; ++i)
            if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) ++c;
    return c;
  }
  static constexpr int C = count();
  int a[C], b[C];
  constexpr OddEvenNet() : a(), b() {
    int c = 0;
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k; ++i)
            if (i + j + k < N && (i + j) / (2 * p) == (i + j + k) / (2 * p)) {
              a[c] = i + j;
              b[c] = i + j + k;
              ++c;
            }
  }
};

// ascending sort of N 32-bit keys in registers (the comparator table above)
template <int N>
__device__ __forceinline__ void regsort_u(uint32_t (&L)[N]) {
  constexpr OddEvenNet<N> net{};
#pragma unroll
  for (int c = 0; c < OddEvenNet<N>::C; ++c) {
    const uint32_t x = L[net.a[c]], y = L[net.b[c]];
    L[net.a[c]] = umin(x, y);
    L[net.b[c]] = umax(x, y);
  }
}
// the same on the first H entries of L (the rest already sorted and not below them)
template <int H, int N>
__device__ __forceinline__ void regsort_head(uint32_t (&L)[N]) {
  static_assert(H <= N, "head within the array");
  constexpr OddEvenNet<H> net{};
#pragma unroll
  for (int c = 0; c < OddEvenNet<H>::C; ++c) {
    const uint32_t x = L[net.a[c]], y = L[net.b[c]];
    L[net.a[c]] = umin(x, y);
    L[net.b[c]] = umax(x, y);
  }
}

// Lref of the score (Eq. 16-17), from the lower-middle r^2 (ra) and upper-middle
// r^2 (rb) of P_2's m points.  Once per leaf by one thread: kept out of line.
static __device__ __noinline__ float leaf_lref(float ra, float rb, uint32_t m, uint32_t keff, float eps_rho) {
  // log2(rho(ra) / rho_med): 0 for odd m, 1 - log2(1 + (ra / rb)^1.5) for even m
  float lr = 0.0f;
  if (!(m & 1u)) {
    const float t = __fdiv_rn(ra, rb);
    lr = __fsub_rn(1.0f, log2f(__fadd_rn(1.0f, __fmul_rn(t, sqrtf(t)))));
  }
  // log2(rho_med) = log2(rho(ra)) - lr, with log2(rho(ra)) = log2(k_eff) - log2(4/3 pi) - 1.5 log2(ra)
  const float l_rho_a =
      __fsub_rn(__fsub_rn(log2f((float)keff), 2.0665336287511624f), __fmul_rn(1.5f, log2f(ra)));
  const float l_med = __fsub_rn(l_rho_a, lr);
  float corr = 0.0f;
  if (eps_rho > 0.0f) {
    const float lx = __fsub_rn(log2f(eps_rho), __fmul_rn(2.0f, l_med));  // log2(eps_rho / rho_med^2)
    corr = (lx > 100.0f) ? __fmul_rn(0.5f, lx) : __fmul_rn(0.5f, log2f(__fadd_rn(1.0f, exp2f(lx))));
  }
  return __fsub_rn(lr, corr);
}

// (d^2)^(gamma/2) for gamma != 2 (the score's common case gamma = 2 needs none): out of line
static __device__ __noinline__ float pow_half_gamma(float d2, float hg) { return exp2f(__fmul_rn(hg, log2f(d2))); }

// Debug and training outputs are indexed by a point's input index g, read from
// the leaf's point data: it is < n whenever the sort and the leaf partition are
// consistent.  Every such write goes through this check first (a failure voids
// the call's results instead of writing out of bounds).
__device__ __forceinline__ bool rec_index_ok(const LeafArgs &A, uint32_t g) {
  if (g < A.n) return true;
  atomicOr(&A.ctr->status, kStInternal);
  return false;
}

template <bool kRec>
__device__ __forceinline__ void write_point(const LeafArgs &A, uint32_t g, uint8_t mk, float sc, uint8_t st) {
  if (g >= A.n) {  // cannot happen with a consistent sort; never write out of bounds
    atomicOr(&A.ctr->status, kStInternal);
    return;
  }
  if (A.mask) A.mask[g] = mk;
  if (A.score) A.score[g] = sc;
  if (A.stage) A.stage[g] = st;
  if (kRec && A.use_train) {
    A.train.stage[g] = st;
    A.train.F[g] = sc;
  }
}

// ---------------------------------------------------------------------------
// one leaf
// ---------------------------------------------------------------------------
template <int KMAX, typename IdxT, bool kRec, bool kXl>
__device__ void process_leaf(const LeafArgs &A, const Leaf lf, const float4 *__restrict__ pts, const LeafMem &M,
                             LeafShared &S) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t NT = blockDim.x, NW = NT >> 5;  // 64 or 128 threads (execution knob)
  const uint32_t nt = lf.count;
  const denoise_params &P = A.p;
  const uint32_t lt = lanemask_lt();
  IdxT *nbr = (IdxT *)M.nbr;
  constexpr bool kPacked = sizeof(IdxT) == 2;  // shared-memory path: neighbour bitmaps
  const uint32_t nbB = nb_bits(M.cap);
  float *const X = M.X;
  float *const Y = M.Y;
  float *const Z = M.Z;
  uint32_t *const W = M.W;

  // ---- Eq. 10-11: the leaf's box origin and voxel size h come from the prep kernel
  if (tid == 0) {
    S.lo[0] = lf.lo[0];
    S.lo[1] = lf.lo[1];
    S.lo[2] = lf.lo[2];
    S.h = lf.h;
    S.delta = A.frames[lf.frame].delta;
    S.run = 0;
  }
  // structural variants (Sec. 4.3.2): stages switched off (A1 voxel gate, A2
  // density gate, A3 score selection) and the score on a kNN within P_2
  const bool a1_on = !(P.stage_off & 1u), a2_on = !(P.stage_off & 2u), a3_on = !(P.stage_off & 4u);
  // ---- Eq. 12: voxel occupancy (hash with warp-aggregated atomics)
  const uint32_t hcap = pow2ceil(2 * nt);  // <= the carved capacity
  for (uint32_t i = tid; i < hcap && a1_on; i += NT) {
    M.hkey[i] = kEmpty;
    M.hcnt[i] = 0;
  }
  __syncthreads();
  const float lo0 = S.lo[0], lo1 = S.lo[1], lo2 = S.lo[2], h = S.h;
  // each point's hash slot, for the gate below (wa is idle until the score weights)
  uint32_t *const vslot = reinterpret_cast<uint32_t *>(M.wa);
  for (uint32_t base = 0; base < nt && a1_on; base += NT) {
    const uint32_t i = base + tid;
    unsigned long long key = kInvalid;
    if (i < nt) {
      const float4 p = pts[i];
      key = ((unsigned long long)vox_index(p.x, lo0, h) << 42) |
            ((unsigned long long)vox_index(p.y, lo1, h) << 21) | (unsigned long long)vox_index(p.z, lo2, h);
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
    uint32_t sl = 0;
    if (i < nt && (peers & lt) == 0) {
      sl = hash_insert(M.hkey, hcap, key, A.ctr);
      atomicAdd(M.hcnt + sl, (uint32_t)__popc(peers));
    }
    sl = __shfl_sync(0xFFFFFFFFu, sl, __ffs(peers) - 1);  // the group's first lane inserted
    if (i < nt) vslot[i] = sl;
  }
  __syncthreads();
  // lookup, gate, compaction of P_1 (order preserved) into the coordinate arrays
  const uint32_t fbeg = A.frames[lf.frame].begin;
  for (uint32_t base = 0; base < nt; base += NT) {
    const uint32_t i = base + tid;
    bool in1 = false;
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t g = 0;
    if (i < nt) {
      p = pts[i];
      g = __float_as_uint(p.w);
      if (g >= A.n) {
        atomicOr(&A.ctr->status, kStInternal);
        g = 0;
      }
      const uint32_t c = a1_on ? M.hcnt[vslot[i]] : 0u;
      in1 = !a1_on || c >= P.min_vox_count;
      if (kXl && A.xphase == 1) A.xflag[lf.start + i] = in1 ? 1 : 0;
      if ((kRec && A.use_dbg) && !(kXl && A.xphase == 3)) {
        if (A.dbg.vox_count) A.dbg.vox_count[g] = c;
        if (A.dbg.leaf_start) A.dbg.leaf_start[g] = lf.start - fbeg;
        if (A.dbg.leaf_count) A.dbg.leaf_count[g] = nt;
        if (A.dbg.leaf_h) A.dbg.leaf_h[g] = h;
        if (A.dbg.leaf_rho_med) A.dbg.leaf_rho_med[g] = 0.0;
        if (A.dbg.r2) A.dbg.r2[g] = 0.0f;
      }
      if (!in1 && !(kXl && A.xphase == 1)) write_point<kRec>(A, g, 0, 0.0f, 1);
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in1);
    if (lane == 0) S.wsum[w] = __popc(bal);
    __syncthreads();
    uint32_t off = S.run;
    for (uint32_t ww = 0; ww < w; ++ww) off += S.wsum[ww];
    if (in1) {
      const uint32_t pos = off + __popc(bal & lt);
      X[pos] = p.x;
      Y[pos] = p.y;
      Z[pos] = p.z;
      W[pos] = g;
      M.spos[pos] = i;
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t t = 0;
      for (uint32_t ww = 0; ww < NW; ++ww) t += S.wsum[ww];
      S.run += t;
    }
    __syncthreads();
  }
  if (kXl && A.xphase == 1) return;  // cross-leaf mode: P_1 is marked, the kNN runs across leaves next
  uint32_t n1 = S.run;  // |P_1|; |P_2| once P_2 is compacted for its own kNN
  for (uint32_t u = tid; u < kPad; u += NT) {  // the NaN padding after P_1
    X[n1 + u] = __int_as_float(0x7FFFFFFF);
    Y[n1 + u] = __int_as_float(0x7FFFFFFF);
    Z[n1 + u] = __int_as_float(0x7FFFFFFF);
    W[n1 + u] = 0u;
  }
  if (!a2_on && !a3_on) {  // no gate or score needs a neighbour: P_1 is kept
    for (uint32_t i = tid; i < n1; i += NT) write_point<kRec>(A, W[i], 1, 0.0f, 0);
    if (tid == 0) {
      atomicAdd(&A.ctr->n_p1, (unsigned long long)n1);
      atomicAdd(&A.ctr->n_p2, (unsigned long long)n1);
    }
    return;
  }
  if (n1 <= 1) {  // no neighbour exists: the density gate cannot keep it
    // without the density gate the lone point is scored, F = 0 (an empty sum):
    // Top-lambda keeps ceil(lambda * 1) = 1 point, ln 0 >= tau never holds
    const bool keep = !a2_on && P.select_mode == DENOISE_SELECT_TOPRATIO;
    for (uint32_t i = tid; i < n1; i += NT)
      write_point<kRec>(A, W[i], keep ? 1 : 0, 0.0f, a2_on ? 2 : (keep ? 0 : 3));
    return;
  }
  uint32_t keff = (P.k < n1 - 1) ? P.k : n1 - 1;
  const bool xl = kXl && A.xphase == 3;  // cross-leaf mode: the kNN ran across leaves
  if (xl) {
    // k_eff is the leaf's (its candidates are shared by its points); 0: no neighbour at all
    keff = A.xkeff[lf.start + M.spos[0]];
    if (keff == 0) {
      for (uint32_t i = tid; i < n1; i += NT) write_point<kRec>(A, W[i], 0, 0.0f, 2);
      return;
    }
    for (uint32_t i = tid; i < n1; i += NT) M.r2[i] = A.xr2[lf.start + M.spos[i]];
  }
  // the neighbour bitmap (shared-memory path): region A if it fits, else the spill area
  auto bitmap_at = [&](uint32_t n) {
    return (bitmap_words(n) * 4u <= M.nbr_bytes) ? reinterpret_cast<uint32_t *>(M.nbr)
                                                  : reinterpret_cast<uint32_t *>(A.big_scratch + (size_t)lf.start * A.big_bpp);
  };
  uint32_t *tbl = bitmap_at(n1);
  if (tid == 0) {
    if (!xl) atomicAdd(&A.ctr->knn_pairs, (unsigned long long)n1 * (unsigned long long)(n1 - 1));
    atomicAdd(&A.ctr->n_p1, (unsigned long long)n1);
  }
  if (tid == NT - 1) {  // Eq. 14 rank (FP64, one thread), taken off the later critical path
    const double pos = __dadd_rn(__ddiv_rn(__dmul_rn((double)n1, (double)P.rho_percentile), 100.0), 0.5);
    const double cc = ceil(pos);
    S.crank = !a2_on ? 1u : (cc < 1.0) ? 1u : (cc > (double)n1) ? n1 : (uint32_t)cc;  // rank 1: nothing removed
    S.qblk = NW;
  }
  uint32_t sn = pow2ceil(n1);
  __syncthreads();  // P_1 and its padding complete
  uint32_t *const vbuf = reinterpret_cast<uint32_t *>(M.sbuf);
  // one kNN on P_1, and with rescore_p2 a second one within P_2 (its own k_eff, r_K, densities)
#pragma unroll 1
  for (uint32_t kpass = 0;; ++kpass) {

  // ---- kNN on P_1 (excluding self), order (d^2, input index): one thread per query,
  // candidates broadcast from shared memory to the warp, four per 16-byte load.
  // The k_eff smallest are found by counting, not by keeping a sorted list
  // (gd_knn_select.cuh): an upper bound theta_0 (the largest d^2 over a window
  // of Morton neighbours holding k_eff others) fixes 32 buckets of an eighth
  // of an octave below it; pass 1 counts every candidate into them (bit-sliced
  // counters), which locates the boundary bucket B and the number of
  // neighbours below it; pass 2 emits those neighbours in position order and
  // parks B's few members, which are sorted to finish the set.  A boundary
  // bucket with more members than the buffer is counted again at 32 times the
  // resolution first.  Ties in d^2 across the cut are broken by input index.
  if (keff > 0 && !xl) {  // (a single point of P_2 has no neighbour to score with: F = 0)
    constexpr int PL = kPacked ? 11 : 21;  // count planes: counts < 2^PL (n1 - 1 candidates)
    if (!kPacked && n1 >= (1u << PL)) {     // beyond the spill path's counters: refuse, do not guess
      if (tid == 0) atomicOr(&A.ctr->status, kStInternal);
      return;
    }
    uint32_t *const pend = M.pend;
    const float delta2 = __fmul_rn(S.delta, S.delta);
    const uint32_t cap = M.cap;
    const uint32_t pbits = nbB;  // position bits of a parked key
    const uint32_t pmask = (1u << pbits) - 1u;
    const uint32_t n16 = (n1 + 15u) >> 4;
    const bool dbg_n = (kRec && A.use_dbg) && A.dbg.nbr, dbg_d = (kRec && A.use_dbg) && A.dbg.nbr_d2;
    const bool use_cm = kPacked && n1 <= 1024u;  // bitmap rows of at most 32 words: chunk masks
    // the queries in blocks of 32, one block per warp at a time, taken first come
    // first served: a warp whose block needed a refinement pass does not hold the
    // next blocks back (warp w starts with block w, then takes S.qblk's next)
    const uint32_t nblk = (n1 + 31u) >> 5;
#pragma unroll 1
    for (uint32_t blk = w; blk < nblk;) {
      const uint32_t q = blk * 32u + lane;
      const bool act = q < n1;
      const uint32_t qq = act ? q : n1 - 1;          // idle lanes shadow a real query, results discarded
      const float xq = X[qq], yq = Y[qq], zq = Z[qq];
      const uint32_t gq = W[qq];
      const f32x2 QX = pk2(xq, xq), QY = pk2(yq, yq), QZ = pk2(zq, zq);
      // theta_0: the largest d^2 over the window [w0, w0 + k_eff] of Morton
      // neighbours (k_eff others at least), read in aligned steps of 4 (NaN padding ignored)
      float t0 = 0.0f;
      {
        uint32_t w0 = (qq > keff / 2) ? qq - keff / 2 : 0u;
        if (w0 > n1 - 1 - keff) w0 = n1 - 1 - keff;
        const uint32_t wa0 = w0 & ~3u, wsteps = (keff + 7u) >> 2;
        for (uint32_t s = 0; s < wsteps; ++s) {
          float d[4];
          sqdist4(X, Y, Z, wa0 + 4u * s, QX, QY, QZ, d);
          t0 = fmaxf(fmaxf(t0, d[0]), fmaxf(fmaxf(d[1], d[2]), d[3]));
        }
      }
      SelLevel L{__float_as_int(t0), -1, kSelS0, 0u, 0};
      SelCut cut;
      {
        // pass 1: every candidate (and the query itself, taken out in the walk) into the buckets
        uint32_t c[PL];
#pragma unroll
        for (int p = 0; p < PL; ++p) c[p] = 0u;
#pragma unroll 1
        for (uint32_t s = 0; s < n16; ++s) {
          uint32_t m[16];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float d[4];
            sqdist4(X, Y, Z, 16u * s + 4u * u, QX, QY, QZ, d);
#pragma unroll
            for (int v = 0; v < 4; ++v) m[4 * u + v] = sel_bucket_bit(L.tb, __float_as_int(d[v]), L.S);
          }
          sel_add16<PL>(c, m);
        }
        cut = sel_walk<PL>(c, L, keff);
        // refinements: count again inside the boundary bucket where it is too full
        // for the buffer (or too wide for a packed key); lanes that are done
        // repeat their own level and get the same result
#pragma unroll 1
        for (int level = 1;; ++level) {
          const bool single = cut.hi == cut.lo + 1;  // one d^2 value: exact ties, resolved below
          const bool again = act && !single && (cut.c_at > kSelBuf || !sel_fits(cut, pbits));
          if (!__any_sync(0xFFFFFFFFu, again)) break;
          if (level > kSelMaxLevels) {  // cannot happen: the range shrinks at every level
            atomicOr(&A.ctr->status, kStInternal);
            break;
          }
          if (again) L = sel_refine(L, cut);
#pragma unroll
          for (int p = 0; p < PL; ++p) c[p] = 0u;
#pragma unroll 1
          for (uint32_t s = 0; s < n16; ++s) {
            uint32_t m[16];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              float d[4];
              sqdist4(X, Y, Z, 16u * s + 4u * u, QX, QY, QZ, d);
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                const int32_t db = __float_as_int(d[v]);
                m[4 * u + v] = (db > L.lo) ? sel_bucket_bit(L.tb, db, L.S) : 0u;
              }
            }
            sel_add16<PL>(c, m);
          }
          cut = sel_walk<PL>(c, L, keff);
        }
      }
      const uint32_t need = keff - cut.c_below;     // 1 <= need <= c_at
      const bool ties_only = cut.c_at > kSelBuf;    // a single d^2 value with more members than the buffer
      const int32_t kbase = cut.lo + 1;              // smallest bits of bucket B's range
      // Record neighbour t of this query (position npos, input index g, distance d2).
      // Ranks come in order t = 0, 1, ...: the packed table is filled through a
      // bit buffer, one word store per 32 bits.
      uint32_t *const nbw = tbl + qq;  // this query's bitmap column: word c at nbw[c * n1]
      // with at most 32 chunks, only the words that hold neighbours are stored, and
      // cm marks them (the score reads those alone); otherwise every word is stored
      uint32_t cm = 0;
      auto set_bit = [&](uint32_t ju) {
        const uint32_t cw = ju >> 5, bit = 1u << (ju & 31u);
        if (!use_cm || ((cm >> cw) & 1u)) {
          nbw[(size_t)cw * n1] |= bit;
        } else {
          nbw[(size_t)cw * n1] = bit;
          cm |= 1u << cw;
        }
      };
      // Record neighbour t (position npos, input index g, distance d2) where the
      // table keeps positions (global path) and in the debug / training outputs.
      auto emit = [&](uint32_t t, uint32_t npos, uint32_t g, float d2) {
        if constexpr (!kPacked) nbr[(size_t)t * cap + qq] = (IdxT)npos;
        if (kRec && (dbg_n || dbg_d || A.use_train) && rec_index_ok(A, gq)) {
          if (dbg_n) A.dbg.nbr[(size_t)gq * P.k + t] = g;
          if (dbg_d) A.dbg.nbr_d2[(size_t)gq * P.k + t] = d2;
          if (A.use_train) {
            A.train.nbr[(size_t)gq * P.k + t] = g;
            A.train.nd2[(size_t)gq * P.k + t] = d2;
          }
        }
      };
      // pass 2, by chunks of 32 candidates: two bit masks (d^2 <= bottom of B's
      // range: a neighbour; d^2 <= top of B's range: B or below).  The
      // comparisons go through the FMA pipe: for IEEE subtraction (no flush to
      // zero) the sign bit of v - d^2 is set exactly when d^2 > v; a funnel shift
      // appends each sign bit, so the chunk's first candidate ends in bit 31.
      const float lo_f = cut.lo >= 0 ? __int_as_float(cut.lo) : -1.0f;
      const float hi_f = __int_as_float(cut.hi);
      const f32x2 LO2 = pk2(lo_f, lo_f), HI2 = pk2(hi_f, hi_f);
      uint32_t a = 0, np = 0;
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < n1; c0 += 32u) {
        uint32_t gtlo = 0, gthi = 0;
#pragma unroll 2
        for (uint32_t st = 0; st < 8; ++st) {
          float d[4];
          sqdist4(X, Y, Z, c0 + 4u * st, QX, QY, QZ, d);
          const f32x2 D0 = pk2(d[0], d[1]), D1 = pk2(d[2], d[3]);
          float e[4], f[4];
          upk2(sub2(LO2, D0), e[0], e[1]);
          upk2(sub2(LO2, D1), e[2], e[3]);
          upk2(sub2(HI2, D0), f[0], f[1]);
          upk2(sub2(HI2, D1), f[2], f[3]);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            gtlo = __funnelshift_l(__float_as_uint(e[u]), gtlo, 1);
            gthi = __funnelshift_l(__float_as_uint(f[u]), gthi, 1);
          }
        }
        const uint32_t le_lo = ~__brev(gtlo), le_hi = ~__brev(gthi);
        // the query itself is no candidate; positions past n1 (NaN padding) are dropped
        uint32_t keep = (qq - c0 < 32u) ? ~(1u << (qq - c0)) : 0xFFFFFFFFu;
        if (n1 - c0 < 32u) keep &= (1u << (n1 - c0)) - 1u;
        uint32_t em = le_lo & keep;
        uint32_t pm = le_hi & ~le_lo & keep;
        a += __popc(em);
        np += __popc(pm);
        if (!act || a > keff) em = 0;                  // nothing to record (a > keff: counts disagree, reported below)
        if (!act || ties_only || np > kSelBuf) pm = 0;
        uint32_t t = a - __popc(em), slot = np - __popc(pm);
        if constexpr (kPacked) {
          // the chunk's neighbours below the boundary bucket, one store
          if (act && (em || !use_cm)) nbw[(size_t)(c0 >> 5) * n1] = em;
          cm |= (em ? 1u : 0u) << ((c0 >> 5) & 31u);
        }
        if constexpr (!kPacked || kRec) {
          while (em) {
            const uint32_t ju = c0 + (uint32_t)(__ffs(em) - 1);
            em &= em - 1u;
            emit(t++, ju, W[ju], (kRec ? sqdist(xq, yq, zq, X[ju], Y[ju], Z[ju]) : 0.0f));
          }
        }
        while (pm) {
          const uint32_t ju = c0 + (uint32_t)(__ffs(pm) - 1);
          pm &= pm - 1u;
          const int32_t db = __float_as_int(sqdist(xq, yq, zq, X[ju], Y[ju], Z[ju]));
          pend[(slot++) * kLeafThreads + tid] = ((uint32_t)(db - kbase) << pbits) | ju;
        }
      }
      if (act && (a != cut.c_below || np != cut.c_at)) atomicOr(&A.ctr->status, kStInternal);  // passes agree
      // the need smallest of bucket B: sort the parked keys ((d^2 offset, position));
      // d^2 ties straddling the cut are ranked by input index
      float theta = hi_f;
      const bool parked = act && !ties_only;
      {
        uint32_t K[kSelBuf];
#pragma unroll
        for (int i = 0; i < (int)kSelBuf; ++i)
          K[i] = (parked && (uint32_t)i < np) ? pend[i * kLeafThreads + tid] : 0xFFFFFFFFu;
        // with at most 8 parked keys in every lane of the warp (the usual case) the
        // padding keys above them stay in place: a network on the first 8 suffices
        if (__reduce_max_sync(0xFFFFFFFFu, parked ? np : 0u) <= kSelBuf / 2) regsort_head<kSelBuf / 2>(K);
        else regsort_u<kSelBuf>(K);
        uint32_t th_off = 0;
#pragma unroll
        for (int i = 0; i < (int)kSelBuf; ++i) {
          th_off = ((uint32_t)i + 1u == need) ? (K[i] >> pbits) : th_off;
          if (parked) pend[i * kLeafThreads + tid] = K[i];  // sorted, for the emission loop below
        }
        uint32_t n_lt = 0, n_eq = 0;
#pragma unroll
        for (int i = 0; i < (int)kSelBuf; ++i) {
          n_lt += (K[i] >> pbits) < th_off;
          n_eq += (K[i] >> pbits) == th_off;  // padding keys have offsets above any real one
        }
        if (parked) theta = __int_as_float(kbase + (int32_t)th_off);
        // take the first `need` sorted keys, unless d^2 ties straddle the cut
        uint32_t take = parked ? ((need >= 32u) ? 0xFFFFFFFFu : ((1u << need) - 1u)) : 0u;
        const uint32_t need_eq = need - n_lt;
        if (parked && n_eq > need_eq) {  // rare: rank the keys at the cut distance by input index
          take = (n_lt >= 32u) ? 0xFFFFFFFFu : ((1u << n_lt) - 1u);
#pragma unroll 1
          for (uint32_t i = n_lt; i < n_lt + n_eq; ++i) {
            const uint32_t gi = W[pend[i * kLeafThreads + tid] & pmask];
            uint32_t before = 0;
#pragma unroll 1
            for (uint32_t j = n_lt; j < n_lt + n_eq; ++j) before += W[pend[j * kLeafThreads + tid] & pmask] < gi;
            if (before < need_eq) take |= 1u << i;
          }
        }
        while (take) {
          const uint32_t i = (uint32_t)(__ffs(take) - 1);
          take &= take - 1u;
          const uint32_t key = pend[i * kLeafThreads + tid], ju = key & pmask;
          if constexpr (kPacked) set_bit(ju);
          emit(a++, ju, W[ju], __int_as_float(kbase + (int32_t)(key >> pbits)));
        }
      }
      // exact ties beyond the buffer (lattices, duplicates): one scan per missing
      // neighbour takes the smallest input index above the last one taken
      const uint32_t rounds = (act && ties_only) ? need : 0u;
      const uint32_t max_rounds = __reduce_max_sync(0xFFFFFFFFu, rounds);
      uint32_t last = 0;
#pragma unroll 1
      for (uint32_t r = 0; r < max_rounds; ++r) {
        uint32_t bg = 0xFFFFFFFFu, bp = 0;
#pragma unroll 1
        for (uint32_t j = 0; j < n1; ++j) {
          const float d2 = sqdist(xq, yq, zq, X[j], Y[j], Z[j]);
          const uint32_t g = W[j];
          if (r < rounds && j != qq && d2 == hi_f && (r == 0 || g > last) && g < bg) {
            bg = g;
            bp = j;
          }
        }
        if (r < rounds) {
          if constexpr (kPacked) set_bit(bp);
          emit(a++, bp, bg, hi_f);
          last = bg;
        }
      }
      if constexpr (!kPacked) {
        // the global path's list in position order (the order of the bitmap rows):
        // the neighbours below the boundary bucket came in order, the rest are inserted
        if (act) {
#pragma unroll 1
          for (uint32_t t = cut.c_below; t < keff && t < a; ++t) {
            const IdxT v = nbr[(size_t)t * cap + qq];
            uint32_t u = t;
            while (u > 0 && nbr[(size_t)(u - 1) * cap + qq] > v) {
              nbr[(size_t)u * cap + qq] = nbr[(size_t)(u - 1) * cap + qq];
              --u;
            }
            nbr[(size_t)u * cap + qq] = v;
          }
        }
      }
      if (act) {
        if (a != keff) atomicOr(&A.ctr->status, kStInternal);
        const float rt = (theta < delta2) ? delta2 : theta;
        M.r2[qq] = rt;
        if (kPacked && use_cm) M.cmask[qq] = cm;
        if (kRec && (A.use_dbg || A.use_train) && rec_index_ok(A, gq)) {
          for (uint32_t t = keff; t < P.k; ++t) {
            if (dbg_n) A.dbg.nbr[(size_t)gq * P.k + t] = 0xFFFFFFFFu;
            if (dbg_d) A.dbg.nbr_d2[(size_t)gq * P.k + t] = 0.0f;
            if (A.use_train) {
              A.train.nbr[(size_t)gq * P.k + t] = 0xFFFFFFFFu;
              A.train.nd2[(size_t)gq * P.k + t] = 0.0f;
            }
          }
          if (A.use_dbg && A.dbg.r2) A.dbg.r2[gq] = rt;
          if (A.use_train) A.train.r2[gq] = rt;
        }
      }
      uint32_t nb = 0;
      if (lane == 0) nb = atomicAdd(&S.qblk, 1u);
      blk = __shfl_sync(0xFFFFFFFFu, nb, 0);
    }
  }
  __syncthreads();

  // ---- Eq. 14: exact percentile cut, as a rank cut on r_K^2 (rho decreasing in r_K);
  // after the kNN within P_2 every point is in P_2 (the sort serves the median)
  for (uint32_t i = tid; i < sn; i += NT) vbuf[i] = (i < n1) ? __float_as_uint(M.r2[i]) : 0xFFFFFFFFu;
  __syncthreads();
  block_sort<uint32_t>(vbuf, sn, 0xFFFFFFFFu);
  const uint32_t Rb = kpass == 0 ? vbuf[n1 - S.crank] : 0xFFFFFFFFu;
  for (uint32_t i = tid; i < n1; i += NT) {
    const uint32_t v = vbuf[i];
    if (v <= Rb && (i + 1 == n1 || vbuf[i + 1] > Rb)) S.m = i + 1;
    M.flag[i] = (__float_as_uint(M.r2[i]) <= Rb) ? 1 : 0;
  }
  __syncthreads();
  if (kpass > 0 || (a3_on && !P.rescore_p2)) break;
  if (!a3_on) {  // no score selection: P_2 is kept with score 0
    for (uint32_t i = tid; i < n1; i += NT) {
      const uint8_t f = M.flag[i];
      write_point<kRec>(A, W[i], f ? 1 : 0, 0.0f, f ? 0 : 2);
    }
    if (tid == 0) atomicAdd(&A.ctr->n_p2, (unsigned long long)S.m);
    return;
  }
  // rescore_p2: the points the density gate removed get their results now, and
  // P_2 is compacted in place (order kept) for its own kNN
  if (tid == 0) S.run = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n1; base += NT) {
    const uint32_t i = base + tid;
    const bool in2 = i < n1 && M.flag[i];
    float x = 0.f, y = 0.f, z = 0.f;
    uint32_t g = 0;
    if (i < n1) {
      x = X[i];
      y = Y[i];
      z = Z[i];
      g = W[i];
      if (!in2) write_point<kRec>(A, g, 0, 0.0f, 2);
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, in2);
    if (lane == 0) S.wsum[w] = __popc(bal);
    __syncthreads();  // every read of this round is done before the writes below
    uint32_t off = S.run;
    for (uint32_t ww = 0; ww < w; ++ww) off += S.wsum[ww];
    if (in2) {
      const uint32_t pos = off + __popc(bal & lt);  // <= i: never ahead of a later round's reads
      X[pos] = x;
      Y[pos] = y;
      Z[pos] = z;
      W[pos] = g;
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t t = 0;
      for (uint32_t ww = 0; ww < NW; ++ww) t += S.wsum[ww];
      S.run += t;
    }
    __syncthreads();
  }
  n1 = S.run;
  for (uint32_t u = tid; u < kPad; u += NT) {
    X[n1 + u] = __int_as_float(0x7FFFFFFF);
    Y[n1 + u] = __int_as_float(0x7FFFFFFF);
    Z[n1 + u] = __int_as_float(0x7FFFFFFF);
    W[n1 + u] = 0u;
  }
  keff = n1 <= 1 ? 0u : (P.k < n1 - 1) ? P.k : n1 - 1;
  tbl = bitmap_at(n1);
  sn = pow2ceil(n1);
  if (tid == 0) S.qblk = NW;
  if (tid == 0 && keff) atomicAdd(&A.ctr->knn_pairs, (unsigned long long)n1 * (unsigned long long)(n1 - 1));
  __syncthreads();
  }  // kpass
  const uint32_t m = S.m;
  // ---- Eq. 16: median density over P_2 and the per-leaf constants of the score.
  // With rho(r2) = k_eff / (4/3 pi r2^1.5), the score needs
  // ell_i = log2(rho_i / sqrt(rho_med^2 + eps_rho)) = Lref - 1.5 log2(r2_i / r2ref)
  // with r2ref the lower-middle r2 of P_2 and Lref = log2(rho(r2ref)) -
  // log2(rho_med) - 0.5 log2(1 + eps_rho / rho_med^2).  Every term is a log2 of a
  // ratio near 1 (or the eps correction), evaluated in FP32 without overflow.
  if (tid == 0) {
    const float ra = __uint_as_float(vbuf[(m - 1) / 2]);
    const float rb = (m & 1u) ? ra : __uint_as_float(vbuf[m / 2]);
    S.r2ref = ra;
    S.Lref = leaf_lref(ra, rb, m, keff, P.eps_rho);
    S.lshift = __fsub_rn(__fsub_rn(__fsub_rn(log2f((float)keff), 2.0665336287511624f), __fmul_rn(1.5f, log2f(ra))),
                         S.Lref);
    S.keep_n = (uint32_t)ceil((double)P.lambda * (double)m);
    if (S.keep_n > m) S.keep_n = m;
    atomicAdd(&A.ctr->n_p2, (unsigned long long)m);
    atomicAdd(&A.ctr->score_terms, (unsigned long long)m * keff);
    if ((kRec && A.use_dbg) && A.dbg.leaf_rho_med) {  // exact FP64 value for the parity output only
      const double k43pi = (4.0 / 3.0) * 3.14159265358979323846;
      auto rho_of = [&](float r2) {
        const double rr = (double)r2;
        return (double)keff / __dmul_rn(k43pi, __dmul_rn(rr, sqrt(rr)));
      };
      S.rho_med = (m & 1u) ? rho_of(ra) : 0.5 * (rho_of(__uint_as_float(vbuf[m / 2 - 1])) + rho_of(rb));
    }
  }
  __syncthreads();
  // distance weight exponent: w_dis = 2^(-d^2 c_i) with c_i = c2 / r2_i, c2 = log2(e) / (2 sigma^2)
  const float c2 = __fdiv_rn(1.4426950408889634f, __fmul_rn(__fmul_rn(2.0f, P.sigma), P.sigma));
  {
    const float r2ref = S.r2ref, Lref = S.Lref;
    const float half_alpha = __fmul_rn(0.5f, P.alpha);
    for (uint32_t i = tid; i < n1; i += NT) {
      const float r2 = M.r2[i];
      const float ell = __fsub_rn(Lref, __fmul_rn(1.5f, log2f(__fdiv_rn(r2, r2ref))));  // log2(rho_i / sqrt(rho_med^2 + eps))
      const float wa = __fmul_rn(half_alpha, ell);
      M.wa[i] = wa;
      // shared-memory leaves: each point's (x, y, z, weight) in one 16-byte word for
      // the score's neighbour reads (region R is idle between the median and Top-lambda)
      if constexpr (kPacked) reinterpret_cast<float4 *>(M.sbuf)[i] = make_float4(X[i], Y[i], Z[i], wa);
      if (kRec && A.use_train) {
        const uint32_t g = W[i];
        if (rec_index_ok(A, g)) A.train.ell[g] = ell;
      }
    }
  }
  __syncthreads();
  // ---- Eq. 15-21: dual-weight gravitational score of every P_2 point.  Every FP32
  // operation of the score, and of the per-leaf and per-point constants above, is an
  // explicit round-to-nearest intrinsic: no contraction is left to the compiler, so
  // the shared-memory and global-memory instantiations give bit-identical scores.
  {
    const bool g2 = (P.gamma == 2.0f);
    const float hg = 0.5f * P.gamma, ek = P.eps_k;
    for (uint32_t i = tid; i < n1; i += NT) {
      if (!M.flag[i]) continue;
      const float xi = X[i], yi = Y[i], zi = Z[i];
      const float ai = M.wa[i], ci = __fdiv_rn(c2, M.r2[i]);  // r2_i's last read: F_i takes its place
      // two neighbours per step into two partial sums (independent chains),
      // F = even-rank terms + odd-rank terms
      float F0 = 0.0f, F1 = 0.0f;
      // neighbours in position order: from the bitmap row (shared memory) or the
      // position-ordered list (global path)
      const uint32_t *row = tbl + i;  // word c at row[c * n1]
      // with chunk masks (at most 32 words) only the words that hold neighbours are
      // read, the next one loaded while the current one is consumed (the row may be
      // in the spill area); otherwise the row is read word by word
      const uint32_t rwords = (n1 + 31u) >> 5;
      const bool cmk_on = !xl && kPacked && n1 <= 1024u;
      // the mask is written by the kNN of this leaf (k_eff > 0); only chunks of the row are taken
      uint32_t cmk = (cmk_on && keff > 0) ? M.cmask[i] & ((rwords >= 32u) ? 0xFFFFFFFFu : ((1u << rwords) - 1u)) : 0u;
      auto pop_chunk = [&]() -> uint32_t {  // next chunk of the mask (32 if none is left)
        const uint32_t c = cmk ? (uint32_t)(__ffs(cmk) - 1) : 32u;
        cmk &= cmk - 1u;
        return c;
      };
      uint32_t rc = 0, rm = 0, pc = 32, pm = 0;
      if (kPacked && !xl && keff > 0) {
        if (cmk_on) {
          rc = pop_chunk();
          rm = rc < 32u ? row[(size_t)rc * n1] : 0u;
          pc = pop_chunk();
          pm = pc < 32u ? row[(size_t)pc * n1] : 0u;
        } else {
          rm = row[0];
        }
      }
      auto next_j = [&](uint32_t t, bool valid) -> uint32_t {  // called for t = 0, 1, ... in order
        if constexpr (kPacked) {
          if (!valid) return 0u;
          if (cmk_on) {
            while (rm == 0u && pc < 32u) {  // take the prefetched word, load the one after it
              rm = pm;
              rc = pc;
              pc = pop_chunk();
              pm = pc < 32u ? row[(size_t)pc * n1] : 0u;
            }
          } else {
            while (rm == 0u && rc + 1 < rwords) rm = row[(size_t)(++rc) * n1];
          }
          const uint32_t j = (rc << 5) + (uint32_t)(__ffs(rm) - 1);  // rm == 0 only if the row is inconsistent
          rm &= rm - 1u;
          return j < n1 ? j : 0u;
        } else {
          return valid ? (uint32_t)nbr[(size_t)t * M.cap + i] : 0u;
        }
      };
      if (xl) {
        // cross-leaf neighbours: coordinates and densities from the global results,
        // ell_j = log2(rho_j) - lshift with rho_j from the neighbour's own k_eff and r_K
        const uint32_t *nl = A.xnbr + (size_t)(lf.start + M.spos[i]) * P.k;
        const float half_alpha = __fmul_rn(0.5f, P.alpha), lsh = S.lshift;
#pragma unroll 1
        for (uint32_t t = 0; t < keff; ++t) {
          const uint32_t j = nl[t];
          const float4 pj = A.spts[j];
          const float d2 = sqdist(xi, yi, zi, pj.x, pj.y, pj.z);
          const float lj = __fsub_rn(__fsub_rn(log2f((float)A.xkeff[j]), 2.0665336287511624f),
                                     __fmul_rn(1.5f, log2f(A.xr2[j])));
          const float waj = __fmul_rn(half_alpha, __fsub_rn(lj, lsh));
          const float wt = ex2_hw(__fmaf_rn(-d2, ci, __fadd_rn(ai, waj)));
          const float D = g2 ? d2 : pow_half_gamma(d2, hg);
          const float e = __fmul_rn(wt, rcp_hw(__fadd_rn(D, ek)));
          if (t & 1u) F1 = __fadd_rn(F1, e);
          else F0 = __fadd_rn(F0, e);
        }
        M.F[i] = __fadd_rn(F0, F1);
        continue;
      }
      // two ranks per step in the two lanes of packed FP32 instructions (even ranks
      // in the low lane, odd in the high: the two partial sums); each lane rounds as
      // the scalar form.  With k_eff odd the last step's second term is computed on
      // the first neighbour again and replaced by +0.
      const f32x2 XI = pk2(xi, xi), YI = pk2(yi, yi), ZI = pk2(zi, zi), AI = pk2(ai, ai);
      const f32x2 NCI = pk2(-ci, -ci), EK = pk2(ek, ek);
      f32x2 FF = pk2(0.0f, 0.0f);
#pragma unroll 1
      for (uint32_t t = 0; t < keff; t += 2) {
        const bool two = t + 1 < keff;
        const uint32_t ja = next_j(t, true);
        uint32_t jb = next_j(t + 1, two);
        jb = two ? jb : ja;
        float4 pa, pb;
        if constexpr (kPacked) {
          pa = reinterpret_cast<const float4 *>(M.sbuf)[ja];
          pb = reinterpret_cast<const float4 *>(M.sbuf)[jb];
        } else {
          pa = make_float4(X[ja], Y[ja], Z[ja], M.wa[ja]);
          pb = make_float4(X[jb], Y[jb], Z[jb], M.wa[jb]);
        }
        const f32x2 DX = sub2(pk2(pa.x, pb.x), XI), DY = sub2(pk2(pa.y, pb.y), YI), DZ = sub2(pk2(pa.z, pb.z), ZI);
        const f32x2 D2 = fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
        float ea, eb, da, db;
        upk2(fma2(D2, NCI, add2(AI, pk2(pa.w, pb.w))), ea, eb);  // -d^2 c_i + (alpha/2)(ell_i + ell_j)
        upk2(D2, da, db);
        const f32x2 DG = g2 ? D2 : pk2(pow_half_gamma(da, hg), pow_half_gamma(db, hg));
        float qa, qb;
        upk2(add2(DG, EK), qa, qb);
        float ta, tb;
        upk2(mul2(pk2(ex2_hw(ea), ex2_hw(eb)), pk2(rcp_hw(qa), rcp_hw(qb))), ta, tb);
        FF = add2(FF, pk2(ta, two ? tb : 0.0f));
      }
      upk2(FF, F0, F1);
      M.F[i] = __fadd_rn(F0, F1);
    }
  }
  __syncthreads();
  // ---- selection: Top-lambda per leaf by (F desc, input index asc), or ln F >= tau.
  if (P.select_mode == DENOISE_SELECT_TOPRATIO) {
    // 32-bit keys ~F (F >= 0: the bit pattern orders like the value) are sorted; the
    // keep_n-th key is the cut value; the P_2 points below it are kept, and of those
    // at it, the ones needed to reach keep_n in input-index order (all of them
    // unless scores tie exactly at the cut).
    uint32_t *const kb = reinterpret_cast<uint32_t *>(M.sbuf);
    for (uint32_t i = tid; i < sn; i += NT)
      kb[i] = (i < n1 && M.flag[i]) ? 0xFFFFFFFFu - __float_as_uint(M.F[i]) : 0xFFFFFFFFu;
    if (tid == 0) S.nless = S.ntied = 0;
    __syncthreads();
    block_sort<uint32_t>(kb, sn, 0xFFFFFFFFu);
    const uint32_t cut = kb[S.keep_n - 1];
    uint32_t nl = 0, nt = 0;
    for (uint32_t i = tid; i < n1; i += NT) {
      if (!M.flag[i]) continue;
      const uint32_t key = 0xFFFFFFFFu - __float_as_uint(M.F[i]);
      nl += key < cut;
      nt += key == cut;
    }
    nl = __reduce_add_sync(0xFFFFFFFFu, nl);
    nt = __reduce_add_sync(0xFFFFFFFFu, nt);
    if (lane == 0) {
      atomicAdd(&S.nless, nl);
      atomicAdd(&S.ntied, nt);
    }
    __syncthreads();
    const uint32_t needed = S.keep_n - S.nless, tied = S.ntied;  // 1 <= needed <= tied
    for (uint32_t i = tid; i < n1; i += NT) {
      if (!M.flag[i]) continue;
      const uint32_t key = 0xFFFFFFFFu - __float_as_uint(M.F[i]);
      bool keep = key < cut;
      if (key == cut) {
        if (needed >= tied) {
          keep = true;
        } else {  // exact score ties at the cut: rank the tied points by input index
          const uint32_t g = W[i];
          uint32_t before = 0;
          for (uint32_t j2 = 0; j2 < n1; ++j2)
            before += (M.flag[j2] && 0xFFFFFFFFu - __float_as_uint(M.F[j2]) == cut &&
                       W[j2] < g);
          keep = before < needed;
        }
      }
      M.flag[i] = keep ? 2 : 1;
    }
  } else {
    for (uint32_t i = tid; i < n1; i += NT)
      if (M.flag[i]) M.flag[i] = (logf(M.F[i]) >= P.tau) ? 2 : 1;
  }
  __syncthreads();
  // ---- Eq. 22: results in input order
  const double rho_med = S.rho_med;
  for (uint32_t i = tid; i < n1; i += NT) {
    const uint32_t g = W[i];
    const uint8_t f = M.flag[i];
    if (f == 0) write_point<kRec>(A, g, 0, 0.0f, 2);
    else write_point<kRec>(A, g, f == 2, M.F[i], f == 2 ? 0 : 3);
    if (kRec && A.use_dbg && A.dbg.leaf_rho_med && g < A.n) A.dbg.leaf_rho_med[g] = rho_med;
  }
}

// ---------------------------------------------------------------------------
// persistent kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Persistent CTAs of 128 threads, GD_LEAF_MIN_CTAS per SM for K <= 32 (a
// 512-point leaf takes 33 KB of shared memory, so 6 fit; the register bound
// follows from the count).  kRec: the debug / training outputs are written (a
// separate instantiation, so that the plain path carries none of their code).
#ifndef GD_LEAF_MIN_CTAS
#define GD_LEAF_MIN_CTAS 6
#endif
template <int KMAX, bool kRec, bool kXl>
__global__ void __launch_bounds__(kLeafThreads, (KMAX >= 64) ? 1 : GD_LEAF_MIN_CTAS) k_leaf(const LeafArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ LeafShared S;
  const uint32_t tid = threadIdx.x;
  const uint32_t lmax = A.lmax;
  LeafMem Ms;
  carve<uint16_t>(smem, lmax, KMAX, &Ms);
  float4 *const s_pts = Ms.raw;  // the raw points land here, P_1 is compacted out of them
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();
  // the part of the largest-first order this launch takes: every leaf, or those
  // before the split (more than kSmallLeaf points), or from it (the small leaves)
  const uint32_t n_all = A.ctr->n_leaves, split = A.ctr->split_leaf;
  const uint32_t w_lo = (A.part == 2) ? split : 0u, w_hi = (A.part == 1) ? split : n_all;
  uint32_t *const wctr = (kXl && A.xphase == 3) ? &A.ctr->leaf_work2
                         : (A.part == 2)         ? &A.ctr->leaf_work3
                                                 : &A.ctr->leaf_work;
  uint32_t phase = 0;
  for (;;) {
    if (tid == 0) S.leaf = (ld_volatile(&A.ctr->status) & kStFatal) ? 0xFFFFFFFFu : w_lo + atomicAdd(wctr, 1u);
    __syncthreads();
    const uint32_t wi = S.leaf;  // block-uniform: one thread decided
    if (wi >= w_hi) break;
    const Leaf lf = A.leaves[A.order[wi]];
    if (lf.count <= lmax) {
      if (tid == 0) {
        const uint32_t bytes = lf.count * 16u;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_pts);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(__cvta_generic_to_global(A.spts + lf.start)), "r"(bytes), "r"(bar)
            : "memory");
      }
      const bool ok = mbar_wait(bar, phase, A.spin_limit);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(&A.ctr->status, kStTimeout);
        (void)mbar_wait(bar, phase, A.spin_limit);  // let the copy in flight land before exiting
        return;
      }
      phase ^= 1u;
      process_leaf<KMAX, uint16_t, kRec, kXl>(A, lf, s_pts, Ms, S);
    } else {
      LeafMem Mg;
      carve<uint32_t>(A.big_scratch + (size_t)lf.start * A.big_bpp, lf.count, KMAX, &Mg);
      Mg.pend = Ms.pend;  // the per-query parked keys live in shared memory on this path too
      process_leaf<KMAX, uint32_t, kRec, kXl>(A, lf, A.spts + lf.start, Mg, S);
    }
    __syncthreads();
  }
}

template <int KMAX, bool kRec, bool kXl>
inline int launch_k(const LeafArgs &a, int num_sms, cudaStream_t st) {
  const size_t smem = leaf_smem_bytes(a.lmax, KMAX);
  // per call (function attributes are per device, and calls may come from several threads)
  if (cudaFuncSetAttribute(k_leaf<KMAX, kRec, kXl>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return -1;
  cudaFuncSetAttribute(k_leaf<KMAX, kRec, kXl>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  const int nt = (a.threads == 64) ? 64 : kLeafThreads;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf<KMAX, kRec, kXl>, nt, smem) != cudaSuccess ||
      per_sm < 1)
    return -1;
  if (a.ctas_per_sm > 0 && (int)a.ctas_per_sm < per_sm) per_sm = (int)a.ctas_per_sm;
  LeafArgs la = a;
  if (la.spin_limit == 0) la.spin_limit = kSpinLimit;
  if (launch_pdl(k_leaf<KMAX, kRec, kXl>, num_sms * per_sm, nt, smem, st, la) != cudaSuccess) return -1;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <bool kRec, bool kXl>
inline int launch_kmax(const LeafArgs &a, int num_sms, cudaStream_t st) {
  switch (leaf_kmax(a.p.k)) {
    case 8: return launch_k<8, kRec, kXl>(a, num_sms, st);
    case 16: return launch_k<16, kRec, kXl>(a, num_sms, st);
    case 32: return launch_k<32, kRec, kXl>(a, num_sms, st);
    default: return launch_k<64, kRec, kXl>(a, num_sms, st);
  }
}

}  // namespace gd
