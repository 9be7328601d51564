// gd_eval.cu -- two cross-set passes over a pair of clouds, on the GPU:
//  - the evaluation metrics of Sec. 4.1: Eq. 29's PSNR (mean squared distance of
//    each clean point to its nearest denoised point, M = the clean cloud's
//    bounding-box diagonal) and Eq. 30's Chamfer distance (both directions);
//  - the gravitational-function baseline of Sec. 2.2 (Eq. 1-9): centroid,
//    extents, radius R, neighbour counts n_i within R, and the keep rule
//    F_i >= T / d_i.
//
// Both need, for every query point, a reduction over every point of another
// set (or the same set): the nearest squared distance, or the count within R.
// Nothing is skipped: each query meets each candidate once, so the pass is
// bound by the FP32 pipe (d^2 = fma(dz,dz,fma(dy,dy,dx*dx)), the method's fixed
// operation order, in packed two-lane form), not by memory.  The candidates are
// packed as structure of arrays and staged through shared memory by TMA bulk
// copies (double-buffered, mbarrier, bounded waits); every thread holds four
// queries in registers, so one broadcast 16-byte load per coordinate feeds
// sixteen query-candidate pairs.  Work units are (1,024 queries, a chunk of
// candidates); the chunks of a query block combine by integer atomics on the
// result (min of non-negative float bits, or a count), which do not depend on
// order.  FP64 sums are taken by fixed-order block reductions, so results are
// deterministic.
#include <cuda_runtime.h>
#include <math.h>

#include "gd_common.cuh"
#include "gd_f32x2.cuh"

namespace gd {

constexpr int kEvThreads = 256;
constexpr int kEvQPT = 4;                         // queries per thread
constexpr int kEvQueries = kEvThreads * kEvQPT;   // queries per work unit
constexpr int kEvTile = 2048;                     // candidates per shared-memory tile
constexpr size_t kEvSmem = 2ull * 3 * kEvTile * sizeof(float);  // two buffers of X, Y, Z: 48 KB
constexpr int kEvRedThreads = 256;

// ---------------------------------------------------------------------------
// packing and reductions
// ---------------------------------------------------------------------------
// xyz [n][3] -> X, Y, Z [npad] (npad = n rounded up to 4), padded with +inf:
// a padding candidate is at infinite distance (never nearest, never within R)
__global__ void k_ev_pack(const float *__restrict__ xyz, uint32_t n, uint32_t npad, float *__restrict__ X,
                          float *__restrict__ Y, float *__restrict__ Z, Counters *ctr) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
    float x = INFINITY, y = INFINITY, z = INFINITY;
    if (i < n) {
      x = xyz[3ull * i];
      y = xyz[3ull * i + 1];
      z = xyz[3ull * i + 2];
      if (!isfinite(x) || !isfinite(y) || !isfinite(z)) atomicOr(&ctr->status, kStNonFinite);
    }
    X[i] = x;
    Y[i] = y;
    Z[i] = z;
  }
}

// Per block: FP64 sums of x, y, z and the FP32 min / max of each axis (stored as
// doubles, exactly).  part[b] = {sx, sy, sz, min x, min y, min z, max x, max y, max z}.
__global__ void __launch_bounds__(kEvRedThreads) k_ev_reduce(const float *__restrict__ X, const float *__restrict__ Y,
                                                             const float *__restrict__ Z, uint32_t n,
                                                             double *__restrict__ part) {
  __shared__ double s_sum[3][kEvRedThreads];
  __shared__ float s_mn[3][kEvRedThreads], s_mx[3][kEvRedThreads];
  const uint32_t t = threadIdx.x;
  double s[3] = {0.0, 0.0, 0.0};
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;  // a contiguous slice per block
  const uint32_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  for (uint32_t i = b0 + t; i < b1; i += kEvRedThreads) {
    const float v[3] = {X[i], Y[i], Z[i]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s[c] = __dadd_rn(s[c], (double)v[c]);
      mn[c] = fminf(mn[c], v[c]);
      mx[c] = fmaxf(mx[c], v[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    s_sum[c][t] = s[c];
    s_mn[c][t] = mn[c];
    s_mx[c][t] = mx[c];
  }
  __syncthreads();
  for (uint32_t h = kEvRedThreads / 2; h > 0; h >>= 1) {  // fixed tree: deterministic
    if (t < h) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s_sum[c][t] = __dadd_rn(s_sum[c][t], s_sum[c][t + h]);
        s_mn[c][t] = fminf(s_mn[c][t], s_mn[c][t + h]);
        s_mx[c][t] = fmaxf(s_mx[c][t], s_mx[c][t + h]);
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    double *o = part + 9ull * blockIdx.x;
    for (int c = 0; c < 3; ++c) {
      o[c] = s_sum[c][0];
      o[3 + c] = (double)s_mn[c][0];
      o[6 + c] = (double)s_mx[c][0];
    }
  }
}

// FP64 sum of the float values v[0..n) (bits of non-negative floats), per block
__global__ void __launch_bounds__(kEvRedThreads) k_ev_sum(const uint32_t *__restrict__ v, uint32_t n,
                                                          double *__restrict__ part) {
  __shared__ double s[kEvRedThreads];
  const uint32_t t = threadIdx.x;
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  double a = 0.0;
  for (uint32_t i = b0 + t; i < b1; i += kEvRedThreads) a = __dadd_rn(a, (double)__uint_as_float(v[i]));
  s[t] = a;
  __syncthreads();
  for (uint32_t h = kEvRedThreads / 2; h > 0; h >>= 1) {
    if (t < h) s[t] = __dadd_rn(s[t], s[t + h]);
    __syncthreads();
  }
  if (t == 0) part[blockIdx.x] = s[0];
}

__global__ void k_ev_fill(uint32_t *__restrict__ v, uint32_t n, uint32_t value) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = value;
}

// ---------------------------------------------------------------------------
// the cross-set pass
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool ev_wait(uint32_t bar, uint32_t phase, uint32_t limit) {
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

__device__ __forceinline__ void ev_issue(uint32_t bar, float *dst, const float *src, uint32_t bytes) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          (uint32_t)__cvta_generic_to_shared(dst)),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
      : "memory");
}

struct CrossArgs {
  const float *qx, *qy, *qz;  // queries (structure of arrays, padded)
  uint32_t nq;
  const float *cx, *cy, *cz;  // candidates (structure of arrays, padded with +inf to a multiple of 4)
  uint32_t ncand;             // candidates incl. padding (multiple of 4)
  uint32_t nchunks;           // candidate chunks per query block
  uint32_t chunk;             // candidates per chunk (multiple of kEvTile)
  float r2f;                  // MODE 1: count d^2 <= r2f ...
  const float *r2f_dev;       // ... or <= *r2f_dev when set (a value computed on the device)
  uint32_t *out;              // [nq]: MODE 0 bits of the min d^2 (preset to +inf), MODE 1 counts (preset to 0)
  Counters *ctr;
  uint32_t spin_limit;
};

// MODE 0: nearest squared distance; MODE 1: count within the radius.
template <int MODE>
__global__ void __launch_bounds__(kEvThreads) k_ev_cross(const CrossArgs A) {
  extern __shared__ __align__(128) float ev_sm[];
  __shared__ __align__(8) unsigned long long s_bar[2];
  const uint32_t tid = threadIdx.x;
  const uint32_t qb = blockIdx.x / A.nchunks, cb = blockIdx.x % A.nchunks;
  const uint32_t c_begin = cb * A.chunk, c_end = min(A.ncand, c_begin + A.chunk);
  if (c_begin >= c_end) return;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&s_bar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // queries in registers (padding queries repeat the last one; their results are dropped)
  f32x2 QX[kEvQPT], QY[kEvQPT], QZ[kEvQPT];
  float best[kEvQPT];
  uint32_t cnt[kEvQPT];
#pragma unroll
  for (int k = 0; k < kEvQPT; ++k) {
    uint32_t q = qb * kEvQueries + tid + k * kEvThreads;
    q = q < A.nq ? q : A.nq - 1;
    QX[k] = pk2(A.qx[q], A.qx[q]);
    QY[k] = pk2(A.qy[q], A.qy[q]);
    QZ[k] = pk2(A.qz[q], A.qz[q]);
    best[k] = INFINITY;
    cnt[k] = 0;
  }
  const float r2 = A.r2f_dev ? *A.r2f_dev : A.r2f;
  const f32x2 R2 = pk2(r2, r2);
  const uint32_t ntiles = (c_end - c_begin + kEvTile - 1) / kEvTile;
  auto issue = [&](uint32_t i) {  // thread 0: tile i of the chunk into buffer i & 1
    const uint32_t c0 = c_begin + i * kEvTile;
    const uint32_t len = min((uint32_t)kEvTile, c_end - c0);  // multiple of 4: 16-byte copies
    const uint32_t bar = (i & 1) ? bar1 : bar0;
    float *buf = ev_sm + (i & 1) * 3 * kEvTile;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(3u * len * 4u) : "memory");
    ev_issue(bar, buf, A.cx + c0, len * 4u);
    ev_issue(bar, buf + kEvTile, A.cy + c0, len * 4u);
    ev_issue(bar, buf + 2 * kEvTile, A.cz + c0, len * 4u);
  };
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(0);
  }
  int failed_at = -1;
  for (uint32_t i = 0; i < ntiles; ++i) {
    if (tid == 0 && i + 1 < ntiles) issue(i + 1);  // the other buffer was released by the barrier below
    const bool ok = ev_wait((i & 1) ? bar1 : bar0, (i >> 1) & 1u, A.spin_limit);
    if (__syncthreads_or(!ok)) {
      failed_at = (int)i;
      break;
    }
    const float *bx = ev_sm + (i & 1) * 3 * kEvTile, *by = bx + kEvTile, *bz = bx + 2 * kEvTile;
    const uint32_t len = min((uint32_t)kEvTile, c_end - (c_begin + i * kEvTile));
#pragma unroll 2
    for (uint32_t c = 0; c < len; c += 4) {
      const float4 x = *reinterpret_cast<const float4 *>(bx + c);
      const float4 y = *reinterpret_cast<const float4 *>(by + c);
      const float4 z = *reinterpret_cast<const float4 *>(bz + c);
      const f32x2 X0 = pk2(x.x, x.y), X1 = pk2(x.z, x.w);
      const f32x2 Y0 = pk2(y.x, y.y), Y1 = pk2(y.z, y.w);
      const f32x2 Z0 = pk2(z.x, z.y), Z1 = pk2(z.z, z.w);
#pragma unroll
      for (int k = 0; k < kEvQPT; ++k) {
        const f32x2 dx0 = sub2(X0, QX[k]), dx1 = sub2(X1, QX[k]);
        const f32x2 dy0 = sub2(Y0, QY[k]), dy1 = sub2(Y1, QY[k]);
        const f32x2 dz0 = sub2(Z0, QZ[k]), dz1 = sub2(Z1, QZ[k]);
        f32x2 s0 = mul2(dx0, dx0), s1 = mul2(dx1, dx1);
        s0 = fma2(dy0, dy0, s0);
        s1 = fma2(dy1, dy1, s1);
        s0 = fma2(dz0, dz0, s0);
        s1 = fma2(dz1, dz1, s1);
        if (MODE == 0) {
          float a0, a1, a2, a3;
          upk2(s0, a0, a1);
          upk2(s1, a2, a3);
          float m;
          asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a0), "f"(a1), "f"(a2));
          asm("min.f32 %0, %1, %2, %3;" : "=f"(best[k]) : "f"(best[k]), "f"(m), "f"(a3));
        } else {
          // sign bit of r2 - d^2 is set exactly when d^2 > r2 (IEEE subtraction, no flush)
          float e0, e1, e2, e3;
          upk2(sub2(R2, s0), e0, e1);
          upk2(sub2(R2, s1), e2, e3);
          cnt[k] += 4u - ((__float_as_uint(e0) >> 31) + (__float_as_uint(e1) >> 31) + (__float_as_uint(e2) >> 31) +
                          (__float_as_uint(e3) >> 31));
        }
      }
    }
    __syncthreads();  // buffer i & 1 may be refilled
  }
  if (failed_at >= 0) {
    if (tid == 0) {  // let the copies in flight (tiles i and i + 1) land before the block exits
      const uint32_t i = (uint32_t)failed_at;
      atomicOr(&A.ctr->status, kStTimeout);
      (void)ev_wait((i & 1) ? bar1 : bar0, (i >> 1) & 1u, A.spin_limit);
      if (i + 1 < ntiles) (void)ev_wait(((i + 1) & 1) ? bar1 : bar0, ((i + 1) >> 1) & 1u, A.spin_limit);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < kEvQPT; ++k) {
    const uint32_t q = qb * kEvQueries + tid + k * kEvThreads;
    if (q >= A.nq) continue;
    if (MODE == 0) {
      if (A.nchunks == 1) A.out[q] = __float_as_uint(best[k]);
      else atomicMin(A.out + q, __float_as_uint(best[k]));  // non-negative floats order like their bits
    } else {
      if (A.nchunks == 1) A.out[q] = cnt[k];
      else atomicAdd(A.out + q, cnt[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// finishing steps
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sum_parts(const double *p, uint32_t n, uint32_t stride) {
  double s = 0.0;
  for (uint32_t i = 0; i < n; ++i) s = __dadd_rn(s, p[(size_t)i * stride]);
  return s;
}

// Eq. 29-30 from the two sums and the clean cloud's extents.
__global__ void k_ev_metrics(const double *part_a, uint32_t nba, const double *part_b, uint32_t nbb,
                             const double *red_clean, uint32_t nbr, uint32_t na, uint32_t nb, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double mse = __ddiv_rn(sum_parts(part_a, nba, 1), (double)na);
  const double back = __ddiv_rn(sum_parts(part_b, nbb, 1), (double)nb);
  double M2 = 0.0;
  for (int c = 0; c < 3; ++c) {
    double lo = INFINITY, hi = -INFINITY;
    for (uint32_t b = 0; b < nbr; ++b) {
      lo = fmin(lo, red_clean[9ull * b + 3 + c]);
      hi = fmax(hi, red_clean[9ull * b + 6 + c]);
    }
    const double e = __dsub_rn(hi, lo);
    M2 = __dadd_rn(M2, __dmul_rn(e, e));
  }
  out[0] = mse;
  out[1] = __dadd_rn(mse, back);
  out[2] = 10.0 * log10(M2 / mse);
}

// Eq. 1-3 and 7 of the baseline: centroid, extents, R (and R^2 rounded down to
// FP32: for a float d^2, d^2 <= R^2 exactly when d^2 <= RD(R^2)), T.
// g[0..2] theta, g[3] R, g[4] T, g[5] bits of RD(R^2) as a double
__global__ void k_bl_params(const double *part, uint32_t nbr, uint32_t n, double G, double alpha, double *g,
                            float *r2f_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double H[3];
  for (int c = 0; c < 3; ++c) {
    g[c] = __ddiv_rn(sum_parts(part + c, nbr, 9), (double)n);
    double lo = INFINITY, hi = -INFINITY;
    for (uint32_t b = 0; b < nbr; ++b) {
      lo = fmin(lo, part[9ull * b + 3 + c]);
      hi = fmax(hi, part[9ull * b + 6 + c]);
    }
    H[c] = __dsub_rn(hi, lo);
  }
  const double area = __dadd_rn(__dadd_rn(__dmul_rn(H[0], H[1]), __dmul_rn(H[0], H[2])), __dmul_rn(H[1], H[2]));
  const double R = __ddiv_rn(__dmul_rn(6.0, area), (double)n);
  const double T = __ddiv_rn(__dmul_rn(__dmul_rn(alpha, G), __dadd_rn(__dadd_rn(H[0], H[1]), H[2])), (double)n);
  g[3] = R;
  g[4] = T;
  *r2f_out = __double2float_rd(__dmul_rn(R, R));
}

// Eq. 4, 6 and 8 per point
__global__ void k_bl_decide(const float *__restrict__ X, const float *__restrict__ Y, const float *__restrict__ Z,
                            uint32_t n, const uint32_t *__restrict__ cnt, const double *__restrict__ g, double G,
                            uint8_t *__restrict__ keep) {
  const double th[3] = {g[0], g[1], g[2]}, T = g[4];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double t0 = __dsub_rn((double)X[i], th[0]), t1 = __dsub_rn((double)Y[i], th[1]),
                 t2 = __dsub_rn((double)Z[i], th[2]);
    const double dd = __dadd_rn(__dadd_rn(__dmul_rn(t0, t0), __dmul_rn(t1, t1)), __dmul_rn(t2, t2));
    const double d = sqrt(dd);
    const double F = __ddiv_rn(__dmul_rn(G, (double)cnt[i]), __dmul_rn(d, d));
    keep[i] = F >= __ddiv_rn(T, d);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t ev_scratch_bytes(uint32_t na, uint32_t nb) {
  const size_t pa = (na + 3u) & ~3u, pb = (nb + 3u) & ~3u;
  const size_t blocks = 2 * ((na + nb) / kEvQueries + 4) + 1024;
  return 4 * 3 * (pa + pb) + 4 * (pa + pb) + 8 * 9 * blocks + 8 * blocks + 256;
}

namespace {
inline uint32_t ev_red_blocks(uint32_t n) { return min(1024u, (n + 4095u) / 4096u + 1u); }

int launch_cross(int mode, const CrossArgs &base, int num_sms, cudaStream_t st) {
  CrossArgs a = base;
  const uint32_t qblocks = (a.nq + kEvQueries - 1) / kEvQueries;
  // enough work units to fill the GPU: split the candidates into chunks of whole tiles
  const uint32_t want = 4u * (uint32_t)num_sms;
  uint32_t nch = (want + qblocks - 1) / qblocks;
  const uint32_t tiles = (a.ncand + kEvTile - 1) / kEvTile;
  if (nch > tiles) nch = tiles;
  if (nch < 1) nch = 1;
  const uint32_t tiles_per = (tiles + nch - 1) / nch;
  a.chunk = tiles_per * kEvTile;
  a.nchunks = (tiles + tiles_per - 1) / tiles_per;
  if (a.nchunks > 1) {
    k_ev_fill<<<min(1024u, (a.nq + 255) / 256), 256, 0, st>>>(a.out, a.nq, mode == 0 ? 0x7F800000u : 0u);
  }
  auto kern = mode == 0 ? k_ev_cross<0> : k_ev_cross<1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEvSmem) != cudaSuccess) return -1;
  kern<<<qblocks * a.nchunks, kEvThreads, kEvSmem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
}  // namespace

int launch_eval_metrics(const EvalArgs &e, int num_sms, cudaStream_t st) {
  unsigned char *p = e.scratch;
  auto take = [&](size_t bytes) { unsigned char *r = p; p += (bytes + 255) & ~size_t(255); return r; };
  const uint32_t pa = (e.na + 3u) & ~3u, pb = (e.nb + 3u) & ~3u;
  float *ax = (float *)take(4ull * pa), *ay = (float *)take(4ull * pa), *az = (float *)take(4ull * pa);
  float *bx = (float *)take(4ull * pb), *by = (float *)take(4ull * pb), *bz = (float *)take(4ull * pb);
  uint32_t *da = (uint32_t *)take(4ull * pa), *db = (uint32_t *)take(4ull * pb);
  const uint32_t ra = ev_red_blocks(e.na), rb = ev_red_blocks(e.nb);
  double *red = (double *)take(8ull * 9 * ra);
  double *pa_sum = (double *)take(8ull * ra), *pb_sum = (double *)take(8ull * rb);
  const uint32_t g = (uint32_t)num_sms * 4;
  k_ev_pack<<<g, 256, 0, st>>>(e.clean, e.na, pa, ax, ay, az, e.ctr);
  k_ev_pack<<<g, 256, 0, st>>>(e.denoised, e.nb, pb, bx, by, bz, e.ctr);
  k_ev_reduce<<<ra, kEvRedThreads, 0, st>>>(ax, ay, az, e.na, red);
  CrossArgs c{};
  c.ctr = e.ctr;
  c.spin_limit = e.spin_limit ? e.spin_limit : kSpinLimit;
  // clean -> denoised (Eq. 29's correspondence and Eq. 30's first term)
  c.qx = ax; c.qy = ay; c.qz = az; c.nq = e.na;
  c.cx = bx; c.cy = by; c.cz = bz; c.ncand = pb;
  c.out = da;
  if (launch_cross(0, c, num_sms, st)) return -1;
  // denoised -> clean (Eq. 30's second term)
  c.qx = bx; c.qy = by; c.qz = bz; c.nq = e.nb;
  c.cx = ax; c.cy = ay; c.cz = az; c.ncand = pa;
  c.out = db;
  if (launch_cross(0, c, num_sms, st)) return -1;
  k_ev_sum<<<ra, kEvRedThreads, 0, st>>>(da, e.na, pa_sum);
  k_ev_sum<<<rb, kEvRedThreads, 0, st>>>(db, e.nb, pb_sum);
  k_ev_metrics<<<1, 32, 0, st>>>(pa_sum, ra, pb_sum, rb, red, ra, e.na, e.nb, e.out);
  if (e.nn_clean) cudaMemcpyAsync(e.nn_clean, da, 4ull * e.na, cudaMemcpyDeviceToDevice, st);
  if (e.nn_denoised) cudaMemcpyAsync(e.nn_denoised, db, 4ull * e.nb, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_baseline(const BaselineArgs &b, int num_sms, cudaStream_t st) {
  unsigned char *p = b.scratch;
  auto take = [&](size_t bytes) { unsigned char *r = p; p += (bytes + 255) & ~size_t(255); return r; };
  const uint32_t pn = (b.n + 3u) & ~3u;
  float *x = (float *)take(4ull * pn), *y = (float *)take(4ull * pn), *z = (float *)take(4ull * pn);
  uint32_t *cnt = b.n_i ? b.n_i : (uint32_t *)take(4ull * pn);
  const uint32_t rn = ev_red_blocks(b.n);
  double *red = (double *)take(8ull * 9 * rn);
  double *gpar = (double *)take(8ull * 8);
  float *r2f = (float *)take(16);
  k_ev_pack<<<(uint32_t)num_sms * 4, 256, 0, st>>>(b.xyz, b.n, pn, x, y, z, b.ctr);
  k_ev_reduce<<<rn, kEvRedThreads, 0, st>>>(x, y, z, b.n, red);
  k_bl_params<<<1, 32, 0, st>>>(red, rn, b.n, b.G, b.alpha, gpar, r2f);
  // the radius is a device value: read it into the pass's arguments on the device side
  CrossArgs c{};
  c.ctr = b.ctr;
  c.spin_limit = b.spin_limit ? b.spin_limit : kSpinLimit;
  c.qx = x; c.qy = y; c.qz = z; c.nq = b.n;
  c.cx = x; c.cy = y; c.cz = z; c.ncand = pn;
  c.out = cnt;
  c.r2f = 0.0f;
  c.r2f_dev = r2f;
  if (launch_cross(1, c, num_sms, st)) return -1;
  k_bl_decide<<<(uint32_t)num_sms * 4, 256, 0, st>>>(x, y, z, b.n, cnt, gpar, b.G, b.keep);
  if (b.params_out) cudaMemcpyAsync(b.params_out, gpar, 8ull * 5, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace gd
