// gd_xleaf.cu -- the cross-leaf kNN variant: neighbours searched over the
// octree cells adjacent to a point's leaf, not only within the leaf (the
// leaf-local search of Sec. 3 gives the points on a leaf's border an r_K
// inflated by the missing points across it).
//
// Candidates of the points of a leaf at level L: the P_1 points of the 27
// cells of level L around (and including) the leaf's cell.  A cell of level L
// is a contiguous range of the Morton-sorted points, found by binary search of
// its key prefix, so the candidate set is at most 27 ranges, shared by every
// query of the leaf.  They are streamed through shared memory in tiles; each
// thread keeps its query's k_eff smallest (d^2, input index) keys in a sorted
// list (d^2 in FP32 with the method's operation order, ties by input index:
// the exact rule).  Outputs by sorted position: the neighbours (sorted
// positions), the floored r_K^2 and k_eff.  The per-leaf gate, median, score and
// selection then run in the fused leaf kernel's cross-leaf phase.
//
// For K <= 32 the work is split into units of (leaf, 32 queries) (k_xleaf_units,
// k_xleaf_knn_warp): a CTA stages the unit's candidates in shared memory tile by
// tile, each warp keeps the sorted lists of 4 queries spread over its lanes (lane
// t holds rank t), tests 32 candidates a step against all 4, and inserts each
// candidate below a query's current k_eff-th key by one shuffle step of that
// list.  Larger K keep the per-thread list (k_xleaf_knn).
#include <cuda_runtime.h>

#include "gd_common.cuh"

namespace gd {

constexpr int kXThreads = 128;
constexpr int kXTile = 1024;  // candidates staged per round

__device__ __forceinline__ uint32_t compact3(unsigned long long k) {  // bits 0, 3, 6, ... -> 0, 1, 2, ...
  k &= 0x1249249249249249ull;
  k = (k | (k >> 2)) & 0x10C30C30C30C30C3ull;
  k = (k | (k >> 4)) & 0x100F00F00F00F00Full;
  k = (k | (k >> 8)) & 0x1F0000FF0000FFull;
  k = (k | (k >> 16)) & 0x1F00000000FFFFull;
  k = (k | (k >> 32)) & 0x1FFFFFull;
  return (uint32_t)k;
}

__device__ __forceinline__ float xsqdist(float xi, float yi, float zi, const float4 &b) {
  const float dx = __fsub_rn(b.x, xi), dy = __fsub_rn(b.y, yi), dz = __fsub_rn(b.z, zi);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// first position in [lo, hi) whose key is >= key
__device__ __forceinline__ uint32_t lower_key(const unsigned long long *keys, uint32_t lo, uint32_t hi,
                                              unsigned long long key) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <int KMAX, bool kRec>
__global__ void __launch_bounds__(kXThreads) k_xleaf_knn(const XleafArgs A) {
  __shared__ float4 s_pts[kXTile];
  __shared__ uint32_t s_pos[kXTile];
  __shared__ uint32_t s_rng[27][2];
  __shared__ uint32_t s_leaf, s_cnt, s_fill;
  const uint32_t tid = threadIdx.x;
  pdl_wait();
  const uint32_t n_leaves = A.ctr->n_leaves;
  for (;;) {
    if (tid == 0) s_leaf = (ld_volatile(&A.ctr->status) & kStFatal) ? 0xFFFFFFFFu : atomicAdd(&A.ctr->xleaf_work, 1u);
    __syncthreads();
    const uint32_t li = s_leaf;
    if (li >= n_leaves) break;
    const Leaf lf = A.leaves[li];
    const FrameInfo fr = A.frames[lf.frame];
    // the 27 cell ranges (level-0 leaf: the whole frame)
    if (tid < 27) {
      uint32_t a = 0, b = 0;
      const uint32_t L = lf.level;
      if (L == 0) {
        if (tid == 13) { a = fr.begin; b = fr.end; }
      } else {
        const unsigned long long k0 = A.keys[lf.start];
        const int sh = 3 * (21 - (int)L);
        const int64_t cx = compact3(k0 >> 2) >> (21 - L), cy = compact3(k0 >> 1) >> (21 - L),
                      cz = compact3(k0) >> (21 - L);
        const int64_t x = cx + (int64_t)(tid / 9) - 1, y = cy + (int64_t)((tid / 3) % 3) - 1,
                      z = cz + (int64_t)(tid % 3) - 1;
        const int64_t side = (int64_t)1 << L;
        if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
          const unsigned long long pre = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
          a = lower_key(A.keys, fr.begin, fr.end, pre << sh);
          b = lower_key(A.keys, a, fr.end, (pre + 1ull) << sh);
        }
      }
      s_rng[tid][0] = a;
      s_rng[tid][1] = b;
    }
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    // |C_t|: the P_1 points of the block
    uint32_t cnt = 0;
    for (int r = 0; r < 27; ++r)
      for (uint32_t p = s_rng[r][0] + tid; p < s_rng[r][1]; p += kXThreads) cnt += A.xflag[p];
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if ((tid & 31) == 0) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    const uint32_t nc = s_cnt;
    const uint32_t keff = nc <= 1 ? 0u : (A.k < nc - 1 ? A.k : nc - 1);
    const float delta2 = __fmul_rn(fr.delta, fr.delta);
    uint32_t nq = 0;
    for (uint32_t qb = 0; qb < lf.count; qb += kXThreads) {
      const uint32_t qi = qb + tid;
      const bool act = qi < lf.count && A.xflag[lf.start + qi];
      const uint32_t qp = lf.start + (qi < lf.count ? qi : 0);
      const float4 me = A.spts[qp];
      unsigned long long L[KMAX];
      uint32_t Pp[KMAX];
#pragma unroll
      for (int s = 0; s < KMAX; ++s) {
        L[s] = ~0ull;
        Pp[s] = 0;
      }
      unsigned long long thr = ~0ull;  // the k_eff-th key so far
      for (int r = 0; r < 27; ++r) {
        for (uint32_t c0 = s_rng[r][0]; c0 < s_rng[r][1]; c0 += kXTile) {
          const uint32_t len = min((uint32_t)kXTile, s_rng[r][1] - c0);
          __syncthreads();
          for (uint32_t u = tid; u < len; u += kXThreads) {
            s_pts[u] = A.spts[c0 + u];
            s_pos[u] = A.xflag[c0 + u] ? c0 + u : 0xFFFFFFFFu;
          }
          __syncthreads();
          if (!act || keff == 0) continue;
          for (uint32_t u = 0; u < len; ++u) {
            const uint32_t pu = s_pos[u];
            if (pu == 0xFFFFFFFFu || pu == qp) continue;
            const float4 c = s_pts[u];
            const float d2 = xsqdist(me.x, me.y, me.z, c);
            const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | __float_as_uint(c.w);
            if (key >= thr) continue;
            // insert into the sorted list of k_eff keys
            int s = (int)keff - 1;
            while (s > 0 && L[s - 1] > key) {
              L[s] = L[s - 1];
              Pp[s] = Pp[s - 1];
              --s;
            }
            L[s] = key;
            Pp[s] = pu;
            thr = L[keff - 1];
          }
        }
      }
      if (act) {
        ++nq;
        A.xkeff[qp] = keff;
        if (keff) {
          const float rk = __uint_as_float((uint32_t)(L[keff - 1] >> 32));
          A.xr2[qp] = rk < delta2 ? delta2 : rk;
        }
        for (uint32_t t = 0; t < keff; ++t) A.xnbr[(size_t)qp * A.k + t] = Pp[t];
        if (kRec && A.use_dbg) {
          const uint32_t g = __float_as_uint(me.w);
          if (g < A.n) {
            for (uint32_t t = 0; t < A.k; ++t) {
              const bool v = t < keff;
              if (A.dbg.nbr) A.dbg.nbr[(size_t)g * A.k + t] = v ? (uint32_t)L[t] : 0xFFFFFFFFu;
              if (A.dbg.nbr_d2) A.dbg.nbr_d2[(size_t)g * A.k + t] = v ? __uint_as_float((uint32_t)(L[t] >> 32)) : 0.f;
            }
            if (A.dbg.r2 && keff) A.dbg.r2[g] = A.xr2[qp];
          } else {
            atomicOr(&A.ctr->status, kStInternal);
          }
        }
      }
    }
    nq = __reduce_add_sync(0xFFFFFFFFu, nq);
    if ((tid & 31) == 0 && nq && nc > 1) atomicAdd(&A.ctr->knn_pairs, (unsigned long long)nq * (nc - 1));
    __syncthreads();
  }
}

// ---- K <= 32: work units of (leaf, 32 queries); one warp keeps 4 queries' lists
constexpr int kXWThreads = 256;                 // 8 warps
constexpr int kXWQ = 4;                         // queries per warp (8 with 2 CTAs per SM: 13.3 vs 9.0 ms)
constexpr int kXWCtas = 4;                      // CTAs per SM (3: 9.6 ms)
constexpr int kXWUnit = kXWQ * kXWThreads / 32; // queries per unit (32)
constexpr int kXWTile = 2048;                   // candidates staged per round

// unit_start[l] = first work unit of leaf l (ceil(count / kXWUnit) units per leaf),
// ctr->x_units = the total: one block scans the leaf table
__global__ void __launch_bounds__(1024) k_xleaf_units(const Leaf *__restrict__ leaves, Counters *ctr,
                                                      uint32_t *__restrict__ unit_start) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_run;
  pdl_wait();
  const uint32_t nl = ctr->n_leaves, tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
  if (tid == 0) s_run = 0;
  __syncthreads();
  for (uint32_t base = 0; base < nl; base += 1024u) {
    const uint32_t i = base + tid;
    const uint32_t c = i < nl ? (leaves[i].count + kXWUnit - 1u) / kXWUnit : 0u;
    uint32_t inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
      uint32_t v = s_w[lane], x = v;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
      }
      s_w[lane] = x - v;  // exclusive prefix of the warps
    }
    __syncthreads();
    const uint32_t run = s_run;
    if (i < nl) unit_start[i] = run + s_w[w] + inc - c;
    __syncthreads();
    if (tid == 1023) s_run = run + s_w[w] + inc;
    __syncthreads();
  }
  if (tid == 0) ctr->x_units = s_run;
}

// insert key K (position P) into the warp-spread sorted list (lane t: rank t) of
// keff <= 32 keys; thr becomes the k_eff-th key
__device__ __forceinline__ void xw_insert(unsigned long long &Lk, uint32_t &Lp, unsigned long long &thr,
                                          unsigned long long K, uint32_t P, uint32_t lane, uint32_t keff) {
  const unsigned long long prev = __shfl_up_sync(0xFFFFFFFFu, Lk, 1);
  const uint32_t pprev = __shfl_up_sync(0xFFFFFFFFu, Lp, 1);
  if (lane < keff) {
    if (lane > 0 && prev > K) {
      Lk = prev;
      Lp = pprev;
    } else if (Lk > K) {
      Lk = K;
      Lp = P;
    }
  }
  thr = __shfl_sync(0xFFFFFFFFu, Lk, keff - 1);
}

template <bool kRec>
__global__ void __launch_bounds__(kXWThreads, kXWCtas) k_xleaf_knn_warp(const XleafArgs A) {
  __shared__ float4 s_c[kXWTile];
  __shared__ uint32_t s_p[kXWTile];   // candidate position, 0xFFFFFFFF: not in P_1
  __shared__ uint32_t s_rng[27][2];
  __shared__ uint32_t s_unit, s_leaf, s_cnt;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
  pdl_wait();
  const uint32_t n_leaves = A.ctr->n_leaves, n_units = A.ctr->x_units;
  for (;;) {
    if (tid == 0) {
      const uint32_t u = (ld_volatile(&A.ctr->status) & kStFatal) ? 0xFFFFFFFFu : atomicAdd(&A.ctr->xleaf_work, 1u);
      uint32_t li = 0;
      if (u < n_units) {  // the leaf whose units hold u: the last start <= u
        uint32_t lo = 0, hi = n_leaves - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (A.unit_start[mid] <= u) lo = mid;
          else hi = mid - 1;
        }
        li = lo;
      }
      s_unit = u;
      s_leaf = li;
    }
    __syncthreads();
    const uint32_t u = s_unit;
    if (u >= n_units) break;
    const uint32_t li = s_leaf;
    const Leaf lf = A.leaves[li];
    const FrameInfo fr = A.frames[lf.frame];
    const uint32_t q0 = (u - A.unit_start[li]) * kXWUnit;  // the unit's first query (leaf offset)
    if (tid < 27) {  // the 27 cell ranges (level-0 leaf: the whole frame)
      uint32_t a = 0, b = 0;
      const uint32_t L = lf.level;
      if (L == 0) {
        if (tid == 13) { a = fr.begin; b = fr.end; }
      } else {
        const unsigned long long k0 = A.keys[lf.start];
        const int sh = 3 * (21 - (int)L);
        const int64_t cx = compact3(k0 >> 2) >> (21 - L), cy = compact3(k0 >> 1) >> (21 - L),
                      cz = compact3(k0) >> (21 - L);
        const int64_t x = cx + (int64_t)(tid / 9) - 1, y = cy + (int64_t)((tid / 3) % 3) - 1,
                      z = cz + (int64_t)(tid % 3) - 1;
        const int64_t side = (int64_t)1 << L;
        if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
          const unsigned long long pre = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
          a = lower_key(A.keys, fr.begin, fr.end, pre << sh);
          b = lower_key(A.keys, a, fr.end, (pre + 1ull) << sh);
        }
      }
      s_rng[tid][0] = a;
      s_rng[tid][1] = b;
    }
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    uint32_t cnt = 0;  // |C_t|: the P_1 points of the block
    for (int r = 0; r < 27; ++r)
      for (uint32_t p = s_rng[r][0] + tid; p < s_rng[r][1]; p += kXWThreads) cnt += A.xflag[p];
    cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if (lane == 0) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    const uint32_t nc = s_cnt;
    const uint32_t keff = nc <= 1 ? 0u : (A.k < nc - 1 ? A.k : nc - 1);  // <= 32 here
    const float delta2 = __fmul_rn(fr.delta, fr.delta);
    // this warp's queries: leaf offsets q0 + 8w .. q0 + 8w + 7 that are in P_1
    uint32_t qpos[kXWQ], act = 0;
    float qx[kXWQ], qy[kXWQ], qz[kXWQ];
    unsigned long long Lk[kXWQ], thr[kXWQ];
    uint32_t Lp[kXWQ];
#pragma unroll
    for (int j = 0; j < kXWQ; ++j) {
      const uint32_t qi = q0 + w * kXWQ + j;
      qpos[j] = lf.start + (qi < lf.count ? qi : 0u);
      if (qi < lf.count && A.xflag[qpos[j]]) act |= 1u << j;
      const float4 me = A.spts[qpos[j]];
      qx[j] = me.x;
      qy[j] = me.y;
      qz[j] = me.z;
      Lk[j] = ~0ull;
      thr[j] = ~0ull;
      Lp[j] = 0;
    }
    if (keff) {
      for (int rr = 0; rr < 27; ++rr) {
        const int r = rr == 0 ? 13 : (rr <= 13 ? rr - 1 : rr);  // the leaf's own cell first
        const uint32_t ra = s_rng[r][0], rb = s_rng[r][1];
        for (uint32_t t0 = ra; t0 < rb; t0 += kXWTile) {
          const uint32_t len = min((uint32_t)kXWTile, rb - t0);
          __syncthreads();  // the previous tile is consumed
          for (uint32_t v = tid; v < len; v += kXWThreads) {
            s_c[v] = A.spts[t0 + v];
            s_p[v] = A.xflag[t0 + v] ? t0 + v : 0xFFFFFFFFu;
          }
          __syncthreads();
          if (!act) continue;
          for (uint32_t c0 = 0; c0 < len; c0 += 32u) {
            const uint32_t v = c0 + lane;
            const bool in = v < len;
            const float4 pc = in ? s_c[v] : make_float4(0.f, 0.f, 0.f, 0.f);
            const uint32_t pp = in ? s_p[v] : 0xFFFFFFFFu;
            const uint32_t gi = __float_as_uint(pc.w);
            // every query's test first (independent), against the high word of its
            // threshold: a candidate with larger d^2 cannot improve the list
            uint32_t db[kXWQ], mm[kXWQ];
#pragma unroll
            for (int j = 0; j < kXWQ; ++j) {
              const float dx = __fsub_rn(pc.x, qx[j]), dy = __fsub_rn(pc.y, qy[j]), dz = __fsub_rn(pc.z, qz[j]);
              db[j] = __float_as_uint(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))));
              const bool ok = ((act >> j) & 1u) && pp != 0xFFFFFFFFu && pp != qpos[j] &&
                              db[j] <= (uint32_t)(thr[j] >> 32);
              mm[j] = __ballot_sync(0xFFFFFFFFu, ok);
            }
#pragma unroll
            for (int j = 0; j < kXWQ; ++j) {
              uint32_t m = mm[j];
              while (m) {  // the exact (d^2, index) keys in lane order; the threshold falls as they go in
                const int b = __ffs(m) - 1;
                m &= m - 1u;
                const unsigned long long K = ((unsigned long long)__shfl_sync(0xFFFFFFFFu, db[j], b) << 32) |
                                             __shfl_sync(0xFFFFFFFFu, gi, b);
                const uint32_t P = __shfl_sync(0xFFFFFFFFu, pp, b);
                if (K < thr[j]) xw_insert(Lk[j], Lp[j], thr[j], K, P, lane, keff);
              }
            }
          }
        }
      }
    }
    uint32_t nq = 0;
#pragma unroll
    for (int j = 0; j < kXWQ; ++j) {
      if (!((act >> j) & 1u)) continue;
      ++nq;
      const uint32_t qp = qpos[j];
      if (lane == 0) {
        A.xkeff[qp] = keff;
        if (keff) {
          const float rk = __uint_as_float((uint32_t)(thr[j] >> 32));
          A.xr2[qp] = rk < delta2 ? delta2 : rk;
        }
      }
      if (lane < keff) A.xnbr[(size_t)qp * A.k + lane] = Lp[j];
      if (kRec && A.use_dbg) {
        const uint32_t g = __float_as_uint(A.spts[qp].w);
        if (g < A.n) {
          if (lane < A.k) {
            const bool v = lane < keff;
            if (A.dbg.nbr) A.dbg.nbr[(size_t)g * A.k + lane] = v ? (uint32_t)Lk[j] : 0xFFFFFFFFu;
            if (A.dbg.nbr_d2)
              A.dbg.nbr_d2[(size_t)g * A.k + lane] = v ? __uint_as_float((uint32_t)(Lk[j] >> 32)) : 0.f;
          }
          if (lane == 0 && A.dbg.r2 && keff) {
            const float rk = __uint_as_float((uint32_t)(thr[j] >> 32));
            A.dbg.r2[g] = rk < delta2 ? delta2 : rk;
          }
        } else if (lane == 0) {
          atomicOr(&A.ctr->status, kStInternal);
        }
      }
    }
    if (lane == 0 && nq && nc > 1) atomicAdd(&A.ctr->knn_pairs, (unsigned long long)nq * (nc - 1));
  }
}

template <bool kRec>
int launch_x(const XleafArgs &a, int num_sms, cudaStream_t st, int *launches) {
  auto go = [&](auto kern) { return launch_pdl(kern, num_sms * 4, kXThreads, 0, st, a); };
  cudaError_t e;
  if (a.k <= 32) {
    e = launch_pdl(k_xleaf_units, 1, 1024, 0, st, a.leaves, a.ctr, a.unit_start);
    if (e == cudaSuccess) e = launch_pdl(k_xleaf_knn_warp<kRec>, num_sms * kXWCtas, kXWThreads, 0, st, a);
    if (launches) *launches += 2;
  } else {
    e = go(k_xleaf_knn<64, kRec>);
    if (launches) *launches += 1;
  }
  return e == cudaSuccess ? 0 : -1;
}

int launch_xleaf_knn(const XleafArgs &a, int num_sms, cudaStream_t st, int *launches) {
  return a.use_dbg ? launch_x<true>(a, num_sms, st, launches) : launch_x<false>(a, num_sms, st, launches);
}

}  // namespace gd
