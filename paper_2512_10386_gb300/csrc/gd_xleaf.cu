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

template <bool kRec>
int launch_x(const XleafArgs &a, int num_sms, cudaStream_t st) {
  auto go = [&](auto kern) { return launch_pdl(kern, num_sms * 4, kXThreads, 0, st, a); };
  cudaError_t e;
  if (a.k <= 8) e = go(k_xleaf_knn<8, kRec>);
  else if (a.k <= 16) e = go(k_xleaf_knn<16, kRec>);
  else if (a.k <= 32) e = go(k_xleaf_knn<32, kRec>);
  else e = go(k_xleaf_knn<64, kRec>);
  return e == cudaSuccess ? 0 : -1;
}

int launch_xleaf_knn(const XleafArgs &a, int num_sms, cudaStream_t st) {
  return a.use_dbg ? launch_x<true>(a, num_sms, st) : launch_x<false>(a, num_sms, st);
}

}  // namespace gd
