// gd_leaf.cu -- the per-leaf part of the method, fused into one persistent kernel
// (device code in gd_leaf_kernel.cuh), its prep kernels and host launchers.
//
// Each CTA pulls octree leaves from a device work counter and runs, for one
// leaf at a time, every per-leaf step of Sec. 3 in shared memory:
//   extents and adaptive voxel size h (Eq. 10-11) -> voxel occupancy counts in a
//   shared hash table with warp-aggregated atomics, voxel gate (Eq. 12) and
//   compaction of P_1 -> kNN of every P_1 point against the leaf's P_1 (seeded
//   register top-K, candidates broadcast from shared memory, ties broken by
//   input index), r_K (Eq. 13) -> exact percentile gate
//   (Eq. 14) as a rank cut on r_K^2 -> median density (Eq. 16) -> dual-weight
//   gravitational score (Eq. 15-21) -> Top-lambda or log-threshold selection,
//   scattered to input order (Eq. 22).
// The leaf's points arrive in shared memory by one TMA bulk copy
// (cp.async.bulk + mbarrier).  Leaves larger than the shared-memory capacity
// (only possible at max depth, i.e. with massive duplicates) run the same code
// on a per-point spill area in global memory.
//
// FP32 steps that decide integers (voxel indices, neighbour order, the density
// rank cut) use explicitly rounded intrinsics so no FMA contraction can change
// them; FP64 per-leaf scalars (V_t, h, rho_med) use explicitly rounded FP64.
#include "gd_leaf_kernel.cuh"

namespace gd {

// ---------------------------------------------------------------------------
// leaf prep: Eq. 10-11 for every leaf (all leaves in parallel)
// ---------------------------------------------------------------------------
// A block takes 32 leaves at a time: each warp reduces the FP32 bounding boxes
// of 4 of them (exact min/max), then lane l of warp 0 evaluates leaf l's
// h = f32(beta * cbrt_spec(V_t / N_t)) with the extents floored at delta and
// V_t in FP64.  One leaf per lane matters: FP64 issue is scarce on this part,
// and a warp instruction costs the same with 1 or 32 lanes active.
constexpr int kPrepThreads = 256;
constexpr int kPrepLeaves = 32;

__device__ __forceinline__ uint32_t leaf_class(uint32_t count, uint32_t lmax) {
  if (count > lmax) return 0;
  const uint32_t b = (count - 1) >> 6;  // 64-point classes, largest first
  return 1 + (kLeafClasses - 2) - (b < kLeafClasses - 2 ? b : kLeafClasses - 2);
}

// warp-aggregated atomicAdd of 1 per lane on ctr[cls]; returns the lane's slot
__device__ __forceinline__ uint32_t class_slot(uint32_t *ctr, uint32_t cls, uint32_t active) {
  const uint32_t peers = __match_any_sync(active, cls);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(&ctr[cls], (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kPrepThreads) k_leaf_prep(const float4 *__restrict__ spts, Leaf *leaves,
                                                            const FrameInfo *__restrict__ frames,
                                                            Counters *ctr, float beta, uint32_t lmax) {
  __shared__ float s_ext[kPrepLeaves][3];
  pdl_wait();
  if (ctr->status & kStFatal) return;
  const uint32_t nl = ctr->n_leaves;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr uint32_t kPerWarp = kPrepLeaves / (kPrepThreads / 32);
  for (uint32_t g = blockIdx.x * kPrepLeaves; g < nl; g += gridDim.x * kPrepLeaves) {
    for (uint32_t t = 0; t < kPerWarp; ++t) {
      const uint32_t slot = w * kPerWarp + t, li = g + slot;
      if (li >= nl) break;
      const uint32_t start = leaves[li].start, cnt = leaves[li].count;
      float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (uint32_t i0 = lane; i0 < cnt; i0 += 128) {  // four loads in flight per lane
        float4 p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t i = i0 + 32u * u;
          if (i < cnt) p[u] = spts[start + i];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (i0 + 32u * u < cnt) {
            mn[0] = fminf(mn[0], p[u].x); mn[1] = fminf(mn[1], p[u].y); mn[2] = fminf(mn[2], p[u].z);
            mx[0] = fmaxf(mx[0], p[u].x); mx[1] = fmaxf(mx[1], p[u].y); mx[2] = fmaxf(mx[2], p[u].z);
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
          mn[a] = fminf(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], o));
          mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], o));
        }
      }
      if (lane < 3) {
        const float lo = lane == 0 ? mn[0] : (lane == 1 ? mn[1] : mn[2]);
        const float hi = lane == 0 ? mx[0] : (lane == 1 ? mx[1] : mx[2]);
        leaves[li].lo[lane] = lo;
        s_ext[slot][lane] = __fsub_rn(hi, lo);
      }
    }
    __syncthreads();
    const uint32_t active = __ballot_sync(0xFFFFFFFFu, g + lane < nl);
    if (w == 0 && g + lane < nl) {
      const uint32_t li = g + lane;
      (void)class_slot(ctr->cls_count, leaf_class(leaves[li].count, lmax), active);
      const float delta = frames[leaves[li].frame].delta;
      double H[3];
      for (int a = 0; a < 3; ++a) {
        float e = s_ext[lane][a];
        if (e < delta) e = delta;
        H[a] = (double)e;
      }
      const double V = __dmul_rn(__dmul_rn(H[0], H[1]), H[2]);
      const double u = __ddiv_rn(V, (double)leaves[li].count);
      leaves[li].h = __double2float_rn(__dmul_rn((double)beta, cbrt_spec(u)));
    }
    __syncthreads();
  }
}

// Scatter the leaf indices into size-class order (class 0 first); the order
// within a class is arbitrary and does not affect any result.
__global__ void __launch_bounds__(256) k_leaf_order(const Leaf *__restrict__ leaves, Counters *ctr,
                                                    uint32_t *__restrict__ order, uint32_t lmax) {
  pdl_wait();
  if (ctr->status & kStFatal) return;
  const uint32_t nl = ctr->n_leaves;
  __shared__ uint32_t s_base[kLeafClasses];
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int c = 0; c < kLeafClasses; ++c) {
      s_base[c] = run;
      run += ctr->cls_count[c];
    }
    // the smallest classes (64 points each, up to kSmallLeaf points) come last
    if (blockIdx.x == 0) ctr->split_leaf = s_base[kLeafClasses - (int)(kSmallLeaf / 64)];
  }
  __syncthreads();
  for (uint32_t b = blockIdx.x * blockDim.x; b < nl; b += gridDim.x * blockDim.x) {
    const uint32_t li = b + threadIdx.x;
    const uint32_t active = __ballot_sync(0xFFFFFFFFu, li < nl);
    if (li >= nl) continue;
    const uint32_t cls = leaf_class(leaves[li].count, lmax);
    const uint32_t slot = s_base[cls] + class_slot(ctr->cls_cursor, cls, active);
    if (slot < nl) order[slot] = li;
    else atomicOr(&ctr->status, kStInternal);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int leaf_kmax(uint32_t k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64; }

size_t leaf_smem_bytes(uint32_t lmax, int kmax) {
  return carve<uint16_t>(nullptr, lmax, kmax, nullptr);
}

namespace {
// max over spill-path leaf sizes (cap > 64) of carve<uint32_t>(cap)/cap, rounded
// up to a multiple of 16 so that every leaf's area starts 16-byte aligned.  The
// ratio is largest for small caps (fixed-size parts); beyond 2^16 points it only
// falls, so scanning 65..65536 bounds every size.
uint32_t big_bpp_scan(int kmax) {
  size_t worst = 4u * ((kLeafSmemMax + 31u) / 32u);
  for (uint32_t cap = 65; cap <= 65536; ++cap) {
    const size_t b = carve<uint32_t>(nullptr, cap, kmax, nullptr);
    const size_t per = (b + cap - 1) / cap;
    if (per > worst) worst = per;
  }
  return (uint32_t)((worst + 15) & ~size_t(15));
}
}  // namespace

uint32_t leaf_big_bpp(int kmax) {
  // computed once, on first use, for the four list sizes (thread-safe static init);
  // at least the neighbour bitmap of a shared-memory leaf (one word a point per
  // 32 points of the leaf), which may be kept in the spill area
  static const uint32_t table[4] = {big_bpp_scan(8), big_bpp_scan(16), big_bpp_scan(32), big_bpp_scan(64)};
  return table[kmax <= 8 ? 0 : kmax <= 16 ? 1 : kmax <= 32 ? 2 : 3];
}

uint32_t leaf_pick_lmax(uint32_t leaf_capacity, int kmax, size_t smem_limit) {
  const uint32_t cap = leaf_capacity < 64 ? 64 : (leaf_capacity > kLeafSmemMax ? kLeafSmemMax : leaf_capacity);
  uint32_t l = pow2ceil(cap);
  while (l > 64 && leaf_smem_bytes(l, kmax) > smem_limit) l >>= 1;
  return l;
}

int launch_leaf_prep(const LeafArgs &a, int num_sms, cudaStream_t st, int *launches) {
  launch_pdl(k_leaf_prep, num_sms * 4, kPrepThreads, 0, st, a.spts, const_cast<Leaf *>(a.leaves), a.frames, a.ctr, a.p.beta,
                                                   a.lmax);
  launch_pdl(k_leaf_order, num_sms * 2, 256, 0, st, a.leaves, a.ctr, a.order, a.lmax);
  if (launches) *launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_leaf(const LeafArgs &a, int num_sms, cudaStream_t st, int *launches, cudaStream_t side, cudaEvent_t fork,
                cudaEvent_t join) {
  if (a.xphase != 0) {  // the cross-leaf phases: their own instantiation
    if (launches) ++*launches;
    return launch_leaf_xl(a, num_sms, st);
  }
  auto go = [&](const LeafArgs &x, cudaStream_t s) {
    return (x.use_dbg || x.use_train) ? launch_leaf_rec(x, num_sms, s) : launch_kmax<false, false>(x, num_sms, s);
  };
  // A small leaf's per-leaf steps keep few warps busy; on 64-thread CTAs of a
  // 64-point shared-memory layout twice as many CTAs share an SM.  The large
  // leaves keep their 128-thread CTAs; the two launches run side by side, and the
  // small-leaf CTAs take the SMs the large-leaf CTAs leave (the order of the
  // leaves and every result are the same as with one launch).
  const bool split = side && fork && join && a.threads != 64 && a.lmax > kSmallLeaf && a.ctas_per_sm == 0;
  if (!split) {
    if (launches) ++*launches;
    return go(a, st);
  }
  LeafArgs big = a, small = a;
  big.part = 1;
  small.part = 2;
  small.threads = 64;  // (32-thread CTAs: dense scan +1.7 %, 64 LiDAR frames -1.4 %)
  small.lmax = kSmallLeaf;
  if (launches) *launches += 2;
  if (cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(side, fork, 0) != cudaSuccess) return -1;
  if (go(big, st) || go(small, side)) return -1;
  if (cudaEventRecord(join, side) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess) return -1;
  return 0;
}

}  // namespace gd
