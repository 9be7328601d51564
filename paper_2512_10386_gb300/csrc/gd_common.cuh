// gd_common.cuh -- device-side types and helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gravdenoise.h"

namespace gd {

constexpr uint32_t kQMax = 2097151u;                  // 2^21 - 1: 21-bit cell index per axis
constexpr float kInvTwo21 = 4.76837158203125e-07f;    // 2^-21
constexpr int kTilePts = 2048;                        // points per front-end tile
constexpr int kFrontThreads = 256;
constexpr int kFrontItems = kTilePts / kFrontThreads; // 8
static_assert(kFrontThreads == 256, "the radix pass maps one thread to each 8-bit digit");
static_assert(kTilePts % kFrontThreads == 0, "whole items per thread");
static_assert(kTilePts % (4 * kFrontThreads) == 0, "whole 4-point groups per thread (bounding-box pass)");
constexpr int kMaxPasses = 8;                         // 8-bit radix digits over <= 63 key bits
// The radix sort runs over the top key bits only (at most kTopPasses digits: the
// octree down to some level DB); below DB the full order is only needed inside the
// level-DB nodes that hold more than leaf_capacity points, sorted one by one.
constexpr int kTopPasses = 4;
constexpr uint32_t kSpinLimit = 1u << 22;             // bounded device-side waits

// device status word bits
enum : uint32_t {
  kStNonFinite = 1u,
  kStTimeout = 2u,
  kStInternal = 4u,  // a bounds or consistency check failed; results are void
};
constexpr uint32_t kStFatal = kStNonFinite | kStTimeout | kStInternal;

// One frame of a batch: its point range and root cube (filled on the device).
struct FrameInfo {
  uint32_t begin, end;
  uint32_t lo_ord[3], hi_ord[3];  // order-preserving integer images of min / max (atomics)
  float lo[3];
  float side, s, delta;
};

// Front-end work tile: [begin, end) of one frame, <= kTilePts points.
struct Tile {
  uint32_t frame, begin, end, first_tile;  // first_tile: index of the frame's first tile
};

// Octree leaf; lo and h (Eq. 10-11) are filled by the leaf-prep kernel.
struct Leaf {
  uint32_t start, count, frame, level;
  float lo[3];
  float h;
};

// The fused leaf kernel takes leaves largest first (longest-processing-time
// order, so that no large leaf starts last and stretches the tail): class 0 =
// leaves above the shared-memory size (global-memory path), then classes of 64
// points from the largest down.
constexpr int kLeafClasses = 9;
// leaves of at most kSmallLeaf points run in their own launch (64-thread CTAs);
// one 64-point size class (measured against 128 and 256: fastest)
constexpr uint32_t kSmallLeaf = 64;

// Programmatic dependent launch: every kernel of a call is launched so that its
// blocks may be scheduled while the previous kernel drains; pdl_wait() (first
// access to global memory) blocks until that kernel has completed and its writes
// are visible, so the stream order of the data is unchanged.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

struct Counters {
  uint32_t status;
  uint32_t n_leaves;
  uint32_t leaf_work;                    // persistent leaf-kernel work counter
  uint32_t leaf_work2;                   // the same for a second leaf-kernel pass (cross-leaf mode)
  uint32_t leaf_work3;                   // the same for the launch that takes the small leaves
  uint32_t split_leaf;                   // first index of the largest-first order with leaves of <= kSmallLeaf points
  uint32_t xleaf_work;                   // cross-leaf kNN work counter
  uint32_t x_units;                      // cross-leaf kNN work units (leaf, 32 queries)
  uint32_t tile_work[kMaxPasses];        // radix-pass tile counters
  uint32_t cls_count[kLeafClasses];      // leaves per size class
  uint32_t cls_cursor[kLeafClasses];     // fill cursors of the class-ordered leaf list
  unsigned long long knn_pairs;
  unsigned long long n_p1;
  unsigned long long n_p2;
  unsigned long long score_terms;        // neighbour terms summed by the score (Eq. 21)
};

// Train-mode cache written by the forward for the backward.
struct TrainCache {
  uint32_t *nbr;    // [n][k] neighbour global indices (P_1 points), 0xFFFFFFFF pad
  float *nd2;       // [n][k] squared neighbour distances (FP32), 0 pad
  float *ell;       // [n] log2(rho_i / sqrt(rho_med^2 + eps_rho)) for P_1 points
  float *r2;        // [n] floored r_K^2 for P_1 points
  float *F;         // [n] score (P_2), 0 otherwise
  uint8_t *stage;   // [n]
  uint32_t k;
};

__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) {  // global memory only
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// FP32 quantisation of one coordinate to a 21-bit cell: min(2^21-1, floor((x - lo) * s)).
__device__ __forceinline__ uint32_t quantise(float x, float lo, float s) {
  float f = floorf(__fmul_rn(__fsub_rn(x, lo), s));
  return (f < 2097151.0f) ? (uint32_t)f : kQMax;
}

// Morton interleave: bit 3b+2 <- x_b, 3b+1 <- y_b, 3b <- z_b.
__device__ __forceinline__ unsigned long long spread3(uint32_t v) {
  unsigned long long x = v & 0x1FFFFFu;
  x = (x | (x << 32)) & 0x1F00000000FFFFull;
  x = (x | (x << 16)) & 0x1F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__device__ __forceinline__ unsigned long long morton3(uint32_t qx, uint32_t qy, uint32_t qz) {
  return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

// Host-side launch helpers (defined in gd_front.cu / gd_leaf.cu).
struct FrontArgs {
  const float *xyz;       // device copy of the points, read after the bounding-box pass
  const float *xyz_src;   // where the bounding-box pass reads them (null: xyz); may be mapped pinned host memory
  float *xyz_copy;        // if set, the bounding-box pass also writes what it read here (= xyz)
  uint32_t n;
  FrameInfo *frames;
  uint32_t nframes;
  const Tile *tiles;
  uint32_t ntiles;
  unsigned long long *keys[2];
  uint32_t *vals[2];
  float4 *spts;
  uint32_t *digit_hist;   // [nframes][kMaxPasses][256]
  uint32_t *digit_base;   // [nframes][kMaxPasses][256]
  uint32_t *lookback;     // [kMaxPasses][ntiles][256]
  Leaf *leaves;
  Counters *ctr;
  uint64_t *dbg_key;
  int max_depth;
  uint32_t leaf_capacity;
  uint32_t spin_limit;      // iterations of a bounded look-back wait (0 = kSpinLimit)
  uint32_t hold_tile1;      // test hook: tile hold_tile1 - 1 of the first radix pass never publishes (0 = off)
  bool full_sort;           // sort by every key bit (the cross-leaf variant searches cells of any level)
};

// Which of the two key buffers holds the sorted keys after launch_front.
int front_sorted_buffer(int max_depth, bool full_sort);
int launch_front(const FrontArgs &a, cudaStream_t st, int *launches, cudaEvent_t *ev_after_keys,
                 cudaEvent_t *ev_after_sort);

struct LeafArgs {
  uint32_t n;                   // total points (bounds check of every output index)
  const float4 *spts;
  const Leaf *leaves;
  uint32_t *order;              // [n_leaves] leaf indices, largest class first (written by the prep step)
  const FrameInfo *frames;
  Counters *ctr;
  denoise_params p;
  uint8_t *mask;
  float *score;
  uint8_t *stage;
  denoise_debug dbg;
  int use_dbg;
  unsigned char *big_scratch;   // per-point spill space for leaves larger than the smem path
  uint32_t big_bpp;             // bytes per point of big_scratch
  uint32_t lmax;                // largest leaf handled in shared memory (power of two)
  TrainCache train;
  int use_train;
  uint32_t ctas_per_sm;         // 0 = occupancy limit
  uint32_t threads;             // threads per leaf CTA: 64 or 128 (0 = 128)
  uint32_t spin_limit;          // iterations of the bounded bulk-copy wait (0 = kSpinLimit)
  uint32_t part;                // leaves taken from the order: 0 all, 1 those before split_leaf, 2 the rest
  // cross-leaf kNN (denoise_params.cross_leaf): phase 1 runs the voxel gate only and
  // marks P_1; phase 3 runs the per-leaf steps after the kNN on the cross-leaf results
  uint32_t xphase;              // 0 (the fused method), 1 or 3
  uint8_t *xflag;               // [n] P_1 membership by sorted position
  const uint32_t *xnbr;         // [n][k] neighbours (sorted positions), by sorted position
  const float *xr2;             // [n] floored r_K^2 by sorted position
  const uint32_t *xkeff;        // [n] k_eff by sorted position (0: no neighbour)
};

// Cross-leaf kNN (gd_xleaf.cu): for the P_1 points of every leaf, the k_eff
// nearest (d^2, input index) among the P_1 points of the 27 same-level octree
// cells around the leaf's cell.
struct XleafArgs {
  uint32_t n;
  const float4 *spts;              // sorted points (x, y, z, input index bits)
  const unsigned long long *keys;  // sorted Morton keys
  const Leaf *leaves;
  const FrameInfo *frames;
  Counters *ctr;
  uint32_t k;
  const uint8_t *xflag;
  uint32_t *xnbr;
  float *xr2;
  uint32_t *xkeff;
  uint32_t *unit_start;  // [n_leaves] scratch: first work unit of each leaf (K <= 32)
  denoise_debug dbg;
  int use_dbg;
};
int launch_xleaf_knn(const XleafArgs &a, int num_sms, cudaStream_t st, int *launches);

int leaf_kmax(uint32_t k);
size_t leaf_smem_bytes(uint32_t lmax, int kmax);
uint32_t leaf_big_bpp(int kmax);
uint32_t leaf_pick_lmax(uint32_t leaf_capacity, int kmax, size_t smem_limit);
// Eq. 10-11 per leaf (box origin lo and voxel size h into the leaf table) and the
// largest-first leaf order; must precede launch_leaf on the same stream.
int launch_leaf_prep(const LeafArgs &a, int num_sms, cudaStream_t st, int *launches);
// With a side stream (and two events), the leaves of more than kSmallLeaf points
// run on `st` and the smaller ones concurrently on `side` (64-thread CTAs of a
// kSmallLeaf-point layout), joined back into `st`; without, one launch takes every leaf.
int launch_leaf(const LeafArgs &a, int num_sms, cudaStream_t st, int *launches, cudaStream_t side = nullptr,
                cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
// the recording instantiation (debug / training outputs), in its own translation unit
int launch_leaf_rec(const LeafArgs &a, int num_sms, cudaStream_t st);
int launch_leaf_xl(const LeafArgs &a, int num_sms, cudaStream_t st);

// Evaluation metrics (Eq. 29-30) and the baseline of Sec. 2.2 (gd_eval.cu).
struct EvalArgs {
  const float *clean, *denoised;  // device xyz [n][3]
  uint32_t na, nb;
  float *nn_clean, *nn_denoised;  // device [na] / [nb] nearest squared distances, or null
  double *out;                    // device [3]: mse, chamfer, psnr
  unsigned char *scratch;         // ev_scratch_bytes(na, nb) bytes, 256-byte aligned
  Counters *ctr;
  uint32_t spin_limit;
};
struct BaselineArgs {
  const float *xyz;               // device xyz [n][3]
  uint32_t n;
  double G, alpha;                // Eq. 6 and Eq. 7 constants
  uint8_t *keep;                  // device [n]
  uint32_t *n_i;                  // device [n] neighbour counts (Eq. 5), or null
  double *params_out;             // device [5]: centroid x, y, z, R, T; or null
  unsigned char *scratch;         // ev_scratch_bytes(n, 0) bytes
  Counters *ctr;
  uint32_t spin_limit;
};
size_t ev_scratch_bytes(uint32_t na, uint32_t nb);
int launch_eval_metrics(const EvalArgs &e, int num_sms, cudaStream_t st);
int launch_baseline(const BaselineArgs &b, int num_sms, cudaStream_t st);

struct BackArgs {
  TrainCache train;
  uint32_t n;
  denoise_params p;
  const float *grad_r;   // [n] dL/dr_i
  float *removal;        // [n] soft removal output
  double *partials;      // [blocks][4]
  double *grad4;         // [4]
};
int launch_soft_removal(const BackArgs &a, cudaStream_t st);
int launch_backward(const BackArgs &a, cudaStream_t st, int *launches);

// Results into pinned host memory (mapped device addresses; a null destination is skipped).
struct OutArgs {
  const uint8_t *mask_d;
  const float *score_d;
  const uint8_t *stage_d;
  uint8_t *mask_h;
  float *score_h;
  uint8_t *stage_h;
  uint32_t n;
  const Counters *ctr_d;
  Counters *ctr_h;
};
int launch_out(const OutArgs &a, int num_sms, cudaStream_t st);

}  // namespace gd
