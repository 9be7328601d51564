// gd_front.cu -- front end of the path: root cube (Eq. 2 extents of each frame),
// 63-bit Morton keys, a segmented LSD radix sort by key (octree order, Sec. 3),
// and the octree leaf finder (leaf = shallowest node holding <= leaf_capacity
// points, or a node at max_depth).
//
// Radix sort design (one kernel per 8-bit digit pass, over the top key bits
// only -- see k_node_sort for the rest): a tile of 2,048 keys is
// ranked stably inside the block with warp match_any, per-digit tile counts are
// published to a look-back array and each tile's exclusive prefix is built by
// decoupled look-back over earlier tiles of the same frame (bounded spins), on
// top of per-frame digit bases taken from one upfront histogram kernel.  The
// frame-major tile layout makes the sort segmented: frames never mix.
#include "gd_common.cuh"

namespace gd {

// ---------------------------------------------------------------------------
// init: reset counters, bbox accumulators and look-back flags
// ---------------------------------------------------------------------------
__global__ void k_init(FrameInfo *frames, uint32_t nframes, Counters *ctr, uint32_t *digit_hist,
                       uint32_t *lookback, uint32_t n_lookback, int passes) {
  pdl_wait();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t stride = gridDim.x * blockDim.x;
  if (tid == 0) {
    ctr->status = 0;
    ctr->n_leaves = 0;
    ctr->leaf_work = 0;
    ctr->leaf_work2 = 0;
    ctr->leaf_work3 = 0;
    ctr->split_leaf = 0;
    ctr->xleaf_work = 0;
    for (int i = 0; i < kMaxPasses; ++i) ctr->tile_work[i] = 0;
    for (int i = 0; i < kLeafClasses; ++i) ctr->cls_count[i] = ctr->cls_cursor[i] = 0;
    ctr->knn_pairs = 0;
    ctr->n_p1 = 0;
    ctr->n_p2 = 0;
    ctr->score_terms = 0;
  }
  for (uint32_t f = tid; f < nframes; f += stride) {
    for (int a = 0; a < 3; ++a) {
      frames[f].lo_ord[a] = 0xFFFFFFFFu;
      frames[f].hi_ord[a] = 0u;
    }
  }
  const uint32_t nh = nframes * kMaxPasses * 256u;
  for (uint32_t i = tid; i < nh; i += stride) digit_hist[i] = 0;
  const uint32_t nl = n_lookback * (uint32_t)passes;
  for (uint32_t i = tid; i < nl; i += stride) lookback[i] = 0;
}

// ---------------------------------------------------------------------------
// bbox: exact FP32 min / max per frame (order-preserving integer atomics);
// flags non-finite coordinates.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFrontThreads) k_bbox(const float *__restrict__ xyz,
                                                        float *__restrict__ xyz_copy,
                                                        FrameInfo *frames, const Tile *__restrict__ tiles,
                                                        Counters *ctr) {
  pdl_wait();
  const Tile t = tiles[blockIdx.x];
  uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0u, 0u, 0u};
  bool bad = false;
  auto take = [&](int a, float v) {
    bad |= !isfinite(v);
    const uint32_t o = f2ord(v);
    mn[a] = min(mn[a], o);
    mx[a] = max(mx[a], o);
  };
  auto point = [&](uint32_t i) {  // one point, scalar loads (and the device copy of host input)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = xyz[3ull * i + a];
      if (xyz_copy) xyz_copy[3ull * i + a] = v;
      take(a, v);
    }
  };
  const bool vec = ((reinterpret_cast<uintptr_t>(xyz) | reinterpret_cast<uintptr_t>(xyz_copy)) & 15u) == 0;
  if (vec) {
    // from the first point index that is a multiple of 4, groups of 4 points (3
    // aligned 16-byte words) are read by consecutive threads -- every warp load
    // covers 512 contiguous bytes, all of a thread's loads issued together (the
    // input may be host memory, read across the link) -- and staged in shared
    // memory; the few points before and after the groups are read one by one.
    __shared__ float4 s_v[kTilePts / 4 * 3];
    const uint32_t p0 = min(t.end, (t.begin + 3u) & ~3u);
    const uint32_t ng = (t.end - p0) >> 2, p1 = p0 + 4u * ng, nv = 3u * ng;
    const float4 *src = reinterpret_cast<const float4 *>(xyz) + 3ull * (p0 >> 2);
    float4 *dst = xyz_copy ? reinterpret_cast<float4 *>(xyz_copy) + 3ull * (p0 >> 2) : nullptr;
    constexpr int kV = kTilePts / 4 * 3 / kFrontThreads;  // words per thread
    float4 v[kV];
#pragma unroll
    for (int it = 0; it < kV; ++it) {
      const uint32_t q = it * kFrontThreads + threadIdx.x;
      if (q < nv) v[it] = src[q];
    }
#pragma unroll
    for (int it = 0; it < kV; ++it) {
      const uint32_t q = it * kFrontThreads + threadIdx.x;
      if (q < nv) {
        s_v[q] = v[it];
        if (dst) dst[q] = v[it];
      }
    }
    const uint32_t nh = p0 - t.begin;  // < 4
    if (threadIdx.x < nh) point(t.begin + threadIdx.x);
    else if (threadIdx.x >= 32u && threadIdx.x - 32u < t.end - p1) point(p1 + threadIdx.x - 32u);
    __syncthreads();
    const float *sf = reinterpret_cast<const float *>(s_v);
    for (uint32_t i = threadIdx.x; i < 4u * ng; i += kFrontThreads) {
      take(0, sf[3u * i]);
      take(1, sf[3u * i + 1u]);
      take(2, sf[3u * i + 2u]);
    }
  } else {
    // a tile holds at most kFrontItems points per thread: unrolled, so that all
    // loads are in flight at once
#pragma unroll
    for (int it = 0; it < kFrontItems; ++it) {
      const uint32_t i = t.begin + it * kFrontThreads + threadIdx.x;
      if (i < t.end) point(i);
    }
  }
  for (int a = 0; a < 3; ++a) {
    for (int off = 16; off; off >>= 1) {
      mn[a] = min(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], off));
      mx[a] = max(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], off));
    }
  }
  bad = __any_sync(0xFFFFFFFFu, bad);
  // block reduction first: one atomic per block and value (all blocks of a
  // frame update the same six words, so per-warp atomics would serialise)
  __shared__ uint32_t s_red[kFrontThreads / 32][6];
  __shared__ int s_bad;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      s_red[w][a] = mn[a];
      s_red[w][3 + a] = mx[a];
    }
    if (bad) s_bad = 1;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int v = threadIdx.x;
    uint32_t r = s_red[0][v];
    for (int ww = 1; ww < kFrontThreads / 32; ++ww) r = (v < 3) ? min(r, s_red[ww][v]) : max(r, s_red[ww][v]);
    FrameInfo &f = frames[t.frame];
    if (v < 3) atomicMin(&f.lo_ord[v], r);
    else atomicMax(&f.hi_ord[v - 3], r);
    if (v == 0 && s_bad) atomicOr(&ctr->status, kStNonFinite);
  }
}

// Root cube of a frame from its reduced extents (reading: anchored at the FP32
// minimum, side = largest FP32 extent, 1 if the frame is a single location).
__device__ __forceinline__ void root_cube(const FrameInfo &f, float lo[3], float &side, float &s) {
  side = 0.0f;
  for (int a = 0; a < 3; ++a) {
    lo[a] = ord2f(f.lo_ord[a]);
    float e = __fsub_rn(ord2f(f.hi_ord[a]), lo[a]);
    side = (e > side) ? e : side;
  }
  if (side == 0.0f) side = 1.0f;
  s = __fdiv_rn(2097152.0f, side);
}

// ---------------------------------------------------------------------------
// keys: 63-bit Morton key per point, value = global point index; the first
// tile of each frame publishes the frame's root cube for later kernels.  The
// digit histograms of every radix pass (per frame) are accumulated on the way.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kFrontThreads) k_keys(const float *__restrict__ xyz, FrameInfo *frames,
                                                        const Tile *__restrict__ tiles,
                                                        unsigned long long *__restrict__ keys,
                                                        uint32_t *__restrict__ vals, uint64_t *dbg_key,
                                                        uint32_t *__restrict__ hist, int lowbit, int passes,
                                                        const Counters *ctr) {
  __shared__ uint32_t sh[kMaxPasses][256];
  pdl_wait();
  if (ctr->status & kStFatal) return;
  for (int i = threadIdx.x; i < passes * 256; i += kFrontThreads) (&sh[0][0])[i] = 0;
  __syncthreads();
  const Tile t = tiles[blockIdx.x];
  float lo[3], side, s;
  root_cube(frames[t.frame], lo, side, s);
  if (blockIdx.x == t.first_tile && threadIdx.x == 0) {
    FrameInfo &f = frames[t.frame];
    f.lo[0] = lo[0];
    f.lo[1] = lo[1];
    f.lo[2] = lo[2];
    f.side = side;
    f.s = s;
    f.delta = __fmul_rn(side, kInvTwo21);
  }
#pragma unroll
  for (int it = 0; it < kFrontItems; ++it) {
    const uint32_t i = t.begin + it * kFrontThreads + threadIdx.x;
    if (i < t.end) {
      const uint32_t q0 = quantise(xyz[3ull * i + 0], lo[0], s);
      const uint32_t q1 = quantise(xyz[3ull * i + 1], lo[1], s);
      const uint32_t q2 = quantise(xyz[3ull * i + 2], lo[2], s);
      const unsigned long long k = morton3(q0, q1, q2);
      keys[i] = k;
      vals[i] = i;
      if (dbg_key) dbg_key[i] = k;
      for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (lowbit + 8 * p)) & 0xFFu], 1u);
    }
  }
  __syncthreads();
  uint32_t *h = hist + (size_t)t.frame * kMaxPasses * 256;
  for (int i = threadIdx.x; i < passes * 256; i += kFrontThreads) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&h[i], v);
  }
}

// exclusive scan of each (frame, pass) digit histogram -> absolute output bases
__global__ void __launch_bounds__(256) k_digit_scan(const uint32_t *__restrict__ hist,
                                                    uint32_t *__restrict__ base,
                                                    const FrameInfo *__restrict__ frames, int passes,
                                                    const Counters *ctr) {
  __shared__ uint32_t warp_tot[8];
  pdl_wait();
  if (ctr->status & kStFatal) return;
  const uint32_t f = blockIdx.x / passes, p = blockIdx.x % passes;
  const size_t off = ((size_t)f * kMaxPasses + p) * 256;
  const uint32_t d = threadIdx.x, lane = d & 31, w = d >> 5;
  uint32_t v = hist[off + d], x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  uint32_t wp = 0;
  for (uint32_t i = 0; i < w; ++i) wp += warp_tot[i];
  base[off + d] = frames[f].begin + wp + x - v;
}

// ---------------------------------------------------------------------------
// one radix pass (stable, segmented by frame, decoupled look-back)
// ---------------------------------------------------------------------------
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kValMask = (1u << 30) - 1u;
constexpr int kLookAhead = 4;  // predecessors read per look-back round

template <bool kLast>
__global__ void __launch_bounds__(kFrontThreads) k_radix_pass(
    const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
    unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, float4 *__restrict__ pout,
    const float *__restrict__ xyz, const Tile *__restrict__ tiles, const FrameInfo *__restrict__ frames,
    const uint32_t *__restrict__ digit_base, uint32_t *__restrict__ lookback, uint32_t *tile_counter,
    int shift, Counters *ctr, uint32_t spin_limit, uint32_t hold_tile1) {
  constexpr int W = kFrontThreads / 32;
  __shared__ uint32_t s_wcnt[W][256];  // per warp and digit: count, then exclusive prefix over warps
  __shared__ uint32_t s_base[256];     // global output base of each digit for this tile
  __shared__ uint32_t s_doff[256];     // first position of each digit in the tile's sorted order
  __shared__ uint32_t s_wsum[W];
  __shared__ unsigned long long s_key[kTilePts];  // the tile in sorted order, for coalesced writes
  __shared__ uint32_t s_val[kTilePts];
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_fail;
  pdl_wait();
  if (ctr->status & kStFatal) return;
  for (int i = threadIdx.x; i < W * 256; i += kFrontThreads) (&s_wcnt[0][0])[i] = 0;
  if (threadIdx.x == 0) {
    s_tile = atomicAdd(tile_counter, 1u);  // dynamic tile order: forward progress of look-back
    s_fail = 0;
  }
  __syncthreads();
  const uint32_t ti = s_tile;
  const Tile t = tiles[ti];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t wbase = t.begin + w * 32 * kFrontItems;

  unsigned long long key[kFrontItems];
  uint32_t val[kFrontItems], dig[kFrontItems], rank[kFrontItems], peers[kFrontItems];
#pragma unroll
  for (int i = 0; i < kFrontItems; ++i) {
    uint32_t idx = wbase + i * 32 + lane;
    bool ok = idx < t.end;
    key[i] = ok ? kin[idx] : ~0ull;
    val[i] = ok ? vin[idx] : 0u;
    dig[i] = ok ? (uint32_t)((key[i] >> shift) & 0xFFu) : 256u;
  }
  // lanes of the warp holding the same 9-bit value (8-bit digit or 256 = no item):
  // one ballot per bit, independent across items
#pragma unroll
  for (int i = 0; i < kFrontItems; ++i) {
    const uint32_t d = dig[i];
    uint32_t pm = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 0; b < 9; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t bb = __ballot_sync(0xFFFFFFFFu, bit);
      pm &= bit ? bb : ~bb;
    }
    peers[i] = pm;
  }
  // stable rank within the warp in (item, lane) order = input order
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int i = 0; i < kFrontItems; ++i) {
    const uint32_t d = dig[i], pm = peers[i];
    uint32_t old = 0;
    if (d < 256u) old = s_wcnt[w][d];
    __syncwarp();
    rank[i] = old + __popc(pm & lt);
    if (d < 256u && (pm & lt) == 0) s_wcnt[w][d] = old + __popc(pm);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, tile total, position in the tile, then look-back
  {
    const uint32_t d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
      uint32_t c = s_wcnt[ww][d];
      s_wcnt[ww][d] = run;
      run += c;
    }
    uint32_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) s_wsum[w] = inc;
    __syncthreads();
    uint32_t wp = 0;
    for (uint32_t ww = 0; ww < w; ++ww) wp += s_wsum[ww];
    s_doff[d] = wp + inc - run;
    uint32_t *lb = lookback + (size_t)ti * 256;
    uint32_t excl = 0;
    // test hook (off unless the host asks): this tile never publishes, so the
    // next tile's bounded wait runs out and the call reports a timeout
    const bool publish = ti + 1u != hold_tile1;
    if (ti == t.first_tile) {
      if (publish) atomicExch(&lb[d], kFlagInc | run);
    } else {
      if (publish) atomicExch(&lb[d], kFlagAgg | run);
      // walk back kLookAhead predecessors per round: their flags are read with
      // independent loads, then consumed in order (a not-yet-published one is
      // re-read until it is); stop at the first inclusive prefix
      bool done = false;
      for (int32_t tp = (int32_t)ti - 1; tp >= (int32_t)t.first_tile && !done; tp -= kLookAhead) {
        const int32_t cnt = min(kLookAhead, tp - (int32_t)t.first_tile + 1);
        uint32_t wv[kLookAhead];
#pragma unroll
        for (int u = 0; u < kLookAhead; ++u)
          if (u < cnt) wv[u] = ld_volatile(lookback + (size_t)(tp - u) * 256 + d);
#pragma unroll
        for (int u = 0; u < kLookAhead; ++u) {
          if (u >= cnt || done) break;
          uint32_t it = 0;
          for (; it < spin_limit && !(wv[u] & (kFlagAgg | kFlagInc)); ++it) {
            if (it > 32) __nanosleep(64);
            wv[u] = ld_volatile(lookback + (size_t)(tp - u) * 256 + d);
          }
          if (it == spin_limit) {
            atomicOr(&ctr->status, kStTimeout);
            s_fail = 1;
            done = true;
            break;
          }
          excl += wv[u] & kValMask;
          if (wv[u] & kFlagInc) done = true;
        }
      }
      if (publish) atomicExch(&lb[d], kFlagInc | (excl + run));
    }
    s_base[d] = digit_base[(size_t)t.frame * kMaxPasses * 256 + d] + excl;
  }
  __syncthreads();
  if (s_fail) return;
  // the tile in sorted order in shared memory ...
#pragma unroll
  for (int i = 0; i < kFrontItems; ++i) {
    const uint32_t d = dig[i];
    if (d >= 256u) continue;
    const uint32_t lp = s_doff[d] + s_wcnt[w][d] + rank[i];  // < tile size by construction
    s_key[lp] = key[i];
    s_val[lp] = val[i];
  }
  __syncthreads();
  // ... then written out: consecutive positions of one digit go to consecutive addresses
  const uint32_t fend = frames[t.frame].end, fbeg = frames[t.frame].begin;
  const uint32_t cnt = t.end - t.begin;
  for (uint32_t j = threadIdx.x; j < cnt; j += kFrontThreads) {
    const unsigned long long k = s_key[j];
    const uint32_t d = (uint32_t)((k >> shift) & 0xFFu);
    const uint32_t pos = s_base[d] + (j - s_doff[d]);
    if (pos < fbeg || pos >= fend) {
      atomicOr(&ctr->status, kStInternal);
      continue;
    }
    kout[pos] = k;
    const uint32_t v = s_val[j];
    if (kLast) {
      if (v >= fend) {  // values are point indices of this batch; never read out of bounds
        atomicOr(&ctr->status, kStInternal);
        continue;
      }
      pout[pos] = make_float4(xyz[3ull * v], xyz[3ull * v + 1], xyz[3ull * v + 2], __uint_as_float(v));
    } else {
      vout[pos] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Order inside the nodes that need it.  The radix passes sort by the key bits
// from `lowbit` up, which places every octree node down to level DB (the sorted
// depth) in one contiguous range; inside a level-DB node the points keep their
// input order.  That is all the leaf partition needs wherever a level-DB node
// holds at most leaf_capacity points (it lies inside one leaf).  A level-DB node
// with more points ("big") is brought into the full order here, (key bits from
// key_low up, input index), by the block of the tile where it starts: in shared
// memory (bitonic network) up to kNodeSmem points, else by stable 8-bit passes
// through the other key buffer.  Its packed points are written again after.
// (The point indices are taken from the packed points: the last radix pass
// writes them there instead of into the value buffer.)
// ---------------------------------------------------------------------------
constexpr uint32_t kNodeSmem = 2048;

__device__ __forceinline__ bool node_less(unsigned long long ka, uint32_t va, unsigned long long kb, uint32_t vb,
                                          int key_low) {
  const unsigned long long a = ka >> key_low, b = kb >> key_low;
  return a < b || (a == b && va < vb);
}

__global__ void __launch_bounds__(kFrontThreads) k_node_sort(
    unsigned long long *__restrict__ keys, uint32_t *__restrict__ vals, unsigned long long *__restrict__ tmpk,
    uint32_t *__restrict__ tmpv, float4 *__restrict__ spts, const float *__restrict__ xyz,
    const Tile *__restrict__ tiles, const FrameInfo *__restrict__ frames, Counters *ctr, uint32_t cap, int DB,
    int key_low) {
  constexpr int W = kFrontThreads / 32;
  __shared__ unsigned long long s_k[kNodeSmem];
  __shared__ uint32_t s_v[kNodeSmem];
  __shared__ uint32_t s_start[kTilePts];
  __shared__ uint32_t s_off[256];
  __shared__ uint32_t s_wc[W][256];
  __shared__ uint32_t s_wsum[W];
  __shared__ uint32_t s_n, s_end;
  pdl_wait();
  if (ctr->status & kStFatal) return;
  const Tile t = tiles[blockIdx.x];
  const uint32_t fb = frames[t.frame].begin, fe = frames[t.frame].end;
  const int sh = 63 - 3 * DB;  // a level-DB node's keys share key >> sh
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) s_n = 0;
  __syncthreads();
  // the big nodes that start in this tile
  for (uint32_t i = t.begin + tid; i < t.end; i += kFrontThreads) {
    const unsigned long long pre = keys[i] >> sh;
    const bool first = (i == fb) || ((keys[i - 1] >> sh) != pre);
    if (first && fe - i > cap && (keys[i + cap] >> sh) == pre) s_start[atomicAdd(&s_n, 1u)] = i;
  }
  __syncthreads();
  const uint32_t nn = s_n;
  for (uint32_t u = 0; u < nn; ++u) {
    const uint32_t s = s_start[u];
    if (tid == 0) {  // the node's end: it holds more than cap points, all sharing the prefix
      const unsigned long long pre = keys[s] >> sh;
      uint32_t lo = s + cap, hi = fe;
      while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if ((keys[mid] >> sh) == pre) lo = mid + 1;
        else hi = mid;
      }
      s_end = lo;
    }
    __syncthreads();
    const uint32_t e = s_end, n = e - s;
    // the last radix pass leaves the point indices in the packed points, not in vals
    for (uint32_t i = s + tid; i < e; i += kFrontThreads) vals[i] = __float_as_uint(spts[i].w);
    __syncthreads();
    if (n <= kNodeSmem) {
      uint32_t n2 = 1;
      while (n2 < n) n2 <<= 1;
      for (uint32_t j = tid; j < n2; j += kFrontThreads) {
        s_k[j] = j < n ? keys[s + j] : ~0ull;  // padding sorts last
        s_v[j] = j < n ? vals[s + j] : 0xFFFFFFFFu;
      }
      __syncthreads();
      for (uint32_t size = 2; size <= n2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t c = tid; c < (n2 >> 1); c += kFrontThreads) {
            const uint32_t a = 2 * stride * (c / stride) + (c % stride), b = a + stride;
            const bool up = (a & size) == 0;
            const unsigned long long ka = s_k[a], kb = s_k[b];
            const uint32_t va = s_v[a], vb = s_v[b];
            if (node_less(kb, vb, ka, va, key_low) == up) {
              s_k[a] = kb;
              s_k[b] = ka;
              s_v[a] = vb;
              s_v[b] = va;
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t j = tid; j < n; j += kFrontThreads) {
        keys[s + j] = s_k[j];
        vals[s + j] = s_v[j];
      }
    } else {
      // stable passes over the digits below the shared prefix, lowest first
      for (uint32_t i = tid; i < W * 256; i += kFrontThreads) (&s_wc[0][0])[i] = 0;
      unsigned long long *sk = keys, *dk = tmpk;
      uint32_t *sv = vals, *dv = tmpv;
      for (int shift = key_low; shift < sh; shift += 8) {
        s_off[tid] = 0;  // one digit per thread (kFrontThreads == 256)
        __syncthreads();
        for (uint32_t i = s + tid; i < e; i += kFrontThreads) atomicAdd(&s_off[(uint32_t)(sk[i] >> shift) & 0xFFu], 1u);
        __syncthreads();
        {  // exclusive scan of the 256 counts, offset by the node's start
          const uint32_t v = s_off[tid];
          uint32_t x = v;
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
          }
          if (lane == 31) s_wsum[w] = x;
          __syncthreads();
          uint32_t wp = 0;
          for (uint32_t ww = 0; ww < w; ++ww) wp += s_wsum[ww];
          s_off[tid] = s + wp + x - v;
        }
        __syncthreads();
        const uint32_t lt = lanemask_lt();
        for (uint32_t c0 = s; c0 < e; c0 += kFrontThreads) {
          const uint32_t i = c0 + tid;
          const bool ok = i < e;
          const unsigned long long k = ok ? sk[i] : 0ull;
          const uint32_t v = ok ? sv[i] : 0u;
          const uint32_t d = ok ? ((uint32_t)(k >> shift) & 0xFFu) : 256u;
          const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
          if (ok && (peers & lt) == 0) s_wc[w][d] = __popc(peers);
          __syncthreads();
          if (ok) {
            uint32_t pos = s_off[d] + __popc(peers & lt);
            for (uint32_t ww = 0; ww < w; ++ww) pos += s_wc[ww][d];
            dk[pos] = k;
            dv[pos] = v;
          }
          __syncthreads();
          {  // digit tid: advance its offset by the chunk's count, clear the warp counts
            uint32_t tot = 0;
            for (int ww = 0; ww < W; ++ww) {
              tot += s_wc[ww][tid];
              s_wc[ww][tid] = 0;
            }
            s_off[tid] += tot;
          }
          __syncthreads();
        }
        unsigned long long *tk = sk;
        sk = dk;
        dk = tk;
        uint32_t *tv = sv;
        sv = dv;
        dv = tv;
      }
      if (sk != keys) {  // an odd number of passes: the result is in the other buffer
        for (uint32_t i = s + tid; i < e; i += kFrontThreads) {
          keys[i] = sk[i];
          vals[i] = sv[i];
        }
      }
    }
    __syncthreads();
    for (uint32_t i = s + tid; i < e; i += kFrontThreads) {
      const uint32_t v = vals[i];
      if (v >= fe) {  // values are point indices of this batch
        atomicOr(&ctr->status, kStInternal);
        continue;
      }
      spts[i] = make_float4(xyz[3ull * v], xyz[3ull * v + 1], xyz[3ull * v + 2], __uint_as_float(v));
    }
    __syncthreads();
  }
}

// Without a sort (max_depth 0: one leaf per frame) the points are packed as is.
__global__ void k_pack(const float *__restrict__ xyz, const Tile *__restrict__ tiles,
                       float4 *__restrict__ pout, const Counters *ctr) {
  pdl_wait();
  if (ctr->status & kStFatal) return;
  const Tile t = tiles[blockIdx.x];
  for (uint32_t i = t.begin + threadIdx.x; i < t.end; i += blockDim.x)
    pout[i] = make_float4(xyz[3ull * i], xyz[3ull * i + 1], xyz[3ull * i + 2], __uint_as_float(i));
}

// ---------------------------------------------------------------------------
// leaf finder
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long prefix_of(unsigned long long k, int level) {
  return level == 0 ? 0ull : (k >> (63 - 3 * level));
}

// Binary searches over sorted keys; kb[idx - koff] is the key of sorted
// position idx (kb = a shared-memory window starting at position koff, or the
// global array with koff = 0).
// first index in [lo, hi) whose level-L prefix is >= pre
__device__ __forceinline__ uint32_t lower_pre(const unsigned long long *kb, uint32_t koff, uint32_t lo,
                                              uint32_t hi, unsigned long long pre, int level) {
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (prefix_of(kb[mid - koff], level) < pre) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
// first index in [lo, hi) whose level-L prefix is > pre
__device__ __forceinline__ uint32_t upper_pre(const unsigned long long *kb, uint32_t koff, uint32_t lo,
                                              uint32_t hi, unsigned long long pre, int level) {
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (prefix_of(kb[mid - koff], level) <= pre) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The leaf finder splits each front-end tile over kLeavesSplit blocks (more
// blocks, fewer items per thread: its binary searches are latency-bound).
constexpr uint32_t kLeavesSplit = 4;
constexpr uint32_t kLeavesPart = kTilePts / kLeavesSplit;
constexpr int kLeavesItems = kFrontItems / kLeavesSplit;
static_assert(kLeavesPart == (uint32_t)kLeavesItems * kFrontThreads, "whole items per thread");
// Largest leaf capacity whose key window fits the leaf finder's shared-memory budget
// (the window and the found-leaf buffer stay within the default 48 KB).
constexpr uint32_t kLeavesSmemKeys = 5600;  // 43.75 KB of keys
constexpr uint32_t kLeavesSmemCap = (kLeavesSmemKeys - kLeavesPart) / 2 - 1;
// static part: found-leaf buffer (kLeavesItems x threads x 5 B) + scan words
static_assert(kLeavesSmemKeys * 8 + kLeavesItems * kFrontThreads * 5 + 64 <= 48 * 1024,
              "leaf finder shared memory above the default 48 KB");

// A sorted position i starts a leaf iff it starts its frame, or every octree
// node shared with position i-1 holds more than leaf_capacity points (so the
// leaf of i is a proper descendant of the deepest shared node, and begins at i).
// Every search below stays within cap + 1 positions of i, except the one at the
// maximum depth D; with cap <= kLeavesSmemCap the block first stages its tile's
// keys plus that halo on both sides in shared memory and searches there.
__global__ void __launch_bounds__(kFrontThreads) k_leaves(const unsigned long long *__restrict__ keys,
                                                          const Tile *__restrict__ tiles,
                                                          const FrameInfo *__restrict__ frames,
                                                          Leaf *__restrict__ leaves, Counters *ctr,
                                                          uint32_t cap, int D, int DB) {
  extern __shared__ unsigned long long s_win[];
  pdl_wait();
  if (ctr->status & kStFatal) return;
  // kLeavesSplit blocks share a tile, each taking a contiguous part of it
  const Tile tile = tiles[blockIdx.x / kLeavesSplit];
  const uint32_t part = blockIdx.x % kLeavesSplit;
  Tile t = tile;
  t.begin = min(tile.end, tile.begin + part * kLeavesPart);
  t.end = min(tile.end, t.begin + kLeavesPart);
  const uint32_t fb = frames[t.frame].begin, fe = frames[t.frame].end;
  const unsigned long long *kb = keys;
  uint32_t koff = 0;
  if (cap <= kLeavesSmemCap) {  // block-uniform
    const uint32_t wb = (t.begin - fb > cap + 1) ? t.begin - cap - 1 : fb;
    const uint32_t we = (fe - t.end > cap + 1) ? t.end + cap + 1 : fe;
    for (uint32_t i = wb + threadIdx.x; i < we; i += kFrontThreads) s_win[i - wb] = keys[i];
    __syncthreads();
    kb = s_win;
    koff = wb;
  }
  // pass 1: each thread finds the leaves that start at its items (count, level)
  __shared__ uint32_t s_cnt[kLeavesItems][kFrontThreads];
  __shared__ uint8_t s_lvl[kLeavesItems][kFrontThreads];
  __shared__ uint32_t s_wsum[kFrontThreads / 32];
  __shared__ uint32_t s_base;
#pragma unroll 1
  for (int it = 0; it < kLeavesItems; ++it) {
    const uint32_t i = t.begin + it * kFrontThreads + threadIdx.x;
    s_cnt[it][threadIdx.x] = 0;
    if (i >= t.end) continue;
    const unsigned long long ki = kb[i - koff];
    int L;  // level of the first node that starts at i
    if (i == fb) {
      L = 0;
    } else {
      const unsigned long long x = kb[i - 1 - koff] ^ ki;
      int l = (x == 0) ? 21 : (__clzll((long long)x) - 1) / 3;  // shared levels below the root
      if (l >= D) continue;                                      // same max-depth node
      if (l > DB) {
        // i-1 and i share a level-DB node; below level DB the keys are in octree
        // order only inside level-DB nodes of more than cap points.  A smaller one
        // lies inside one leaf, which cannot start at i.
        const unsigned long long preB = prefix_of(ki, DB);
        const uint32_t wlo = (i - fb > cap + 1) ? i - cap - 1 : fb;
        const uint32_t whi = (fe - i > cap + 1) ? i + cap + 1 : fe;
        if (upper_pre(kb, koff, i, whi, preB, DB) - lower_pre(kb, koff, wlo, i, preB, DB) <= cap) continue;
      }
      // count of the level-l node containing i-1 and i, decided within a window
      bool big;
      if (l == 0) {
        big = (fe - fb) > cap;
      } else {
        const unsigned long long pre = prefix_of(ki, l);
        const uint32_t wlo = (i - fb > cap + 1) ? i - cap - 1 : fb;
        const uint32_t whi = (fe - i > cap + 1) ? i + cap + 1 : fe;
        const uint32_t a = lower_pre(kb, koff, wlo, i, pre, l);
        const uint32_t b = upper_pre(kb, koff, i, whi, pre, l);
        big = (b - a) > cap;
      }
      if (!big) continue;
      L = l + 1;
    }
    // descend from the level-L node starting at i to the leaf containing i
    for (;; ++L) {
      const unsigned long long pre = prefix_of(ki, L);
      uint32_t e;
      if (L < D) {
        const uint32_t whi = (fe - i > cap + 1) ? i + cap + 1 : fe;
        e = upper_pre(kb, koff, i, whi, pre, L);
        if (e - i > cap) continue;
      } else {
        e = upper_pre(keys, 0, i, fe, pre, L);  // a max-depth node may be of any size
      }
      s_cnt[it][threadIdx.x] = e - i;  // >= 1: position i is in its own leaf
      s_lvl[it][threadIdx.x] = (uint8_t)L;
      break;
    }
  }
  // pass 2: one atomic per block reserves the block's leaf slots
  uint32_t mine = 0;
#pragma unroll
  for (int it = 0; it < kLeavesItems; ++it) mine += s_cnt[it][threadIdx.x] ? 1u : 0u;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) s_wsum[w] = inc;
  __syncthreads();
  uint32_t wp = 0, total = 0;
  for (int ww = 0; ww < kFrontThreads / 32; ++ww) {
    if (ww < (int)w) wp += s_wsum[ww];
    total += s_wsum[ww];
  }
  if (threadIdx.x == 0) s_base = total ? atomicAdd(&ctr->n_leaves, total) : 0u;
  __syncthreads();
  uint32_t slot = s_base + wp + inc - mine;
#pragma unroll
  for (int it = 0; it < kLeavesItems; ++it) {
    const uint32_t c = s_cnt[it][threadIdx.x];
    if (!c) continue;
    Leaf lf{};
    lf.start = t.begin + it * kFrontThreads + threadIdx.x;
    lf.count = c;
    lf.frame = t.frame;
    lf.level = s_lvl[it][threadIdx.x];
    leaves[slot++] = lf;
  }
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------
namespace {
// The passes of a call: all ceil(3 D / 8) digits of the key's 3 D bits, or the top
// kTopPasses of them; *sorted_depth receives the deepest level whose nodes are
// contiguous after them (D when every bit is sorted), *key_low the key's lowest bit.
int front_plan(int max_depth, bool full_sort, int *lowbit, int *sorted_depth, int *key_low) {
  const int all = (3 * max_depth + 7) / 8;
  const int passes = (full_sort || all <= kTopPasses) ? all : kTopPasses;
  *key_low = 63 - 3 * max_depth;
  *lowbit = *key_low + 8 * (all - passes);  // lowest sorted bit
  *sorted_depth = (passes == all) ? max_depth : (63 - *lowbit) / 3;
  return passes;
}
}  // namespace

int front_sorted_buffer(int max_depth, bool full_sort) {
  int lowbit, db, kl;
  return front_plan(max_depth, full_sort, &lowbit, &db, &kl) & 1;
}

int launch_front(const FrontArgs &a, cudaStream_t st, int *launches, cudaEvent_t *ev_after_keys,
                 cudaEvent_t *ev_after_sort) {
  int lowbit = 0, DB = 0, key_low = 0;
  const int passes = front_plan(a.max_depth, a.full_sort, &lowbit, &DB, &key_low);
  const uint32_t spin = a.spin_limit ? a.spin_limit : kSpinLimit;
  const uint32_t nlb = a.ntiles * 256u;
  int nl = 0;
  {
    uint32_t work = a.nframes * kMaxPasses * 256u;
    if (nlb * (uint32_t)passes > work) work = nlb * (uint32_t)passes;
    uint32_t blocks = (work + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    launch_pdl(k_init, blocks, 256, 0, st, a.frames, a.nframes, a.ctr, a.digit_hist, a.lookback, nlb, passes);
    ++nl;
  }
  launch_pdl(k_bbox, a.ntiles, kFrontThreads, 0, st, a.xyz_src ? a.xyz_src : a.xyz, a.xyz_copy, a.frames, a.tiles,
             a.ctr);
  launch_pdl(k_keys, a.ntiles, kFrontThreads, 0, st, a.xyz, a.frames, a.tiles, a.keys[0], a.vals[0], a.dbg_key,
                                             a.digit_hist, lowbit, passes, a.ctr);
  nl += 2;
  if (ev_after_keys) cudaEventRecord(*ev_after_keys, st);
  int cur = 0;
  if (passes > 0) {
    launch_pdl(k_digit_scan, a.nframes * passes, 256, 0, st, a.digit_hist, a.digit_base, a.frames, passes, a.ctr);
    ++nl;
    for (int p = 0; p < passes; ++p) {
      const int shift = lowbit + 8 * p;
      const uint32_t *base = a.digit_base + p * 256;
      uint32_t *lb = a.lookback + (size_t)p * nlb;
      if (p == passes - 1) {
        launch_pdl(k_radix_pass<true>, a.ntiles, kFrontThreads, 0, st,
            a.keys[cur], a.vals[cur], a.keys[cur ^ 1], a.vals[cur ^ 1], a.spts, a.xyz, a.tiles, a.frames,
            base, lb, &a.ctr->tile_work[p], shift, a.ctr, spin, p == 0 ? a.hold_tile1 : 0u);
      } else {
        launch_pdl(k_radix_pass<false>, a.ntiles, kFrontThreads, 0, st,
            a.keys[cur], a.vals[cur], a.keys[cur ^ 1], a.vals[cur ^ 1], a.spts, a.xyz, a.tiles, a.frames,
            base, lb, &a.ctr->tile_work[p], shift, a.ctr, spin, p == 0 ? a.hold_tile1 : 0u);
      }
      cur ^= 1;
      ++nl;
    }
  } else {
    launch_pdl(k_pack, a.ntiles, kFrontThreads, 0, st, a.xyz, a.tiles, a.spts, a.ctr);
    ++nl;
  }
  // a capacity above any frame's size means the same as "the root is a leaf"; clamped
  // so that the finder's window arithmetic (cap + 1) cannot wrap
  const uint32_t cap = a.leaf_capacity < (1u << 30) ? a.leaf_capacity : (1u << 30);
  if (DB < a.max_depth) {  // the big level-DB nodes in full octree order
    launch_pdl(k_node_sort, a.ntiles, kFrontThreads, 0, st, a.keys[cur], a.vals[cur], a.keys[cur ^ 1], a.vals[cur ^ 1],
               a.spts, a.xyz, a.tiles, a.frames, a.ctr, cap, DB, key_low);
    ++nl;
  }
  if (ev_after_sort) cudaEventRecord(*ev_after_sort, st);
  const size_t win = (a.leaf_capacity <= kLeavesSmemCap)
                        ? sizeof(unsigned long long) * (kLeavesPart + 2 * ((size_t)a.leaf_capacity + 1))
                        : 0;
  launch_pdl(k_leaves, a.ntiles * kLeavesSplit, kFrontThreads, win, st, a.keys[cur], a.tiles, a.frames, a.leaves, a.ctr,
             cap, a.max_depth, DB);
  ++nl;
  if (launches) *launches += nl;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace gd
