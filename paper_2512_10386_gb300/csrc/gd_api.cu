// gd_api.cu -- the C ABI declared in include/gravdenoise.h: contexts, argument
// checks, host/device staging, kernel sequencing, optional CUDA-graph capture.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "gd_common.cuh"

using namespace gd;

struct denoise_ctx {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  size_t max_points = 0;
  uint32_t max_frames = 0;
  uint32_t max_tiles = 0;
  // device memory
  float *d_xyz = nullptr;
  uint8_t *d_mask = nullptr;
  float *d_score = nullptr;
  uint8_t *d_stage = nullptr;
  float *d_gin = nullptr;
  unsigned long long *d_keys[2] = {nullptr, nullptr};
  uint32_t *d_vals[2] = {nullptr, nullptr};
  float4 *d_spts = nullptr;
  FrameInfo *d_frames = nullptr;
  Tile *d_tiles = nullptr;
  uint32_t *d_hist = nullptr;
  uint32_t *d_base = nullptr;
  uint32_t *d_lookback = nullptr;
  Leaf *d_leaves = nullptr;
  uint32_t *d_order = nullptr;
  Counters *d_ctr = nullptr;
  unsigned char *d_big = nullptr;
  uint32_t big_bpp = 0;
  double *d_partials = nullptr;
  double *d_grad = nullptr;
  // training cache (allocated by denoise_set_training)
  TrainCache train{};
  bool train_alloc = false;
  // cross-leaf tables (allocated by denoise_set_cross_leaf), by sorted position
  uint32_t *x_nbr = nullptr;  // [max_points][64]
  float *x_r2 = nullptr;
  uint32_t *x_keff = nullptr;
  uint8_t *x_flag = nullptr;
  // pinned host memory
  // pinned tile/frame tables: a ring of slots, so that a call with a new frame
  // layout does not wait for the calls still in flight (each slot is rewritten
  // only after the call that last copied from it has passed `staged`)
  static constexpr int kSlots = 4;
  Tile *h_tiles[kSlots] = {};
  FrameInfo *h_frames[kSlots] = {};
  cudaEvent_t staged[kSlots] = {};
  bool staged_rec[kSlots] = {};
  int slot = 0;
  Counters *h_ctr = nullptr;
  Counters *h_ctr_dev = nullptr;  // mapped device address of h_ctr (null: copied by the copy engine)
  double *h_grad = nullptr;
  // options
  int sync = 1, graphs = 0, profiling = 0, training = 0;
  uint32_t leaf_ctas_per_sm = 0;
  uint32_t leaf_smem_points = 0;
  uint32_t leaf_threads = 0;
  uint32_t wait_limit = 0;   // bounded device waits (0 = built-in limit)
  uint32_t hold_tile1 = 0;   // test hook of the radix look-back (0 = off)
  // last call
  size_t last_n = 0;
  uint32_t last_nframes = 0;
  denoise_params last_p{};
  bool last_trained = false;
  int last_launches = 0;
  int last_status_read = 0;
  float stage_ms[8] = {0};
  int n_stage_ms = 0;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // graph cache (captured on a private stream, launched on the caller's)
  cudaStream_t cap_stream = nullptr;
  // the small-leaf launch runs on a side stream, forked from and joined into the call's stream
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  // frame layout cache
  std::vector<uint64_t> layout;
  uint32_t ntiles = 0;
  uint64_t layout_gen = 0;        // bumped at every layout change
  uint64_t tables_gen = ~0ull;    // layout generation that d_tiles / d_frames hold (after a direct call)
};

namespace {

constexpr size_t kBackPartials = 1024;

// Where a caller's buffer lives: host memory (staged through the context), device
// memory of the context's GPU, or unusable (device memory of another GPU, which
// the kernels could not read without peer access).
enum class Loc { kHost, kDevice, kOtherDevice };

// For pinned host memory `mapped` (if given) receives its device address, else null.
Loc locate(const void *p, int device, void **mapped = nullptr) {
  cudaPointerAttributes at;
  if (mapped) *mapped = nullptr;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return Loc::kHost;
  }
  if (at.type == cudaMemoryTypeManaged) return Loc::kDevice;
  if (at.type == cudaMemoryTypeDevice) return at.device == device ? Loc::kDevice : Loc::kOtherDevice;
  if (mapped && at.type == cudaMemoryTypeHost) *mapped = at.devicePointer;
  return Loc::kHost;
}

// Device address of pinned (page-locked, mapped) host memory, or null for anything else.
const float *mapped_host(const float *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? static_cast<const float *>(at.devicePointer) : nullptr;
}

int check_params(const denoise_params *p) {
  if (!p) return DENOISE_E_INVAL;
  if (p->k == 0 || p->k > 64) return DENOISE_E_INVAL;
  if (p->leaf_capacity == 0) return DENOISE_E_INVAL;
  if (p->max_depth > 21) return DENOISE_E_INVAL;
  if (!(p->beta > 0.0f) || !isfinite(p->beta)) return DENOISE_E_INVAL;
  if (!(p->rho_percentile >= 0.0f && p->rho_percentile <= 100.0f)) return DENOISE_E_INVAL;
  if (!(p->lambda > 0.0f && p->lambda <= 1.0f)) return DENOISE_E_INVAL;
  if (!(p->gamma > 0.0f) || !isfinite(p->gamma)) return DENOISE_E_INVAL;
  if (!(p->sigma > 0.0f) || !isfinite(p->sigma)) return DENOISE_E_INVAL;
  if (!isfinite(p->alpha) || !(p->eps_rho >= 0.0f) || !(p->eps_k >= 0.0f)) return DENOISE_E_INVAL;
  if (!isfinite(p->eps_rho) || !isfinite(p->eps_k) || !isfinite(p->tau)) return DENOISE_E_INVAL;
  if (p->select_mode > 1) return DENOISE_E_INVAL;
  if (!(p->temperature > 0.0f) || !isfinite(p->temperature)) return DENOISE_E_INVAL;
  if (p->stage_off > 7u || p->rescore_p2 > 1u || p->cross_leaf > 1u) return DENOISE_E_INVAL;
  if (p->cross_leaf && (p->stage_off || p->rescore_p2)) return DENOISE_E_INVAL;
  return DENOISE_OK;
}

template <typename T>
int dalloc(T **p, size_t count) {
  if (count == 0) count = 1;
  return cudaMalloc((void **)p, sizeof(T) * count) == cudaSuccess ? 0 : -1;
}

void free_ctx(denoise_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  void *dptrs[] = {c->d_xyz, c->d_mask, c->d_score, c->d_stage, c->d_gin, c->d_keys[0], c->d_keys[1],
                   c->d_vals[0], c->d_vals[1], c->d_spts, c->d_frames, c->d_tiles, c->d_hist, c->d_base,
                   c->d_lookback, c->d_leaves, c->d_order, c->d_ctr, c->d_big, c->d_partials, c->d_grad,
                   c->train.nbr, c->train.nd2, c->train.ell, c->train.r2, c->train.F, c->train.stage,
                   c->x_nbr, c->x_r2, c->x_keff, c->x_flag};
  for (void *p : dptrs)
    if (p) cudaFree(p);
  void *hptrs[] = {c->h_ctr, c->h_grad};
  for (void *p : hptrs)
    if (p) cudaFreeHost(p);
  for (int i = 0; i < denoise_ctx::kSlots; ++i) {
    if (c->h_tiles[i]) cudaFreeHost(c->h_tiles[i]);
    if (c->h_frames[i]) cudaFreeHost(c->h_frames[i]);
    if (c->staged[i]) cudaEventDestroy(c->staged[i]);
  }
  for (auto &e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  cudaGetLastError();
  delete c;
}

// A failed runtime call leaves a "last error" in the process-wide runtime that
// the next caller (e.g. PyTorch) would report as its own: clear it here.
int cuda_fail() {
  cudaGetLastError();
  return DENOISE_E_CUDA;
}

int map_status(uint32_t st) {
  if (st & kStNonFinite) return DENOISE_E_NONFINITE;
  if (st & kStTimeout) return DENOISE_E_TIMEOUT;
  if (st & kStInternal) return DENOISE_E_CUDA;
  return DENOISE_OK;
}

// Front-end tiles of a frame layout (host); returns the tile count.
uint32_t build_tiles(denoise_ctx *c, const uint64_t *offsets, uint32_t nframes) {
  uint32_t nt = 0;
  for (uint32_t f = 0; f < nframes; ++f) {
    const uint32_t b = (uint32_t)offsets[f], e = (uint32_t)offsets[f + 1];
    FrameInfo &fi = c->h_frames[c->slot][f];
    fi = FrameInfo{};
    fi.begin = b;
    fi.end = e;
    const uint32_t first = nt;
    for (uint32_t s = b; s < e; s += kTilePts) {
      const uint32_t te = (e - s > (uint32_t)kTilePts) ? s + kTilePts : e;
      c->h_tiles[c->slot][nt++] = Tile{f, s, te, first};
    }
  }
  return nt;
}

// Enqueue one whole call on `st`.  Returns a DENOISE status (host-side errors only).
int enqueue(denoise_ctx *c, const float *xyz_dev, uint32_t n, uint32_t nframes, const denoise_params &p,
            uint8_t *mask, float *score, uint8_t *stage, const denoise_debug *dbg, bool use_events,
            cudaStream_t st, const float *xyz_host, uint8_t *mask_h, float *score_h, uint8_t *stage_h,
            void *const out_mapped[3]) {
  int launches = 0;
  // Pinned host input is read in place by the bounding-box pass, which writes the
  // device copy on the way (one pass over the link, overlapped with the reduction);
  // other host memory is copied first.
  const float *xyz_mapped = xyz_host ? mapped_host(xyz_host) : nullptr;
  if (xyz_host && !xyz_mapped) {
    if (cudaMemcpyAsync(c->d_xyz, xyz_host, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return cuda_fail();
  }
  // The tile and frame tables go up when the layout changed since the last direct
  // call that uploaded them (no kernel writes a tile or a frame's bounds; a frame's
  // per-call fields are reset on the device), and always into a captured graph,
  // which has to stand alone.
  const bool capturing = st == c->cap_stream;
  const bool upload = capturing || c->tables_gen != c->layout_gen;
  if (upload) {
    if (!capturing) c->tables_gen = ~0ull;  // valid again only once this call is enqueued
    cudaMemcpyAsync(c->d_tiles, c->h_tiles[c->slot], sizeof(Tile) * c->ntiles, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(c->d_frames, c->h_frames[c->slot], sizeof(FrameInfo) * nframes, cudaMemcpyHostToDevice, st);
  }
  if (use_events) cudaEventRecord(c->ev[0], st);
  FrontArgs fa{};
  fa.xyz = xyz_dev;
  fa.xyz_src = xyz_mapped;
  fa.xyz_copy = xyz_mapped ? c->d_xyz : nullptr;
  fa.n = n;
  fa.frames = c->d_frames;
  fa.nframes = nframes;
  fa.tiles = c->d_tiles;
  fa.ntiles = c->ntiles;
  fa.keys[0] = c->d_keys[0];
  fa.keys[1] = c->d_keys[1];
  fa.vals[0] = c->d_vals[0];
  fa.vals[1] = c->d_vals[1];
  fa.spts = c->d_spts;
  fa.digit_hist = c->d_hist;
  fa.digit_base = c->d_base;
  fa.lookback = c->d_lookback;
  fa.leaves = c->d_leaves;
  fa.ctr = c->d_ctr;
  fa.dbg_key = dbg ? dbg->key : nullptr;
  fa.max_depth = (int)p.max_depth;
  fa.leaf_capacity = p.leaf_capacity;
  fa.full_sort = p.cross_leaf != 0;
  fa.spin_limit = c->wait_limit;
  fa.hold_tile1 = c->hold_tile1;
  if (launch_front(fa, st, &launches, use_events ? &c->ev[1] : nullptr, use_events ? &c->ev[2] : nullptr))
    return cuda_fail();
  if (use_events) cudaEventRecord(c->ev[3], st);
  LeafArgs la{};
  la.n = n;
  la.spts = c->d_spts;
  la.leaves = c->d_leaves;
  la.order = c->d_order;
  la.frames = c->d_frames;
  la.ctr = c->d_ctr;
  la.p = p;
  la.mask = mask;
  la.score = score;
  la.stage = stage;
  if (dbg) {
    la.dbg = *dbg;
    la.use_dbg = 1;
  }
  la.big_scratch = c->d_big;
  la.big_bpp = c->big_bpp;
  la.ctas_per_sm = c->leaf_ctas_per_sm;
  la.threads = c->leaf_threads;
  la.spin_limit = c->wait_limit;
  const int kmax = leaf_kmax(p.k);
  la.lmax = leaf_pick_lmax(p.leaf_capacity, kmax, c->smem_optin - 2048);
  if (c->leaf_smem_points) {
    uint32_t l = 64;
    while (l * 2 <= c->leaf_smem_points) l *= 2;
    if (l < la.lmax) la.lmax = l;
  }
  if (c->training) {
    la.train = c->train;
    la.train.k = p.k;
    la.use_train = 1;
  }
  if (launch_leaf_prep(la, c->num_sms, st, &launches)) return cuda_fail();
  if (use_events) cudaEventRecord(c->ev[4], st);
  if (p.cross_leaf) {
    // phase 1 (voxel gates: P_1), the cross-leaf kNN, phase 3 (the per-leaf steps after the kNN)
    la.xflag = c->x_flag;
    la.xnbr = c->x_nbr;
    la.xr2 = c->x_r2;
    la.xkeff = c->x_keff;
    la.xphase = 1;
    if (launch_leaf(la, c->num_sms, st, &launches)) return cuda_fail();
    XleafArgs xa{};
    xa.n = n;
    xa.spts = c->d_spts;
    xa.keys = c->d_keys[front_sorted_buffer((int)p.max_depth, true)];
    xa.leaves = c->d_leaves;
    xa.frames = c->d_frames;
    xa.ctr = c->d_ctr;
    xa.k = p.k;
    xa.xflag = c->x_flag;
    xa.xnbr = c->x_nbr;
    xa.xr2 = c->x_r2;
    xa.xkeff = c->x_keff;
    if (dbg) {
      xa.dbg = *dbg;
      xa.use_dbg = 1;
    }
    xa.unit_start = c->d_vals[0];  // free after the front end
    if (launch_xleaf_knn(xa, c->num_sms, st, &launches)) return cuda_fail();
    la.xphase = 3;
  }
  if (launch_leaf(la, c->num_sms, st, &launches, c->side_stream, c->fork_ev, c->join_ev)) return cuda_fail();
  if (use_events) cudaEventRecord(c->ev[5], st);
  // Results into host buffers: pinned ones and the counters by one kernel through
  // their mapped addresses; other host memory (and everything, where the counters
  // have no mapped address) by the copy engine.
  const bool by_sms = c->h_ctr_dev != nullptr;
  uint8_t *mask_m = by_sms && mask_h ? static_cast<uint8_t *>(out_mapped[0]) : nullptr;
  float *score_m = by_sms && score_h ? static_cast<float *>(out_mapped[1]) : nullptr;
  uint8_t *stage_m = by_sms && stage_h ? static_cast<uint8_t *>(out_mapped[2]) : nullptr;
  if (mask_h && !mask_m) cudaMemcpyAsync(mask_h, c->d_mask, n, cudaMemcpyDeviceToHost, st);
  if (score_h && !score_m) cudaMemcpyAsync(score_h, c->d_score, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (stage_h && !stage_m) cudaMemcpyAsync(stage_h, c->d_stage, n, cudaMemcpyDeviceToHost, st);
  if (by_sms) {
    const OutArgs oa{c->d_mask, c->d_score, c->d_stage, mask_m, score_m, stage_m, n, c->d_ctr, c->h_ctr_dev};
    if (launch_out(oa, c->num_sms, st)) return cuda_fail();
    ++launches;
  } else {
    cudaMemcpyAsync(c->h_ctr, c->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
  }
  c->last_launches = launches;
  if (cudaGetLastError() != cudaSuccess) return DENOISE_E_CUDA;
  if (upload && !capturing) c->tables_gen = c->layout_gen;
  return DENOISE_OK;
}

int finish(denoise_ctx *c, cudaStream_t st, bool events) {
  if (!c->sync) return DENOISE_OK;
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail();
  if (events) {
    c->n_stage_ms = 5;
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&c->stage_ms[i], c->ev[i], c->ev[i + 1]);
  }
  return map_status(c->h_ctr->status);
}

int run_impl(denoise_ctx *c, const float *xyz, const uint64_t *offsets, uint32_t nframes, const denoise_params *p,
             uint8_t *mask, float *score, uint8_t *stage, const denoise_debug *dbg, void *stream) {
  if (!c || !offsets) return DENOISE_E_INVAL;
  int s = check_params(p);
  if (s) return s;
  if (nframes == 0) return DENOISE_E_INVAL;
  if (nframes > c->max_frames) return DENOISE_E_CAPACITY;
  if (offsets[0] != 0) return DENOISE_E_INVAL;
  for (uint32_t f = 0; f < nframes; ++f)
    if (offsets[f + 1] < offsets[f]) return DENOISE_E_INVAL;
  const uint64_t n64 = offsets[nframes];
  if (n64 > c->max_points) return DENOISE_E_CAPACITY;
  if (cudaSetDevice(c->device) != cudaSuccess) return DENOISE_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  c->last_n = (size_t)n64;
  c->last_nframes = nframes;
  c->last_p = *p;
  c->last_trained = false;
  if (n64 == 0) {
    memset(c->h_ctr, 0, sizeof(Counters));
    c->last_launches = 0;
    return DENOISE_OK;
  }
  if (!xyz) return DENOISE_E_INVAL;
  const uint32_t n = (uint32_t)n64;
  if (c->training && !c->train_alloc) return DENOISE_E_STATE;
  if (c->training && p->k > 64) return DENOISE_E_INVAL;
  if (p->cross_leaf && !c->x_nbr) return DENOISE_E_STATE;

  // resolve host / device buffers (device memory of another GPU is rejected)
  const Loc lx = locate(xyz, c->device);
  void *out_mapped[3] = {nullptr, nullptr, nullptr};  // device addresses of pinned host outputs
  const Loc lm = mask ? locate(mask, c->device, &out_mapped[0]) : Loc::kDevice;
  const Loc ls = score ? locate(score, c->device, &out_mapped[1]) : Loc::kDevice;
  const Loc lg = stage ? locate(stage, c->device, &out_mapped[2]) : Loc::kDevice;
  if (lx == Loc::kOtherDevice || lm == Loc::kOtherDevice || ls == Loc::kOtherDevice || lg == Loc::kOtherDevice)
    return DENOISE_E_INVAL;
  const bool xyz_dev = lx == Loc::kDevice;
  const float *xyz_d = xyz_dev ? xyz : c->d_xyz;
  const float *xyz_h = xyz_dev ? nullptr : xyz;
  uint8_t *mask_d = mask, *mask_h = nullptr;
  float *score_d = score, *score_h = nullptr;
  uint8_t *stage_d = stage, *stage_h = nullptr;
  if (mask && lm == Loc::kHost) { mask_h = mask; mask_d = c->d_mask; }
  if (score && ls == Loc::kHost) { score_h = score; score_d = c->d_score; }
  if (stage && lg == Loc::kHost) { stage_h = stage; stage_d = c->d_stage; }

  // frame layout -> tiles (re-built only when it changes)
  bool layout_changed = c->layout.size() != nframes + 1 ||
                        memcmp(c->layout.data(), offsets, sizeof(uint64_t) * (nframes + 1)) != 0;
  if (layout_changed) {
    const int ns = (c->slot + 1) % denoise_ctx::kSlots;
    if (c->staged_rec[ns] && cudaEventSynchronize(c->staged[ns]) != cudaSuccess)  // slot still being copied
      return cuda_fail();
    c->slot = ns;
    c->layout.assign(offsets, offsets + nframes + 1);
    c->ntiles = build_tiles(c, offsets, nframes);
    ++c->layout_gen;
  }
  const bool events = c->profiling && !c->graphs && c->sync;
  int rc;
  if (c->graphs && !dbg) {
    // graph key: everything the captured work depends on
    std::vector<unsigned char> key;
    auto put = [&](const void *v, size_t b) {
      const unsigned char *q = (const unsigned char *)v;
      key.insert(key.end(), q, q + b);
    };
    put(p, sizeof(*p));
    put(&xyz, sizeof(xyz));
    put(&mask, sizeof(mask));
    put(&score, sizeof(score));
    put(&stage, sizeof(stage));
    put(&c->training, sizeof(c->training));
    put(&c->leaf_ctas_per_sm, sizeof(c->leaf_ctas_per_sm));
    put(&c->leaf_smem_points, sizeof(c->leaf_smem_points));
    put(&c->leaf_threads, sizeof(c->leaf_threads));
    put(&c->wait_limit, sizeof(c->wait_limit));
    put(&c->hold_tile1, sizeof(c->hold_tile1));
    put(offsets, sizeof(uint64_t) * (nframes + 1));
    put(&c->slot, sizeof(c->slot));  // the staging slot the graph's table copies read (rewritten for other layouts)
    if (!c->gexec || key != c->gkey) {
      if (c->gexec) {
        cudaStreamSynchronize(st);
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail();
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return cuda_fail();
      rc = enqueue(c, xyz_d, n, nframes, *p, mask_d, score_d, stage_d, nullptr, false, c->cap_stream, xyz_h, mask_h,
                   score_h, stage_h, out_mapped);
      const cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
      if (rc || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : DENOISE_E_CUDA;
      }
      const cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail();
      }
      c->gkey.swap(key);
    }
    if (cudaGraphLaunch(c->gexec, st) != cudaSuccess) return cuda_fail();
  } else {
    rc = enqueue(c, xyz_d, n, nframes, *p, mask_d, score_d, stage_d, dbg, events, st, xyz_h, mask_h, score_h,
                 stage_h, out_mapped);
    if (rc) return rc;
  }
  if (cudaEventRecord(c->staged[c->slot], st) != cudaSuccess) return cuda_fail();
  c->staged_rec[c->slot] = true;
  c->last_trained = c->training != 0;
  c->last_status_read = 0;
  return finish(c, st, events);
}

}  // namespace

extern "C" {

const char *denoise_strerror(int s) {
  switch (s) {
    case DENOISE_OK: return "ok";
    case DENOISE_E_INVAL: return "invalid argument or parameter";
    case DENOISE_E_NONFINITE: return "input contains a NaN or infinite coordinate";
    case DENOISE_E_CAPACITY: return "more points or frames than the context was created for";
    case DENOISE_E_NOMEM: return "out of device or pinned host memory";
    case DENOISE_E_TIMEOUT: return "a bounded device-side wait ran out";
    case DENOISE_E_CUDA: return "CUDA runtime error";
    case DENOISE_E_STATE: return "call out of order (no training forward to differentiate)";
    default: return "unknown status";
  }
}

int denoise_create(denoise_ctx **out, int device, size_t max_points, uint32_t max_frames) {
  if (!out) return DENOISE_E_INVAL;
  *out = nullptr;
  if (max_points == 0 || max_frames == 0 || max_points >= (1u << 30)) return DENOISE_E_INVAL;
  if (cudaSetDevice(device) != cudaSuccess) return DENOISE_E_CUDA;
  denoise_ctx *c = new (std::nothrow) denoise_ctx();
  if (!c) return DENOISE_E_NOMEM;
  c->device = device;
  c->max_points = max_points;
  c->max_frames = max_frames;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    free_ctx(c);
    return DENOISE_E_CUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  c->max_tiles = (uint32_t)(max_points / kTilePts) + max_frames + 1;
  c->big_bpp = leaf_big_bpp(64);
  const size_t N = max_points;
  int e = 0;
  // largest first: a context too large for the GPU fails before it holds anything
  e |= dalloc(&c->d_big, N * c->big_bpp);
  if (!e) e |= dalloc(&c->d_xyz, 3 * N);
  e |= dalloc(&c->d_mask, N);
  e |= dalloc(&c->d_score, N);
  e |= dalloc(&c->d_stage, N);
  e |= dalloc(&c->d_gin, N);
  e |= dalloc(&c->d_keys[0], N);
  e |= dalloc(&c->d_keys[1], N);
  e |= dalloc(&c->d_vals[0], N);
  e |= dalloc(&c->d_vals[1], N);
  e |= dalloc(&c->d_spts, N);
  e |= dalloc(&c->d_frames, max_frames);
  e |= dalloc(&c->d_tiles, c->max_tiles);
  e |= dalloc(&c->d_hist, (size_t)max_frames * kMaxPasses * 256);
  e |= dalloc(&c->d_base, (size_t)max_frames * kMaxPasses * 256);
  e |= dalloc(&c->d_lookback, (size_t)kMaxPasses * c->max_tiles * 256);
  e |= dalloc(&c->d_leaves, N);
  e |= dalloc(&c->d_order, N);
  e |= dalloc(&c->d_ctr, 1);
  e |= dalloc(&c->d_partials, kBackPartials * 4);
  e |= dalloc(&c->d_grad, 4);
  if (e) {
    cudaGetLastError();
    free_ctx(c);
    return DENOISE_E_NOMEM;
  }
  bool pinned_ok = true;
  for (int i = 0; i < denoise_ctx::kSlots; ++i)
    pinned_ok = pinned_ok && cudaMallocHost((void **)&c->h_tiles[i], sizeof(Tile) * c->max_tiles) == cudaSuccess &&
                cudaMallocHost((void **)&c->h_frames[i], sizeof(FrameInfo) * max_frames) == cudaSuccess;
  if (!pinned_ok || cudaMallocHost((void **)&c->h_ctr, sizeof(Counters)) != cudaSuccess ||
      cudaMallocHost((void **)&c->h_grad, sizeof(double) * 4) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(c);
    return DENOISE_E_NOMEM;
  }
  memset(c->h_ctr, 0, sizeof(Counters));
  if (cudaHostGetDevicePointer((void **)&c->h_ctr_dev, c->h_ctr, 0) != cudaSuccess) {
    cudaGetLastError();
    c->h_ctr_dev = nullptr;
  }
  for (auto &ev : c->ev) {
    if (cudaEventCreate(&ev) != cudaSuccess) {
      free_ctx(c);
      return DENOISE_E_CUDA;
    }
  }
  for (auto &ev : c->staged) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      free_ctx(c);
      return DENOISE_E_CUDA;
    }
  }
  if (cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    free_ctx(c);
    return DENOISE_E_CUDA;
  }
  *out = c;
  return DENOISE_OK;
}

int denoise_destroy(denoise_ctx *ctx) {
  if (!ctx) return DENOISE_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  free_ctx(ctx);
  return DENOISE_OK;
}

int denoise_run(denoise_ctx *ctx, const float *xyz, size_t n, const denoise_params *p, uint8_t *mask, float *score,
                uint8_t *stage, void *stream) {
  const uint64_t off[2] = {0, (uint64_t)n};
  return run_impl(ctx, xyz, off, 1, p, mask, score, stage, nullptr, stream);
}

int denoise_run_debug(denoise_ctx *ctx, const float *xyz, size_t n, const denoise_params *p, uint8_t *mask,
                      float *score, uint8_t *stage, const denoise_debug *dbg, void *stream) {
  const uint64_t off[2] = {0, (uint64_t)n};
  return run_impl(ctx, xyz, off, 1, p, mask, score, stage, dbg, stream);
}

int denoise_run_batch(denoise_ctx *ctx, const float *xyz, const uint64_t *offsets, uint32_t nframes,
                      const denoise_params *p, uint8_t *mask, float *score, uint8_t *stage, void *stream) {
  return run_impl(ctx, xyz, offsets, nframes, p, mask, score, stage, nullptr, stream);
}

int denoise_set_sync(denoise_ctx *ctx, int synchronous) {
  if (!ctx) return DENOISE_E_INVAL;
  ctx->sync = synchronous ? 1 : 0;
  return DENOISE_OK;
}

int denoise_set_graphs(denoise_ctx *ctx, int enable) {
  if (!ctx) return DENOISE_E_INVAL;
  ctx->graphs = enable ? 1 : 0;
  return DENOISE_OK;
}

int denoise_set_profiling(denoise_ctx *ctx, int enable) {
  if (!ctx) return DENOISE_E_INVAL;
  ctx->profiling = enable ? 1 : 0;
  return DENOISE_OK;
}

int denoise_set_tuning(denoise_ctx *ctx, const denoise_tuning *t) {
  if (!ctx || !t) return DENOISE_E_INVAL;
  if (t->leaf_threads != 0 && t->leaf_threads != 64 && t->leaf_threads != 128) return DENOISE_E_INVAL;
  ctx->leaf_ctas_per_sm = t->leaf_ctas_per_sm;
  ctx->leaf_smem_points = t->leaf_smem_points;
  ctx->leaf_threads = t->leaf_threads;
  return DENOISE_OK;
}

// Host or device input of an evaluation call: device pointers pass through,
// host arrays are copied into `stage` (context scratch) first.
static const float *stage_points(const float *p, size_t n, int device, float *stage, cudaStream_t st, int *rc) {
  const Loc l = locate(p, device);
  if (l == Loc::kOtherDevice) {
    *rc = DENOISE_E_INVAL;
    return nullptr;
  }
  if (l == Loc::kDevice) return p;
  if (cudaMemcpyAsync(stage, p, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st) != cudaSuccess) *rc = cuda_fail();
  return stage;
}

int denoise_eval_metrics(denoise_ctx *ctx, const float *clean, size_t n_clean, const float *denoised,
                         size_t n_denoised, double *metrics, float *nn_clean, float *nn_denoised, void *stream) {
  if (!ctx || !clean || !denoised || !metrics || n_clean == 0 || n_denoised == 0) return DENOISE_E_INVAL;
  if (n_clean > ctx->max_points || n_denoised > ctx->max_points) return DENOISE_E_CAPACITY;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t na = (uint32_t)n_clean, nb = (uint32_t)n_denoised;
  // context scratch: the spill area holds the passes' arrays and any host staging
  const size_t need = ev_scratch_bytes(na, nb);
  const size_t stage_a = (need + 255) & ~size_t(255), stage_b = stage_a + ((12ull * na + 255) & ~size_t(255));
  const size_t total = stage_b + 12ull * nb;
  if (total > ctx->max_points * (size_t)ctx->big_bpp) return DENOISE_E_CAPACITY;
  int rc = DENOISE_OK;
  const float *a = stage_points(clean, na, ctx->device, (float *)(ctx->d_big + stage_a), st, &rc);
  const float *b = rc ? nullptr : stage_points(denoised, nb, ctx->device, (float *)(ctx->d_big + stage_b), st, &rc);
  if (rc) return rc;
  const Loc la = nn_clean ? locate(nn_clean, ctx->device) : Loc::kDevice;
  const Loc lb = nn_denoised ? locate(nn_denoised, ctx->device) : Loc::kDevice;
  if (la == Loc::kOtherDevice || lb == Loc::kOtherDevice) return DENOISE_E_INVAL;
  EvalArgs e{};
  e.clean = a;
  e.denoised = b;
  e.na = na;
  e.nb = nb;
  e.nn_clean = nn_clean ? (la == Loc::kDevice ? nn_clean : ctx->d_score) : nullptr;
  e.nn_denoised = nn_denoised ? (lb == Loc::kDevice ? nn_denoised : (float *)ctx->d_gin) : nullptr;
  e.out = ctx->d_grad;
  e.scratch = ctx->d_big;
  e.ctr = ctx->d_ctr;
  e.spin_limit = ctx->wait_limit;
  if (cudaMemsetAsync(&ctx->d_ctr->status, 0, sizeof(uint32_t), st) != cudaSuccess) return cuda_fail();
  if (launch_eval_metrics(e, ctx->num_sms, st)) return cuda_fail();
  if (nn_clean && la == Loc::kHost) cudaMemcpyAsync(nn_clean, e.nn_clean, 4ull * na, cudaMemcpyDeviceToHost, st);
  if (nn_denoised && lb == Loc::kHost)
    cudaMemcpyAsync(nn_denoised, e.nn_denoised, 4ull * nb, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(ctx->h_grad, ctx->d_grad, sizeof(double) * 3, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&ctx->h_ctr->status, &ctx->d_ctr->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail();
  const int s2 = map_status(ctx->h_ctr->status);
  if (s2) return s2;
  for (int i = 0; i < 3; ++i) metrics[i] = ctx->h_grad[i];
  return DENOISE_OK;
}

int denoise_run_baseline(denoise_ctx *ctx, const float *xyz, size_t n, double G, double alpha, uint8_t *mask,
                         uint32_t *n_i, double *params, void *stream) {
  if (!ctx || !xyz || !mask || n == 0 || !(G > 0.0) || !isfinite(G) || !(alpha > 0.0) || !isfinite(alpha))
    return DENOISE_E_INVAL;
  if (n > ctx->max_points) return DENOISE_E_CAPACITY;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t nn = (uint32_t)n;
  const size_t need = ev_scratch_bytes(nn, 0);
  const size_t stage = (need + 255) & ~size_t(255);
  if (stage + 12ull * nn > ctx->max_points * (size_t)ctx->big_bpp) return DENOISE_E_CAPACITY;
  int rc = DENOISE_OK;
  const float *x = stage_points(xyz, nn, ctx->device, (float *)(ctx->d_big + stage), st, &rc);
  if (rc) return rc;
  const Loc lm = locate(mask, ctx->device), ln = n_i ? locate(n_i, ctx->device) : Loc::kDevice;
  if (lm == Loc::kOtherDevice || ln == Loc::kOtherDevice) return DENOISE_E_INVAL;
  BaselineArgs b{};
  b.xyz = x;
  b.n = nn;
  b.G = G;
  b.alpha = alpha;
  b.keep = lm == Loc::kDevice ? mask : ctx->d_mask;
  b.n_i = n_i ? (ln == Loc::kDevice ? n_i : (uint32_t *)ctx->d_gin) : nullptr;
  b.params_out = ctx->d_partials;
  b.scratch = ctx->d_big;
  b.ctr = ctx->d_ctr;
  b.spin_limit = ctx->wait_limit;
  if (cudaMemsetAsync(&ctx->d_ctr->status, 0, sizeof(uint32_t), st) != cudaSuccess) return cuda_fail();
  if (launch_baseline(b, ctx->num_sms, st)) return cuda_fail();
  if (lm == Loc::kHost) cudaMemcpyAsync(mask, b.keep, nn, cudaMemcpyDeviceToHost, st);
  if (n_i && ln == Loc::kHost) cudaMemcpyAsync(n_i, b.n_i, 4ull * nn, cudaMemcpyDeviceToHost, st);
  double hp[5] = {0, 0, 0, 0, 0};
  if (params) cudaMemcpyAsync(hp, ctx->d_partials, sizeof(hp), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&ctx->h_ctr->status, &ctx->d_ctr->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail();
  const int s2 = map_status(ctx->h_ctr->status);
  if (s2) return s2;
  if (params)
    for (int i = 0; i < 5; ++i) params[i] = hp[i];
  return DENOISE_OK;
}

int denoise_set_wait_limit(denoise_ctx *ctx, uint32_t iterations) {
  if (!ctx) return DENOISE_E_INVAL;
  ctx->wait_limit = iterations;
  return DENOISE_OK;
}

int denoise_test_hold_lookback(denoise_ctx *ctx, int32_t tile) {
  if (!ctx || tile < -1) return DENOISE_E_INVAL;
  ctx->hold_tile1 = (uint32_t)(tile + 1);
  return DENOISE_OK;
}

int denoise_get_status(denoise_ctx *ctx, void *stream) {
  if (!ctx) return DENOISE_E_INVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DENOISE_E_CUDA;
  return map_status(ctx->h_ctr->status);
}

int denoise_get_stats(denoise_ctx *ctx, denoise_stats *out) {
  if (!ctx || !out) return DENOISE_E_INVAL;
  memset(out, 0, sizeof(*out));
  out->n_points = ctx->last_n;
  out->n_leaves = ctx->h_ctr->n_leaves;
  out->knn_pairs = ctx->h_ctr->knn_pairs;
  out->n_p1 = ctx->h_ctr->n_p1;
  out->n_p2 = ctx->h_ctr->n_p2;
  out->score_terms = ctx->h_ctr->score_terms;
  out->launches = (uint32_t)ctx->last_launches;
  out->n_stages = (uint32_t)ctx->n_stage_ms;
  for (int i = 0; i < ctx->n_stage_ms && i < 8; ++i) out->stage_ms[i] = ctx->stage_ms[i];
  return DENOISE_OK;
}

int denoise_set_training(denoise_ctx *ctx, int enable) {
  if (!ctx) return DENOISE_E_INVAL;
  if (enable && !ctx->train_alloc) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
    const size_t N = ctx->max_points;
    int e = 0;
    e |= dalloc(&ctx->train.nbr, N * 64);
    e |= dalloc(&ctx->train.nd2, N * 64);
    e |= dalloc(&ctx->train.ell, N);
    e |= dalloc(&ctx->train.r2, N);
    e |= dalloc(&ctx->train.F, N);
    e |= dalloc(&ctx->train.stage, N);
    if (e) {
      cudaGetLastError();
      return DENOISE_E_NOMEM;
    }
    ctx->train_alloc = true;
  }
  ctx->training = enable ? 1 : 0;
  return DENOISE_OK;
}

int denoise_set_cross_leaf(denoise_ctx *ctx, int enable) {
  if (!ctx) return DENOISE_E_INVAL;
  if (enable && !ctx->x_nbr) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
    const size_t N = ctx->max_points;
    int e = 0;
    e |= dalloc(&ctx->x_nbr, N * 64);
    e |= dalloc(&ctx->x_r2, N);
    e |= dalloc(&ctx->x_keff, N);
    e |= dalloc(&ctx->x_flag, N);
    if (e) {
      void *ps[] = {ctx->x_nbr, ctx->x_r2, ctx->x_keff, ctx->x_flag};
      for (void *q : ps)
        if (q) cudaFree(q);
      ctx->x_nbr = nullptr;
      ctx->x_r2 = nullptr;
      ctx->x_keff = nullptr;
      ctx->x_flag = nullptr;
      cudaGetLastError();
      return DENOISE_E_NOMEM;
    }
  }
  return DENOISE_OK;
}

int denoise_soft_removal(denoise_ctx *ctx, float *removal, void *stream) {
  if (!ctx || !removal) return DENOISE_E_INVAL;
  if (!ctx->last_trained) return DENOISE_E_STATE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const Loc lr = locate(removal, ctx->device);
  if (lr == Loc::kOtherDevice) return DENOISE_E_INVAL;
  const bool dev = lr == Loc::kDevice;
  BackArgs a{};
  a.train = ctx->train;
  a.train.k = ctx->last_p.k;
  a.n = (uint32_t)ctx->last_n;
  a.p = ctx->last_p;
  a.removal = dev ? removal : ctx->d_score;
  if (a.n == 0) return DENOISE_OK;
  if (launch_soft_removal(a, st)) return DENOISE_E_CUDA;
  if (!dev) {
    cudaMemcpyAsync(removal, ctx->d_score, sizeof(float) * a.n, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return DENOISE_E_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? DENOISE_OK : DENOISE_E_CUDA;
}

int denoise_backward(denoise_ctx *ctx, const float *grad_removal, double *grad4, void *stream) {
  if (!ctx || !grad_removal || !grad4) return DENOISE_E_INVAL;
  if (!ctx->last_trained) return DENOISE_E_STATE;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DENOISE_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  BackArgs a{};
  a.train = ctx->train;
  a.train.k = ctx->last_p.k;
  a.n = (uint32_t)ctx->last_n;
  a.p = ctx->last_p;
  if (a.n == 0) {
    for (int i = 0; i < 4; ++i) grad4[i] = 0.0;
    return DENOISE_OK;
  }
  const float *g = grad_removal;
  const Loc lgr = locate(grad_removal, ctx->device);
  if (lgr == Loc::kOtherDevice) return DENOISE_E_INVAL;
  if (lgr == Loc::kHost) {
    cudaMemcpyAsync(ctx->d_gin, grad_removal, sizeof(float) * a.n, cudaMemcpyHostToDevice, st);
    g = ctx->d_gin;
  }
  a.grad_r = g;
  a.partials = ctx->d_partials;
  a.grad4 = ctx->d_grad;
  int launches = 0;
  if (launch_backward(a, st, &launches)) return DENOISE_E_CUDA;
  cudaMemcpyAsync(ctx->h_grad, ctx->d_grad, sizeof(double) * 4, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return DENOISE_E_CUDA;
  for (int i = 0; i < 4; ++i) grad4[i] = ctx->h_grad[i];
  return DENOISE_OK;
}

}  // extern "C"
