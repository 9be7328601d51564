// gd_noalloc.cu -- denoise_run_noalloc: the path of denoise_run for one cloud of
// at most DENOISE_NOALLOC_MAX_POINTS points, with every scratch buffer carved
// out of one file-scope device array instead of context allocations.
//
// For callers that cannot allocate device memory (a host framework that owns
// all allocations, a loop whose policy forbids cudaMalloc): nothing here calls
// cudaMalloc, cudaFree, cudaMallocHost or any allocating library routine.  The
// array is shared by all calls and keeps the last call's contents; k_init of
// the front end clears the counters, histograms and look-back flags each call,
// and k_noalloc_tables rewrites the frame and tile tables.  Overlapping calls
// race on the array.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "gd_common.cuh"

using namespace gd;

namespace {

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kN = DENOISE_NOALLOC_MAX_POINTS;
constexpr size_t kTiles = (kN + kTilePts - 1) / kTilePts;
constexpr uint32_t kSpillBpp = 320;  // leaf_big_bpp(64): checked against the library at first use
// carve of the scratch array
constexpr size_t kOffKeys0 = 0;
constexpr size_t kOffKeys1 = kOffKeys0 + al256(8 * kN);
constexpr size_t kOffVals0 = kOffKeys1 + al256(8 * kN);
constexpr size_t kOffVals1 = kOffVals0 + al256(4 * kN);
constexpr size_t kOffSpts = kOffVals1 + al256(4 * kN);
constexpr size_t kOffLeaves = kOffSpts + al256(16 * kN);
constexpr size_t kOffOrder = kOffLeaves + al256(sizeof(Leaf) * kN);
constexpr size_t kOffFrames = kOffOrder + al256(4 * kN);
constexpr size_t kOffTiles = kOffFrames + al256(sizeof(FrameInfo));
constexpr size_t kOffHist = kOffTiles + al256(sizeof(Tile) * kTiles);
constexpr size_t kOffBase = kOffHist + al256(4 * kMaxPasses * 256);
constexpr size_t kOffLookback = kOffBase + al256(4 * kMaxPasses * 256);
constexpr size_t kOffCtr = kOffLookback + al256(4 * kMaxPasses * kTiles * 256);
constexpr size_t kOffSpill = kOffCtr + al256(sizeof(Counters));
constexpr size_t kScratchBytes = kOffSpill + al256((size_t)kSpillBpp * kN);

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  size_t smem_optin = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// device memory the kernels on `dev` can read: managed memory, or device memory
// of that GPU (not of another GPU, which would need peer access)
bool dev_ptr(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

int params_ok(const denoise_params *p) {
  if (!p || p->k == 0 || p->k > 64 || p->leaf_capacity == 0 || p->max_depth > 21) return 0;
  if (!(p->beta > 0.0f) || !isfinite(p->beta)) return 0;
  if (!(p->rho_percentile >= 0.0f && p->rho_percentile <= 100.0f)) return 0;
  if (!(p->lambda > 0.0f && p->lambda <= 1.0f)) return 0;
  if (!(p->gamma > 0.0f) || !isfinite(p->gamma) || !(p->sigma > 0.0f) || !isfinite(p->sigma)) return 0;
  if (!isfinite(p->alpha) || !(p->eps_rho >= 0.0f) || !(p->eps_k >= 0.0f)) return 0;
  if (!isfinite(p->eps_rho) || !isfinite(p->eps_k) || !isfinite(p->tau)) return 0;
  if (p->select_mode > 1 || !(p->temperature > 0.0f) || !isfinite(p->temperature)) return 0;
  if (p->stage_off > 7u || p->rescore_p2 > 1u || p->cross_leaf) return 0;  // (no cross-leaf tables here)
  return 1;
}

int fail_cuda() {
  cudaGetLastError();
  return DENOISE_E_CUDA;
}

}  // namespace

// The scratch: one array per GPU that loads the library, alive until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// one frame [0, n) and its tiles, written on the device (no host staging memory)
__global__ void k_noalloc_tables(FrameInfo *frames, Tile *tiles, uint32_t n) {
  const uint32_t t = threadIdx.x;
  if (t == 0) {
    FrameInfo f{};
    f.begin = 0;
    f.end = n;
    frames[0] = f;
  }
  const uint32_t ntiles = (n + kTilePts - 1) / kTilePts;
  for (uint32_t i = t; i < ntiles; i += blockDim.x) {
    const uint32_t b = i * (uint32_t)kTilePts;
    tiles[i] = Tile{0u, b, (n - b > (uint32_t)kTilePts) ? b + (uint32_t)kTilePts : n, 0u};
  }
}

extern "C" size_t denoise_noalloc_scratch_bytes(void) {
  return leaf_big_bpp(64) <= kSpillBpp ? kScratchBytes : 0;
}

extern "C" int denoise_run_noalloc(const float *xyz, size_t n, const denoise_params *p, uint8_t *mask, float *score,
                                   uint8_t *stage, void *stream) {
  if (!params_ok(p)) return DENOISE_E_INVAL;
  if (n > kN) return DENOISE_E_CAPACITY;
  if (n == 0) return DENOISE_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail_cuda();
  if (dev < 0 || dev >= kMaxDevices) return DENOISE_E_INVAL;
  if (!xyz || !dev_ptr(xyz, dev)) return DENOISE_E_INVAL;
  if ((mask && !dev_ptr(mask, dev)) || (score && !dev_ptr(score, dev)) || (stage && !dev_ptr(stage, dev)))
    return DENOISE_E_INVAL;
  if (leaf_big_bpp(64) > kSpillBpp) return DENOISE_E_INVAL;  // carve no longer covers the spill stride
  {
    // the call reads the device status back, which a capturing stream cannot do
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) return fail_cuda();
    if (cs != cudaStreamCaptureStatusNone) return DENOISE_E_INVAL;
  }
  DeviceSetup su;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_setup[dev].ready) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return fail_cuda();
      int sms = 0, optin = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return fail_cuda();
      g_setup[dev].base = (unsigned char *)ptr;
      g_setup[dev].num_sms = sms;
      g_setup[dev].smem_optin = (size_t)optin;
      g_setup[dev].ready = true;
    }
    su = g_setup[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *b = su.base;
  const uint32_t nn = (uint32_t)n;
  const uint32_t ntiles = (nn + kTilePts - 1) / kTilePts;
  FrameInfo *frames = (FrameInfo *)(b + kOffFrames);
  Tile *tiles = (Tile *)(b + kOffTiles);
  Counters *ctr = (Counters *)(b + kOffCtr);
  k_noalloc_tables<<<1, 32, 0, st>>>(frames, tiles, nn);

  FrontArgs fa{};
  fa.xyz = xyz;
  fa.n = nn;
  fa.frames = frames;
  fa.nframes = 1;
  fa.tiles = tiles;
  fa.ntiles = ntiles;
  fa.keys[0] = (unsigned long long *)(b + kOffKeys0);
  fa.keys[1] = (unsigned long long *)(b + kOffKeys1);
  fa.vals[0] = (uint32_t *)(b + kOffVals0);
  fa.vals[1] = (uint32_t *)(b + kOffVals1);
  fa.spts = (float4 *)(b + kOffSpts);
  fa.digit_hist = (uint32_t *)(b + kOffHist);
  fa.digit_base = (uint32_t *)(b + kOffBase);
  fa.lookback = (uint32_t *)(b + kOffLookback);
  fa.leaves = (Leaf *)(b + kOffLeaves);
  fa.ctr = ctr;
  fa.dbg_key = nullptr;
  fa.max_depth = (int)p->max_depth;
  fa.leaf_capacity = p->leaf_capacity;
  if (launch_front(fa, st, nullptr, nullptr, nullptr)) return fail_cuda();

  LeafArgs la{};
  la.n = nn;
  la.spts = fa.spts;
  la.leaves = fa.leaves;
  la.order = (uint32_t *)(b + kOffOrder);
  la.frames = frames;
  la.ctr = ctr;
  la.p = *p;
  la.mask = mask;
  la.score = score;
  la.stage = stage;
  la.big_scratch = b + kOffSpill;
  la.big_bpp = leaf_big_bpp(64);
  la.lmax = leaf_pick_lmax(p->leaf_capacity, leaf_kmax(p->k), su.smem_optin - 2048);
  if (launch_leaf_prep(la, su.num_sms, st, nullptr) || launch_leaf(la, su.num_sms, st, nullptr)) return fail_cuda();

  uint32_t status = 0;
  if (cudaMemcpyAsync(&status, &ctr->status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail_cuda();
  if (cudaStreamSynchronize(st) != cudaSuccess) return fail_cuda();
  if (status & kStNonFinite) return DENOISE_E_NONFINITE;
  if (status & kStTimeout) return DENOISE_E_TIMEOUT;
  if (status & kStInternal) return DENOISE_E_CUDA;
  return DENOISE_OK;
}
