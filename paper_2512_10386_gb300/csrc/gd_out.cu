// gd_out.cu -- a call's results written into the caller's pinned host buffers by
// the SMs: one kernel after the leaf stage stores mask, score, stage and the
// counters (the status word the host reads) through the buffers' mapped device
// addresses, 16 bytes a store where source and destination share their offset
// within 16 bytes.  It replaces one copy-engine transfer per buffer (each with
// its own setup latency) by a single launch that all SMs share.
#include <cuda_runtime.h>

#include "gd_common.cuh"

namespace gd {

constexpr int kOutThreads = 256;

__device__ __forceinline__ void out_copy(unsigned char *dst, const unsigned char *src, size_t nbytes, size_t gt,
                                         size_t gs) {
  const size_t head = (16u - ((uintptr_t)dst & 15u)) & 15u;  // bytes before dst is 16-byte aligned
  if (((((uintptr_t)dst) ^ ((uintptr_t)src)) & 15u) == 0 && nbytes >= head + 16u) {
    const size_t nv = (nbytes - head) >> 4;
    for (size_t i = gt; i < head; i += gs) dst[i] = src[i];
    const uint4 *s = reinterpret_cast<const uint4 *>(src + head);
    uint4 *d = reinterpret_cast<uint4 *>(dst + head);
    for (size_t i = gt; i < nv; i += gs) d[i] = s[i];
    for (size_t i = head + (nv << 4) + gt; i < nbytes; i += gs) dst[i] = src[i];
  } else {
    for (size_t i = gt; i < nbytes; i += gs) dst[i] = src[i];
  }
}

__global__ void __launch_bounds__(kOutThreads) k_out(const OutArgs a) {
  const size_t gt = (size_t)blockIdx.x * kOutThreads + threadIdx.x, gs = (size_t)gridDim.x * kOutThreads;
  if (a.mask_h) out_copy(a.mask_h, a.mask_d, a.n, gt, gs);
  if (a.score_h)
    out_copy(reinterpret_cast<unsigned char *>(a.score_h), reinterpret_cast<const unsigned char *>(a.score_d),
             sizeof(float) * (size_t)a.n, gt, gs);
  if (a.stage_h) out_copy(a.stage_h, a.stage_d, a.n, gt, gs);
  if (blockIdx.x == 0) {  // every kernel of the call is done: the counters are final
    const uint32_t *s = reinterpret_cast<const uint32_t *>(a.ctr_d);
    uint32_t *d = reinterpret_cast<uint32_t *>(a.ctr_h);
    for (uint32_t i = threadIdx.x; i < sizeof(Counters) / 4; i += kOutThreads) d[i] = s[i];
  }
}

int launch_out(const OutArgs &a, int num_sms, cudaStream_t st) {
  // an ordinary launch (no programmatic dependency): the call's stream may hold
  // an event wait (the small-leaf stream's join) right before it
  const bool any = a.mask_h || a.score_h || a.stage_h;  // else only the counters: one block
  k_out<<<any ? num_sms * 2 : 1, kOutThreads, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace gd
