// gd_backward.cu -- differentiable form of the score selection.
//
// Soft removal probability of a scored point (Eq. 21 score F_i, threshold tau,
// temperature T):  r_i = 1 - sigmoid((ln F_i - tau) / T); points removed by the
// voxel or density gate have r_i = 1 (constant).  The backward pass takes
// dL/dr_i and returns dL/d(alpha, sigma, gamma, tau) with the neighbour sets,
// gates and densities held fixed: none of them depends on these parameters.
//
// Per neighbour term t_ij = W^(alpha/2) exp(-d^2/(2 sigma^2 r_K^2)) / ((d^2)^(gamma/2) + eps_k):
//   dt/dalpha = t * ln(W)/2,  dt/dsigma = t * d^2 / (sigma^3 r_K^2),
//   dt/dgamma = -t * (d^2)^(gamma/2) * ln(d^2) / 2 / ((d^2)^(gamma/2) + eps_k)   (0 at d^2 = 0),
//   dr/dF = -m(1-m)/(T F),  dr/dtau = m(1-m)/T,  m = sigmoid((ln F - tau)/T).
// Terms are evaluated in FP32, sums in FP64; the grid reduction is a fixed
// two-level tree, so the result does not depend on scheduling.
#include "gd_common.cuh"

namespace gd {

constexpr int kBackThreads = 256;
constexpr int kBackBlocks = 1024;

__device__ __forceinline__ bool scored(uint8_t st) { return st == 0 || st == 3; }

__global__ void k_soft_removal(const BackArgs a) {
  const float T = a.p.temperature, tau = a.p.tau;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += gridDim.x * blockDim.x) {
    float r = 1.0f;
    const float F = a.train.F[g];
    if (scored(a.train.stage[g]) && F > 0.0f) {
      const float z = (logf(F) - tau) / T;
      r = 1.0f - 1.0f / (1.0f + expf(-z));
    }
    a.removal[g] = r;
  }
}

__global__ void __launch_bounds__(kBackThreads) k_backward(const BackArgs a) {
  __shared__ double red[kBackThreads / 32][4];
  const float T = a.p.temperature, tau = a.p.tau;
  const float alpha = a.p.alpha, sigma = a.p.sigma, gamma = a.p.gamma, ek = a.p.eps_k;
  const float c2 = 1.4426950408889634f / (2.0f * sigma * sigma);
  const float ln2 = 0.6931471805599453f;
  const uint32_t k = a.train.k;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n; g += gridDim.x * blockDim.x) {
    const float F = a.train.F[g];
    const float u = a.grad_r[g];
    if (!scored(a.train.stage[g]) || !(F > 0.0f) || u == 0.0f) continue;
    const float z = (logf(F) - tau) / T;
    const float m = 1.0f / (1.0f + expf(-z));
    const double dm = (double)m * (1.0 - (double)m) / (double)T;
    const float r2i = a.train.r2[g];
    const float elli = a.train.ell[g];
    const float ci = c2 / r2i;
    double dA = 0.0, dS = 0.0, dG = 0.0;
    for (uint32_t t = 0; t < k; ++t) {
      const uint32_t j = a.train.nbr[(size_t)g * k + t];
      if (j == 0xFFFFFFFFu) break;
      const float d2 = a.train.nd2[(size_t)g * k + t];
      const float lw2 = elli + a.train.ell[j];           // log2 W_ij
      const float D = (gamma == 2.0f) ? d2 : exp2f(0.5f * gamma * log2f(d2));
      const float tt = exp2f(0.5f * alpha * lw2 - d2 * ci) / (D + ek);
      dA += (double)tt * 0.5 * (double)(lw2 * ln2);
      dS += (double)tt * (double)d2 / ((double)sigma * sigma * sigma * r2i);
      if (d2 > 0.0f) dG -= (double)tt * (double)D * 0.5 * (double)logf(d2) / ((double)D + ek);
    }
    const double dr_dF = -dm / (double)F;
    acc[0] += (double)u * dr_dF * dA;
    acc[1] += (double)u * dr_dF * dS;
    acc[2] += (double)u * dr_dF * dG;
    acc[3] += (double)u * dm;
  }
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = acc[q];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int ww = 0; ww < kBackThreads / 32; ++ww) s += red[ww][threadIdx.x];
    a.partials[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

__global__ void k_backward_final(const double *__restrict__ partials, uint32_t blocks, double *grad4) {
  __shared__ double red[32][4];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t b = threadIdx.x; b < blocks; b += blockDim.x)
    for (int q = 0; q < 4; ++q) acc[q] += partials[(size_t)b * 4 + q];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    double v = acc[q];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[w][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (uint32_t ww = 0; ww < blockDim.x / 32; ++ww) s += red[ww][threadIdx.x];
    grad4[threadIdx.x] = s;
  }
}

int launch_soft_removal(const BackArgs &a, cudaStream_t st) {
  uint32_t blocks = (a.n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks == 0) blocks = 1;
  k_soft_removal<<<blocks, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_backward(const BackArgs &a, cudaStream_t st, int *launches) {
  k_backward<<<kBackBlocks, kBackThreads, 0, st>>>(a);
  k_backward_final<<<1, 256, 0, st>>>(a.partials, kBackBlocks, a.grad4);
  if (launches) *launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace gd
