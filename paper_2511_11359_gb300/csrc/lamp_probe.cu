// Measurement helper: the sustained MUFU ex2 rate of this GPU, in ex2 results
// per SM per clock, from a kernel that issues nothing but dependent chains of
// ex2.approx.ftz.f32 (eight independent chains per thread, all SMs busy) and
// reads each SM's cycle counter around its loop.  The rate is the denominator
// of the roofline of the tensor-core sweeps, whose epilogue needs two ex2 per
// cost entry.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/lamp.h"
#include "lamp_common.cuh"

namespace {

constexpr int kChains = 8;

__global__ void k_ex2_rate(int iters, float seed, float* sink, long long* cycles) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = seed * (0.25f + 0.01f * c) + 0.001f * threadIdx.x;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float y;
      // y = 2^(-v): stays in (0, 1) and keeps each chain dependent
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-v[c]));
      v[c] = y;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == 12345.0f) sink[0] = s;  // keeps the chains live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" int lamp_measure_ex2_rate(double* ex2_per_clk_per_sm) {
  if (!ex2_per_clk_per_sm) return LAMP_E_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LAMP_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LAMP_E_CUDA;
  const int threads = 512, blocks = sms * 4, iters = 4096;
  float* sink = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return LAMP_E_NOMEM;
  if (cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess) {
    cudaFree(sink);
    return LAMP_E_NOMEM;
  }
  k_ex2_rate<<<blocks, threads>>>(64, 0.5f, sink, cyc);  // warm-up
  k_ex2_rate<<<blocks, threads>>>(iters, 0.5f, sink, cyc);
  std::vector<long long> h(blocks);
  cudaError_t e = cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) return LAMP_E_CUDA;
  // 4 resident blocks per SM run concurrently: each SM executes 4 * threads * iters * chains ex2
  // in (about) the longest of its blocks' cycle counts
  long long mx = 0;
  for (long long c : h) mx = c > mx ? c : mx;
  const double per_sm = 4.0 * threads * (double)iters * kChains;
  *ex2_per_clk_per_sm = per_sm / (double)mx;
  return LAMP_OK;
}
