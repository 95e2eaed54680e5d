// Arithmetic peak of this GPU measured by a kernel of the library's own (acm_fma_rate): the
// roofline denominator of the FP64 stage kernel, which on GB300 is bound by the FP64 pipe rather
// than by HBM.  No counterpart in the paper.
//
// Every thread runs kChains independent chains of kIters dependent fused multiply-adds x = x a + b
// (a just below 1, so the values stay finite); the grid covers every SM several times over.
// flops = 2 x threads x kChains x kIters over the CUDA-event time of the launch (median of
// several launches after a warm-up).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/acm.h"
#include "kernels.hpp"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T a, T b, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot drop; it never executes for these inputs (s stays finite)
  if (s == T(-1)) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" acm_status acm_fma_rate(int precision, double* flops_out, void* stream) {
  if (!flops_out || (precision != 32 && precision != 64)) return ACM_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = acm::sm_count() * 8;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return ACM_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ACM_ECUDA;
  }
  std::vector<float> ms;
  acm_status s = ACM_OK;
  for (int r = 0; r < 6 && s == ACM_OK; ++r) {
    cudaEventRecord(e0, st);
    if (precision == 64)
      k_fma_chains<double><<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, nullptr);
    else
      k_fma_chains<float><<<blocks, kThreads, 0, st>>>(0.9999f, 1e-4f, nullptr);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      s = ACM_ECUDA;
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (r > 0) ms.push_back(t);                 // the first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != ACM_OK) return s;
  std::sort(ms.begin(), ms.end());
  const double sec = ms[ms.size() / 2] * 1e-3;
  *flops_out = 2.0 * blocks * kThreads * (double)kChains * kIters / sec;
  return ACM_OK;
}
