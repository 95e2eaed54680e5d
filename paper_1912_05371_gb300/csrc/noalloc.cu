// Allocation-free variant of the max-norm reduction (entry point acm_max_norms_noalloc).
//
// Scratch memory for the per-block partial maxima is a file-scope __device__ array, so the
// entry point never allocates.  Host code must not pass the array's name to a kernel (on the
// host it names a shadow object, not device memory): its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first call made there.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/acm.h"

namespace {

constexpr int kNT = 256;
constexpr int kMaxDevices = 64;

// [block][5]: max |u|, |v|, |w|, |p|, |(u,v,w)| of each block.  Every call writes the entries
// of all its blocks before reading them back, so nothing needs clearing between calls.
static __device__ __align__(256) double g_block_max[ACM_NOALLOC_MAX_BLOCKS * 5];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

template <typename T>
__device__ __forceinline__ T absval(T v) { return v < T(0) ? -v : v; }
__device__ __forceinline__ float root(float v) { return sqrtf(v); }
__device__ __forceinline__ double root(double v) { return sqrt(v); }

// One CTA per block of the dense block-order array (component-major, then z, y, x).
template <typename T>
__global__ void __launch_bounds__(kNT) k_block_max(const T* __restrict__ fields, int Bs, double* partials) {
  const int n3 = Bs * Bs * Bs;
  const T* b = fields + (size_t)blockIdx.x * 4 * n3;
  T m[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int i = threadIdx.x; i < n3; i += kNT) {
    T v[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      v[f] = b[(size_t)f * n3 + i];
      const T a = absval(v[f]);
      m[f] = a > m[f] ? a : m[f];
    }
    const T mag = root(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    m[4] = mag > m[4] ? mag : m[4];
  }
  __shared__ double red[5][kNT / 32];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double mk = (double)m[k];
    for (int o = 16; o > 0; o >>= 1) mk = fmax(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = mk;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double mk = 0.0;
    for (int w = 0; w < kNT / 32; ++w) mk = fmax(mk, red[threadIdx.x][w]);
    partials[(size_t)blockIdx.x * 5 + threadIdx.x] = mk;
  }
}

__global__ void __launch_bounds__(1024) k_final_max(const double* partials, int n, double* out) {
  __shared__ double red[5][32];
  double m[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < n; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k] = fmax(m[k], partials[(size_t)b * 5 + k]);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    for (int o = 16; o > 0; o >>= 1) m[k] = fmax(m[k], __shfl_xor_sync(0xffffffffu, m[k], o));
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = m[k];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double mk = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mk = fmax(mk, red[threadIdx.x][w]);
    out[threadIdx.x] = mk;
  }
}

}  // namespace

extern "C" acm_status acm_max_norms_noalloc(const void* fields, int64_t n_blocks, int Bs, int precision,
                                            double* norms_out, void* stream) {
  if (!fields || !norms_out || n_blocks < 1) return ACM_EINVAL;
  if (Bs != 9 && Bs != 17) return ACM_EINVAL;
  if (precision != 32 && precision != 64) return ACM_EINVAL;
  if (n_blocks > ACM_NOALLOC_MAX_BLOCKS) return ACM_ECAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ACM_ECUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_block_max) != cudaSuccess || !p) return ACM_ECUDA;
      g_scratch[dev] = p;
    }
    scratch = g_scratch[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* partials = static_cast<double*>(scratch);
  if (precision == 64)
    k_block_max<double><<<(unsigned)n_blocks, kNT, 0, st>>>(static_cast<const double*>(fields), Bs, partials);
  else
    k_block_max<float><<<(unsigned)n_blocks, kNT, 0, st>>>(static_cast<const float*>(fields), Bs, partials);
  k_final_max<<<1, 1024, 0, st>>>(partials, (int)n_blocks, norms_out);
  return cudaGetLastError() == cudaSuccess ? ACM_OK : ACM_ECUDA;
}
