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

// Maximum that keeps NaN: a comparison with NaN is false, so a plain maximum (or fmax) would
// drop it; with this one a non-finite state gives a non-finite norm, as in the forest's own
// reduction, and NaN wins over infinity once it is in m.
template <typename T>
__device__ __forceinline__ T keep_max(T a, T m) { return (a > m || a != a) ? a : m; }

// Squared velocity magnitude in the same rounding sequence as the forest's max norm (u*u, then
// fma(v, v, .), then fma(w, w, .)), so both give bitwise the same largest magnitude.
template <typename T>
__device__ __forceinline__ T speed2(T u, T v, T w) {
  T s = u * u;
  s = fma(v, v, s);
  return fma(w, w, s);
}

// One CTA per block of the dense block-order array (component-major, then z, y, x).
template <typename T>
__global__ void __launch_bounds__(kNT) k_block_max(const T* __restrict__ fields, int Bs, double* partials) {
  const int n3 = Bs * Bs * Bs;
  const T* b = fields + (size_t)blockIdx.x * 4 * n3;
  // m[4] holds the squared speed; its root is taken once per block, in the field precision
  T m[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int i = threadIdx.x; i < n3; i += kNT) {
    T v[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      v[f] = b[(size_t)f * n3 + i];
      m[f] = keep_max(absval(v[f]), m[f]);
    }
    m[4] = keep_max(speed2(v[0], v[1], v[2]), m[4]);
  }
  __shared__ T red[5][kNT / 32];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    T mk = m[k];
    for (int o = 16; o > 0; o >>= 1) mk = keep_max(__shfl_xor_sync(0xffffffffu, mk, o), mk);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = mk;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    T mk = T(0);
    for (int w = 0; w < kNT / 32; ++w) mk = keep_max(red[threadIdx.x][w], mk);
    // the root is monotone and correctly rounded: the root of the largest square is the
    // largest root
    partials[(size_t)blockIdx.x * 5 + threadIdx.x] = threadIdx.x == 4 ? (double)root(mk) : (double)mk;
  }
}

__global__ void __launch_bounds__(1024) k_final_max(const double* partials, int n, double* out) {
  __shared__ double red[5][32];
  double m[5] = {0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < n; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 5; ++k) m[k] = keep_max(partials[(size_t)b * 5 + k], m[k]);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    for (int o = 16; o > 0; o >>= 1) m[k] = keep_max(__shfl_xor_sync(0xffffffffu, m[k], o), m[k]);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = m[k];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double mk = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) mk = keep_max(red[threadIdx.x][w], mk);
    out[threadIdx.x] = mk;
  }
}

}  // namespace

extern "C" acm_status acm_max_norms_noalloc(const void* fields, int64_t n_blocks, int Bs, int precision,
                                            double* norms_out, void* stream) {
  if (!fields || !norms_out || n_blocks < 1) return ACM_EINVAL;
  if (Bs != 9 && Bs != 17 && Bs != 33) return ACM_EINVAL;
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
