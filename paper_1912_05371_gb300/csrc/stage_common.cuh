// Device helpers shared by the fused stage kernels (stage.cu: one point per thread, any
// precision; stage_pair.cu: two points per thread, FP32 with packed arithmetic).
#pragma once

#include <atomic>

#include "common.cuh"
#include "kernels.hpp"

namespace acm {
namespace {

// Opt `kernel` in to `bytes` of dynamic shared memory (above the default 48 KB) on the current
// device, once per device (the attribute belongs to the device's context).
template <typename K>
void smem_opt_in_stage(K kernel, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_relaxed) & bit) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done.fetch_or(bit);
}

// faces: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z ; box index of the face neighbour
__constant__ int kFaceBox[6] = {12, 14, 10, 16, 4, 22};

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(T) == 4) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  }
}
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Packed FP32x2 operations, round to nearest.  a - b is fma(b, -1, a): b * -1 is exact, so it
// rounds once, like a subtraction.
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
// Bulk prefetch of a contiguous range into L2 (address and size multiples of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// mbarrier-tracked bulk copies (the Blackwell TMA engine's 1D form): one thread announces the
// bytes a phase expects and issues the copies; every thread waits for the phase.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// makes the initialised barriers visible to the copy engine (before the CTA-wide barrier)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// orders this thread's earlier shared-memory accesses (and those the CTA barrier published)
// before later bulk copies into the same memory
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy of `bytes` (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// Waits for the phase of the given parity; gives up after a bounded number of polls (each poll
// may suspend the thread for a while), sets err |= 1 (a bounded wait expired) and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  unsigned done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  if (!done && err) atomicOr(err, 1);
  return done != 0;
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Address of one halo value: face F, distance l = 1..3 from the face plane, tangential
// coordinates (t0, t1) = (y, z) for x-faces, (x, z) for y-faces, (x, y) for z-faces.
template <typename T, int BS>
__device__ __forceinline__ const T* halo_ptr(const int (&ftype)[6], const int (&fs)[6][4],
                                             const T* __restrict__ in, const T* __restrict__ slab,
                                             int F, int l, int t0, int t1, int f) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int ax = F >> 1;
  const bool plus = F & 1;
  const int ty = ftype[F];
  int s, nl, u0 = t0, u1 = t1;
  if (ty == kTypeLeaf) {
    s = fs[F][0];
    nl = plus ? l : M - l;
  } else if (ty == kTypeRefined) {
    const int c0 = t0 > M / 2, c1 = t1 > M / 2;
    s = fs[F][c0 + 2 * c1];
    nl = plus ? 2 * l : M - 2 * l;
    u0 = 2 * t0 - c0 * M;
    u1 = 2 * t1 - c1 * M;
  } else {
    return slab + ((((size_t)fs[F][0] * 4 + f) * 3 + (l - 1)) * BS + t1) * BS + t0;
  }
  int x, y, z;
  if (ax == 0) { x = nl; y = u0; z = u1; }
  else if (ax == 1) { x = u0; y = nl; z = u1; }
  else { x = u0; y = u1; z = nl; }
  return in + (size_t)s * L::BLK + (size_t)f * L::FS + L::idx(x, y, z);
}


// Face table of one block: for each face F (0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z) the type of the
// neighbour across it (leaf, refined: the four children touching the face, or coarser: the halo
// slab the coarse-face kernel predicted) and the slots / slab index in fs[F][0..3].  Threads
// 0..23 fill it; the caller synchronises.
__device__ __forceinline__ void stage_faces(int tid, const int* __restrict__ nbh, const int32_t* __restrict__ slabidx,
                                            int rank, int (&ftype)[6], int (&fs)[6][4]) {
  if (tid < 24) {
    const int F = tid >> 2, j = tid & 3;
    const int c0 = j & 1, c1 = j >> 1;
    const int d = kFaceBox[F];
    int ty = nbh[kNbhType + d] & 15;
    int s;
    if (ty == kTypeLeaf) {
      s = nbh[8 * d];
    } else if (ty == kTypeRefined) {
      const int nbit = (F & 1) ? 0 : 1;
      const int ax = F >> 1;
      int c;
      if (ax == 0) c = nbit | (c0 << 1) | (c1 << 2);
      else if (ax == 1) c = c0 | (nbit << 1) | (c1 << 2);
      else c = c0 | (c1 << 1) | (nbit << 2);
      s = nbh[8 * d + c];
    } else {
      ty = kTypeCoarser;                 // halo slab predicted by the coarse-face kernel
      s = slabidx[(size_t)rank * 8 + F];
    }
    fs[F][j] = s;
    if (j == 0) ftype[F] = ty;
  }
}

// Sponge profile of one block along each axis (Sec. 2.2, sponge terms; the profile's reading is
// the tanh of the distance to the nearest box face minus L_sp), in the field precision: threads
// 0..3 Bs - 1 fill sp[axis][i]; the caller synchronises.
template <typename T, int BS>
__device__ __forceinline__ void stage_sponge(int tid, const PhysK& ph, int4 bi, T (&sp)[3][BS]) {
  constexpr int M = BS - 1;
  if (ph.sponge && tid < 3 * BS) {
    const double h = ph.h[bi.x];
    const int ax = tid / BS, i = tid % BS;
    const int g = ax == 0 ? bi.y : (ax == 1 ? bi.z : bi.w);
    const long long N = ((long long)ph.nroot[ax] << bi.x) * M;
    long long gi = (long long)g * M + i;        // in [0, N]; the seam x = L is taken as 0
    if (gi >= N) gi -= N;
    const double c = (double)gi * h;
    // the profile in the field precision (FP32 fields keep tanh off the FP64 pipe)
    const T dist = T(fmin(c, ph.sp_L[ax] - c));
    sp[ax][i] = T(0.5) * (T(1) - ttanh((dist - T(ph.sp_width)) / T(ph.sp_delta)));
  }
}

}  // namespace
}  // namespace acm
