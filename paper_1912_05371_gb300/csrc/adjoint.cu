// Discrete adjoint of the RK4 steps on a frozen grid (kernels in adjoint_kernels.cuh, one
// translation unit per precision and block size): the launchers of kernels.hpp, dispatching on
// the block size.
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace acm {
namespace adj {

template <typename T, int BS>
void stage(const AdjStageK<T>& a, const TopoK& t, const PhysK& ph, const MaskK& m, const FwTasks& fw, int* err,
           cudaStream_t st);
template <typename T, int BS>
void fw_T(T* r, const FwTasks& fw, const int32_t* blist, const int32_t* nbh, cudaStream_t st);
template <typename T, int BS>
void sum3(T* out, const T* x, const T* y, const T* z, const int32_t* blist, int64_t n, cudaStream_t st);
template <typename T, int BS>
void objective(const T* U, const T* chi, T* lam, T* gchi, const int32_t* blist, const int4* binfo,
               int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m, double* dtheta, cudaStream_t st);
template <typename T, int BS>
void theta(const T* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph, const MaskK& m,
           double* out, cudaStream_t st);
template <typename T, int BS>
void gather(const T* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st);
template <typename T, int BS>
void put(const double* dense, T* r, const int32_t* blist, int64_t n, cudaStream_t st);

}  // namespace adj

// Blocks of 33^3 are FP32 only (the forest refuses FP64 with them).
#define ACM_ADJ_BS(Bs, FN, ...)                                       \
  do {                                                                \
    if ((Bs) == 33) {                                                 \
      if constexpr (sizeof(T) == 4) adj::FN<T, 33>(__VA_ARGS__);      \
    } else if ((Bs) == 17) {                                          \
      adj::FN<T, 17>(__VA_ARGS__);                                    \
    } else {                                                          \
      adj::FN<T, 9>(__VA_ARGS__);                                     \
    }                                                                 \
  } while (0)

template <typename T>
void launch_adj_stage(int Bs, const AdjStageK<T>& a, const TopoK& t, const PhysK& ph, const MaskK& m,
                      const FwTasks& fw, int* err, cudaStream_t st) {
  if (t.n <= 0) return;
  ACM_ADJ_BS(Bs, stage, a, t, ph, m, fw, err, st);
}

template <typename T>
void launch_adj_fw_T(int Bs, T* r, const FwTasks& fw, const int32_t* blist, const int32_t* nbh, int64_t n,
                     cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, fw_T, r, fw, blist, nbh, st);
}

template <typename T>
void launch_adj_sum3(int Bs, T* out, const T* x, const T* y, const T* z, const int32_t* blist, int64_t n,
                     cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, sum3, out, x, y, z, blist, n, st);
}

template <typename T>
void launch_adj_objective(int Bs, const T* U, const T* chi, T* lam, T* gchi, const int32_t* blist,
                          const int4* binfo, int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m,
                          double* dtheta, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, objective, U, chi, lam, gchi, blist, binfo, n, ph, wN, wE, m, dtheta, st);
}

template <typename T>
void launch_adj_theta(int Bs, const T* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph,
                      const MaskK& m, double* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, theta, gchi, blist, binfo, n, ph, m, out, st);
}

template <typename T>
void launch_adj_gather(int Bs, const T* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, gather, r, dense, blist, n, st);
}

template <typename T>
void launch_adj_put(int Bs, const double* dense, T* r, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, put, dense, r, blist, n, st);
}

#define ACM_ADJ_INST(T)                                                                                        \
  template void launch_adj_stage<T>(int, const AdjStageK<T>&, const TopoK&, const PhysK&, const MaskK&,         \
                                    const FwTasks&, int*, cudaStream_t);                                      \
  template void launch_adj_fw_T<T>(int, T*, const FwTasks&, const int32_t*, const int32_t*, int64_t, cudaStream_t); \
  template void launch_adj_sum3<T>(int, T*, const T*, const T*, const T*, const int32_t*, int64_t, cudaStream_t); \
  template void launch_adj_objective<T>(int, const T*, const T*, T*, T*, const int32_t*, const int4*, int64_t,  \
                                        const PhysK&, double, double, const MaskK&, double*, cudaStream_t);  \
  template void launch_adj_theta<T>(int, const T*, const int32_t*, const int4*, int64_t, const PhysK&,         \
                                    const MaskK&, double*, cudaStream_t);                                     \
  template void launch_adj_gather<T>(int, const T*, double*, const int32_t*, int64_t, cudaStream_t);             \
  template void launch_adj_put<T>(int, const double*, T*, const int32_t*, int64_t, cudaStream_t);
ACM_ADJ_INST(float)
ACM_ADJ_INST(double)

}  // namespace acm
