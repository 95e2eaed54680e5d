// Discrete adjoint of the RK4 steps on a frozen grid (kernels in adjoint_kernels.cuh, one
// translation unit per precision and block size): the launchers of kernels.hpp, dispatching on
// the block size.
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.hpp"

namespace acm {
namespace adj {

template <typename T, int BS>
void jgt(const T* Y, const double* kap, const T* chi, double* gchi, double* wgt, double* nu, const int32_t* blist,
         const int4* binfo, const int32_t* nbh, const uint8_t* finer, int64_t n, const PhysK& ph, const MaskK& m,
         double* dtheta, int* err, cudaStream_t st);
template <typename T, int BS>
void fw_T(double* r, const int32_t* blist, const int32_t* nbh, const uint8_t* finer, int64_t n, cudaStream_t st);
template <typename T, int BS>
void lin(double* out, double a, const double* x, double b, const double* y, const int32_t* blist, int64_t n,
         cudaStream_t st);
template <typename T, int BS>
void objective(const T* U, const T* chi, double* lam, double* gchi, const int32_t* blist, const int4* binfo,
               int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m, double* dtheta, cudaStream_t st);
template <typename T, int BS>
void theta(const double* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph, const MaskK& m,
           double* out, cudaStream_t st);
template <typename T, int BS>
void gather(const double* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st);
template <typename T, int BS>
void put(const double* dense, double* r, const int32_t* blist, int64_t n, cudaStream_t st);

}  // namespace adj

#define ACM_ADJ_BS(Bs, FN, ...)            \
  do {                                     \
    if ((Bs) == 17) adj::FN<T, 17>(__VA_ARGS__); \
    else adj::FN<T, 9>(__VA_ARGS__);       \
  } while (0)

size_t adj_weight_doubles(int Bs, int64_t nblocks) {
  return (size_t)kAdjWeightsPerPoint * Bs * Bs * Bs * (size_t)nblocks;
}

template <typename T>
void launch_adj_jgt(int Bs, const T* Y, const double* kap, const T* chi, double* gchi, double* wgt, double* nu,
                    const int32_t* blist, const int4* binfo, const int32_t* nbh, const uint8_t* finer, int64_t n,
                    const PhysK& ph, const MaskK& m, double* dtheta, int* err, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, jgt, Y, kap, chi, gchi, wgt, nu, blist, binfo, nbh, finer, n, ph, m, dtheta, err, st);
}

template <typename T>
void launch_adj_fw_T(int Bs, double* r, const int32_t* blist, const int32_t* nbh, const uint8_t* finer, int64_t n,
                     cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, fw_T, r, blist, nbh, finer, n, st);
}

template <typename T>
void launch_adj_lin(int Bs, double* out, double a, const double* x, double b, const double* y, const int32_t* blist,
                    int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, lin, out, a, x, b, y, blist, n, st);
}

template <typename T>
void launch_adj_objective(int Bs, const T* U, const T* chi, double* lam, double* gchi, const int32_t* blist,
                          const int4* binfo, int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m,
                          double* dtheta, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, objective, U, chi, lam, gchi, blist, binfo, n, ph, wN, wE, m, dtheta, st);
}

template <typename T>
void launch_adj_theta(int Bs, const double* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph,
                      const MaskK& m, double* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, theta, gchi, blist, binfo, n, ph, m, out, st);
}

template <typename T>
void launch_adj_gather(int Bs, const double* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, gather, r, dense, blist, n, st);
}

template <typename T>
void launch_adj_put(int Bs, const double* dense, double* r, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_ADJ_BS(Bs, put, dense, r, blist, n, st);
}

#define ACM_ADJ_INST(T)                                                                                        \
  template void launch_adj_jgt<T>(int, const T*, const double*, const T*, double*, double*, double*, const int32_t*, \
                                  const int4*, const int32_t*, const uint8_t*, int64_t, const PhysK&, const MaskK&, \
                                  double*, int*, cudaStream_t);                                              \
  template void launch_adj_fw_T<T>(int, double*, const int32_t*, const int32_t*, const uint8_t*, int64_t, cudaStream_t); \
  template void launch_adj_lin<T>(int, double*, double, const double*, double, const double*, const int32_t*, int64_t, \
                                  cudaStream_t);                                                              \
  template void launch_adj_objective<T>(int, const T*, const T*, double*, double*, const int32_t*, const int4*, int64_t, \
                                        const PhysK&, double, double, const MaskK&, double*, cudaStream_t);  \
  template void launch_adj_theta<T>(int, const double*, const int32_t*, const int4*, int64_t, const PhysK&,   \
                                    const MaskK&, double*, cudaStream_t);                                     \
  template void launch_adj_gather<T>(int, const double*, double*, const int32_t*, int64_t, cudaStream_t);         \
  template void launch_adj_put<T>(int, const double*, double*, const int32_t*, int64_t, cudaStream_t);
ACM_ADJ_INST(float)
ACM_ADJ_INST(double)

}  // namespace acm
