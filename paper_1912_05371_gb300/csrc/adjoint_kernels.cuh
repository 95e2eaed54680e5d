// Discrete adjoint of the RK4 steps on a frozen grid: kernels of libacm.  The forward state and
// the mask are in the forest's precision T; every adjoint variable, coefficient and sum is FP64
// (indexed like a register of T: same block, component and point offsets).
//
// One RK4 step (Sec. 2.3) maps U to U' = V + dt/6 (K1 + 2 K2 + 2 K3 + K4), V = W U, with
// K_s = G(Y_s) the right-hand side of eqs. (u_eqn-1, p_eqn-1) (Sec. 2.1-2.2) of the synchronised
// stage state.  G(Y) = loc(E W Y): W is fine wins on the block boundaries, E fills each block's
// face halos (3 layers) from the finest leaf holding a point, else by the tensor DD-4 prediction
// (Sec. 3.1, 4.2), and loc is the block-local stencil arithmetic.  Its transpose applied to an
// adjoint stage variable kappa is built in three launches:
//   k_adj_weights   per interior point the coefficients of loc^T (from Y's values and kappa),
//   k_adj_scatter   per halo or interior point of every block the sum of the stencil terms that
//                   read it (loc^T), added to the point's source in the register (E^T: the
//                   block's own point, the leaf holding it, or the DD-4 stencil's sources),
//   k_adj_fw_T      W^T: a boundary point held by a finer leaf passes its value to that leaf's
//                   point and is cleared.
// The elementwise RK4 adjoint combination, the objective's direct terms and the reduction of the
// mask sensitivity onto the sphere's centre and radius complete the step (host side in api.cu).
//
// This header holds the kernels and one launcher per kernel and (T, BS); each of the
// translation units adjoint_{f,d}{9,17}.cu instantiates one pair (they compile in parallel),
// and adjoint.cu dispatches on the block size.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.hpp"

namespace acm {
namespace {

constexpr int kNA = 256;
constexpr int kNW = kAdjWeightsPerPoint;   // loc^T coefficients per interior point (layout in k_adj_weights)

__device__ __forceinline__ double lattice_coord(const PhysK& ph, int4 bi, int a, int i, int M, double h) {
  const int g = a == 0 ? bi.y : (a == 1 ? bi.z : bi.w);
  const long long N = ((long long)ph.nroot[a] << bi.x) * M;
  const long long gi = (long long)g * M + i;              // in [0, N]; the seam x = L is taken as 0
  return (double)(gi >= N ? gi - N : gi) * h;
}

// Sponge profile (the stage kernel's, in FP64): the largest of the three axis profiles.
__device__ __forceinline__ double sponge_at(const PhysK& ph, int4 bi, int x, int y, int z, int M, double h) {
  const int q[3] = {x, y, z};
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double c = lattice_coord(ph, bi, a, q[a], M, h);
    const double dist = fmin(c, ph.sp_L[a] - c);
    const double v = 0.5 * (1.0 - tanh((dist - ph.sp_width) / ph.sp_delta));
    s = v > s ? v : s;
  }
  return s;
}

// Value of the stage state at local point (x, y, z) of a block: its own point inside, else the
// ghost value (finest leaf holding it, else the DD-4 prediction).
template <typename T, int BS>
__device__ __forceinline__ double yval(const T* Y, const int* nbh, size_t own, int x, int y, int z, int f) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  if (x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M) return (double)Y[own + (size_t)f * L::FS + L::idx(x, y, z)];
  return (double)point_value<T, BS>(Y, nbh, x, y, z, f);
}

// Moving rigid box (mask kind 2) at offset r = x - x_0 from its pivot: the solid velocity
// u_s = omega x r, its derivative d u_s/dtheta = (d omega/dtheta) x r, and d chi/dtheta through
// the body coordinates x_b = R^T r (d x_b/dtheta = dR^T r) and the gradient of the box's signed
// distance (outside: from the nearest box point; inside: the nearest face's normal).
struct BoxPoint {
  double us[3], dus[3], dchi;
};
__device__ __forceinline__ BoxPoint box_point(const MaskK& m, double rx, double ry, double rz) {
  BoxPoint o;
  const double* w = m.p + 19;
  const double* dw = m.p + 33;
  o.us[0] = w[1] * rz - w[2] * ry;
  o.us[1] = w[2] * rx - w[0] * rz;
  o.us[2] = w[0] * ry - w[1] * rx;
  o.dus[0] = dw[1] * rz - dw[2] * ry;
  o.dus[1] = dw[2] * rx - dw[0] * rz;
  o.dus[2] = dw[0] * ry - dw[1] * rx;
  double q[3], sg[3], dxb[3], n2 = 0.0, qmax = -1e300;
  int kmax = 0;
  for (int k = 0; k < 3; ++k) {
    const double xb = m.p[k] * rx + m.p[3 + k] * ry + m.p[6 + k] * rz;
    dxb[k] = m.p[24 + k] * rx + m.p[27 + k] * ry + m.p[30 + k] * rz;
    const double dv = xb - m.p[12 + k];
    sg[k] = dv >= 0.0 ? 1.0 : -1.0;
    q[k] = fabs(dv) - m.p[15 + k];
    if (q[k] > 0.0) n2 += q[k] * q[k];
    if (q[k] > qmax) { qmax = q[k]; kmax = k; }
  }
  const double nout = sqrt(n2);
  double gd = 0.0;                                     // grad d . d x_b / dtheta
  if (nout > 0.0) {
    for (int k = 0; k < 3; ++k)
      if (q[k] > 0.0) gd += q[k] / nout * sg[k] * dxb[k];
  } else {
    gd = sg[kmax] * dxb[kmax];
  }
  const double d = nout + (qmax < 0.0 ? qmax : 0.0);
  const double th = tanh(d / m.p[18]);
  o.dchi = -0.5 / m.p[18] * (1.0 - th * th) * gd;
  return o;
}

// Block reduction of one double per thread into *out (one atomic per CTA).
__device__ __forceinline__ void block_add(double v, double* out) {
  __shared__ double red[kNA / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kNA / 32; ++k) t += red[k];
    atomicAdd(out, t);
  }
}

// Coefficients of loc^T at each interior point p of block `rank` (kappa: the adjoint stage
// variable, Y: the synchronised stage state):
//   [3i + j]  A_ij = -u_j kappa_i      (i, j < 3; weight of D1_j applied to field i)
//   [9]       P    = -c0^2 kappa_p     (weight of D1_j applied to field j, from the p equation)
//   [10 + i]  V_i  = nu kappa_i        (weight of every D2 applied to field i)
//   [13 + i]  G_i  = -kappa_i          (weight of D1_i applied to p)
//   [16 + j]  pointwise term of field j: -sum_i kappa_i D1_j u_i - (chi/C_eta + chi_sp/C_sp) kappa_j,
//             and for p: -(C_gamma + chi_sp/C_sp) kappa_p
// The mask sensitivity -sum_i kappa_i u_i / C_eta is added to gchi.
// With a moving box (m.kind == 2) the mask's and the solid velocity's sensitivities are turned into
// d/dtheta at once (the pose is the stage's) and summed into *dtheta instead of gchi.
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_weights(const T* Y, const double* kap, const T* chi,
                                                     double* gchi, double* wgt, const int32_t* blist,
                                                     const int4* binfo, const int32_t* nbh_all, const PhysK ph,
                                                     const MaskK m, double* dtheta) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, N3 = BS * BS * BS;
  __shared__ int nbh[kNbhStride];
  const int rank = blockIdx.x;
  for (int i = threadIdx.x; i < kNbhStride; i += kNA) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  __syncthreads();
  const int slot = blist[rank];
  const int4 bi = binfo[rank];
  const double h = ph.h[bi.x], ih = 1.0 / h;
  const double a[3] = {ph.a1, ph.a2, ph.a3};
  const size_t own = (size_t)slot * L::BLK;
  double* w = wgt + (size_t)rank * kNW * N3;
  const bool moving = m.kind == 2;
  double dth = 0.0;
  for (int t = threadIdx.x; t < N3; t += kNA) {
    const int x = t % BS, y = (t / BS) % BS, z = t / (BS * BS);
    const int pi = L::idx(x, y, z);
    double u[3], k[4], du[3][3];
    for (int f = 0; f < 3; ++f) u[f] = (double)Y[own + (size_t)f * L::FS + pi];
    for (int f = 0; f < 4; ++f) k[f] = kap[own + (size_t)f * L::FS + pi];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int m = 1; m <= 3; ++m) {
          const int dx = j == 0 ? m : 0, dy = j == 1 ? m : 0, dz = j == 2 ? m : 0;
          s += a[m - 1] * (yval<T, BS>(Y, nbh, own, x + dx, y + dy, z + dz, i) -
                           yval<T, BS>(Y, nbh, own, x - dx, y - dy, z - dz, i));
        }
        du[i][j] = s * ih;
      }
    const double c = ph.mask ? (double)chi[(size_t)slot * L::FS + pi] : 0.0;
    const double cs = ph.sponge ? sponge_at(ph, bi, x, y, z, M, h) : 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) w[(size_t)(3 * i + j) * N3 + t] = -u[j] * k[i];
    w[(size_t)9 * N3 + t] = -ph.c0sq * k[3];
    for (int i = 0; i < 3; ++i) {
      w[(size_t)(10 + i) * N3 + t] = ph.nu * k[i];
      w[(size_t)(13 + i) * N3 + t] = -k[i];
    }
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int i = 0; i < 3; ++i) s -= k[i] * du[i][j];
      w[(size_t)(16 + j) * N3 + t] = s - (c * ph.inv_ceta + cs * ph.inv_csp) * k[j];
    }
    w[(size_t)19 * N3 + t] = -(ph.cgamma + cs * ph.inv_csp) * k[3];
    if (moving) {
      const BoxPoint bp = box_point(m, lattice_coord(ph, bi, 0, x, M, h) - m.p[9],
                                    lattice_coord(ph, bi, 1, y, M, h) - m.p[10],
                                    lattice_coord(ph, bi, 2, z, M, h) - m.p[11]);
      double gc = 0.0, gu = 0.0;
      for (int i = 0; i < 3; ++i) {
        gc -= k[i] * (u[i] - bp.us[i]) * ph.inv_ceta;      // d/dchi of -chi (u - u_s) / C_eta
        gu += c * k[i] * ph.inv_ceta * bp.dus[i];          // d/du_s, times d u_s / dtheta
      }
      dth += gc * bp.dchi + gu;
    } else if (ph.mask) {
      gchi[(size_t)slot * L::FS + pi] -= (k[0] * u[0] + k[1] * u[1] + k[2] * u[2]) * ph.inv_ceta;
    }
  }
  if (moving) block_add(dth, dtheta);
}

// loc^T and E^T: for every point q of block `rank`'s extended region (interior and the six face
// halos of depth 3) and component f, the sum of the stencil terms of the interior points that
// read q, added to q's source in `nu` (FP64 atomics: several blocks reach one point).
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_scatter(const double* wgt, double* nu, const int32_t* blist,
                                                     const int4* binfo, const int32_t* nbh_all, const PhysK ph,
                                                     int* err) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, N3 = BS * BS * BS, NH = 6 * 3 * BS * BS;
  __shared__ int nbh[kNbhStride];
  const int rank = blockIdx.x;
  for (int i = threadIdx.x; i < kNbhStride; i += kNA) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  __syncthreads();
  const int slot = blist[rank];
  const int4 bi = binfo[rank];
  const double h = ph.h[bi.x], ih = 1.0 / h, ih2 = 1.0 / (12.0 * h * h);
  const double a[3] = {ph.a1, ph.a2, ph.a3};
  const double d2[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
  const double* w = wgt + (size_t)rank * kNW * N3;
  const size_t own = (size_t)slot * L::BLK;
  auto inside = [](int x, int y, int z) { return x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M; };
  auto wat = [&](int k, int x, int y, int z) { return w[(size_t)k * N3 + (z * BS + y) * BS + x]; };
  for (int t = threadIdx.x; t < 4 * (N3 + NH); t += kNA) {
    const int f = t / (N3 + NH), r = t % (N3 + NH);
    int q[3];
    if (r < N3) {
      q[0] = r % BS; q[1] = (r / BS) % BS; q[2] = r / (BS * BS);
    } else {
      const int e = r - N3, F = e / (3 * BS * BS), l = (e / (BS * BS)) % 3, uv = e % (BS * BS);
      const int ax = F >> 1, side = F & 1;
      const int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
      q[ax] = side ? M + 1 + l : -1 - l;
      q[o1] = uv % BS;
      q[o2] = uv / BS;
    }
    double de = 0.0;
    for (int j = 0; j < 3; ++j) {
      // D1_j: point p = q - m e_j reads q with +a_m/h, p = q + m e_j with -a_m/h
      const int kidx = f < 3 ? 3 * f + j : 13 + j;
      for (int m = 1; m <= 3; ++m) {
        int p[3] = {q[0], q[1], q[2]};
        p[j] = q[j] - m;
        if (inside(p[0], p[1], p[2])) {
          double wv = wat(kidx, p[0], p[1], p[2]);
          if (f < 3 && f == j) wv += wat(9, p[0], p[1], p[2]);
          de += a[m - 1] * ih * wv;
        }
        p[j] = q[j] + m;
        if (inside(p[0], p[1], p[2])) {
          double wv = wat(kidx, p[0], p[1], p[2]);
          if (f < 3 && f == j) wv += wat(9, p[0], p[1], p[2]);
          de -= a[m - 1] * ih * wv;
        }
      }
      // D2_j on the velocity: p = q - k e_j reads q with d2[k + 2]
      if (f < 3)
        for (int kk = -2; kk <= 2; ++kk) {
          int p[3] = {q[0], q[1], q[2]};
          p[j] = q[j] - kk;
          if (inside(p[0], p[1], p[2])) de += d2[kk + 2] * ih2 * wat(10 + f, p[0], p[1], p[2]);
        }
    }
    if (r < N3) {
      de += wat(16 + f, q[0], q[1], q[2]);
      atomicAdd(&nu[own + (size_t)f * L::FS + L::idx(q[0], q[1], q[2])], de);
      continue;
    }
    if (de == 0.0) continue;
    const long long o = direct_offset<T, BS>(nbh, q[0], q[1], q[2], f);
    if (o >= 0) {
      atomicAdd(&nu[o], de);
      continue;
    }
    // predicted ghost: the tensor DD-4 weights (x, then y, then z) of its even stencil points
    const double wd[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
    const int off[4] = {-3, -1, 1, 3};
    const int nx = (q[0] & 1) ? 4 : 1, ny = (q[1] & 1) ? 4 : 1, nz = (q[2] & 1) ? 4 : 1;
    for (int kz = 0; kz < nz; ++kz)
      for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < nx; ++kx) {
          const int xx = nx == 4 ? q[0] + off[kx] : q[0];
          const int yy = ny == 4 ? q[1] + off[ky] : q[1];
          const int zz = nz == 4 ? q[2] + off[kz] : q[2];
          const double wt = (nx == 4 ? wd[kx] : 1.0) * (ny == 4 ? wd[ky] : 1.0) * (nz == 4 ? wd[kz] : 1.0);
          const long long o2 = direct_offset<T, BS>(nbh, xx, yy, zz, f);
          if (o2 < 0) {
            atomicOr(err, 8);
            continue;
          }
          atomicAdd(&nu[o2], wt * de);
        }
  }
}

// W^T on register r: a boundary point of block `rank` that a finer leaf holds (the first refined
// box among those containing it, in the order the forward search uses) adds its value to that
// leaf's point and is cleared.
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_fw_T(double* r, const int32_t* blist, const int32_t* nbh_all,
                                                  const uint8_t* finer) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, N3 = BS * BS * BS;
  const int rank = blockIdx.x;
  if (!finer[rank]) return;
  __shared__ int nbh[kNbhStride];
  for (int i = threadIdx.x; i < kNbhStride; i += kNA) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  __syncthreads();
  const size_t own = (size_t)blist[rank] * L::BLK;
  for (int t = threadIdx.x; t < N3; t += kNA) {
    const int p[3] = {t % BS, (t / BS) % BS, t / (BS * BS)};
    if (p[0] != 0 && p[0] != M && p[1] != 0 && p[1] != M && p[2] != 0 && p[2] != M) continue;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = p[a] == 0 ? -1 : 0;
      hi[a] = p[a] == M ? 1 : 0;
    }
    long long src = -1;
    for (int dz = lo[2]; dz <= hi[2] && src < 0; ++dz)
      for (int dy = lo[1]; dy <= hi[1] && src < 0; ++dy)
        for (int dx = lo[0]; dx <= hi[0] && src < 0; ++dx) {
          const int d = box_index(dx, dy, dz);
          if ((nbh[kNbhType + d] & 15) != kTypeRefined) continue;
          const int bd[3] = {dx, dy, dz};
          int c = 0, l[3];
          for (int a = 0; a < 3; ++a) {
            const int qa = p[a] - bd[a] * M;                 // in [0, M] inside box d
            const int ca = qa > M / 2 ? 1 : (qa < M / 2 ? 0 : (bd[a] < 0 ? 1 : 0));
            c |= ca << a;
            l[a] = 2 * qa - ca * M;
          }
          const int s = nbh[8 * d + c];
          if (s >= 0) src = (long long)s * L::BLK + L::idx(l[0], l[1], l[2]);
        }
    if (src < 0) continue;
    for (int f = 0; f < 4; ++f) {
      const size_t o = own + (size_t)f * L::FS + L::idx(p[0], p[1], p[2]);
      const double v = r[o];
      r[o] = 0.0;
      if (v != 0.0) atomicAdd(&r[(size_t)src + (size_t)f * L::FS], v);
    }
  }
}

// out = a x + b y over the blocks of the list (whole block strides); y may be null.
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_lin(double* out, double a, const double* x, double b, const double* y,
                                                 const int32_t* blist) {
  using L = Lay<T, BS>;
  const size_t base = (size_t)blist[blockIdx.x] * L::BLK;
  for (int i = threadIdx.x; i < L::BLK; i += kNA)
    out[base + i] = a * x[base + i] + (y ? b * y[base + i] : 0.0);
}

// Direct terms of (1/N) [F_x(U) + w_E E(U)] (Sec. 2.2, half-open points, weight h^3): into lam
// and, for the mask, into gchi.
// With a moving box the force integrates chi (u - u_s) at the state's time (pose in m): the direct
// d/dtheta of the force is summed into *dtheta.
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_objective(const T* U, const T* chi, double* lam, double* gchi,
                                                       const int32_t* blist, const int4* binfo, const PhysK ph,
                                                       double wN, double wE, const MaskK m, double* dtheta) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const double h = ph.h[bi.x], h3 = h * h * h;
  const size_t own = (size_t)slot * L::BLK;
  const bool moving = m.kind == 2;
  double dth = 0.0;
  for (int t = threadIdx.x; t < M * M * M; t += kNA) {
    const int x = t % M, y = (t / M) % M, z = t / (M * M);
    const int pi = L::idx(x, y, z);
    const double u = (double)U[own + pi];
    const double c = ph.mask ? (double)chi[(size_t)slot * L::FS + pi] : 0.0;
    lam[own + pi] += wN * (c * ph.inv_ceta + wE * u) * h3;
    for (int f = 1; f < 3; ++f)
      lam[own + (size_t)f * L::FS + pi] += wN * wE * (double)U[own + (size_t)f * L::FS + pi] * h3;
    if (moving) {
      const BoxPoint bp = box_point(m, lattice_coord(ph, bi, 0, x, M, h) - m.p[9],
                                    lattice_coord(ph, bi, 1, y, M, h) - m.p[10],
                                    lattice_coord(ph, bi, 2, z, M, h) - m.p[11]);
      dth += wN * h3 * ph.inv_ceta * ((u - bp.us[0]) * bp.dchi - c * bp.dus[0]);
    } else if (ph.mask) {
      gchi[(size_t)slot * L::FS + pi] += wN * u * h3 * ph.inv_ceta;
    }
  }
  if (moving) block_add(dth, dtheta);
}

// sum over all points of gchi * d chi / d (cx, cy, cz, R) for the sphere mask
// chi = (1 - tanh((|x - c| - R)/delta))/2 (Sec. 2.2), into out[0..3].
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_theta(const double* gchi, const int32_t* blist, const int4* binfo,
                                                   const PhysK ph, const MaskK m, double* out) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, N3 = BS * BS * BS;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const double h = ph.h[bi.x];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < N3; t += kNA) {
    const int x = t % BS, y = (t / BS) % BS, z = t / (BS * BS);
    const double g = gchi[(size_t)slot * L::FS + L::idx(x, y, z)];
    if (g == 0.0) continue;
    const double rx = lattice_coord(ph, bi, 0, x, M, h) - m.p[0];
    const double ry = lattice_coord(ph, bi, 1, y, M, h) - m.p[1];
    const double rz = lattice_coord(ph, bi, 2, z, M, h) - m.p[2];
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    const double th = tanh((r - m.p[3]) / m.p[4]);
    const double sg = 0.5 / m.p[4] * (1.0 - th * th) * g;        // -d chi / d d, times gchi
    const double rs = r > 0.0 ? r : 1.0;
    s[0] += sg * rx / rs;
    s[1] += sg * ry / rs;
    s[2] += sg * rz / rs;
    s[3] += sg;
  }
  __shared__ double red[4][kNA / 32];
  for (int k = 0; k < 4; ++k)
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x >> 5] = s[k];
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int wi = 0; wi < kNA / 32; ++wi) v += red[threadIdx.x][wi];
    atomicAdd(&out[threadIdx.x], v);
  }
}

// Block-order copy of an FP64 register indexed like a register of T: dense[rank][f][z][y][x].
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_gather(const double* r, double* dense, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int N3 = BS * BS * BS;
  const size_t own = (size_t)blist[blockIdx.x] * L::BLK;
  double* d = dense + (size_t)blockIdx.x * 4 * N3;
  for (int t = threadIdx.x; t < 4 * N3; t += kNA) {
    const int f = t / N3, r3 = t % N3;
    d[t] = r[own + (size_t)f * L::FS + L::idx(r3 % BS, (r3 / BS) % BS, r3 / (BS * BS))];
  }
}

// The inverse copy: dense[rank][f][z][y][x] into the register's interior points (the register's
// padding is left as it is).
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_put(const double* dense, double* r, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int N3 = BS * BS * BS;
  const size_t own = (size_t)blist[blockIdx.x] * L::BLK;
  const double* d = dense + (size_t)blockIdx.x * 4 * N3;
  for (int t = threadIdx.x; t < 4 * N3; t += kNA) {
    const int f = t / N3, r3 = t % N3;
    r[own + (size_t)f * L::FS + L::idx(r3 % BS, (r3 / BS) % BS, r3 / (BS * BS))] = d[t];
  }
}

inline dim3 g1(int64_t n) { return dim3((unsigned)n); }

}  // namespace

namespace adj {

template <typename T, int BS>
void jgt(const T* Y, const double* kap, const T* chi, double* gchi, double* wgt, double* nu, const int32_t* blist,
         const int4* binfo, const int32_t* nbh, const uint8_t* finer, int64_t n, const PhysK& ph, const MaskK& m,
         double* dtheta, int* err, cudaStream_t st) {
  k_adj_weights<T, BS><<<g1(n), kNA, 0, st>>>(Y, kap, chi, gchi, wgt, blist, binfo, nbh, ph, m, dtheta);
  k_adj_scatter<T, BS><<<g1(n), kNA, 0, st>>>(wgt, nu, blist, binfo, nbh, ph, err);
  k_adj_fw_T<T, BS><<<g1(n), kNA, 0, st>>>(nu, blist, nbh, finer);
}

template <typename T, int BS>
void fw_T(double* r, const int32_t* blist, const int32_t* nbh, const uint8_t* finer, int64_t n, cudaStream_t st) {
  k_adj_fw_T<T, BS><<<g1(n), kNA, 0, st>>>(r, blist, nbh, finer);
}

template <typename T, int BS>
void lin(double* out, double a, const double* x, double b, const double* y, const int32_t* blist, int64_t n,
         cudaStream_t st) {
  k_adj_lin<T, BS><<<g1(n), kNA, 0, st>>>(out, a, x, b, y, blist);
}

template <typename T, int BS>
void objective(const T* U, const T* chi, double* lam, double* gchi, const int32_t* blist, const int4* binfo,
               int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m, double* dtheta, cudaStream_t st) {
  k_adj_objective<T, BS><<<g1(n), kNA, 0, st>>>(U, chi, lam, gchi, blist, binfo, ph, wN, wE, m, dtheta);
}

template <typename T, int BS>
void theta(const double* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph, const MaskK& m,
           double* out, cudaStream_t st) {
  k_adj_theta<T, BS><<<g1(n), kNA, 0, st>>>(gchi, blist, binfo, ph, m, out);
}

template <typename T, int BS>
void gather(const double* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st) {
  k_adj_gather<T, BS><<<g1(n), kNA, 0, st>>>(r, dense, blist);
}

template <typename T, int BS>
void put(const double* dense, double* r, const int32_t* blist, int64_t n, cudaStream_t st) {
  k_adj_put<T, BS><<<g1(n), kNA, 0, st>>>(dense, r, blist);
}

}  // namespace adj
}  // namespace acm

// Explicit instantiation of every launcher for one (T, BS).
#define ACM_ADJ_INSTANTIATE(T, BS)                                                                                 \
  namespace acm {                                                                                                  \
  namespace adj {                                                                                                  \
  template void jgt<T, BS>(const T*, const double*, const T*, double*, double*, double*, const int32_t*, const int4*, \
                           const int32_t*, const uint8_t*, int64_t, const PhysK&, const MaskK&, double*, int*,       \
                           cudaStream_t);                                                                          \
  template void fw_T<T, BS>(double*, const int32_t*, const int32_t*, const uint8_t*, int64_t, cudaStream_t);         \
  template void lin<T, BS>(double*, double, const double*, double, const double*, const int32_t*, int64_t,           \
                           cudaStream_t);                                                                          \
  template void objective<T, BS>(const T*, const T*, double*, double*, const int32_t*, const int4*, int64_t,         \
                                 const PhysK&, double, double, const MaskK&, double*, cudaStream_t);               \
  template void theta<T, BS>(const double*, const int32_t*, const int4*, int64_t, const PhysK&, const MaskK&,        \
                             double*, cudaStream_t);                                                               \
  template void gather<T, BS>(const double*, double*, const int32_t*, int64_t, cudaStream_t);                        \
  template void put<T, BS>(const double*, double*, const int32_t*, int64_t, cudaStream_t);                           \
  }                                                                                                                \
  }
