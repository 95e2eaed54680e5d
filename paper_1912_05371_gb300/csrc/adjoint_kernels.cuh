// Discrete adjoint of the RK4 steps on a frozen grid: kernels of libacm.  The forward state, the
// mask and the adjoint variables are in the forest's precision T; the sums over the grid that make
// the gradient with respect to the mask parameters are FP64, and so is the gradient with respect
// to U_0 handed to the caller.
//
// One RK4 step (Sec. 2.3) maps U to U' = V + dt/6 (K1 + 2 K2 + 2 K3 + K4), V = W U, with
// K_s = G(Y_s) the right-hand side of eqs. (u_eqn-1, p_eqn-1) (Sec. 2.1-2.2) of the synchronised
// stage state.  G(Y) = loc(E W Y): W is fine wins on the block boundaries, E fills each block's
// face halos (3 layers) from the finest leaf holding a point, else by the tensor DD-4 prediction
// (Sec. 3.1, 4.2), and loc is the block-local stencil arithmetic.  The adjoint of one stage,
// nu = W^T E^T loc^T kappa with kappa = c_lam lam + c_nu nu' (the RK4 adjoint combination), takes
// four launches:
//   k_adj_stage      loc^T at every block's own interior points, in gather form (a z-march like
//                    the forward stage kernel), with the combination for kappa, the running sum
//                    of the stage nus and the mask sensitivity fused in;
//   k_adj_samelevel  E^T of the face-halo targets that same-level neighbours read from a block,
//                    gathered by that block (no atomics);
//   k_adj_halo       loc^T at the face-halo points toward finer and coarser faces and E^T: added
//                    to the points they were read from (the finest leaf holding the point, or its
//                    DD-4 prediction's even points);
//   k_adj_fw_T       W^T: a boundary point held by a finer leaf passes its value to that leaf's
//                    point and is cleared.
// The objective's direct terms and the reduction of the mask sensitivity onto the sphere's centre
// and radius complete the sweep (host side in api.cu).
//
// This header holds the kernels and one launcher per kernel and (T, BS); each of the
// translation units adjoint_{f,d}{9,17}.cu instantiates one pair (they compile in parallel),
// and adjoint.cu dispatches on the block size.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "stage_common.cuh"

namespace acm {
namespace {

constexpr int kNA = 256;

__device__ __forceinline__ double lattice_coord(const PhysK& ph, int4 bi, int a, int i, int M, double h) {
  const int g = a == 0 ? bi.y : (a == 1 ? bi.z : bi.w);
  const long long N = ((long long)ph.nroot[a] << bi.x) * M;
  const long long gi = (long long)g * M + i;              // in [0, N]; the seam x = L is taken as 0
  return (double)(gi >= N ? gi - N : gi) * h;
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

// A float estimate of the box's signed distance at offset r (the distance part of box_point, in
// float): it decides which points are so far from the surface that tanh(d/delta) is +-1 in the
// field precision (exactly in FP64 beyond 19.1 delta), where d chi/dtheta vanishes and chi is 0
// (outside) or 1 (inside), and the FP64 distance and tanh need not be evaluated.
__device__ __forceinline__ float box_distance_f(const MaskK& m, float rx, float ry, float rz) {
  float n2 = 0.f, qmax = -1e30f;
  for (int k = 0; k < 3; ++k) {
    const float xb = (float)m.p[k] * rx + (float)m.p[3 + k] * ry + (float)m.p[6 + k] * rz;
    const float q = fabsf(xb - (float)m.p[12 + k]) - (float)m.p[15 + k];
    if (q > 0.f) n2 += q * q;
    qmax = fmaxf(qmax, q);
  }
  return sqrtf(n2) + fminf(qmax, 0.f);
}
// d u_s/dtheta = (d omega/dtheta) x r, as box_point computes it.
__device__ __forceinline__ void box_dus(const MaskK& m, double rx, double ry, double rz, double (&dus)[3]) {
  const double* dw = m.p + 33;
  dus[0] = dw[1] * rz - dw[2] * ry;
  dus[1] = dw[2] * rx - dw[0] * rz;
  dus[2] = dw[0] * ry - dw[1] * rx;
}
// Beyond this distance from the surface the box's chi is exactly 0 or 1 and its derivative 0
// (FP64: tanh rounds to +-1 beyond 19.1 delta; FP32 fields: tanhf beyond 9.1 delta, the FP64
// derivative left out there is below 1e-8 of its value at the surface).
template <typename T>
__device__ __forceinline__ double box_far(const MaskK& m) {
  return (sizeof(T) == 8 ? 20.0 : 10.0) * m.p[18];
}

// Block reduction of one double per thread of an NT-thread CTA into *out (one atomic per CTA).
template <int NT>
__device__ __forceinline__ void block_add_n(double v, double* out) {
  __shared__ double red[NT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < NT / 32; ++k) t += red[k];
    atomicAdd(out, t);
  }
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

// ---- the adjoint of one RK stage: nu = W^T E^T loc(E W Y)^T kappa ------------------------------------
// loc^T kappa at a target point q, for the weights at the block's interior sources p (zero
// outside the interior; h-free first differences Dt_j g(q) = sum_m a_m [g(q - m e_j) - g(q + m e_j)],
// the symmetric second difference D2_j g(q) = sum_k d2_k g(q + k e_j), d2 = (-1, 16, -30, 16, -1)):
//   nu_i(q) = -1/h [sum_j Dt_j(u_j kappa_i) + c0^2 Dt_i(kappa_p)] + nu/(12 h^2) sum_j D2_j(kappa_i)
//             - 1/h sum_k kappa_k(q) Dh_i u_k(q) - (chi/C_eta + chi_sp/C_sp) kappa_i(q)      (i < 3)
//   nu_p(q) = -1/h sum_j Dt_j(kappa_j) - (C_gamma + chi_sp/C_sp) kappa_p(q)
// (Dh_i: the forward's h-free first difference along i, of the stage state with its ghost values).
// The first two lines are the transposed stencils of the convective, pressure, divergence and
// viscous terms, the last ones the pointwise terms of the linearisation.
//
// k_adj_stage evaluates this at the block's own interior targets in gather form (one CTA per
// block, a thread per (x, y) pencil marching in z, as the forward stage kernel): kappa and u of
// the current plane in shared memory with a zero halo (sources outside the interior weigh
// nothing), kappa and u of the planes z - 3 .. z + 3 in a register ring, and for the pointwise
// term the stage state's x/y halos by cp.async from the neighbours (copy or decimation) or from
// the coarse-face slabs, as the forward reads them.  kappa = c_lam lam + c_nu nu' is formed as it
// is read (nu': the next RK stage's nu), and the running sum of the stage nus is updated from nu'
// in the same pass.  The own targets are stored with plain writes; the targets in the face halos
// (k_adj_halo) go to other blocks' points through E^T afterwards.
// A block of 33^3 points is split by rows over three CTAs (as the forward stage kernel): the
// kappa rows of the CTA next to this one are sources inside the block, loaded like a halo.
template <typename T, int BS>
struct AdjCfg {
  static constexpr int RY = BS <= 17 ? BS : 11;                  // rows (y) per CTA
  static constexpr int NS = (BS + RY - 1) / RY;                  // CTAs per block
  static constexpr int NT = ((BS * RY + 31) / 32) * 32;
  static constexpr int H = RY + 6;
  static constexpr int W = sizeof(T) == 4 && BS <= 17 ? BS + 32 : BS + 6;   // bank-conflict-free rows (FP32)
  static constexpr int PW = H * W;
  static constexpr int NC = 7;                                   // planes: u, v, w, kappa_0..3
  static constexpr int NHC = 6 * (RY + BS);                      // x/y halo values of one component
  static constexpr int NH = 3 * NHC;                             // x/y halo values of u, v, w per plane
  static constexpr int HPT = (NH + NT - 1) / NT;
  static constexpr size_t BUF = (size_t)2 * NC * PW * sizeof(T);
  static constexpr size_t bytes = BUF + (size_t)NH * 12;
  static constexpr int MINB = sizeof(T) == 4 ? 2 : 1;
  static_assert(NC * PW < 0x8000, "plane buffer offsets must fit 15 bits");
  static_assert(NS == 1 || sizeof(T) == 4, "row-split blocks are FP32 only");
};

// MOVING: the moving box's parameter sensitivity (kind 2), compiled apart from the static masks'
// form so that its FP64 pose arithmetic costs the static form no registers.
template <typename T, int BS, bool MOVING>
__global__ void __launch_bounds__(AdjCfg<T, BS>::NT, AdjCfg<T, BS>::MINB)
k_adj_stage(const AdjStageK<T> a, const TopoK tp, const PhysK ph, const MaskK m) {
  using L = Lay<T, BS>;
  using C = AdjCfg<T, BS>;
  constexpr int M = L::M;
  constexpr int NT = C::NT, W = C::W, PW = C::PW, NH = C::NH, HPT = C::HPT;
  extern __shared__ __align__(16) unsigned char smem[];
  T* buf = reinterpret_cast<T*>(smem);                                       // [2][7][PW]
  unsigned* hlo = reinterpret_cast<unsigned*>(smem + C::BUF);
  unsigned* hhi = hlo + NH;
  unsigned* hzd = hhi + NH;
  __shared__ int ftype[6];
  __shared__ int fs[6][4];
  __shared__ T sp[3][BS];

  constexpr int RY = C::RY, NHC = C::NHC;
  const int tid = threadIdx.x;
  const int rank = blockIdx.x / C::NS, part = blockIdx.x % C::NS;
  const int slot = tp.blist[rank];
  const int4 bi = tp.binfo[rank];
  const int* nbh = tp.nbh + (size_t)rank * kNbhStride;
  const int y0 = part * RY, ny = BS - y0 < RY ? BS - y0 : RY;    // this CTA's rows
  stage_faces(tid, nbh, tp.slabidx, rank, ftype, fs);
  stage_sponge<T, BS>(tid, ph, bi, sp);
  // the kappa planes' halos stay zero (sources outside the block weigh nothing)
  for (int i = tid; i < 2 * C::NC * PW; i += NT) buf[i] = T(0);
  __syncthreads();

  const T a1 = T(ph.a1), a2 = T(ph.a2), a3 = T(ph.a3);
  const T ih = T(1.0 / ph.h[bi.x]);
  const T nu_ih2 = T(ph.nu / (12.0 * ph.h[bi.x] * ph.h[bi.x]));
  const T c0sq = T(ph.c0sq), inv_ceta = T(ph.inv_ceta), inv_csp = T(ph.inv_csp), cgam = T(ph.cgamma);
  const T c_lam = T(a.c_lam), c_nu = T(a.c_nu);
  const bool act = tid < BS * ny;
  const int x = act ? tid % BS : 0, y = y0 + (act ? tid / BS : 0);
  const size_t bo = (size_t)slot * L::BLK;
  const T* __restrict__ Yb = a.Y + bo;

  auto y_value = [&](int zz, int f) -> T {
    if (zz >= 0 && zz <= M) return Yb[(size_t)f * L::FS + L::idx(x, y, zz)];
    if (zz < 0) return *halo_ptr<T, BS>(ftype, fs, a.Y, a.slab, 4, -zz, x, y, f);
    return *halo_ptr<T, BS>(ftype, fs, a.Y, a.slab, 5, zz - M, x, y, f);
  };
  auto kappa = [&](int zz, int f) -> T {
    if (zz < 0 || zz > M) return T(0);
    const size_t o = bo + (size_t)f * L::FS + L::idx(x, y, zz);
    T k = c_lam * a.lam[o];
    if (a.nup) k += c_nu * a.nup[o];
    return k;
  };

  // x/y halo values of u, v, w of every plane as affine functions of z (the forward kernel's
  // table): entry i is read at (z <= M/2 ? lo : hi) + z * stride from Y (or the slab buffer,
  // flag bit 15) and lands at dst: hzd = stride << 16 | slab << 15 | dst (0: unused entry).
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int i = tid + k * NT;
    if (i < NH) {
      const int f = i / NHC;
      int el = i % NHC, F, l, t;
      if (el < 6 * RY) {
        F = el / (3 * RY);
        el %= 3 * RY;
        l = el % 3 + 1;
        t = y0 + el / 3;
      } else {
        el -= 6 * RY;
        F = 2 + el / (3 * BS);
        el %= 3 * BS;
        t = el % BS;
        l = el / BS + 1;
      }
      int hx, hy;                                   // plane coordinates, rows from y0
      if (F == 0) { hx = -l; hy = t - y0; }
      else if (F == 1) { hx = M + l; hy = t - y0; }
      else if (F == 2) { hx = t; hy = -l; }
      else { hx = t; hy = ny - 1 + l; }
      const unsigned dst = (unsigned)(f * PW + (hy + 3) * W + hx + 3);
      const int ty = ftype[F];
      const bool plus = F & 1;
      const int ax = F >> 1;
      if (F < 2 && t >= y0 + ny) {
        hlo[i] = 0; hhi[i] = 0; hzd[i] = 0;
      } else if ((F == 2 && y0 > 0) || (F == 3 && y0 + ny - 1 < M)) {
        const int yy = F == 2 ? y0 - l : y0 + ny - 1 + l;       // a row of this block
        const unsigned o = (unsigned)(bo + (size_t)f * L::FS + L::idx(t, yy, 0));
        hlo[i] = o; hhi[i] = o; hzd[i] = ((unsigned)L::PP << 16) | dst;
      } else if (ty == kTypeCoarser) {
        const unsigned o = (unsigned)((((size_t)fs[F][0] * 4 + f) * 3 + (l - 1)) * BS * BS + t);
        hlo[i] = o; hhi[i] = o; hzd[i] = ((unsigned)BS << 16) | 0x8000u | dst;
      } else if (ty == kTypeLeaf) {
        const int nl = plus ? l : M - l;
        const int xx = ax == 0 ? nl : t, yy = ax == 0 ? t : nl;
        const unsigned o = (unsigned)((size_t)fs[F][0] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0));
        hlo[i] = o; hhi[i] = o; hzd[i] = ((unsigned)L::PP << 16) | dst;
      } else {
        const int c0 = t > M / 2;
        const int nl = plus ? 2 * l : M - 2 * l;
        const int u0 = 2 * t - c0 * M;
        const int xx = ax == 0 ? nl : u0, yy = ax == 0 ? u0 : nl;
        const unsigned lo = (unsigned)((size_t)fs[F][c0] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0));
        const unsigned hi = (unsigned)((size_t)fs[F][c0 + 2] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0)) -
                            (unsigned)(M * L::PP);
        hlo[i] = lo; hhi[i] = hi; hzd[i] = ((unsigned)(2 * L::PP) << 16) | dst;
      }
    }
  }
  auto issue_halos = [&](int zz, T* B) {
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
      const int i = tid + k * NT;
      if (i < NH) {
        const unsigned zd = hzd[i];
        if (C::NS > 1 && zd == 0) continue;
        const unsigned off = (zz > M / 2 ? hhi[i] : hlo[i]) + (unsigned)zz * (zd >> 16);
        cp_async_elem(B + (zd & 0x7fffu), ((zd & 0x8000u) ? a.slab : a.Y) + (size_t)off);
      }
    }
    cp_async_commit();
  };
  // kappa of plane zz in the rows the CTAs next to this one own (3 each side that has one)
  auto fill_kappa_rows = [&](int zz, T* B) {
    if constexpr (C::NS > 1) {
      for (int j = tid; j < 2 * 3 * BS; j += NT) {
        const int side = j / (3 * BS), l = (j / BS) % 3 + 1, t = j % BS;
        if (side == 0 ? y0 == 0 : y0 + ny - 1 == M) continue;
        const int yy = side == 0 ? y0 - l : y0 + ny - 1 + l, hy = side == 0 ? -l : ny - 1 + l;
        const size_t o = bo + L::idx(t, yy, zz);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          T k = c_lam * a.lam[o + (size_t)f * L::FS];
          if (a.nup) k += c_nu * a.nup[o + (size_t)f * L::FS];
          B[(3 + f) * PW + (hy + 3) * W + t + 3] = k;
        }
      }
    }
  };

  // register rings: qy[c][k] = u_c of plane z + k - 3, qk[f][k] = kappa_f of plane z + k - 3
  T qy[3][8], qk[4][8];
#pragma unroll
  for (int k = 0; k < 7; ++k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) qy[c][k] = act ? y_value(k - 3, c) : T(0);
#pragma unroll
    for (int f = 0; f < 4; ++f) qk[f][k] = act ? kappa(k - 3, f) : T(0);
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) qk[f][7] = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) qy[c][7] = T(0);
  fill_kappa_rows(0, buf);
  __syncthreads();
  issue_halos(0, buf);

  const int ci = (y - y0 + 3) * W + x + 3;
  constexpr bool moving = MOVING;
  double dth = 0.0;
  const double hd = ph.h[bi.x];
  for (int z = 0; z <= M; ++z) {
    T* B = buf + (z & 1) * C::NC * PW;
    if (act) {
#pragma unroll
      for (int c = 0; c < 3; ++c) B[c * PW + ci] = qy[c][3];
#pragma unroll
      for (int f = 0; f < 4; ++f) B[(3 + f) * PW + ci] = qk[f][3];
    }
    cp_async_wait_all();
    __syncthreads();
    if (z < M) {
      issue_halos(z + 1, buf + ((z + 1) & 1) * C::NC * PW);
      fill_kappa_rows(z + 1, buf + ((z + 1) & 1) * C::NC * PW);
    }
    if (act) {
      if (z + 4 <= M + 3) {
#pragma unroll
        for (int c = 0; c < 3; ++c) qy[c][7] = y_value(z + 4, c);
#pragma unroll
        for (int f = 0; f < 4; ++f) qk[f][7] = kappa(z + 4, f);
      }
      const size_t pi = (size_t)L::idx(x, y, z);
      // h-free first differences Dh_j u_i of the stage state (with its ghost values)
      T du[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T* s = B + c * PW;
        du[c][0] = a1 * (s[ci + 1] - s[ci - 1]) + a2 * (s[ci + 2] - s[ci - 2]) + a3 * (s[ci + 3] - s[ci - 3]);
        du[c][1] = a1 * (s[ci + W] - s[ci - W]) + a2 * (s[ci + 2 * W] - s[ci - 2 * W]) +
                   a3 * (s[ci + 3 * W] - s[ci - 3 * W]);
        du[c][2] = a1 * (qy[c][4] - qy[c][2]) + a2 * (qy[c][5] - qy[c][1]) + a3 * (qy[c][6] - qy[c][0]);
      }
      // transposed first differences of the products u_j kappa_i and of kappa, and the second
      // differences of kappa, along x (shared plane), y (shared plane) and z (register rings)
      T tconv[3] = {T(0), T(0), T(0)};     // sum_j Dt_j(u_j kappa_i)
      T tk[4];                              // Dt_j(kappa_f) along j = f (f < 3); for p: sum_j Dt_j(kappa_j)
      T d2k[3] = {T(0), T(0), T(0)};       // sum_j D2_j(kappa_i)
      T tkp[3];                             // Dt_i(kappa_p)
      tk[3] = T(0);
      const T* su = B;
      const T* sk[4] = {B + 3 * PW, B + 4 * PW, B + 5 * PW, B + 6 * PW};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // tap values at offsets -3..3 (index o + 3) along direction j
        T uj[7], kf[4][7];
#pragma unroll
        for (int o = -3; o <= 3; ++o) {
          if (j < 2) {
            const int st = j == 0 ? o : o * W;
            uj[o + 3] = su[j * PW + ci + st];
#pragma unroll
            for (int f = 0; f < 4; ++f) kf[f][o + 3] = sk[f][ci + st];
          } else {
            uj[o + 3] = qy[2][o + 3];
#pragma unroll
            for (int f = 0; f < 4; ++f) kf[f][o + 3] = qk[f][o + 3];
          }
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T g1 = uj[2] * kf[i][2] - uj[4] * kf[i][4];
          const T g2 = uj[1] * kf[i][1] - uj[5] * kf[i][5];
          const T g3 = uj[0] * kf[i][0] - uj[6] * kf[i][6];
          tconv[i] += a1 * g1 + a2 * g2 + a3 * g3;
          d2k[i] += T(16) * (kf[i][2] + kf[i][4]) - (kf[i][1] + kf[i][5]) - T(30) * kf[i][3];
        }
        tkp[j] = a1 * (kf[3][2] - kf[3][4]) + a2 * (kf[3][1] - kf[3][5]) + a3 * (kf[3][0] - kf[3][6]);
        tk[3] += a1 * (kf[j][2] - kf[j][4]) + a2 * (kf[j][1] - kf[j][5]) + a3 * (kf[j][0] - kf[j][6]);
      }
      const T k0 = qk[0][3], k1 = qk[1][3], k2 = qk[2][3], k3 = qk[3][3];
      const T chiv = ph.mask ? a.chi[(size_t)slot * L::FS + pi] : T(0);
      const T cs = ph.sponge ? tmax(tmax(sp[0][x], sp[1][y]), sp[2][z]) : T(0);
      const T damp = chiv * inv_ceta + cs * inv_csp;
      T out[4];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        out[i] = -ih * (tconv[i] + c0sq * tkp[i]) + nu_ih2 * d2k[i] -
                 ih * (k0 * du[0][i] + k1 * du[1][i] + k2 * du[2][i]) - damp * qk[i][3];
      out[3] = -ih * tk[3] - (cgam + cs * inv_csp) * k3;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const size_t o = bo + (size_t)f * L::FS + pi;
        a.nu[o] = out[f];
        if (a.sum_mode == 1) a.sum[o] = a.nup[o];
        else if (a.sum_mode == 2) a.sum[o] += a.nup[o];
      }
      const T u = qy[0][3], v = qy[1][3], w = qy[2][3];
      if constexpr (MOVING) {
        const double rx = lattice_coord(ph, bi, 0, x, M, hd) - m.p[9];
        const double ry = lattice_coord(ph, bi, 1, y, M, hd) - m.p[10];
        const double rz = lattice_coord(ph, bi, 2, z, M, hd) - m.p[11];
        const double kk[3] = {(double)k0, (double)k1, (double)k2};
        const float df = box_distance_f(m, (float)rx, (float)ry, (float)rz);
        const double far = box_far<T>(m);
        if (df < -far) {
          // inside, away from the surface: chi = 1 and d chi = 0, only d u_s/dtheta acts
          double dus[3], gu = 0.0;
          box_dus(m, rx, ry, rz, dus);
          for (int i = 0; i < 3; ++i) gu += (double)chiv * kk[i] * ph.inv_ceta * dus[i];
          dth += gu;
        } else if (!(df > far)) {
          const BoxPoint bp = box_point(m, rx, ry, rz);
          const double uu[3] = {(double)u, (double)v, (double)w};
          double gc = 0.0, gu = 0.0;
          for (int i = 0; i < 3; ++i) {
            gc -= kk[i] * (uu[i] - bp.us[i]) * ph.inv_ceta;     // d/dchi of -chi (u - u_s) / C_eta
            gu += (double)chiv * kk[i] * ph.inv_ceta * bp.dus[i]; // d/du_s, times d u_s / dtheta
          }
          dth += gc * bp.dchi + gu;
        }                                                       // outside, far: no term
      } else if (ph.mask && a.gchi) {
        a.gchi[(size_t)slot * L::FS + pi] -= (k0 * u + k1 * v + k2 * w) * inv_ceta;
      }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
#pragma unroll
      for (int c = 0; c < 3; ++c) qy[c][k] = qy[c][k + 1];
#pragma unroll
      for (int f = 0; f < 4; ++f) qk[f][k] = qk[f][k + 1];
    }
  }
  if (moving) {
    __syncthreads();
    block_add_n<AdjCfg<T, BS>::NT>(dth, a.dtheta);
  }
}

// The targets of loc^T in block `rank`'s face halos (3 layers beyond each face): only sources
// along the face normal are inside the block, so a halo point q at distance l gets
//   nu_i(q) = -1/h sum_{m=l..3} (+-a_m) [u_n kappa_i + delta_{in} c0^2 kappa_p](q -+ m e_n)
//             + nu/(12 h^2) sum_{k=l..2} d2_k kappa_i(q -+ k e_n)                      (i < 3)
//   nu_p(q) = -1/h sum_{m=l..3} (+-a_m) kappa_n(q -+ m e_n)
// (n the normal axis, the sign that of the face), added through E^T to the point q was read from.
// One CTA per (block, face); faces toward a same-level neighbour are left to that neighbour,
// which gathers them (k_adj_samelevel).  Across a finer face q goes to the child's coinciding
// point (the forward's decimation); fine wins' copies
// between leaves are W's part (k_adj_fw_T).  Across a coarser face, q is held by a leaf if it lies
// on one's lattice (its point gets the value), else it was predicted by the tensor DD-4 from the
// even points of the 5 x (M/2 + 3)^2 coarse patch around the face: the predicted targets are kept
// in shared memory and the transposed prediction is applied one axis at a time (along the face,
// then across it) as gathers, each coarse point summing the fine points its prediction weights
// reach; then each patch point goes to the leaf holding it.  FP atomics in global memory only:
// several blocks reach one point.  Runs after k_adj_stage.
//
// The face-halo targets of the four components at one tangential point: de[f][l - 1] for the
// halo layers l = 1..3 beyond a face with normal axis ax (sg: +1 for the upper face, -1 for the
// lower), from the three source points next to it (po[k]: element offset of the source at normal
// distance k = 0, 1, 2 inside the face, component 0).  Each source value is read once for all
// four components.
template <typename T, int BS>
__device__ __forceinline__ void face_targets(const AdjStageK<T>& a, const size_t (&po)[3], int ax, T sg, T ih,
                                             T nu_ih2, T c0sq, const T (&am)[3], T c_lam, T c_nu, T (&de)[4][3]) {
  using L = Lay<T, BS>;
  const T d2[2] = {T(16), T(-1)};
  T kap[4][3], uax[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    uax[k] = a.Y[po[k] + (size_t)ax * L::FS];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      T kv = c_lam * a.lam[po[k] + (size_t)g * L::FS];
      if (a.nup) kv += c_nu * a.nup[po[k] + (size_t)g * L::FS];
      kap[g][k] = kv;
    }
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T Wk[3], Kk[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (f < 3) {
        Kk[k] = kap[f][k];
        Wk[k] = uax[k] * Kk[k];
        if (f == ax) Wk[k] += c0sq * kap[3][k];
      } else {
        Kk[k] = T(0);
        Wk[k] = kap[ax][k];
      }
    }
#pragma unroll
    for (int l = 1; l <= 3; ++l) {
      T e = T(0), dd = T(0);
#pragma unroll
      for (int k = 0; k + l <= 3; ++k) {
        e += sg * am[l + k - 1] * Wk[k];
        if (l + k <= 2) dd += d2[l + k - 1] * Kk[k];
      }
      de[f][l - 1] = -ih * e + (f < 3 ? nu_ih2 * dd : T(0));
    }
  }
}

// E^T across same-level faces in gather form: block A adds to its own points the face-halo
// targets of its same-level face neighbours that the forward read from A (the neighbour N's
// halo point at distance l beyond the shared face is A's point at distance l inside it), each
// computed from N's sources next to the face as k_adj_halo computes a halo target.  One CTA per
// block walks its six faces in turn (a point near an edge takes one face's value at a time), so
// the additions need no atomics; a thread per tangential point of a face, all four components.
// It runs after k_adj_stage and before k_adj_halo's atomics.
template <int BS>
struct SameCfg {
  static constexpr int NT = BS * BS <= 1024 ? ((BS * BS + 31) / 32) * 32 : 384;
};

template <typename T, int BS>
__global__ void __launch_bounds__(SameCfg<BS>::NT)
k_adj_samelevel(const AdjStageK<T> a, const TopoK tp, const PhysK ph, int* err) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, NT = SameCfg<BS>::NT;
  __shared__ int types[6], slots[6];
  const int rank = blockIdx.x;
  if (threadIdx.x < 6) {
    const int d = kFaceBox[threadIdx.x];
    const int* nbh = tp.nbh + (size_t)rank * kNbhStride;
    types[threadIdx.x] = nbh[kNbhType + d] & 15;
    slots[threadIdx.x] = nbh[8 * d];
  }
  __syncthreads();
  const size_t bo = (size_t)tp.blist[rank] * L::BLK;
  const int4 bi = tp.binfo[rank];
  const T ih = T(1.0 / ph.h[bi.x]);
  const T nu_ih2 = T(ph.nu / (12.0 * ph.h[bi.x] * ph.h[bi.x]));
  const T c0sq = T(ph.c0sq);
  const T am[3] = {T(ph.a1), T(ph.a2), T(ph.a3)};
  const T c_lam = T(a.c_lam), c_nu = T(a.c_nu);
  for (int F = 0; F < 6; ++F) {
    if (types[F] != kTypeLeaf) continue;                        // uniform over the CTA
    if (slots[F] < 0) {
      if (threadIdx.x == 0) atomicOr(err, 8);
      continue;
    }
    const int ax = F >> 1, side = F & 1;
    const int o1 = ax == 0 ? 1 : 0, o2 = 3 - ax - o1;
    const size_t nb = (size_t)slots[F] * L::BLK;
    // the shared face is the neighbour's opposite face: its sources at distance k inside it sit
    // at neighbour coordinate k (this block's upper face) or M - k (its lower face), and its
    // halo stencils take the sign of that face
    const T sg = side ? T(-1) : T(1);
    for (int uv = threadIdx.x; uv < BS * BS; uv += NT) {
      int p[3] = {0, 0, 0};
      p[o1] = uv % BS;
      p[o2] = uv / BS;
      size_t po[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        p[ax] = side ? k : M - k;
        po[k] = nb + L::idx(p[0], p[1], p[2]);
      }
      T de[4][3];
      face_targets<T, BS>(a, po, ax, sg, ih, nu_ih2, c0sq, am, c_lam, c_nu, de);
#pragma unroll
      for (int l = 1; l <= 3; ++l) {
        p[ax] = side ? M - l : l;
        const size_t o = bo + L::idx(p[0], p[1], p[2]);
#pragma unroll
        for (int f = 0; f < 4; ++f) a.nu[o + (size_t)f * L::FS] += de[f][l - 1];
      }
    }
    __syncthreads();
  }
}

template <typename T, int BS>
struct HaloCfg {
  static constexpr int M = BS - 1;
  static constexpr int NTG = M / 2 + 3;               // even fine tangential coordinates -2 .. M + 2
  static constexpr int NPATCH = 5 * NTG * NTG;        // normal: 5 even fine coordinates beyond the face
  // shared memory of a coarse face: the predicted halo targets h [f][l][t2][t1], then after the
  // transposed prediction along t1, t2 and the normal a [f][l][t2][c1], b [f][l][c2][c1] (in h's
  // place) and the patch [f][n][c2][c1] (in a's place)
  static constexpr int NH3 = 3 * BS * BS, NA = 3 * BS * NTG, NB = 3 * NTG * NTG;
  static constexpr int U0 = 4 * (NH3 > NB ? NH3 : NB);
  static constexpr int U1 = 4 * (NA > NPATCH ? NA : NPATCH);
  static constexpr size_t bytes = (size_t)(U0 + U1) * sizeof(T);
};

template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_halo(const AdjStageK<T> a, const TopoK tp, const PhysK ph, int* err) {
  using L = Lay<T, BS>;
  using H = HaloCfg<T, BS>;
  constexpr int M = L::M, NTG = H::NTG, NP = H::NPATCH;
  __shared__ int nbh[kNbhStride];
  extern __shared__ __align__(16) unsigned char hsm[];
  T* hv = reinterpret_cast<T*>(hsm);                  // h, later b
  T* acc = hv + H::U0;                                // a, later the patch
  const int rank = blockIdx.x / 6, F = blockIdx.x % 6;
  const int ax = F >> 1, side = F & 1;
  const int d = kFaceBox[F];
  // a same-level neighbour gathers these targets itself (k_adj_samelevel): its CTA reads the
  // face's type word only
  if ((tp.nbh[(size_t)rank * kNbhStride + kNbhType + d] & 15) == kTypeLeaf) return;
  for (int i = threadIdx.x; i < kNbhStride; i += kNA) nbh[i] = tp.nbh[(size_t)rank * kNbhStride + i];
  __syncthreads();
  const int ty = nbh[kNbhType + d] & 15;
  const bool coarse = ty != kTypeLeaf && ty != kTypeRefined;
  if (coarse) {
    for (int i = threadIdx.x; i < 4 * H::NH3; i += kNA) hv[i] = T(0);
    __syncthreads();
  }
  const size_t bo = (size_t)tp.blist[rank] * L::BLK;
  const int4 bi = tp.binfo[rank];
  const T ih = T(1.0 / ph.h[bi.x]);
  const T nu_ih2 = T(ph.nu / (12.0 * ph.h[bi.x] * ph.h[bi.x]));
  const T c0sq = T(ph.c0sq);
  const T am[3] = {T(ph.a1), T(ph.a2), T(ph.a3)};
  const T c_lam = T(a.c_lam), c_nu = T(a.c_nu);
  // threads run along the tangential axis with the smaller memory stride (x for y and z faces)
  const int o1 = ax == 0 ? 1 : 0, o2 = 3 - ax - o1;
  const T sg = side ? T(1) : T(-1);
  const T wd[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  // E^T of one halo target q of component f with value de
  auto scatter = [&](const int (&q)[3], int f, int l, T de) {
    if (!coarse) {
      // a finer face: the child's coinciding point (the forward's decimation)
      int c = (side ? 0 : 1) << ax;
      const int b1 = q[o1] > M / 2, b2 = q[o2] > M / 2;
      c |= (b1 << o1) | (b2 << o2);
      const int s = nbh[8 * d + c];
      int lc[3];
      lc[ax] = side ? 2 * l : M - 2 * l;
      lc[o1] = 2 * q[o1] - b1 * M;
      lc[o2] = 2 * q[o2] - b2 * M;
      if (s < 0) {
        atomicOr(err, 8);
        return;
      }
      if (de != T(0)) atomicAdd(&a.nu[(size_t)s * L::BLK + (size_t)f * L::FS + L::idx(lc[0], lc[1], lc[2])], de);
      return;
    }
    if (de == T(0)) return;
    if (ty != kTypeCoarser || q[o1] == 0 || q[o1] == M || q[o2] == 0 || q[o2] == M) {
      // on the face's boundary lines a leaf of this level or finer may hold q
      const long long o = direct_offset<T, BS>(nbh, q[0], q[1], q[2], f);
      if (o >= 0) {
        atomicAdd(&a.nu[o], de);
        return;
      }
    } else if (!((q[0] | q[1] | q[2]) & 1)) {
      // strictly inside the face's box only the coarser leaf holds q, on its lattice here
      const int oct = nbh[kNbhType + d] >> 4;
      int lc[3];
#pragma unroll
      for (int ac = 0; ac < 3; ++ac) {
        const int qb = q[ac] - (ac == ax ? (side ? M : -M) : 0);      // in box d's frame
        lc[ac] = (((oct >> ac) & 1) * M + qb) >> 1;
      }
      const int s = nbh[8 * d];
      if (s < 0) {
        atomicOr(err, 8);
        return;
      }
      atomicAdd(&a.nu[(size_t)s * L::BLK + (size_t)f * L::FS + L::idx(lc[0], lc[1], lc[2])], de);
      return;
    }
    // a predicted ghost: kept for the transposed prediction below (each target has one thread)
    hv[((f * 3 + l - 1) * BS + q[o2]) * BS + q[o1]] = de;
  };
  // a thread per tangential point, all four components: the three halo layers from the three
  // sources next to the face, p_k at normal distance k = 0, 1, 2 inside it (q at layer l reads
  // p_k with weight a_{l+k}, and its second difference d2_{l+k} for l + k <= 2)
  for (int uv = threadIdx.x; uv < BS * BS; uv += kNA) {
    int q[3] = {0, 0, 0};
    q[o1] = uv % BS;
    q[o2] = uv / BS;
    size_t po[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int p[3] = {q[0], q[1], q[2]};
      p[ax] = side ? M - k : k;
      po[k] = bo + L::idx(p[0], p[1], p[2]);
    }
    T de[4][3];
    face_targets<T, BS>(a, po, ax, sg, ih, nu_ih2, c0sq, am, c_lam, c_nu, de);
#pragma unroll
    for (int l = 1; l <= 3; ++l) {
      q[ax] = side ? M + l : -l;
#pragma unroll
      for (int f = 0; f < 4; ++f) scatter(q, f, l, de[f][l - 1]);
    }
  }
  if (!coarse) return;
  __syncthreads();
  // the transposed tensor DD-4 prediction, one axis at a time as gathers: a coarse point c (fine
  // coordinate 2c - 2 along the face, nbase + 2n across it) takes the fine point it coincides
  // with (weight 1) and the odd fine points at distance 1 and 3 (9/16, -1/16)
  auto gather_line = [&](const T* src, int stride, int tc, int lo, int hi) -> T {
    T v = T(0);
    if (tc >= lo && tc <= hi) v += src[tc * stride];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int t = tc - (2 * k - 3);           // t + off_k = tc with off_k = -3, -1, 1, 3
      if (t >= lo && t <= hi && (t & 1)) v += wd[k] * src[t * stride];
    }
    return v;
  };
  T* pa = acc;
  for (int i = threadIdx.x; i < 4 * H::NA; i += kNA) {        // along t1: a[f][l][t2][c1]
    const int c1 = i % NTG, r = i / NTG;                      // r = (f * 3 + l) * BS + t2
    pa[i] = gather_line(hv + (size_t)r * BS, 1, 2 * c1 - 2, 0, M);
  }
  __syncthreads();
  T* pb = hv;
  for (int i = threadIdx.x; i < 4 * H::NB; i += kNA) {        // along t2: b[f][l][c2][c1]
    const int c1 = i % NTG, c2 = (i / NTG) % NTG, fl = i / (NTG * NTG);
    pb[i] = gather_line(pa + (size_t)fl * BS * NTG + c1, NTG, 2 * c2 - 2, 0, M);
  }
  __syncthreads();
  const int nbase = side ? M - 2 : -6;
  for (int i = threadIdx.x; i < 4 * NP; i += kNA) {           // across the face: patch[f][n][c2][c1]
    const int c = i % (NTG * NTG), n = (i / (NTG * NTG)) % 5, f = i / NP;
    // layer l sits at fine normal coordinate side ? M + l : -l, i.e. index l - 1 of b's rows at
    // coordinate (side ? M + 1 : -1) + (side ? 1 : -1) (l - 1)
    const int pn = nbase + 2 * n;
    T v = T(0);
#pragma unroll
    for (int l = 1; l <= 3; ++l) {
      const int qn = side ? M + l : -l;
      const int off = pn - qn;
      T w = T(0);
      if (off == 0) w = T(1);
      else if (qn & 1) w = off == -3 ? wd[0] : (off == -1 ? wd[1] : (off == 1 ? wd[2] : (off == 3 ? wd[3] : T(0))));
      if (w != T(0)) v += w * pb[((size_t)(f * 3 + l - 1) * NTG * NTG) + c];
    }
    acc[i] = v;
  }
  __syncthreads();
  // each patch point to the leaf holding it (the prediction's sources are held directly)
  for (int i = threadIdx.x; i < 4 * NP; i += kNA) {
    const T v = acc[i];
    if (v == T(0)) continue;
    const int f = i / NP, r = i % NP;
    const int kn = r / (NTG * NTG), k2 = (r / NTG) % NTG, k1 = r % NTG;
    int c[3];
    c[ax] = nbase + 2 * kn;
    c[o2] = 2 * k2 - 2;
    c[o1] = 2 * k1 - 2;
    const long long o = direct_offset<T, BS>(nbh, c[0], c[1], c[2], f);
    if (o < 0) {
      atomicOr(err, 8);
      continue;
    }
    atomicAdd(&a.nu[o], v);
  }
}

// W^T on register r, over the forward's fine-wins task list (rank, refined box d): every boundary
// point of block `rank` that the forward overwrote with the value of a point of box d's child
// hands its value to that point and is cleared.  A point on an edge or corner may appear in two
// tasks (the forward wrote it twice, the same value): the atomic exchange gives it to the first
// task that reaches it, the other moves zero.  CTAs walk the list, whose length is on the device.
template <typename T>
__device__ __forceinline__ T exch_zero(T* p) {
  if constexpr (sizeof(T) == 4) {
    return __int_as_float(atomicExch(reinterpret_cast<int*>(p), 0));
  } else {
    return __longlong_as_double(
        (long long)atomicExch(reinterpret_cast<unsigned long long*>(p), 0ull));
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_fw_T(T* r, const int2* tasks, const int32_t* ntasks,
                                                  const int32_t* nbh_all, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int nt = *ntasks;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const int2 tk = tasks[ti];
    const int* nbh = nbh_all + (size_t)tk.x * kNbhStride;
    const int me = blist[tk.x];
    const int d = tk.y;
    const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    int n[3], o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      n[a] = dd[a] == 0 ? BS : 1;
      o[a] = dd[a] < 0 ? 0 : (dd[a] > 0 ? M : 0);
    }
    const int tot = n[0] * n[1] * n[2];
    for (int i = threadIdx.x; i < tot; i += kNA) {
      const int p[3] = {o[0] + i % n[0], o[1] + (i / n[0]) % n[1], o[2] + i / (n[0] * n[1])};
      int c = 0, l[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = p[a] - dd[a] * M;
        const int ca = q > M / 2 ? 1 : (q < M / 2 ? 0 : (dd[a] < 0 ? 1 : 0));
        c |= ca << a;
        l[a] = 2 * q - ca * M;
      }
      const int s = nbh[8 * d + c];
      if (s < 0) continue;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T v = exch_zero(&r[(size_t)me * L::BLK + (size_t)f * L::FS + L::idx(p[0], p[1], p[2])]);
        if (v != T(0)) atomicAdd(&r[(size_t)s * L::BLK + (size_t)f * L::FS + L::idx(l[0], l[1], l[2])], v);
      }
    }
  }
}

// out = x + y + z over the blocks of the list (whole block strides).
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_sum3(T* out, const T* x, const T* y, const T* z, const int32_t* blist) {
  using L = Lay<T, BS>;
  const size_t base = (size_t)blist[blockIdx.x] * L::BLK;
  for (int i = threadIdx.x; i < L::BLK; i += kNA) out[base + i] = x[base + i] + y[base + i] + z[base + i];
}

// Direct terms of (1/N) [F_x(U) + w_E E(U)] (Sec. 2.2, half-open points, weight h^3): into lam
// and, for the mask, into gchi.
// With a moving box the force integrates chi (u - u_s) at the state's time (pose in m): the direct
// d/dtheta of the force is summed into *dtheta.
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_objective(const T* U, const T* chi, T* lam, T* gchi,
                                                       const int32_t* blist, const int4* binfo, const PhysK ph,
                                                       double wN, double wE, const MaskK m, double* dtheta) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const double h = ph.h[bi.x], h3 = h * h * h;
  const size_t own = (size_t)slot * L::BLK;
  const bool moving = m.kind == 2;
  // the terms' weights of this block in FP64, the per-point products in the field precision
  const T a_chi = T(wN * h3 * ph.inv_ceta), a_e = T(wN * wE * h3);
  double dth = 0.0;
  for (int t = threadIdx.x; t < M * M * M; t += kNA) {
    const int x = t % M, y = (t / M) % M, z = t / (M * M);
    const int pi = L::idx(x, y, z);
    const T uT = U[own + pi];
    const T cT = ph.mask ? chi[(size_t)slot * L::FS + pi] : T(0);
    lam[own + pi] += a_chi * cT + a_e * uT;
    for (int f = 1; f < 3; ++f) lam[own + (size_t)f * L::FS + pi] += a_e * U[own + (size_t)f * L::FS + pi];
    if (moving) {
      const double u = (double)uT, c = (double)cT;
      const double rx = lattice_coord(ph, bi, 0, x, M, h) - m.p[9];
      const double ry = lattice_coord(ph, bi, 1, y, M, h) - m.p[10];
      const double rz = lattice_coord(ph, bi, 2, z, M, h) - m.p[11];
      const float df = box_distance_f(m, (float)rx, (float)ry, (float)rz);
      const double far = box_far<T>(m);
      if (df < -far) {                          // chi = 1, d chi = 0: the u_s term only
        double dus[3];
        box_dus(m, rx, ry, rz, dus);
        dth += wN * h3 * ph.inv_ceta * (0.0 - c * dus[0]);
      } else if (!(df > far)) {
        const BoxPoint bp = box_point(m, rx, ry, rz);
        dth += wN * h3 * ph.inv_ceta * ((u - bp.us[0]) * bp.dchi - c * bp.dus[0]);
      }
    } else if (ph.mask) {
      gchi[(size_t)slot * L::FS + pi] += a_chi * uT;
    }
  }
  if (moving) block_add(dth, dtheta);
}

// sum over all points of gchi * d chi / d (cx, cy, cz, R) for the sphere mask
// chi = (1 - tanh((|x - c| - R)/delta))/2 (Sec. 2.2), into out[0..3].
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_theta(const T* gchi, const int32_t* blist, const int4* binfo,
                                                   const PhysK ph, const MaskK m, double* out) {
  using L = Lay<T, BS>;
  constexpr int M = L::M, N3 = BS * BS * BS;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const double h = ph.h[bi.x];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < N3; t += kNA) {
    const int x = t % BS, y = (t / BS) % BS, z = t / (BS * BS);
    const double g = (double)gchi[(size_t)slot * L::FS + L::idx(x, y, z)];
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
__global__ void __launch_bounds__(kNA) k_adj_gather(const T* r, double* dense, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int N3 = BS * BS * BS;
  const size_t own = (size_t)blist[blockIdx.x] * L::BLK;
  double* d = dense + (size_t)blockIdx.x * 4 * N3;
  for (int t = threadIdx.x; t < 4 * N3; t += kNA) {
    const int f = t / N3, r3 = t % N3;
    d[t] = (double)r[own + (size_t)f * L::FS + L::idx(r3 % BS, (r3 / BS) % BS, r3 / (BS * BS))];
  }
}

// The inverse copy: dense[rank][f][z][y][x] into the register's interior points (the register's
// padding is left as it is).
template <typename T, int BS>
__global__ void __launch_bounds__(kNA) k_adj_put(const double* dense, T* r, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int N3 = BS * BS * BS;
  const size_t own = (size_t)blist[blockIdx.x] * L::BLK;
  const double* d = dense + (size_t)blockIdx.x * 4 * N3;
  for (int t = threadIdx.x; t < 4 * N3; t += kNA) {
    const int f = t / N3, r3 = t % N3;
    r[own + (size_t)f * L::FS + L::idx(r3 % BS, (r3 / BS) % BS, r3 / (BS * BS))] = T(d[t]);
  }
}

inline dim3 g1(int64_t n) { return dim3((unsigned)n); }

}  // namespace

namespace adj {

// CTAs of the task-list kernel: enough to fill the GPU, at most one per task.
inline unsigned fw_ctas(int64_t max_tasks) {
  const int64_t c = (int64_t)sm_count() * 8;
  return (unsigned)(max_tasks < c ? (max_tasks > 0 ? max_tasks : 1) : c);
}

template <typename T, int BS>
void stage(const AdjStageK<T>& a, const TopoK& t, const PhysK& ph, const MaskK& m, const FwTasks& fw, int* err,
           cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0}, opted_m{0};
  if (m.kind == 2) {
    smem_opt_in_stage(k_adj_stage<T, BS, true>, AdjCfg<T, BS>::bytes, opted_m);
    k_adj_stage<T, BS, true><<<g1(t.n * AdjCfg<T, BS>::NS), AdjCfg<T, BS>::NT, AdjCfg<T, BS>::bytes, st>>>(a, t, ph, m);
  } else {
    smem_opt_in_stage(k_adj_stage<T, BS, false>, AdjCfg<T, BS>::bytes, opted);
    k_adj_stage<T, BS, false><<<g1(t.n * AdjCfg<T, BS>::NS), AdjCfg<T, BS>::NT, AdjCfg<T, BS>::bytes, st>>>(a, t, ph, m);
  }
  k_adj_samelevel<T, BS><<<g1(t.n), SameCfg<BS>::NT, 0, st>>>(a, t, ph, err);
  static std::atomic<unsigned long long> opted_h{0};
  smem_opt_in_stage(k_adj_halo<T, BS>, HaloCfg<T, BS>::bytes, opted_h);
  k_adj_halo<T, BS><<<g1(6 * t.n), kNA, HaloCfg<T, BS>::bytes, st>>>(a, t, ph, err);
  k_adj_fw_T<T, BS><<<fw_ctas(fw.max_tasks), kNA, 0, st>>>(a.nu, fw.tasks, fw.ntasks, t.nbh, t.blist);
}

template <typename T, int BS>
void fw_T(T* r, const FwTasks& fw, const int32_t* blist, const int32_t* nbh, cudaStream_t st) {
  k_adj_fw_T<T, BS><<<fw_ctas(fw.max_tasks), kNA, 0, st>>>(r, fw.tasks, fw.ntasks, nbh, blist);
}

template <typename T, int BS>
void sum3(T* out, const T* x, const T* y, const T* z, const int32_t* blist, int64_t n, cudaStream_t st) {
  k_adj_sum3<T, BS><<<g1(n), kNA, 0, st>>>(out, x, y, z, blist);
}

template <typename T, int BS>
void objective(const T* U, const T* chi, T* lam, T* gchi, const int32_t* blist, const int4* binfo,
               int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m, double* dtheta, cudaStream_t st) {
  k_adj_objective<T, BS><<<g1(n), kNA, 0, st>>>(U, chi, lam, gchi, blist, binfo, ph, wN, wE, m, dtheta);
}

template <typename T, int BS>
void theta(const T* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph, const MaskK& m,
           double* out, cudaStream_t st) {
  k_adj_theta<T, BS><<<g1(n), kNA, 0, st>>>(gchi, blist, binfo, ph, m, out);
}

template <typename T, int BS>
void gather(const T* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st) {
  k_adj_gather<T, BS><<<g1(n), kNA, 0, st>>>(r, dense, blist);
}

template <typename T, int BS>
void put(const double* dense, T* r, const int32_t* blist, int64_t n, cudaStream_t st) {
  k_adj_put<T, BS><<<g1(n), kNA, 0, st>>>(dense, r, blist);
}

}  // namespace adj
}  // namespace acm

// Explicit instantiation of every launcher for one (T, BS).
#define ACM_ADJ_INSTANTIATE(T, BS)                                                                                 \
  namespace acm {                                                                                                  \
  namespace adj {                                                                                                  \
  template void stage<T, BS>(const AdjStageK<T>&, const TopoK&, const PhysK&, const MaskK&, const FwTasks&, int*,  \
                             cudaStream_t);                                                                        \
  template void fw_T<T, BS>(T*, const FwTasks&, const int32_t*, const int32_t*, cudaStream_t);                       \
  template void sum3<T, BS>(T*, const T*, const T*, const T*, const int32_t*, int64_t, cudaStream_t);                \
  template void objective<T, BS>(const T*, const T*, T*, T*, const int32_t*, const int4*, int64_t,                   \
                                 const PhysK&, double, double, const MaskK&, double*, cudaStream_t);               \
  template void theta<T, BS>(const T*, const int32_t*, const int4*, int64_t, const PhysK&, const MaskK&,             \
                             double*, cudaStream_t);                                                               \
  template void gather<T, BS>(const T*, double*, const int32_t*, int64_t, cudaStream_t);                             \
  template void put<T, BS>(const double*, T*, const int32_t*, int64_t, cudaStream_t);                                \
  }                                                                                                                \
  }
