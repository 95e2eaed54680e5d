// Fused right-hand side + RK4 stage kernel of libacm (the hot path).
//
// One CTA updates one block.  Paper, eqs. (u_eqn-1, p_eqn-1):
//   du/dt = -(u.grad)u - grad p + nu lap u - chi/C_eta u - chi_sp/C_sp (u - u_inf)     (u_s = 0)
//   dp/dt = -C_0^2 div u - C_gamma p - chi_sp/C_sp (p - p_inf)
// with the Tam-Webb (or classical) 4th-order first derivative and the classical 4th-order
// second derivative (Sec. 2.3), and one stage of classical RK4 (Sec. 2.3):
//   stage 1: acc = Y + dt/6 K,  out = Y + dt/2 K     (Y = U^n)
//   stage 2: acc += dt/3 K,     out = U + dt/2 K
//   stage 3: acc += dt/3 K,     out = U + dt K
//   stage 4:                    out = acc + dt/6 K  (= U^{n+1})
//   stage 0 (checks only):      acc = K
//
// Work layout: a thread owns one (x, y) pencil of the block and marches in z (a block of up to
// 17^3 points is one CTA; a 33^3 block is split by rows over three CTAs, which read the rows
// next to their own from the block like a halo).  The z-stencil
// (7 points) lives in a register queue fed one plane ahead from global memory; the x/y
// stencils read a shared-memory plane with a 3-point halo on each side, double-buffered, whose
// halo is brought in by cp.async one plane ahead.  Halo points come straight from the
// neighbour's stored interior (same level: copy; finer: decimation, Sec. 3.1 restriction) or,
// across a face to a coarser neighbour, from the halo slab that the coarse-face kernel
// predicted for this stage.  No ghost layer is written to HBM.
#include <algorithm>

#include "stage_common.cuh"

namespace acm {

namespace {

template <typename T, int BS, int RYT = 0>
struct Cfg {
  // rows (y) of the block one CTA updates: all of them up to Bs = 17; a CTA may have at most
  // 1024 threads, so a Bs = 33 block goes to three CTAs of 11 rows; RYT != 0 chooses the rows
  // per CTA (the autotuner's tile shape: a 17^3 block over two CTAs of 9 and 8 rows)
  static constexpr int RY = RYT ? RYT : (BS <= 17 ? BS : 11);
  static constexpr int NS = (BS + RY - 1) / RY;    // CTAs per block
  static constexpr int NT = ((BS * RY + 31) / 32) * 32;
  static constexpr int H = RY + 6;       // plane rows: 3 halo rows each side
  // row stride: a warp covers consecutive pencils of about two rows; with a stride congruent
  // to BS modulo the bank count (32 words for FP32) the second row continues on the next
  // banks and the plane is read without bank conflicts (Bs = 33 keeps the narrow stride: a
  // warp is one row there, and the wide one would not fit the static shared memory)
  static constexpr int W = sizeof(T) == 4 && BS <= 17 ? BS + 32 : BS + 6;
  static constexpr int PW = H * W;
  // x/y halo values per plane and component: x faces 2 x 3 x RY, y faces 2 x 3 x BS
  static constexpr int NHC = 6 * (RY + BS);
  static constexpr int NH = 4 * NHC;
  static constexpr int HPT = (NH + NT - 1) / NT;   // halo values per thread
  static constexpr int MINB = sizeof(T) == 4 ? (NT <= 160 ? 6 : (NT <= 352 ? 3 : 2)) : 1;   // CTAs per SM
  static_assert(4 * PW < 0x8000, "plane buffer offsets must fit 15 bits");
  static_assert(NS == 1 || sizeof(T) == 4, "row-split blocks are FP32 only");
};


// Planes of U, the accumulator and chi a stage reads besides its input (TMA variant: staged in
// shared memory by bulk copies).
template <int STAGE>
__host__ __device__ constexpr int staged_planes(bool mask) {
  return (STAGE == 2 || STAGE == 3 ? 8 : (STAGE == 4 ? 4 : 0)) + (mask ? 1 : 0);
}

// TMA = true: the planes of U, the accumulator and chi of plane z + 1 are brought into a
// two-slot shared-memory ring by 1D bulk copies (one thread issues them after the plane
// barrier of iteration z, completion on an mbarrier per slot), instead of per-thread loads at
// the point of use.
// The update of one block (rank `rank` of the topology tp), rows part * RY .. of it; a: the
// arrays, kc: the constants.
template <typename T, int BS, int STAGE, bool TMA, int RYT = 0>
__device__ __forceinline__ void stage_block(const StagePtrs<T>& a, const StageConst<T>& kc, const TopoK& tp,
                                            const PhysK& ph, int* err, const int rank, const int part) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  constexpr int NT = Cfg<T, BS, RYT>::NT;
  constexpr int RY = Cfg<T, BS, RYT>::RY, NHC = Cfg<T, BS, RYT>::NHC;
  static_assert(!TMA || Cfg<T, BS, RYT>::NS == 1, "the bulk-copy ring stages whole planes");
  constexpr int W = Cfg<T, BS, RYT>::W;
  constexpr int PW = Cfg<T, BS, RYT>::PW;
  constexpr int HPT = Cfg<T, BS, RYT>::HPT;

  __shared__ __align__(16) T buf[2][4][PW];
  __shared__ int ftype[6];
  __shared__ int fs[6][4];
  __shared__ T sp[3][BS];
  // x/y halo values of every plane as affine functions of z (see below)
  constexpr int NH = Cfg<T, BS, RYT>::NH;
  __shared__ unsigned hlo[NH], hhi[NH], hzd[NH];

  const int tid = threadIdx.x;
  const int slot = tp.blist[rank];
  const int4 bi = tp.binfo[rank];
  const int* nbh = tp.nbh + (size_t)rank * kNbhStride;

  stage_faces(tid, nbh, tp.slabidx, rank, ftype, fs);
  stage_sponge<T, BS>(tid, ph, bi, sp);
  __syncthreads();

  // model and RK constants are read from the kernel parameters (constant bank), not registers;
  // so are the level's 1/h and 1/(12 h^2) (no per-thread FP64 division)
  // 1/h is applied once per right-hand side term, not to every difference
  const T ih = kc.ih[bi.x], nu_ih2 = kc.nu * kc.ih2[bi.x], c0sq_ih = kc.c0sq * ih;
  // RK coefficients: kernel parameters, or (steps with the time step on the device) the values
  // the time-step kernel left in device memory
  T c_acc = kc.c_acc, c_out = kc.c_out;
  if (STAGE >= 1 && a.coefp) {
    c_acc = T(a.coefp[2 * (STAGE - 1)]);
    c_out = T(a.coefp[2 * (STAGE - 1) + 1]);
  }
  const int y0 = part * RY, ny = BS - y0 < RY ? BS - y0 : RY;   // this CTA's rows
  const bool act = tid < BS * ny;
  const int x = act ? tid % BS : 0, y = y0 + (act ? tid / BS : 0);
  (void)err;   // this kernel has no waits that can expire
  const T* __restrict__ inb = a.in + (size_t)slot * L::BLK;
  const size_t bo = (size_t)slot * L::BLK;

  auto plane_value = [&](int zz, int f) -> T {
    if (zz >= 0 && zz <= M) return inb[(size_t)f * L::FS + L::idx(x, y, zz)];
    if (zz < 0) return *halo_ptr<T, BS>(ftype, fs, a.in, a.slab, 4, -zz, x, y, f);
    return *halo_ptr<T, BS>(ftype, fs, a.in, a.slab, 5, zz - M, x, y, f);
  };
  // this thread's x/y halo values of every plane, as affine functions of z: element
  // (component f, face F, layer l, tangential t) of plane z is read at offset
  // (z <= M/2 ? lo : hi) + z * hz from the state (or from the slab buffer, flag bit 15) and
  // lands at dst of the plane buffer: hzd = hz << 16 | slab << 15 | dst.  The offsets are
  // element indices (32-bit: pool and slab sizes are checked at forest creation); hi differs
  // from lo for the upper child of a finer face.  Thread tid owns entries tid + k NT.  A CTA
  // holding part of the rows reads the rows beyond its own from the block itself, and its
  // x-face entries past its last row are unused (hzd = 0; every used dst is at least 3).
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int i = tid + k * NT;
    if (i < NH) {
      const int f = i / NHC;
      int el = i % NHC, F, l, t;
      // x-faces take the 3 layers of a row as consecutive elements (one sector), y-faces a row
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
        // a row of this block held by the CTA next to this one
        const int yy = F == 2 ? y0 - l : y0 + ny - 1 + l;
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
        // upper child: its plane 2z - M sits at 2z * PP - M * PP from its base (the sum with
        // z * hz is taken modulo 2^32 and is non-negative)
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
        if (Cfg<T, BS, RYT>::NS > 1 && zd == 0) continue;
        const unsigned off = (zz > M / 2 ? hhi[i] : hlo[i]) + (unsigned)zz * (zd >> 16);
        cp_async_elem(B + (zd & 0x7fffu), ((zd & 0x8000u) ? a.slab : a.in) + (size_t)off);
      }
    }
    cp_async_commit();
  };

  // TMA ring: stg[slot][k][PP], component k of the staged arrays (U 0..3 and acc 4..7 in stages
  // 2, 3; acc 0..3 in stage 4; chi last if a mask is set)
  extern __shared__ __align__(128) unsigned char dsm[];
  T* stg = reinterpret_cast<T*>(dsm);
  __shared__ __align__(8) unsigned long long mbar[2];
  const int nstg = staged_planes<STAGE>(ph.mask != 0);
  auto stage_src = [&](int k) -> const T* {
    if (STAGE == 2 || STAGE == 3) {
      if (k < 4) return a.U + bo + (size_t)k * L::FS;
      if (k < 8) return a.acc + bo + (size_t)(k - 4) * L::FS;
    } else if (STAGE == 4) {
      if (k < 4) return a.acc + bo + (size_t)k * L::FS;
    }
    return a.chi + (size_t)slot * L::FS;
  };
  auto issue_staged = [&](int zz) {          // thread 0 only
    const int sl = zz & 1;
    constexpr unsigned pb = (unsigned)(L::PP * sizeof(T));
    mbar_expect_tx(&mbar[sl], pb * (unsigned)nstg);
    for (int k = 0; k < nstg; ++k)
      bulk_g2s(stg + ((size_t)sl * nstg + k) * L::PP, stage_src(k) + (size_t)zz * L::PP, pb, &mbar[sl]);
  };
  if (TMA && nstg > 0) {
    if (tid == 0) {
      mbar_init(&mbar[0], 1);
      mbar_init(&mbar[1], 1);
      mbar_init_fence();
    }
    __syncthreads();
    if (tid == 0) issue_staged(0);
  }

  T nm[5] = {T(0), T(0), T(0), T(0), T(0)};   // stage 4: max |u|,|v|,|w|,|p|, |(u,v,w)|^2
  // L2 prefetch of the planes an iteration reads kPf iterations ahead: one thread per array
  // (stage input planes z + 4 + kPf, U, acc and chi planes z + kPf), one bulk request each
  // (this CTA's rows of the plane, widened to 16-byte boundaries inside the padded plane)
  constexpr int kPf = 2;
  const int pf0 = Cfg<T, BS, RYT>::NS == 1 ? 0 : ((y0 * BS) & ~(L::VEC - 1));
  const int pf1 = Cfg<T, BS, RYT>::NS == 1 ? L::PP : (((y0 + ny) * BS + L::VEC - 1) & ~(L::VEC - 1));
  const unsigned kPlaneBytes = (unsigned)((pf1 - pf0) * sizeof(T));
  auto prefetch_planes = [&](int zin, int zo) {
    const size_t pz = (size_t)zin * L::PP + pf0, po = (size_t)zo * L::PP + pf0;
    if (tid < 4) {
      if (zin <= M) prefetch_l2(inb + (size_t)tid * L::FS + pz, kPlaneBytes);
    } else if (tid < 8) {
      if ((STAGE == 2 || STAGE == 3) && zo <= M)
        prefetch_l2(a.U + bo + (size_t)(tid - 4) * L::FS + po, kPlaneBytes);
    } else if (tid < 12) {
      if (STAGE >= 2 && zo <= M) prefetch_l2(a.acc + bo + (size_t)(tid - 8) * L::FS + po, kPlaneBytes);
    } else if (tid == 12) {
      if (ph.mask && zo <= M) prefetch_l2(a.chi + (size_t)slot * L::FS + po, kPlaneBytes);
    }
  };
  for (int k = 0; k < kPf; ++k) prefetch_planes(4 + k, k);
  T q[4][8];
#pragma unroll
  for (int k = 0; k < 7; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f) q[f][k] = act ? plane_value(k - 3, f) : T(0);
#pragma unroll
  for (int f = 0; f < 4; ++f) q[f][7] = T(0);
  issue_halos(0, &buf[0][0][0]);

  const int ci = (y - y0 + 3) * W + x + 3;
  const T sp_xy = ph.sponge ? tmax(sp[0][x], sp[1][y]) : T(0);   // the sponge profile's x/y part
  for (int z = 0; z <= M; ++z) {
    T(*B)[PW] = buf[z & 1];
    if (act) {
#pragma unroll
      for (int f = 0; f < 4; ++f) B[f][ci] = q[f][3];
    }
    cp_async_wait_all();
    __syncthreads();
    if (z < M) issue_halos(z + 1, &buf[(z + 1) & 1][0][0]);
    if (TMA && nstg > 0 && tid == 0 && z < M) {
      // the slot of plane z + 1 held plane z - 1, which every thread finished before the barrier
      fence_async_shared();
      issue_staged(z + 1);
    }
    prefetch_planes(z + 4 + kPf, z + kPf);
    if (TMA && nstg > 0) mbar_wait(&mbar[z & 1], (unsigned)((z >> 1) & 1), err);
    if (act) {
      if (z + 4 <= M + 3) {
#pragma unroll
        for (int f = 0; f < 4; ++f) q[f][7] = plane_value(z + 4, f);
      }
      const size_t pi = (size_t)L::idx(x, y, z);
      T Uv[4], Av[4], chiv = T(0);
      if constexpr (TMA) {
        const T* sg = stg + (size_t)(z & 1) * nstg * L::PP + (size_t)L::idx(x, y, 0);
        if (STAGE == 2 || STAGE == 3) {
#pragma unroll
          for (int f = 0; f < 4; ++f) Uv[f] = sg[(size_t)f * L::PP];
#pragma unroll
          for (int f = 0; f < 4; ++f) Av[f] = sg[(size_t)(4 + f) * L::PP];
        } else if (STAGE == 4) {
#pragma unroll
          for (int f = 0; f < 4; ++f) Av[f] = sg[(size_t)f * L::PP];
        }
        if (ph.mask) chiv = sg[(size_t)(nstg - 1) * L::PP];
      } else {
        if (STAGE == 2 || STAGE == 3) {
#pragma unroll
          for (int f = 0; f < 4; ++f) Uv[f] = a.U[bo + (size_t)f * L::FS + pi];
        }
        if (STAGE != 1) {
#pragma unroll
          for (int f = 0; f < 4; ++f) Av[f] = a.acc[bo + (size_t)f * L::FS + pi];
        }
        if (ph.mask) chiv = a.chi[(size_t)slot * L::FS + pi];
      }

      T dx[4], dy[4], dz[4], lap[3];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T* s = B[f];
        const T c = q[f][3];
        const T xp1 = s[ci + 1], xm1 = s[ci - 1], xp2 = s[ci + 2], xm2 = s[ci - 2];
        const T xp3 = s[ci + 3], xm3 = s[ci - 3];
        const T yp1 = s[ci + W], ym1 = s[ci - W], yp2 = s[ci + 2 * W], ym2 = s[ci - 2 * W];
        const T yp3 = s[ci + 3 * W], ym3 = s[ci - 3 * W];
        // h dx, h dy, h dz and 12 h^2 lap (the spacing factors are applied in K below)
        dx[f] = kc.a1 * (xp1 - xm1) + kc.a2 * (xp2 - xm2) + kc.a3 * (xp3 - xm3);
        dy[f] = kc.a1 * (yp1 - ym1) + kc.a2 * (yp2 - ym2) + kc.a3 * (yp3 - ym3);
        dz[f] = kc.a1 * (q[f][4] - q[f][2]) + kc.a2 * (q[f][5] - q[f][1]) + kc.a3 * (q[f][6] - q[f][0]);
        if (f < 3) {
          const T lx = T(16) * (xp1 + xm1) - (xp2 + xm2) - T(30) * c;
          const T ly = T(16) * (yp1 + ym1) - (yp2 + ym2) - T(30) * c;
          const T lz = T(16) * (q[f][4] + q[f][2]) - (q[f][5] + q[f][1]) - T(30) * c;
          lap[f] = lx + ly + lz;
        }
      }
      const T u = q[0][3], v = q[1][3], w = q[2][3], p = q[3][3];
      T K[4];
      K[0] = -(u * dx[0] + v * dy[0] + w * dz[0] + dx[3]) * ih + nu_ih2 * lap[0];
      K[1] = -(u * dx[1] + v * dy[1] + w * dz[1] + dy[3]) * ih + nu_ih2 * lap[1];
      K[2] = -(u * dx[2] + v * dy[2] + w * dz[2] + dz[3]) * ih + nu_ih2 * lap[2];
      K[3] = -c0sq_ih * (dx[0] + dy[1] + dz[2]) - kc.cgam * p;
      if (ph.mask) {
        const T cm = chiv * kc.inv_ceta;
        K[0] -= cm * u;
        K[1] -= cm * v;
        K[2] -= cm * w;
      }
      if (ph.sponge) {
        const T cs = tmax(sp_xy, sp[2][z]) * kc.inv_csp;
        K[0] -= cs * (u - kc.uinf[0]);
        K[1] -= cs * (v - kc.uinf[1]);
        K[2] -= cs * (w - kc.uinf[2]);
        K[3] -= cs * (p - kc.pinf);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const size_t o = bo + (size_t)f * L::FS + pi;
        if (STAGE == 0) {
          a.acc[o] = K[f];
        } else if (STAGE == 1) {
          a.acc[o] = q[f][3] + c_acc * K[f];
          a.out[o] = q[f][3] + c_out * K[f];
        } else if (STAGE == 4) {
          const T nv = Av[f] + c_out * K[f];
          a.out[o] = nv;
          const T av = nv < T(0) ? -nv : nv;
          nm[f] = av > nm[f] ? av : nm[f];
          Uv[f] = nv;
        } else {
          a.acc[o] = Av[f] + c_acc * K[f];
          a.out[o] = Uv[f] + c_out * K[f];
        }
      }
      if (STAGE == 4) {
        const T m2 = mag2(Uv[0], Uv[1], Uv[2]);
        nm[4] = m2 > nm[4] ? m2 : nm[4];
      }
    }
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int k = 0; k < 7; ++k) q[f][k] = q[f][k + 1];
  }
  if (STAGE == 4 && a.norms) {
    // block maxima (buf is free now), then one atomic maximum per norm and block
    __syncthreads();
    T* red = &buf[0][0][0];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      T m = nm[k];
      for (int o = 16; o > 0; o >>= 1) {
        const T t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
      }
      if ((tid & 31) == 0) red[k * (NT / 32) + (tid >> 5)] = m;
    }
    __syncthreads();
    if (tid < 5) {
      T m = T(0);
      for (int w = 0; w < NT / 32; ++w) m = red[tid * (NT / 32) + w] > m ? red[tid * (NT / 32) + w] : m;
      const double d = tid == 4 ? (double)tsqrt(m) : (double)m;
      atomicMax(a.norms + tid, (unsigned long long)__double_as_longlong(d));
    }
  }
}

template <typename T, int BS, int STAGE, bool TMA = false, int RYT = 0>
__global__ void __launch_bounds__(Cfg<T, BS, RYT>::NT, Cfg<T, BS, RYT>::MINB)
k_stage(const StageK<T> a, const TopoK tp, const PhysK ph, int* err) {
  const StagePtrs<T> p{a.in, a.U, a.acc, a.out, a.chi, a.slab, a.norms, a.coefp};
  constexpr int NS = Cfg<T, BS, RYT>::NS;
  stage_block<T, BS, STAGE, TMA, RYT>(p, a.kc, tp, ph, err, blockIdx.x / NS, blockIdx.x % NS);
}

// Persistent form over several independent instances: the CTAs walk the work list of
// (instance, rank) pairs, each instance with its own arrays and topology (desc) and the same
// physics and constants; every block gets bitwise the update k_stage gives it.
template <typename T, int BS, int STAGE, int RYT = 0>
__global__ void __launch_bounds__(Cfg<T, BS, RYT>::NT, Cfg<T, BS, RYT>::MINB)
k_stage_multi(const StageConst<T> kc, const PhysK ph, const StageInst<T>* desc, const int2* work, int nwork,
              int* err) {
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 it = work[w];
    const StageInst<T> d = desc[it.x];
    stage_block<T, BS, STAGE, false>(d.p, kc, d.tp, ph, err, it.y, 0);
    __syncthreads();                   // the next block reuses the shared arrays
  }
}

// Time step of one RK4 step on the device (Sec. 2.3): dt_fixed if > 0, else the CFL rule from the
// velocity max norm of the last reduction (maxbits[4]); writes rk[0] = dt, rk[1] += dt (time)
// and the stage coefficients rk[2..9] = (c_acc, c_out) of stages 1..4, in double, by the same
// expressions as the host path.
__global__ void k_rk_coefs(const unsigned long long* maxbits, RkK p, double* rk) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double dt = p.dt_fixed;
  if (!(dt > 0.0)) {
    const double u = __longlong_as_double((long long)maxbits[4]);
    const double ueig = fabs(u) + sqrt(u * u + p.c0 * p.c0);
    dt = p.cfl * p.h / ueig;
    if (p.mask) dt = fmin(dt, p.cfl_eta * p.C_eta);
    if (p.nu > 0) dt = fmin(dt, p.cfl_nu * p.h * p.h / p.nu);
  }
  rk[0] = dt;
  rk[1] += dt;
  rk[2] = dt / 6.0; rk[3] = dt / 2.0;
  rk[4] = dt / 3.0; rk[5] = dt / 2.0;
  rk[6] = dt / 3.0; rk[7] = dt;
  rk[8] = dt / 3.0; rk[9] = dt / 6.0;
}

template <typename T, int BS, int STAGE, bool TMA, int RYT = 0>
void launch_one(const StageK<T>& s, const TopoK& t, const PhysK& p, int* err, cudaStream_t st) {
  const dim3 grid((unsigned)(t.n * Cfg<T, BS, RYT>::NS)), block(Cfg<T, BS, RYT>::NT);
  const size_t dyn = TMA ? (size_t)2 * staged_planes<STAGE>(p.mask != 0) * Lay<T, BS>::PP * sizeof(T) : 0;
  if (TMA) {
    // the ring comes on top of the kernel's static shared memory: opt in to its largest size
    static std::atomic<unsigned long long> opted{0};
    smem_opt_in_stage(k_stage<T, BS, STAGE, TMA, RYT>, (size_t)2 * staged_planes<STAGE>(true) * Lay<T, BS>::PP * sizeof(T),
                      opted);
  }
  k_stage<T, BS, STAGE, TMA, RYT><<<grid, block, dyn, st>>>(s, t, p, err);
}

template <typename T, int BS, bool TMA, int RYT = 0>
void launch_stage_bs(int stage, const StageK<T>& s, const TopoK& t, const PhysK& p, int* err, cudaStream_t st) {
  if (t.n <= 0) return;
  switch (stage) {
    case 0: launch_one<T, BS, 0, TMA, RYT>(s, t, p, err, st); break;
    case 1: launch_one<T, BS, 1, TMA, RYT>(s, t, p, err, st); break;
    case 2: launch_one<T, BS, 2, TMA, RYT>(s, t, p, err, st); break;
    case 3: launch_one<T, BS, 3, TMA, RYT>(s, t, p, err, st); break;
    default: launch_one<T, BS, 4, TMA, RYT>(s, t, p, err, st); break;
  }
}

}  // namespace

template <typename T>
StageConst<T> stage_constants(const PhysK& p, double c_acc, double c_out) {
  StageConst<T> c{};
  c.a1 = T(p.a1); c.a2 = T(p.a2); c.a3 = T(p.a3);
  c.nu = T(p.nu); c.c0sq = T(p.c0sq); c.cgam = T(p.cgamma);
  c.inv_ceta = T(p.inv_ceta); c.inv_csp = T(p.inv_csp);
  for (int i = 0; i < 3; ++i) c.uinf[i] = T(p.uinf[i]);
  c.pinf = T(p.pinf);
  c.c_acc = T(c_acc); c.c_out = T(c_out);
  for (int J = 0; J <= kMaxLevel; ++J) {
    c.ih[J] = T(1.0 / p.h[J]);
    c.ih2[J] = T(1.0 / (12.0 * p.h[J] * p.h[J]));
  }
  return c;
}

template <typename T>
void launch_stage_multi(int stage, int Bs, const PhysK& p, const StageInst<T>* desc, const int2* work, int64_t nwork,
                        int ctas, int* err, cudaStream_t st) {
  if (nwork <= 0 || Bs == 33) return;     // the persistent form takes whole blocks (Bs <= 17)
  const StageConst<T> kc = stage_constants<T>(p, 0.0, 0.0);
  const int nb = (int)std::min<int64_t>(nwork, (int64_t)std::max(ctas, 1));
  auto go = [&](auto kern, int nt) { kern<<<nb, nt, 0, st>>>(kc, p, desc, work, (int)nwork, err); };
  if (Bs == 17) {
    constexpr int NT = Cfg<T, 17>::NT;
    switch (stage) {
      case 1: go(k_stage_multi<T, 17, 1>, NT); break;
      case 2: go(k_stage_multi<T, 17, 2>, NT); break;
      case 3: go(k_stage_multi<T, 17, 3>, NT); break;
      default: go(k_stage_multi<T, 17, 4>, NT); break;
    }
  } else {
    constexpr int NT = Cfg<T, 9>::NT;
    switch (stage) {
      case 1: go(k_stage_multi<T, 9, 1>, NT); break;
      case 2: go(k_stage_multi<T, 9, 2>, NT); break;
      case 3: go(k_stage_multi<T, 9, 3>, NT); break;
      default: go(k_stage_multi<T, 9, 4>, NT); break;
    }
  }
}

template <typename T>
void launch_stage(int stage, int Bs, const StageK<T>& s, const TopoK& t, const PhysK& p, int* err,
                  cudaStream_t st, int variant) {
  if constexpr (sizeof(T) == 4) {
    if (variant == kStagePair && Bs != 33) {
      launch_stage_pair(stage, Bs, s, t, p, st);
      return;
    }
  }
  StageK<T> a = s;
  a.kc = stage_constants<T>(p, s.c_acc, s.c_out);
  if constexpr (sizeof(T) == 4) {
    if (Bs == 33) {              // the point form, rows split over three CTAs (or four of 9 rows)
      if (variant == kStagePointRows) launch_stage_bs<T, 33, false, 9>(stage, a, t, p, err, st);
      else launch_stage_bs<T, 33, false>(stage, a, t, p, err, st);
      return;
    }
    if (variant == kStagePointRows && Bs == 17) {   // a block over two CTAs of 9 and 8 rows
      launch_stage_bs<T, 17, false, 9>(stage, a, t, p, err, st);
      return;
    }
    if (variant == kStagePointTMA) {
      if (Bs == 17) launch_stage_bs<T, 17, true>(stage, a, t, p, err, st);
      else launch_stage_bs<T, 9, true>(stage, a, t, p, err, st);
      return;
    }
  }
  if (Bs == 17) launch_stage_bs<T, 17, false>(stage, a, t, p, err, st);
  else launch_stage_bs<T, 9, false>(stage, a, t, p, err, st);
}

void launch_rk_coefs(const unsigned long long* maxbits, const RkK& p, double* rk, cudaStream_t st) {
  k_rk_coefs<<<1, 32, 0, st>>>(maxbits, p, rk);
}

template void launch_stage<float>(int, int, const StageK<float>&, const TopoK&, const PhysK&, int*, cudaStream_t, int);
template void launch_stage_multi<float>(int, int, const PhysK&, const StageInst<float>*, const int2*, int64_t, int, int*,
                                        cudaStream_t);
template void launch_stage_multi<double>(int, int, const PhysK&, const StageInst<double>*, const int2*, int64_t, int,
                                         int*, cudaStream_t);
template void launch_stage<double>(int, int, const StageK<double>&, const TopoK&, const PhysK&, int*, cudaStream_t, int);

}  // namespace acm
