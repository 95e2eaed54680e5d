// Fused right-hand side + RK4 stage kernel for FP32 fields: two points per thread, packed
// FP32x2 arithmetic (the hot path of libacm in FP32).
//
// Same update as the one-point kernel of stage.cu.  Paper, eqs. (u_eqn-1, p_eqn-1):
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
// Work layout: one CTA per block; thread t < NPR * Bs owns the x-adjacent points (x0, x0 + 1),
// x0 = 2 (t mod NPR), y = t / NPR, NPR = (Bs + 1) / 2, of every z-plane and marches in z.  Bs
// is odd, so the last pair of a row holds x = M and a dummy lane: it reads valid data (the
// point x = M again from global memory) and its results are never stored.  Both points go
// through one instruction stream of packed FP32x2 operations (add/mul/fma .rn.f32x2), which are
// lane by lane the IEEE operations of a scalar evaluation in a fixed order: a point's value
// does not depend on its lane, its thread or its block, so redundant face points of same-level
// neighbours stay bitwise equal.
//
// Data movement per plane z:
//   * the z-stencil (7 planes) lives in a register ring of 8 plane pairs per component, fed
//     from global memory four planes ahead (z + 4); the loop over z is unrolled by 8 so that
//     ring positions are compile-time register names (no shifting);
//   * the x/y stencils read a shared-memory plane (3 halo rows, 4 columns on each side; row
//     pitch W even, W/2 = NPR mod 16, so a warp's 8-byte reads of pairs hit 16 distinct bank
//     pairs per half-warp), double-buffered; its halo values arrive by cp.async one plane
//     ahead straight from the neighbours' stored interiors (same level: copy; finer:
//     decimation, Sec. 3.1 restriction) or from the coarse-face halo slab of this stage;
//   * the planes two iterations ahead are requested into L2 with one bulk prefetch per array.
// No ghost layer is written to HBM.
#include "stage_common.cuh"

namespace acm {

namespace {

// Smallest even row pitch >= Bs + 8 columns (x = -4 .. M + 4) with (W / 2) mod 16 = NPR mod 16.
constexpr int pair_pitch(int BS) {
  const int npr = (BS + 1) / 2;
  int w2 = (BS + 9) / 2;
  while (w2 % 16 != npr % 16) ++w2;
  return 2 * w2;
}

template <int BS>
struct PCfg {
  static constexpr int M = BS - 1;
  static constexpr int NPR = (BS + 1) / 2;           // pairs per row
  static constexpr int NACT = NPR * BS;              // threads that own a pair
  static constexpr int NT = ((NACT + 31) / 32) * 32;
  static constexpr int R = BS + 6;                   // plane rows y = -3 .. M + 3
  static constexpr int W = pair_pitch(BS);           // row pitch (floats)
  static constexpr int PW = R * W;                   // one component's plane
  static constexpr int NH = 48 * BS;                 // x/y halo values per plane
  static constexpr int HPT = (NH + NT - 1) / NT;     // halo values per thread
  static constexpr int MINB = BS <= 17 ? 3 : 1;      // resident CTAs per SM the kernel is built for
  static constexpr size_t BUF_BYTES = (size_t)2 * 4 * PW * sizeof(float);
  static constexpr size_t bytes = BUF_BYTES + (size_t)NH * (8 + 8 + 4);
  static_assert(4 * PW < 0x8000, "plane buffer offsets must fit 15 bits");
};

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float keep_max(float a, float m) { return (a > m || a != a) ? a : m; }

template <int BS, int STAGE>
__global__ void __launch_bounds__(PCfg<BS>::NT, PCfg<BS>::MINB)
k_stage_pair(const StageK<float> a, const PairConst pc, const TopoK tp, const PhysK ph) {
  using L = Lay<float, BS>;
  using C = PCfg<BS>;
  constexpr int M = C::M;
  constexpr int NT = C::NT;
  constexpr int W = C::W;
  constexpr int PW = C::PW;
  constexpr int NH = C::NH;
  constexpr int HPT = C::HPT;

  extern __shared__ __align__(16) unsigned char smem[];
  float* buf = reinterpret_cast<float*>(smem);                               // [2][4][PW]
  unsigned long long* alo = reinterpret_cast<unsigned long long*>(smem + C::BUF_BYTES);   // [NH]
  unsigned long long* ahi = alo + NH;                                        // [NH]
  unsigned* hzd = reinterpret_cast<unsigned*>(ahi + NH);                     // [NH]
  __shared__ int ftype[6];
  __shared__ int fs[6][4];
  __shared__ float sp[3][BS];

  const int tid = threadIdx.x;
  const int slot = tp.blist[blockIdx.x];
  const int4 bi = tp.binfo[blockIdx.x];
  const int* nbh = tp.nbh + (size_t)blockIdx.x * kNbhStride;

  stage_faces(tid, nbh, tp.slabidx, blockIdx.x, ftype, fs);
  stage_sponge<float, BS>(tid, ph, bi, sp);
  // plane cells that no halo copy writes (corners, the dummy lane's outer columns) read as 0
  for (int i = tid; i < 2 * 4 * PW; i += NT) buf[i] = 0.f;
  __syncthreads();

  const float ih = pc.ih[bi.x];
  const float2 mih = make_float2(-ih, -ih);                                   // -1/h
  const float2 nu_ih2 = make_float2(pc.nu * pc.ih2[bi.x], pc.nu * pc.ih2[bi.x]);
  const float2 mc0sq_ih = make_float2(-pc.c0sq * ih, -pc.c0sq * ih);
  float c_acc = pc.c_acc, c_out = pc.c_out;
  if (STAGE >= 1 && a.coefp) {
    c_acc = float(a.coefp[2 * (STAGE - 1)]);
    c_out = float(a.coefp[2 * (STAGE - 1) + 1]);
  }
  const float2 cacc2 = make_float2(c_acc, c_acc), cout2 = make_float2(c_out, c_out);

  const bool act = tid < C::NACT;
  const int y = act ? tid / C::NPR : 0;
  const int x0 = act ? 2 * (tid % C::NPR) : 0;
  const bool two = x0 < M;                 // false: the second lane is the dummy
  const int x1 = two ? x0 + 1 : x0;        // the dummy re-reads x = M
  const float* __restrict__ inb = a.in + (size_t)slot * L::BLK;
  const size_t bo = (size_t)slot * L::BLK;
  const int ci = (y + 3) * W + x0 + 4;     // this pair in the plane buffer (even)

  // pair of plane zz of component f (z-halo planes from the z-face neighbours)
  auto own_pair = [&](int zz, int f) -> float2 {
    if (zz >= 0 && zz <= M) {
      const float* p = inb + (size_t)f * L::FS + (size_t)zz * L::PP + y * BS;
      return make_float2(p[x0], p[x1]);
    }
    const int F = zz < 0 ? 4 : 5, l = zz < 0 ? -zz : zz - M;
    return make_float2(*halo_ptr<float, BS>(ftype, fs, a.in, a.slab, F, l, x0, y, f),
                       *halo_ptr<float, BS>(ftype, fs, a.in, a.slab, F, l, x1, y, f));
  };

  // x/y halo values of every plane as affine functions of z: entry i (component f, face F,
  // layer l, tangential t) of plane z is read from alo[i] (z <= M/2) or ahi[i] (z > M/2, the
  // upper child of a finer face) plus z * stride elements and lands at dst of the plane
  // buffer: hzd = stride << 16 | dst.  Thread tid owns entries tid + k NT.
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    const int i = tid + k * NT;
    if (i < NH) {
      const int g = i / (3 * BS), el = i % (3 * BS);
      const int F = g & 3, f = g >> 2;
      int l, t;
      // x-faces take the 3 layers of a row as consecutive entries, y-faces a row
      if (F < 2) { l = el % 3 + 1; t = el / 3; }
      else { t = el % BS; l = el / BS + 1; }
      int hx, hy;
      if (F == 0) { hx = -l; hy = t; }
      else if (F == 1) { hx = M + l; hy = t; }
      else if (F == 2) { hx = t; hy = -l; }
      else { hx = t; hy = M + l; }
      const unsigned dst = (unsigned)(f * PW + (hy + 3) * W + hx + 4);
      const int ty = ftype[F];
      const bool plus = F & 1;
      const int ax = F >> 1;
      const float *lo, *hi;
      unsigned stride;
      if (ty == kTypeCoarser) {
        lo = hi = a.slab + (((size_t)fs[F][0] * 4 + f) * 3 + (l - 1)) * BS * BS + t;
        stride = BS;
      } else if (ty == kTypeLeaf) {
        const int nl = plus ? l : M - l;
        const int xx = ax == 0 ? nl : t, yy = ax == 0 ? t : nl;
        lo = hi = a.in + (size_t)fs[F][0] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0);
        stride = L::PP;
      } else {
        const int c0 = t > M / 2;
        const int nl = plus ? 2 * l : M - 2 * l;
        const int u0 = 2 * t - c0 * M;
        const int xx = ax == 0 ? nl : u0, yy = ax == 0 ? u0 : nl;
        lo = a.in + (size_t)fs[F][c0] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0);
        // upper child: its plane 2z - M is at (2z - M) PP from its base
        hi = a.in + (size_t)fs[F][c0 + 2] * L::BLK + (size_t)f * L::FS + L::idx(xx, yy, 0) - (ptrdiff_t)M * L::PP;
        stride = 2 * L::PP;
      }
      alo[i] = reinterpret_cast<unsigned long long>(lo);
      ahi[i] = reinterpret_cast<unsigned long long>(hi);
      hzd[i] = (stride << 16) | dst;
    }
  }
  __syncthreads();
  auto issue_halos = [&](int zz, float* B) {
    const unsigned long long* A = zz > M / 2 ? ahi : alo;
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
      const int i = tid + k * NT;
      if (i < NH) {
        const unsigned zd = hzd[i];
        const float* src = reinterpret_cast<const float*>(A[i]) + (size_t)zz * (zd >> 16);
        cp_async_elem(B + (zd & 0x7fffu), src);
      }
    }
    cp_async_commit();
  };

  float nm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // stage 4: max |u|,|v|,|w|,|p|, |(u,v,w)|^2
  constexpr int kPf = 2;
  constexpr unsigned kPlaneBytes = (unsigned)(L::PP * sizeof(float));
  auto prefetch_planes = [&](int zin, int zo) {
    if (tid < 4) {
      if (zin <= M) prefetch_l2(inb + (size_t)tid * L::FS + (size_t)zin * L::PP, kPlaneBytes);
    } else if (tid < 8) {
      if ((STAGE == 2 || STAGE == 3) && zo <= M)
        prefetch_l2(a.U + bo + (size_t)(tid - 4) * L::FS + (size_t)zo * L::PP, kPlaneBytes);
    } else if (tid < 12) {
      if (STAGE >= 2 && zo <= M) prefetch_l2(a.acc + bo + (size_t)(tid - 8) * L::FS + (size_t)zo * L::PP, kPlaneBytes);
    } else if (tid == 12) {
      if (ph.mask && zo <= M) prefetch_l2(a.chi + (size_t)slot * L::FS + (size_t)zo * L::PP, kPlaneBytes);
    }
  };
  for (int k = 0; k < kPf; ++k) prefetch_planes(4 + k, k);

  // register ring: q[f][(zz + 3) & 7] holds plane zz
  float2 q[4][8];
#pragma unroll
  for (int k = 0; k < 7; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f) q[f][k] = act ? own_pair(k - 3, f) : make_float2(0.f, 0.f);
#pragma unroll
  for (int f = 0; f < 4; ++f) q[f][7] = make_float2(0.f, 0.f);
  issue_halos(0, buf);

  float2 sp_xy = make_float2(0.f, 0.f);        // the sponge profile's x/y part
  if (ph.sponge) sp_xy = make_float2(fmaxf(sp[0][x0], sp[1][y]), fmaxf(sp[0][x1], sp[1][y]));

#pragma unroll 1
  for (int z0 = 0; z0 <= M; z0 += 8) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int z = z0 + j;
      if (z > M) break;
      float* B = buf + (j & 1) * 4 * PW;
#define QR(f, k) q[f][(j + 3 + (k)) & 7]
      if (act) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (two) *reinterpret_cast<float2*>(B + f * PW + ci) = QR(f, 0);
          else B[f * PW + ci] = QR(f, 0).x;
        }
      }
      cp_async_wait_all();
      __syncthreads();
      if (z < M) issue_halos(z + 1, buf + ((j + 1) & 1) * 4 * PW);
      prefetch_planes(z + 4 + kPf, z + kPf);
      if (act) {
        if (z + 4 <= M + 3) {
#pragma unroll
          for (int f = 0; f < 4; ++f) QR(f, 4) = own_pair(z + 4, f);
        }
        const size_t pz = (size_t)z * L::PP + y * BS;
        float2 Uv[4], Av[4], chiv = make_float2(0.f, 0.f);
        if (STAGE == 2 || STAGE == 3) {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const float* p = a.U + bo + (size_t)f * L::FS + pz;
            Uv[f] = make_float2(p[x0], p[x1]);
          }
        }
        if (STAGE >= 2) {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            const float* p = a.acc + bo + (size_t)f * L::FS + pz;
            Av[f] = make_float2(p[x0], p[x1]);
          }
        }
        if (ph.mask) {
          const float* p = a.chi + (size_t)slot * L::FS + pz;
          chiv = make_float2(p[x0], p[x1]);
        }

        // The right-hand side is accumulated component by component, so that only one
        // component's derivatives are live at a time: for velocity component i,
        // T_i = u h d_x u_i + v h d_y u_i + w h d_z u_i and L_i = 12 h^2 lap u_i; the pressure
        // then adds h d_i p to T_i; div = h (d_x u + d_y v + d_z w).  (Spacing factors are
        // applied once per term.)
        const float2 u = QR(0, 0), v = QR(1, 0), w = QR(2, 0), p = QR(3, 0);
        float2 T[3], Lp[3], div;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float* s = B + f * PW + ci;
          const float2 c = QR(f, 0);
          const float2 Am = ld2(s - 2), Ap = ld2(s + 2);       // x0-2, x0-1 | x0+2, x0+3
          const float em = s[-3], ep = s[4];                   // x0-3 | x0+4
          // x0 + 1 from the plane: the second point, or for the last pair of a row the halo
          // value at x = M + 1 (the dummy lane's own value is a copy of x = M)
          const float cr = s[1];
          // right minus left neighbour at distance 1, 2, 3, lane by lane
          const float2 d1x = make_float2(cr - Am.y, Ap.x - c.x);
          const float2 d2x = psub(Ap, Am);
          const float2 d3x = make_float2(Ap.y - em, ep - Am.x);
          const float2 yp1 = ld2(s + W), ym1 = ld2(s - W), yp2 = ld2(s + 2 * W), ym2 = ld2(s - 2 * W);
          const float2 yp3 = ld2(s + 3 * W), ym3 = ld2(s - 3 * W);
          const float2 dx = pfma(pc.a1, d1x, pfma(pc.a2, d2x, pmul(pc.a3, d3x)));
          const float2 dy = pfma(pc.a1, psub(yp1, ym1), pfma(pc.a2, psub(yp2, ym2), pmul(pc.a3, psub(yp3, ym3))));
          const float2 dz = pfma(pc.a1, psub(QR(f, 1), QR(f, -1)),
                                 pfma(pc.a2, psub(QR(f, 2), QR(f, -2)), pmul(pc.a3, psub(QR(f, 3), QR(f, -3)))));
          if (f < 3) {
            T[f] = pfma(w, dz, pfma(v, dy, pmul(u, dx)));
            // 16 (sum of the six distance-1 neighbours) - (sum of the six at distance 2) - 90 c
            const float2 s1x = make_float2(cr + Am.y, Ap.x + c.x);
            const float2 s2x = padd(Ap, Am);
            const float2 S1 = padd(padd(s1x, padd(yp1, ym1)), padd(QR(f, 1), QR(f, -1)));
            const float2 S2 = padd(padd(s2x, padd(yp2, ym2)), padd(QR(f, 2), QR(f, -2)));
            Lp[f] = psub(pfma(pc.k16, S1, pmul(pc.km90, c)), S2);
            const float2 dd = f == 0 ? dx : (f == 1 ? dy : dz);
            div = f == 0 ? dd : padd(div, dd);
          } else {
            T[0] = padd(T[0], dx);
            T[1] = padd(T[1], dy);
            T[2] = padd(T[2], dz);
          }
        }
        float2 K[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) K[i] = pfma(nu_ih2, Lp[i], pmul(mih, T[i]));
        K[3] = pfma(mc0sq_ih, div, pmul(pc.mcgam, p));
        if (ph.mask) {
          const float2 cm = pmul(chiv, pc.minv_ceta);
          K[0] = pfma(cm, u, K[0]);
          K[1] = pfma(cm, v, K[1]);
          K[2] = pfma(cm, w, K[2]);
        }
        if (ph.sponge) {
          const float spz = sp[2][z];
          const float2 cs = pmul(make_float2(fmaxf(sp_xy.x, spz), fmaxf(sp_xy.y, spz)), pc.minv_csp);
          K[0] = pfma(cs, psub(u, pc.uinf0), K[0]);
          K[1] = pfma(cs, psub(v, pc.uinf1), K[1]);
          K[2] = pfma(cs, psub(w, pc.uinf2), K[2]);
          K[3] = pfma(cs, psub(p, pc.pinf), K[3]);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const size_t o = bo + (size_t)f * L::FS + pz;
          float2 r_acc, r_out;
          if (STAGE == 0) {
            r_acc = K[f];
          } else if (STAGE == 1) {
            r_acc = pfma(cacc2, K[f], QR(f, 0));
            r_out = pfma(cout2, K[f], QR(f, 0));
          } else if (STAGE == 4) {
            r_out = pfma(cout2, K[f], Av[f]);
            nm[f] = keep_max(fabsf(r_out.x), nm[f]);
            if (two) nm[f] = keep_max(fabsf(r_out.y), nm[f]);
            Uv[f] = r_out;
          } else {
            r_acc = pfma(cacc2, K[f], Av[f]);
            r_out = pfma(cout2, K[f], Uv[f]);
          }
          if (STAGE != 4) {
            a.acc[o + x0] = r_acc.x;
            if (two) a.acc[o + x1] = r_acc.y;
          }
          if (STAGE != 0) {
            a.out[o + x0] = r_out.x;
            if (two) a.out[o + x1] = r_out.y;
          }
        }
        if (STAGE == 4) {
          nm[4] = keep_max(mag2(Uv[0].x, Uv[1].x, Uv[2].x), nm[4]);
          if (two) nm[4] = keep_max(mag2(Uv[0].y, Uv[1].y, Uv[2].y), nm[4]);
        }
      }
#undef QR
    }
  }
  if (STAGE == 4 && a.norms) {
    // block maxima (the plane buffer is free now), then one atomic maximum per norm and block
    __syncthreads();
    float* red = buf;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float m = nm[k];
      for (int o = 16; o > 0; o >>= 1) m = keep_max(__shfl_xor_sync(0xffffffffu, m, o), m);
      if ((tid & 31) == 0) red[k * (NT / 32) + (tid >> 5)] = m;
    }
    __syncthreads();
    if (tid < 5) {
      float m = 0.f;
      for (int w = 0; w < NT / 32; ++w) m = keep_max(red[tid * (NT / 32) + w], m);
      const double d = tid == 4 ? (double)sqrtf(m) : (double)m;
      atomicMax(a.norms + tid, (unsigned long long)__double_as_longlong(d));
    }
  }
}

template <int BS, int STAGE>
void launch_one(const StageK<float>& s, const PairConst& pc, const TopoK& t, const PhysK& p, cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0};
  smem_opt_in_stage(k_stage_pair<BS, STAGE>, PCfg<BS>::bytes, opted);
  k_stage_pair<BS, STAGE><<<(unsigned)t.n, PCfg<BS>::NT, PCfg<BS>::bytes, st>>>(s, pc, t, p);
}

template <int BS>
void launch_bs(int stage, const StageK<float>& s, const PairConst& pc, const TopoK& t, const PhysK& p,
               cudaStream_t st) {
  switch (stage) {
    case 0: launch_one<BS, 0>(s, pc, t, p, st); break;
    case 1: launch_one<BS, 1>(s, pc, t, p, st); break;
    case 2: launch_one<BS, 2>(s, pc, t, p, st); break;
    case 3: launch_one<BS, 3>(s, pc, t, p, st); break;
    default: launch_one<BS, 4>(s, pc, t, p, st); break;
  }
}

}  // namespace

void launch_stage_pair(int stage, int Bs, const StageK<float>& s, const TopoK& t, const PhysK& p, cudaStream_t st) {
  if (t.n <= 0) return;
  PairConst pc{};
  auto two = [](double v) { return make_float2(float(v), float(v)); };
  pc.a1 = two(p.a1); pc.a2 = two(p.a2); pc.a3 = two(p.a3);
  pc.k16 = two(16.0); pc.km90 = two(-90.0);
  pc.mcgam = two(-p.cgamma);
  pc.minv_ceta = two(-p.inv_ceta); pc.minv_csp = two(-p.inv_csp);
  pc.uinf0 = two(p.uinf[0]); pc.uinf1 = two(p.uinf[1]); pc.uinf2 = two(p.uinf[2]); pc.pinf = two(p.pinf);
  pc.nu = float(p.nu); pc.c0sq = float(p.c0sq);
  pc.c_acc = float(s.c_acc); pc.c_out = float(s.c_out);
  for (int J = 0; J <= kMaxLevel; ++J) {
    pc.ih[J] = float(1.0 / p.h[J]);
    pc.ih2[J] = float(1.0 / (12.0 * p.h[J] * p.h[J]));
  }
  if (Bs == 17) launch_bs<17>(stage, s, pc, t, p, st);
  else if (Bs == 33) launch_bs<33>(stage, s, pc, t, p, st);
  else launch_bs<9>(stage, s, pc, t, p, st);
}

}  // namespace acm
