// Synchronisation, wavelet-detail, adaptation and diagnostic kernels of libacm.
//
// Paper: Sec. 3.1 (DD-4 prediction, decimation, details u - P R u), Sec. 3.3-3.4 (block
// indicator: largest detail normalised per component by its global max norm), Sec. 3.5
// (refine by prediction, coarsen by merging sister blocks), Sec. 4.2 (ghost synchronisation:
// restrict or predict, then copy), Sec. 2.2 (smoothed mask, force by midpoint rule).
#include "common.cuh"
#include "kernels.hpp"

namespace acm {

namespace {

constexpr int kNT = 256;

template <typename T>
__device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }

// Gather n values v(i) into dst[i] with U independent loads in flight per thread.
template <typename T, int U, typename F>
__device__ __forceinline__ void gather(T* dst, int n, F&& val) {
  for (int base = threadIdx.x; base < n; base += kNT * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * kNT;
      v[u] = i < n ? val(i) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * kNT;
      if (i < n) dst[i] = v[u];
    }
  }
}

// ---- (1) fine wins: block boundary points held by a finer neighbour take its value -----------
// task = (rank, box index d of a REFINED neighbour box).  Points of the block's boundary lying
// in box d: coordinate 0 / M where d is -1 / +1, the whole range where d is 0.
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_fine_wins(T* reg, const int2* tasks, const int32_t* nbh_all,
                                                    const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int2 tk = tasks[blockIdx.x];
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
  for (int i = threadIdx.x; i < tot; i += kNT) {
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
    for (int f = 0; f < 4; ++f)
      reg[(size_t)me * L::BLK + (size_t)f * L::FS + L::idx(p[0], p[1], p[2])] =
          reg[(size_t)s * L::BLK + (size_t)f * L::FS + L::idx(l[0], l[1], l[2])];
  }
}

// ---- (2) coarse-face halo slabs ------------------------------------------------------------------
// task = (rank, face F, slab index, -); one CTA per (task, component).  The 3 x Bs x Bs halo
// points beyond face F take the value of the finest leaf holding them, else the tensor DD-4
// prediction from the coarse lattice (Sec. 3.1).  Only points on the face's tangential boundary
// lines (t0 or t1 = 0 or M) can be held by a leaf of the block's level or finer; all others lie
// in the coarser leaf alone.  The coarse patch the predictions need (even local coordinates
// [M-2, M+6] or [-6, 2] across the face, [-2, M+2] along it) is gathered once, then predicted
// separably: along t0, then t1, then across the face (a fixed order per face orientation, so
// every block that needs a halo point gets bitwise the same value).
// Slab layout [slab][comp][layer l-1][t1][t0] with (t0, t1) as in the stage kernel.
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_coarse_slabs(const T* reg, T* slab, const int4* tasks,
                                                       const int32_t* nbh_all) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  constexpr int NC = M / 2 + 3;                     // coarse samples along the face: -2..M+2 step 2
  constexpr int NN = 5;                             // coarse planes across the face
  __shared__ int nbh[kNbhStride];
  __shared__ T P[NN][NC][NC];                       // [n][t1 coarse][t0 coarse]
  __shared__ T A[NN][NC][BS];                       // predicted along t0
  __shared__ T B[NN][BS][BS];                       // predicted along t0 and t1
  const int4 tk = tasks[blockIdx.x >> 2];
  const int f = blockIdx.x & 3;
  for (int i = threadIdx.x; i < kNbhStride; i += kNT) nbh[i] = nbh_all[(size_t)tk.x * kNbhStride + i];
  __syncthreads();
  const int F = tk.y, ax = F >> 1;
  const bool plus = F & 1;
  const int n0 = plus ? M - 2 : -6;                 // first coarse plane (even local coordinate)
  auto place = [&](int nl, int t0, int t1, int* x, int* y, int* z) {
    if (ax == 0) { *x = nl; *y = t0; *z = t1; }
    else if (ax == 1) { *x = t0; *y = nl; *z = t1; }
    else { *x = t0; *y = t1; *z = nl; }
  };
  const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  gather<T, 4>(&P[0][0][0], NN * NC * NC, [&](int i) {
    const int a0 = i % NC, a1 = (i / NC) % NC, an = i / (NC * NC);
    int x, y, z;
    place(n0 + 2 * an, 2 * a0 - 2, 2 * a1 - 2, &x, &y, &z);
    T v;
    if (!direct_value<T, BS>(reg, nbh, x, y, z, f, &v)) v = T(__longlong_as_double(0x7ff8000000000000ll));
    return v;
  });
  __syncthreads();
  for (int i = threadIdx.x; i < NN * NC * BS; i += kNT) {
    const int t0 = i % BS, a1 = (i / BS) % NC, an = i / (BS * NC);
    T acc = T(0);
    if (t0 & 1) {
      const int c = (t0 - 3 + 2) >> 1;              // coarse index of t0 - 3
      for (int k = 0; k < 4; ++k) acc = acc + w[k] * P[an][a1][c + k];
    } else {
      acc = P[an][a1][(t0 + 2) >> 1];
    }
    A[an][a1][t0] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NN * BS * BS; i += kNT) {
    const int t0 = i % BS, t1 = (i / BS) % BS, an = i / (BS * BS);
    T acc = T(0);
    if (t1 & 1) {
      const int c = (t1 - 3 + 2) >> 1;
      for (int k = 0; k < 4; ++k) acc = acc + w[k] * A[an][c + k][t0];
    } else {
      acc = A[an][(t1 + 2) >> 1][t0];
    }
    B[an][t1][t0] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * BS * BS; i += kNT) {
    const int t0 = i % BS, t1 = (i / BS) % BS, l = i / (BS * BS) + 1;
    const int nl = plus ? M + l : -l;
    const bool edge = t0 == 0 || t0 == M || t1 == 0 || t1 == M;
    T v;
    bool have = false;
    if (edge) {
      int x, y, z;
      place(nl, t0, t1, &x, &y, &z);
      have = direct_value<T, BS>(reg, nbh, x, y, z, f, &v);
    }
    if (!have) {
      const int c = nl - n0;                        // fine offset from the first coarse plane
      if (c & 1) {
        const int k0 = (c - 3) >> 1;
        v = T(0);
        for (int k = 0; k < 4; ++k) v = v + w[k] * B[k0 + k][t1][t0];
      } else {
        v = B[c >> 1][t1][t0];
      }
    }
    slab[((((size_t)tk.z * 4 + f) * 3 + (l - 1)) * BS + t1) * BS + t0] = v;
  }
}

// ---- (3) extended arrays (interior + g ghost layers) ---------------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_sync_ext(const T* reg, T* out, int g, const int32_t* blist,
                                                   const int32_t* nbh_all, int by_rank) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  __shared__ int nbh[kNbhStride];
  const int slot = blist[blockIdx.x];
  for (int i = threadIdx.x; i < kNbhStride; i += kNT) nbh[i] = nbh_all[(size_t)blockIdx.x * kNbhStride + i];
  __syncthreads();
  const int ne = BS + 2 * g;
  const size_t ne3 = (size_t)ne * ne * ne;
  T* o = out + (size_t)(by_rank ? blockIdx.x : slot) * 4 * ne3;
  const T* me = reg + (size_t)slot * L::BLK;
  for (size_t i = threadIdx.x; i < 4 * ne3; i += kNT) {
    const int f = (int)(i / ne3);
    const int r = (int)(i % ne3);
    const int x = r % ne - g, y = (r / ne) % ne - g, z = r / (ne * ne) - g;
    T v;
    if (x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M)
      v = me[(size_t)f * L::FS + L::idx(x, y, z)];
    else
      v = point_value<T, BS>(reg, nbh, x, y, z, f);
    o[i] = v;
  }
}

// ---- (4) block indicators: details (Sec. 3.1) and mask range ----------------------------------
// The coarse samples are the block's even points, local coordinates -2..M+2 (those outside the
// block are held directly by a neighbour leaf); they are predicted back to every interior point
// separably (x, then y, then z: the tensor DD-4 sum in that nesting) and subtracted.
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_details(const T* reg, const T* chi, const int32_t* blist,
                                                  const int32_t* ranks, const int32_t* nbh_all,
                                                  const unsigned long long* norm_bits, double* ind,
                                                  double* chirange) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  constexpr int NC = M / 2 + 3;                 // coarse samples -1..M/2+1
  constexpr int RA = (NC * NC * NC > NC * BS * BS) ? NC * NC * NC : NC * BS * BS;
  __shared__ int nbh[kNbhStride];
  __shared__ __align__(16) T ra[RA];            // coarse samples c, later the y-pass py
  __shared__ __align__(16) T rb[NC * NC * BS];  // x-pass px
  T(&c)[NC][NC][NC] = *reinterpret_cast<T(*)[NC][NC][NC]>(ra);
  T(&py)[NC][BS][BS] = *reinterpret_cast<T(*)[NC][BS][BS]>(ra);
  T(&px)[NC][NC][BS] = *reinterpret_cast<T(*)[NC][NC][BS]>(rb);
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  for (int i = threadIdx.x; i < kNbhStride; i += kNT) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  double best = 0.0;
  for (int f = 0; f < 4; ++f) {
    // global max norm of component f, as left by the max-norm reduction (non-negative double bits)
    const double nf = __longlong_as_double((long long)norm_bits[f]);
    const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
    if (inv == 0.0) continue;
    T dmax = T(0);      // max |detail| in the field precision; max(|d| inv) = max|d| inv exactly
    __syncthreads();
    gather<T, 4>(ra, NC * NC * NC, [&](int i) {
      const int x = 2 * (i % NC) - 2, y = 2 * ((i / NC) % NC) - 2, z = 2 * (i / (NC * NC)) - 2;
      T v;
      if (x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M)
        v = reg[(size_t)slot * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)];
      else if (!direct_value<T, BS>(reg, nbh, x, y, z, f, &v))
        v = T(__longlong_as_double(0x7ff8000000000000ll));
      return v;
    });
    __syncthreads();
    for (int i = threadIdx.x; i < NC * NC * BS; i += kNT) {
      const int x = i % BS, yc = (i / BS) % NC, zc = i / (BS * NC);
      T acc = T(0);
      if (x & 1) {
        const int k0 = (x - 1) >> 1;            // coarse index of x - 3
        for (int k = 0; k < 4; ++k) acc = acc + w[k] * c[zc][yc][k0 + k];
      } else {
        acc = acc + T(1) * c[zc][yc][(x + 2) >> 1];
      }
      px[zc][yc][x] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NC * BS * BS; i += kNT) {
      const int x = i % BS, y = (i / BS) % BS, zc = i / (BS * BS);
      T acc = T(0);
      if (y & 1) {
        const int k0 = (y - 1) >> 1;
        for (int k = 0; k < 4; ++k) acc = acc + w[k] * px[zc][k0 + k][x];
      } else {
        acc = acc + T(1) * px[zc][(y + 2) >> 1][x];
      }
      py[zc][y][x] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
      const int x = i % BS, y = (i / BS) % BS, z = i / (BS * BS);
      if (((x | y | z) & 1) == 0) continue;          // all-even points: detail is zero
      T acc = T(0);
      if (z & 1) {
        const int k0 = (z - 1) >> 1;
        for (int k = 0; k < 4; ++k) acc = acc + w[k] * py[k0 + k][y][x];
      } else {
        acc = acc + T(1) * py[(z + 2) >> 1][y][x];
      }
      const T dv = tabs(reg[(size_t)slot * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)] - acc);
      dmax = dv > dmax ? dv : dmax;
    }
    const double r = (double)dmax * inv;
    best = r > best ? r : best;
  }
  double cmin = 1e300, cmax = -1e300;
  if (chi) {
    T tmin = T(1e30), tmax = T(-1e30);
    for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
      const int x = i % BS, y = (i / BS) % BS, z = i / (BS * BS);
      const T cv = chi[(size_t)slot * L::FS + L::idx(x, y, z)];
      tmin = cv < tmin ? cv : tmin;
      tmax = cv > tmax ? cv : tmax;
    }
    cmin = (double)tmin;
    cmax = (double)tmax;
  }
  __shared__ double red[3][kNT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    cmin = fmin(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
    cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][wid] = best; red[1][wid] = cmin; red[2][wid] = cmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0, mn = 1e300, mx = -1e300;
    for (int k = 0; k < kNT / 32; ++k) {
      b = fmax(b, red[0][k]);
      mn = fmin(mn, red[1][k]);
      mx = fmax(mx, red[2][k]);
    }
    ind[rank] = b;
    chirange[rank] = chi ? mx - mn : 0.0;
  }
}

// ---- (5) max norms (Sec. 2.3 u_max, Sec. 3.4 normalisation) ------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_maxnorm(const T* reg, const int32_t* blist, unsigned long long* out) {
  using L = Lay<T, BS>;
  const int slot = blist[blockIdx.x];
  const T* b = reg + (size_t)slot * L::BLK;
  // arithmetic in the field precision (an FP32 field gives an FP32 norm, stored as double)
  T m[5] = {T(0), T(0), T(0), T(0), T(0)};
  for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
    const int x = i % BS, y = (i / BS) % BS, z = i / (BS * BS);
    const int pi = L::idx(x, y, z);
    T v[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      v[f] = b[(size_t)f * L::FS + pi];
      const T a = tabs(v[f]);
      m[f] = a > m[f] ? a : m[f];
    }
    const T mag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    m[4] = mag > m[4] ? mag : m[4];
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double mk = (double)m[k];
    for (int o = 16; o > 0; o >>= 1) mk = fmax(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + k, (unsigned long long)__double_as_longlong(mk));
  }
}

// ---- (6) refinement: 8 children predicted from the synchronised parent (Sec. 3.5 step 1) -------
// One CTA per (parent, component); task = [parent rank in the old grid, new slots of children
// 0..7].  src is
// a copy of the state taken before any child is written (children may reuse the parent's slot).
// Per component: the parent's samples over local [-1, M+1]^3 (its ghost layer with the
// finest-leaf rule, else the DD-4 prediction from the even lattice [-4, M+4]) are gathered into
// shared memory once; each child is then predicted separably (x, then y, then z).
// Dynamic shared memory: pp (M+3)^3 + ev/qx + qy, in T.
template <typename T, int BS>
struct RefSmem {
  static constexpr int M = BS - 1;
  static constexpr int NPP = M + 3;                 // parent samples per axis: -1..M+1
  static constexpr int NEV = M / 2 + 5;             // even lattice per axis: -4..M+4
  static constexpr int NP = M / 2 + 3;              // samples per axis one child uses
  static constexpr int PP = NPP * NPP * NPP;
  static constexpr int EQ = (NEV * NEV * NEV > NP * NP * BS) ? NEV * NEV * NEV : NP * NP * BS;
  static constexpr int QY = NP * BS * BS;
  static constexpr size_t bytes = (size_t)(PP + EQ + QY) * sizeof(T) + kNbhStride * sizeof(int);
};

template <typename T, int BS>
__global__ void __launch_bounds__(kNT, 4) k_refine(const T* src, T* dst, const int32_t* tasks, const int32_t* blist,
                                                    const int32_t* nbh_all) {
  using L = Lay<T, BS>;
  using S = RefSmem<T, BS>;
  constexpr int M = L::M, NPP = S::NPP, NEV = S::NEV, NP = S::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pp = reinterpret_cast<T*>(smem_raw);
  T* eq = pp + S::PP;                           // even lattice ev, later the x-pass qx
  T* qy = eq + S::EQ;
  int* nbh = reinterpret_cast<int*>(qy + S::QY);
  const int32_t* tk = tasks + (size_t)(blockIdx.x >> 2) * 9;
  const int f = blockIdx.x & 3;
  const int prank = tk[0];
  const int pslot = blist[prank];
  for (int i = threadIdx.x; i < kNbhStride; i += kNT) nbh[i] = nbh_all[(size_t)prank * kNbhStride + i];
  const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  const int off[4] = {-3, -1, 1, 3};
  auto PPI = [&](int x, int y, int z) { return ((z + 1) * NPP + (y + 1)) * NPP + (x + 1); };
  {
    __syncthreads();
    // even-lattice points -4..M+4 (held directly by some leaf)
    gather<T, 4>(eq, NEV * NEV * NEV, [&](int i) {
      const int x = 2 * (i % NEV) - 4, y = 2 * ((i / NEV) % NEV) - 4, z = 2 * (i / (NEV * NEV)) - 4;
      T v;
      if (x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M)
        v = src[(size_t)pslot * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)];
      else if (!direct_value<T, BS>(src, nbh, x, y, z, f, &v))
        v = T(__longlong_as_double(0x7ff8000000000000ll));
      return v;
    });
    __syncthreads();
    // parent samples: interior, else the finest leaf holding the point, else the tensor DD-4
    // prediction from the even lattice (z outer, then y, then x)
    for (int i = threadIdx.x; i < S::PP; i += kNT) {
      const int x = i % NPP - 1, y = (i / NPP) % NPP - 1, z = i / (NPP * NPP) - 1;
      T v;
      if (x >= 0 && x <= M && y >= 0 && y <= M && z >= 0 && z <= M) {
        v = src[(size_t)pslot * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)];
      } else if (!direct_value<T, BS>(src, nbh, x, y, z, f, &v)) {
        const int p[3] = {x, y, z};
        int cnt[3];
        for (int a = 0; a < 3; ++a) cnt[a] = (p[a] & 1) ? 4 : 1;
        T accz = T(0);
        for (int kz = 0; kz < cnt[2]; ++kz) {
          const int zz = ((cnt[2] == 4 ? z + off[kz] : z) + 4) >> 1;
          T accy = T(0);
          for (int ky = 0; ky < cnt[1]; ++ky) {
            const int yy = ((cnt[1] == 4 ? y + off[ky] : y) + 4) >> 1;
            T accx = T(0);
            for (int kx = 0; kx < cnt[0]; ++kx) {
              const int xx = ((cnt[0] == 4 ? x + off[kx] : x) + 4) >> 1;
              accx = accx + (cnt[0] == 4 ? w[kx] : T(1)) * eq[(zz * NEV + yy) * NEV + xx];
            }
            accy = accy + (cnt[1] == 4 ? w[ky] : T(1)) * accx;
          }
          accz = accz + (cnt[2] == 4 ? w[kz] : T(1)) * accy;
        }
        v = accz;
      }
      pp[i] = v;
    }
    for (int c = 0; c < 8; ++c) {
      const int cb[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
      const int o[3] = {cb[0] * (M / 2) - 1, cb[1] * (M / 2) - 1, cb[2] * (M / 2) - 1};
      T* qx = eq;
      __syncthreads();
      // along x: qx[zz][yy][ix], zz, yy over the child's samples o..o+NP-1
      for (int i = threadIdx.x; i < NP * NP * BS; i += kNT) {
        const int ix = i % BS, yy = (i / BS) % NP, zz = i / (BS * NP);
        const int px = cb[0] * M + ix;             // parent-local fine index (twice the parent index)
        const int y = o[1] + yy, z = o[2] + zz;
        T acc = T(0);
        if (px & 1) {
          for (int k = 0; k < 4; ++k) acc = acc + w[k] * pp[PPI((px + off[k]) / 2, y, z)];
        } else {
          acc = acc + T(1) * pp[PPI(px / 2, y, z)];
        }
        qx[(zz * NP + yy) * BS + ix] = acc;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < NP * BS * BS; i += kNT) {
        const int ix = i % BS, iy = (i / BS) % BS, zz = i / (BS * BS);
        const int py = cb[1] * M + iy;
        T acc = T(0);
        if (py & 1) {
          for (int k = 0; k < 4; ++k) acc = acc + w[k] * qx[(zz * NP + ((py + off[k]) / 2 - o[1])) * BS + ix];
        } else {
          acc = acc + T(1) * qx[(zz * NP + (py / 2 - o[1])) * BS + ix];
        }
        qy[(zz * BS + iy) * BS + ix] = acc;
      }
      __syncthreads();
      T* out = dst + (size_t)tk[1 + c] * L::BLK + (size_t)f * L::FS;
      for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
        const int ix = i % BS, iy = (i / BS) % BS, iz = i / (BS * BS);
        const int pz = cb[2] * M + iz;
        T acc = T(0);
        if (pz & 1) {
          for (int k = 0; k < 4; ++k) acc = acc + w[k] * qy[(((pz + off[k]) / 2 - o[2]) * BS + iy) * BS + ix];
        } else {
          acc = acc + T(1) * qy[((pz / 2 - o[2]) * BS + iy) * BS + ix];
        }
        out[L::idx(ix, iy, iz)] = acc;
      }
    }
  }
}

// ---- (7) coarsening: parent by decimation of its 8 children (Sec. 3.1 R, Sec. 3.5 step 3) ----
// task = [new parent slot, old child slots 0..7]; src is a copy of the state taken before the
// merge (the parent may reuse a child's slot).
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_coarsen(const T* src, T* dst, const int32_t* tasks) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int32_t* tk = tasks + (size_t)blockIdx.x * 9;
  for (int i = threadIdx.x; i < 4 * BS * BS * BS; i += kNT) {
    const int f = i / (BS * BS * BS);
    const int r = i % (BS * BS * BS);
    const int x = r % BS, y = (r / BS) % BS, z = r / (BS * BS);
    const int cx = x > M / 2, cy = y > M / 2, cz = z > M / 2;
    const int lx = 2 * x - cx * M, ly = 2 * y - cy * M, lz = 2 * z - cz * M;
    const int cs = tk[1 + (cx | (cy << 1) | (cz << 2))];
    dst[(size_t)tk[0] * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)] =
        src[(size_t)cs * L::BLK + (size_t)f * L::FS + L::idx(lx, ly, lz)];
  }
}

// ---- copy of whole blocks (same slots) between two registers --------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_copy_blocks(const T* src, T* dst, const int32_t* blist) {
  using L = Lay<T, BS>;
  const size_t base = (size_t)blist[blockIdx.x] * L::BLK;
  const float4* s4 = reinterpret_cast<const float4*>(src + base);
  float4* d4 = reinterpret_cast<float4*>(dst + base);
  constexpr int n4 = (int)(L::BLK * sizeof(T) / 16);
  for (int i = threadIdx.x; i < n4; i += kNT) d4[i] = s4[i];
}

// ---- (8) analytic initial conditions and masks, FP64 at integer-derived coordinates ------------
__device__ __forceinline__ int lattice(const PhysK& ph, int4 bi, int a, int i, int M) {
  const int g = a == 0 ? bi.y : (a == 1 ? bi.z : bi.w);
  const int N = (ph.nroot[a] << bi.x) * M;
  const int gi = g * M + i;                               // in [0, N]
  return gi >= N ? gi - N : gi;                           // periodic seam x = L taken as 0
}

__device__ __forceinline__ double coord(const PhysK& ph, int4 bi, int a, int i, int M, double h) {
  const int g = a == 0 ? bi.y : (a == 1 ? bi.z : bi.w);
  const long long N = ((long long)ph.nroot[a] << bi.x) * M;
  const long long gi = (long long)g * M + i;             // in [0, N]
  return (double)(gi >= N ? gi - N : gi) * h;             // periodic seam x = L taken as 0
}

template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_ic(T* reg, const int32_t* blist, const int32_t* ranks, const int4* binfo,
                                             const PhysK ph, const IcK ic) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  const int4 bi = binfo[rank];
  const double h = ph.root_len / ((double)(1 << bi.x) * M);
  for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
    const int ix = i % BS, iy = (i / BS) % BS, iz = i / (BS * BS);
    const double X = coord(ph, bi, 0, ix, M, h), Y = coord(ph, bi, 1, iy, M, h), Z = coord(ph, bi, 2, iz, M, h);
    double v[4] = {0, 0, 0, 0};
    if (ic.kind == 1) {          // Taylor-Green
      const double k = ic.p[0], A = ic.p[1];
      v[0] = A * sin(k * X) * cos(k * Y) * cos(k * Z);
      v[1] = -A * cos(k * X) * sin(k * Y) * cos(k * Z);
    } else if (ic.kind == 2) {   // uniform
      v[0] = ic.p[0]; v[1] = ic.p[1]; v[2] = ic.p[2]; v[3] = ic.p[3];
    } else if (ic.kind == 3) {   // Gaussian pressure pulse, nearest periodic image
      const double c[3] = {ic.p[0], ic.p[1], ic.p[2]}, Lb[3] = {ic.p[5], ic.p[6], ic.p[7]};
      const double P[3] = {X, Y, Z};
      double r2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        double d = P[a] - c[a];
        d = d - Lb[a] * rint(d / Lb[a]);
        r2 += d * d;
      }
      v[3] = ic.p[4] * exp(-r2 / (ic.p[3] * ic.p[3]));
    }
    const int pi = L::idx(ix, iy, iz);
#pragma unroll
    for (int f = 0; f < 4; ++f) reg[(size_t)slot * L::BLK + (size_t)f * L::FS + pi] = T(v[f]);
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_mask(T* chi, const int32_t* blist, const int32_t* ranks, const int4* binfo,
                                               const PhysK ph, const MaskK m) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  const int4 bi = binfo[rank];
  const double h = ph.root_len / ((double)(1 << bi.x) * M);
  // A block that lies entirely farther than 40 delta from the sphere surface has tanh(d/delta)
  // = +-1 exactly in double precision at all its points (1 - tanh(40) < 1e-34): chi is exactly
  // 0 or 1 there and needs no transcendental.  Blocks on the periodic seam are evaluated fully.
  int uniform = -1;
  if (m.kind == 1) {
    const double lo[3] = {(double)bi.y * M * h, (double)bi.z * M * h, (double)bi.w * M * h};
    const double L[3] = {ph.nroot[0] * ph.root_len, ph.nroot[1] * ph.root_len, ph.nroot[2] * ph.root_len};
    bool seam = false;
    double dmin2 = 0.0, dmax2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double hi = lo[a] + M * h;
      if (hi >= L[a]) seam = true;
      const double c = m.p[a];
      const double near = c < lo[a] ? lo[a] - c : (c > hi ? c - hi : 0.0);
      const double far = fmax(fabs(c - lo[a]), fabs(hi - c));
      dmin2 += near * near;
      dmax2 += far * far;
    }
    if (!seam) {
      if (sqrt(dmin2) - m.p[3] > 40.0 * m.p[4]) uniform = 0;
      else if (sqrt(dmax2) - m.p[3] < -40.0 * m.p[4]) uniform = 1;
    }
  }
  for (int i = threadIdx.x; i < BS * BS * BS; i += kNT) {
    const int ix = i % BS, iy = (i / BS) % BS, iz = i / (BS * BS);
    // evaluated in the field precision: FP64 fields in double, FP32 fields in float
    T c = T(0);
    if (uniform >= 0) {
      c = T(uniform);
    } else if (m.kind == 1) {
      // coordinates in the field precision: i h with i the wrapped lattice index (exact when h
      // is dyadic, as for power-of-two root sides)
      const T X = T(lattice(ph, bi, 0, ix, M)) * T(h), Y = T(lattice(ph, bi, 1, iy, M)) * T(h),
              Z = T(lattice(ph, bi, 2, iz, M)) * T(h);
      const T dx = X - T(m.p[0]), dy = Y - T(m.p[1]), dz = Z - T(m.p[2]);
      const T d = sqrt(dx * dx + dy * dy + dz * dz) - T(m.p[3]);
      // beyond 10 delta (FP32) / 20 delta (FP64) tanh(d/delta) rounds to exactly +-1
      const T cut = T(sizeof(T) == 4 ? 10.0 : 20.0) * T(m.p[4]);
      if (d > cut) c = T(0);
      else if (d < -cut) c = T(1);
      else c = T(0.5) * (T(1) - tanh(d / T(m.p[4])));
    }
    chi[(size_t)slot * L::FS + L::idx(ix, iy, iz)] = c;
  }
}

// ---- (9) diagnostics: raw per-block sums over the half-open points [0, M-1]^3 -----------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_diag(const T* reg, const T* chi, const int32_t* blist, double* out) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int slot = blist[blockIdx.x];
  const T* b = reg + (size_t)slot * L::BLK;
  double s[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < M * M * M; i += kNT) {
    const int x = i % M, y = (i / M) % M, z = i / (M * M);
    const int pi = L::idx(x, y, z);
    const double u = b[pi], v = b[L::FS + pi], w = b[2 * L::FS + pi];
    if (chi) {
      const double c = chi[(size_t)slot * L::FS + pi];
      s[0] += c * u;
      s[1] += c * v;
      s[2] += c * w;
    }
    s[3] += u * u + v * v + w * w;
  }
  __shared__ double red[4][kNT / 32];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x >> 5] = s[k];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < kNT / 32; ++w) t += red[threadIdx.x][w];
    out[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

// ---- (10) dense <-> pool ---------------------------------------------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_gather(const T* reg, T* dense, const int32_t* blist, int ncomp, int comp_stride_blk) {
  using L = Lay<T, BS>;
  const int slot = blist[blockIdx.x];
  const int n = ncomp * BS * BS * BS;
  for (int i = threadIdx.x; i < n; i += kNT) {
    const int f = i / (BS * BS * BS), r = i % (BS * BS * BS);
    const int x = r % BS, y = (r / BS) % BS, z = r / (BS * BS);
    dense[(size_t)blockIdx.x * n + i] = reg[(size_t)slot * comp_stride_blk + (size_t)f * L::FS + L::idx(x, y, z)];
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_scatter(const T* dense, T* reg, const int32_t* blist) {
  using L = Lay<T, BS>;
  const int slot = blist[blockIdx.x];
  const int n = 4 * BS * BS * BS;
  for (int i = threadIdx.x; i < n; i += kNT) {
    const int f = i / (BS * BS * BS), r = i % (BS * BS * BS);
    const int x = r % BS, y = (r / BS) % BS, z = r / (BS * BS);
    reg[(size_t)slot * L::BLK + (size_t)f * L::FS + L::idx(x, y, z)] = dense[(size_t)blockIdx.x * n + i];
  }
}

inline dim3 grid1(int64_t n) { return dim3((unsigned)n); }

}  // namespace

LayoutInfo layout_info(int precision, int Bs) {
  LayoutInfo li{};
#define ACM_FILL(T, B)                                                                             \
  li.PP = Lay<T, B>::PP; li.FS = Lay<T, B>::FS; li.BLK = Lay<T, B>::BLK; li.NE = Lay<T, B>::NE;  \
  li.NE3 = Lay<T, B>::NE3; li.EBLK = Lay<T, B>::EBLK;
  if (precision == 64) {
    if (Bs == 17) { ACM_FILL(double, 17) } else { ACM_FILL(double, 9) }
  } else {
    if (Bs == 17) { ACM_FILL(float, 17) } else { ACM_FILL(float, 9) }
  }
#undef ACM_FILL
  return li;
}

#define ACM_BS_DISPATCH(Bs, KERNEL, ...)                 \
  do {                                                   \
    if ((Bs) == 17) { KERNEL<T, 17> __VA_ARGS__; }       \
    else { KERNEL<T, 9> __VA_ARGS__; }                   \
  } while (0)

template <typename T>
void launch_fine_wins(int Bs, T* reg, const int2* tasks, int64_t n, const int32_t* nbh, const int32_t* blist,
                      cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_fine_wins, <<<grid1(n), kNT, 0, st>>>(reg, tasks, nbh, blist));
}
template <typename T>
void launch_coarse_slabs(int Bs, const T* reg, T* slab, const int4* tasks, int64_t n, const int32_t* nbh, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_coarse_slabs, <<<grid1(4 * n), kNT, 0, st>>>(reg, slab, tasks, nbh));
}
template <typename T>
void launch_sync_ext(int Bs, const T* reg, T* out, int g, const int32_t* list, int64_t n, const int32_t* nbh, int by_rank, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_sync_ext, <<<grid1(n), kNT, 0, st>>>(reg, out, g, list, nbh, by_rank));
}
template <typename T>
void launch_details(int Bs, const T* reg, const T* chi, const int32_t* blist, const int32_t* ranks,
                    const int32_t* nbh, int64_t n, const unsigned long long* norm_bits, double* ind,
                    double* chirange, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_details, <<<grid1(n), kNT, 0, st>>>(reg, chi, blist, ranks, nbh, norm_bits, ind, chirange));
}
template <typename T>
void launch_maxnorm(int Bs, const T* reg, const int32_t* blist, int64_t n, unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_maxnorm, <<<grid1(n), kNT, 0, st>>>(reg, blist, out));
}
template <typename T, int BS>
void launch_refine_bs(const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* blist,
                      const int32_t* nbh, cudaStream_t st) {
  static bool attr = false;             // opt in to more than 48 KB of dynamic shared memory once
  if (!attr) {
    cudaFuncSetAttribute(k_refine<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RefSmem<T, BS>::bytes);
    attr = true;
  }
  k_refine<T, BS><<<grid1(4 * n), kNT, RefSmem<T, BS>::bytes, st>>>(src, dst, tasks, blist, nbh);
}
template <typename T>
void launch_refine(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* blist,
                   const int32_t* nbh, cudaStream_t st) {
  if (n <= 0) return;
  if (Bs == 17) launch_refine_bs<T, 17>(src, dst, tasks, n, blist, nbh, st);
  else launch_refine_bs<T, 9>(src, dst, tasks, n, blist, nbh, st);
}
template <typename T>
void launch_coarsen(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_coarsen, <<<grid1(n), kNT, 0, st>>>(src, dst, tasks));
}
template <typename T>
void launch_copy_blocks(int Bs, const T* src, T* dst, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_copy_blocks, <<<grid1(n), kNT, 0, st>>>(src, dst, blist));
}
template <typename T>
void launch_ic(int Bs, T* reg, const int32_t* blist, const int32_t* ranks, int64_t n, const int4* binfo,
               const PhysK& p, const IcK& ic, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_ic, <<<grid1(n), kNT, 0, st>>>(reg, blist, ranks, binfo, p, ic));
}
template <typename T>
void launch_mask(int Bs, T* chi, const int32_t* blist, const int32_t* ranks, int64_t n, const int4* binfo,
                 const PhysK& p, const MaskK& m, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_mask, <<<grid1(n), kNT, 0, st>>>(chi, blist, ranks, binfo, p, m));
}
template <typename T>
void launch_diag(int Bs, const T* reg, const T* chi, const int32_t* blist, int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_diag, <<<grid1(n), kNT, 0, st>>>(reg, chi, blist, out));
}
template <typename T>
void launch_gather(int Bs, const T* reg, T* dense, const int32_t* blist, int64_t n, int ncomp, cudaStream_t st) {
  if (n <= 0) return;
  const int stride = (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).BLK;
  const int cstride = ncomp == 1 ? (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).FS : stride;
  ACM_BS_DISPATCH(Bs, k_gather, <<<grid1(n), kNT, 0, st>>>(reg, dense, blist, ncomp, cstride));
}
template <typename T>
void launch_scatter(int Bs, const T* dense, T* reg, const int32_t* blist, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_scatter, <<<grid1(n), kNT, 0, st>>>(dense, reg, blist));
}

#define ACM_INST(T)                                                                                        \
  template void launch_fine_wins<T>(int, T*, const int2*, int64_t, const int32_t*, const int32_t*, cudaStream_t);          \
  template void launch_coarse_slabs<T>(int, const T*, T*, const int4*, int64_t, const int32_t*, cudaStream_t); \
  template void launch_sync_ext<T>(int, const T*, T*, int, const int32_t*, int64_t, const int32_t*, int, cudaStream_t); \
  template void launch_details<T>(int, const T*, const T*, const int32_t*, const int32_t*, const int32_t*, int64_t, const unsigned long long*, double*, double*, cudaStream_t); \
  template void launch_maxnorm<T>(int, const T*, const int32_t*, int64_t, unsigned long long*, cudaStream_t); \
  template void launch_refine<T>(int, const T*, T*, const int32_t*, int64_t, const int32_t*, const int32_t*, cudaStream_t); \
  template void launch_coarsen<T>(int, const T*, T*, const int32_t*, int64_t, cudaStream_t);               \
  template void launch_copy_blocks<T>(int, const T*, T*, const int32_t*, int64_t, cudaStream_t);          \
  template void launch_ic<T>(int, T*, const int32_t*, const int32_t*, int64_t, const int4*, const PhysK&, const IcK&, cudaStream_t); \
  template void launch_mask<T>(int, T*, const int32_t*, const int32_t*, int64_t, const int4*, const PhysK&, const MaskK&, cudaStream_t); \
  template void launch_diag<T>(int, const T*, const T*, const int32_t*, int64_t, double*, cudaStream_t);   \
  template void launch_gather<T>(int, const T*, T*, const int32_t*, int64_t, int, cudaStream_t);          \
  template void launch_scatter<T>(int, const T*, T*, const int32_t*, int64_t, cudaStream_t);
ACM_INST(float)
ACM_INST(double)

}  // namespace acm
