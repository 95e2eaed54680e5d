// Device-side layout and point lookup shared by the libacm kernels.
//
// Field storage (per register): block slot -> component (u, v, w, p) -> z -> y -> x, x fastest.
// A z-plane of Bs*Bs values is padded to a multiple of 16 bytes (so every plane of every
// block starts 16-byte aligned and can be moved by one bulk copy), and a component to a
// multiple of 32 elements (every component starts 128-byte aligned).
//
// Neighbourhood table (one per slot, built on the host after every grid change): the 27
// level-J boxes around a block, box index d = (dx+1) + 3(dy+1) + 9(dz+1), centre 13 = the
// block itself.  Entries 8d..8d+7: LEAF -> [0] = slot; COARSER -> [0] = slot of the covering
// leaf one level up; REFINED -> [c] = slot of child c = cx + 2cy + 4cz (-1 if not a leaf).
// Entry 216 + d: box type (low 4 bits) | octant of the box inside its coarser leaf << 4.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace acm {

constexpr int kNbhStride = 256;      // int32 per slot in the neighbourhood table
constexpr int kNbhType = 216;        // offset of the 27 type words
constexpr int kGE = 2;               // ghost depth of the adaptation buffer (details, refine)
constexpr int kTypeLeaf = 0, kTypeCoarser = 1, kTypeRefined = 2, kTypeNone = 3;

template <typename T, int BS>
struct Lay {
  static constexpr int M = BS - 1;
  static constexpr int PLANE = BS * BS;
  static constexpr int VEC = 16 / (int)sizeof(T);
  static constexpr int PP = ((PLANE + VEC - 1) / VEC) * VEC;   // plane pitch (elements)
  static constexpr int FS = ((BS * PP + 31) / 32) * 32;         // component stride
  static constexpr int BLK = 4 * FS;                            // block stride
  static constexpr int NE = BS + 2 * kGE;                       // adaptation buffer extent
  static constexpr int NE3 = NE * NE * NE;
  static constexpr int EBLK = 4 * NE3;
  __host__ __device__ static constexpr int idx(int x, int y, int z) { return z * PP + y * BS + x; }
};

// Host-side copy of the layout numbers for a runtime (precision, Bs).
struct LayoutInfo {
  int64_t PP, FS, BLK, NE, NE3, EBLK;
};
LayoutInfo layout_info(int precision, int Bs);

__host__ __device__ constexpr int box_index(int dx, int dy, int dz) {
  return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

// Element offset (from the start of the register, component f) of local lattice point p of the
// block whose neighbourhood is nbh (level-J lattice, local coordinates in [-M, 2M]) in the
// finest leaf that holds p as a grid point: a finer leaf (decimation), else a same-level leaf
// (copy), else a coarser leaf if p lies on its lattice.  Returns -1 if p is covered by coarser
// leaves only and is not on their lattice (it must then be predicted).  Only shared/constant
// data is read, so callers can find several offsets first and then issue their loads together.
template <typename T, int BS>
__device__ __forceinline__ long long direct_offset(const int* __restrict__ nbh, int px, int py, int pz, int f) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int p[3] = {px, py, pz};
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = p[a] <= 0 ? -1 : (p[a] <= M ? 0 : 1);
    hi[a] = p[a] < 0 ? -1 : (p[a] < M ? 0 : 1);
  }
  int best = -1, bestp = 0, bd[3] = {0, 0, 0};
  for (int dz = lo[2]; dz <= hi[2]; ++dz)
    for (int dy = lo[1]; dy <= hi[1]; ++dy)
      for (int dx = lo[0]; dx <= hi[0]; ++dx) {
        const int d = box_index(dx, dy, dz);
        const int t = nbh[kNbhType + d] & 15;
        const int pr = t == kTypeRefined ? 3 : (t == kTypeLeaf ? 2 : (t == kTypeCoarser ? 1 : 0));
        if (pr > bestp) {
          bestp = pr;
          best = d;
          bd[0] = dx; bd[1] = dy; bd[2] = dz;
        }
      }
  if (bestp == 0) return -1;
  int q[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a] = p[a] - bd[a] * M;   // in [0, M] inside box `best`
  int s, l[3];
  if (bestp == 3) {
    int c = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ca = q[a] > M / 2 ? 1 : (q[a] < M / 2 ? 0 : (bd[a] < 0 ? 1 : 0));
      c |= ca << a;
      l[a] = 2 * q[a] - ca * M;
    }
    s = nbh[8 * best + c];
  } else if (bestp == 2) {
    s = nbh[8 * best];
    l[0] = q[0]; l[1] = q[1]; l[2] = q[2];
  } else {
    const int oct = nbh[kNbhType + best] >> 4;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int r = ((oct >> a) & 1) * M + q[a];
      if (r & 1) return -1;
      l[a] = r >> 1;
    }
    s = nbh[8 * best];
  }
  if (s < 0) return -1;
  return (long long)s * L::BLK + (long long)f * L::FS + L::idx(l[0], l[1], l[2]);
}

// Value at local lattice point p from the finest leaf holding it (see direct_offset); false if
// it must be predicted.
template <typename T, int BS>
__device__ __forceinline__ bool direct_value(const T* __restrict__ reg, const int* __restrict__ nbh,
                                             int px, int py, int pz, int f, T* out) {
  const long long o = direct_offset<T, BS>(nbh, px, py, pz, f);
  if (o < 0) return false;
  *out = reg[o];
  return true;
}

// Square root and tanh in the argument's own precision (float arguments never take the double
// routines, which run on the much slower FP64 pipe).
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float ttanh(float x) { return tanhf(x); }
__device__ __forceinline__ double ttanh(double x) { return tanh(x); }

// Squared velocity magnitude with one fixed rounding sequence, so every kernel that takes the
// max norm of (u, v, w) gets bitwise the same value (sqrt of the max = max of the sqrt).
template <typename T>
__device__ __forceinline__ T mag2(T u, T v, T w) {
  T s = u * u;
  s = fma(v, v, s);
  return fma(w, w, s);
}

// DD-4 prediction of one line (Sec. 3.1): from NC = M/2 + 3 coarse samples c[k] at coarse
// index k - 1 (fine index 2k - 2), the fine value at fine index i = 0..M: the sample itself at
// even i, the 4-point stencil (-1, 9, 9, -1)/16 around it at odd i.  The sum runs left to right.
template <typename T, int BS>
__device__ __forceinline__ T dd4_line(const T (&c)[BS / 2 + 3], int i) {
  if (i & 1) {
    const int k0 = (i - 1) >> 1;            // coarse sample at fine index i - 3
    T acc = T(0);
    acc = acc + (T(-1) / T(16)) * c[k0];
    acc = acc + (T(9) / T(16)) * c[k0 + 1];
    acc = acc + (T(9) / T(16)) * c[k0 + 2];
    acc = acc + (T(-1) / T(16)) * c[k0 + 3];
    return acc;
  }
  return c[(i + 2) >> 1];
}

// Point value with the DD-4 fallback (Sec. 3.1): points held only by coarser leaves are the
// tensor-product prediction from the coarse lattice, along x, then y, then z.  Every stencil
// point has even coordinates, so it is held directly by some leaf.
template <typename T, int BS>
__device__ __forceinline__ T point_value(const T* __restrict__ reg, const int* __restrict__ nbh,
                                         int px, int py, int pz, int f) {
  T v;
  if (direct_value<T, BS>(reg, nbh, px, py, pz, f, &v)) return v;
  const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  const int off[4] = {-3, -1, 1, 3};
  const int nx = (px & 1) ? 4 : 1, ny = (py & 1) ? 4 : 1, nz = (pz & 1) ? 4 : 1;
  T accz = T(0);
  for (int kz = 0; kz < nz; ++kz) {
    const int zz = nz == 4 ? pz + off[kz] : pz;
    const T wz = nz == 4 ? w[kz] : T(1);
    T accy = T(0);
    for (int ky = 0; ky < ny; ++ky) {
      const int yy = ny == 4 ? py + off[ky] : py;
      const T wy = ny == 4 ? w[ky] : T(1);
      T accx = T(0);
      for (int kx = 0; kx < nx; ++kx) {
        const int xx = nx == 4 ? px + off[kx] : px;
        const T wx = nx == 4 ? w[kx] : T(1);
        T c;
        if (!direct_value<T, BS>(reg, nbh, xx, yy, zz, f, &c)) c = T(__longlong_as_double(0x7ff8000000000000ll));
        accx = accx + wx * c;
      }
      accy = accy + wy * accx;
    }
    accz = accz + wz * accy;
  }
  return accz;
}

}  // namespace acm
