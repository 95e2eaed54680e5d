// Synchronisation, wavelet-detail, adaptation and diagnostic kernels of libacm.
//
// Paper: Sec. 3.1 (DD-4 prediction, decimation, details u - P R u), Sec. 3.3-3.4 (block
// indicator: largest detail normalised per component by its global max norm), Sec. 3.5
// (refine by prediction, coarsen by merging sister blocks), Sec. 4.2 (ghost synchronisation:
// restrict or predict, then copy), Sec. 2.2 (smoothed mask, force by midpoint rule).
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.hpp"

namespace acm {

namespace {

constexpr int kNT = 256;

// Opt `kernel` in to `bytes` of dynamic shared memory (above the default 48 KB) on the current
// device, once per device (the attribute belongs to the device's context).
template <typename K>
void smem_opt_in(K kernel, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_relaxed) & bit) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done.fetch_or(bit);
}

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
// in box d: coordinate 0 / M where d is -1 / +1, the whole range where d is 0.  The CTAs walk
// the task list (its length is on the device).
template <typename T, int BS>
__device__ __forceinline__ void fine_wins_task(T* reg, const int2 tk, const int32_t* nbh_all, const int32_t* blist) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
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

template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_fine_wins(T* reg, const int2* tasks, const int32_t* ntasks,
                                                    const int32_t* nbh_all, const int32_t* blist) {
  const int nt = *ntasks;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) fine_wins_task<T, BS>(reg, tasks[t], nbh_all, blist);
}

// ---- (2) coarse-face halo slabs ------------------------------------------------------------------
// task = (rank, face F, slab index, -); a CTA per task at a time, all four components (the CTAs
// walk the task list, whose length is on the device).  The 3 x Bs x Bs
// halo points beyond face F take the value of the finest leaf holding them, else the tensor DD-4
// prediction from the coarse lattice (Sec. 3.1).  Only points on the face's tangential boundary
// lines (t0 or t1 = 0 or M) can be held by a leaf of the block's level or finer; all others lie
// in the coarser leaf alone.  The coarse patch the predictions need (even local coordinates
// [M-2, M+6] or [-6, 2] across the face, [-2, M+2] along it) is gathered once, then predicted
// separably: along t0, then t1, then across the face (a fixed order per face orientation, so
// every block that needs a halo point gets bitwise the same value).  The leaf lookups are done
// once per point for all components; each separable pass gives a thread one whole line, and
// the last pass one halo column (t0, t1).
// Slab layout [slab][comp][layer l-1][t1][t0] with (t0, t1) as in the stage kernel.
// The leaf lookups depend on the grid only: with `offc` set, a launch with use_cache = 0 stores
// them per slab (SlabSmem::NOFF words: the patch, then 3 layers of the 4M edge columns) and a
// later launch on the same grid with use_cache = 1 reads them back instead of searching again.
// Dynamic shared memory: P, A, B below in T, then the neighbourhood.
template <typename T, int BS>
struct SlabSmem {
  // a thread per halo column (t0, t1); above 1024 columns (Bs = 33) a thread takes two
  static constexpr int NT = BS * BS <= 1024 ? ((BS * BS + 31) / 32) * 32 : 1024;
  static constexpr bool ONE = BS * BS <= NT;        // one column per thread
  static constexpr int MINB = BS <= 17 ? 3 : 1;     // CTAs per SM
  static constexpr int M = BS - 1;
  static constexpr int NC = M / 2 + 3;              // coarse samples along the face: -2..M+2 step 2
  static constexpr int NN = 5;                      // coarse planes across the face
  static constexpr int P = 4 * NN * NC * NC;        // [f][n][t1 coarse][t0 coarse]
  static constexpr int A = 4 * NN * NC * BS;        // [f][n][t1 coarse][t0]: predicted along t0
  static constexpr int B = 4 * NN * BS * BS;        // [f][n][t1][t0]: predicted along t0 and t1
  static constexpr size_t bytes = (size_t)(P + A + B) * sizeof(T) + kNbhStride * sizeof(int);
  static constexpr int NEDGE = 4 * M;                 // halo columns on the face's boundary lines
  static constexpr int NOFF = NN * NC * NC + 3 * NEDGE;
};

// Compact index of an edge column (t0 or t1 on the boundary), 0..4M-1.
template <int BS>
__device__ __forceinline__ int edge_index(int t0, int t1) {
  constexpr int M = BS - 1;
  if (t1 == 0) return t0;
  if (t1 == M) return BS + t0;
  if (t0 == 0) return 2 * BS + t1 - 1;
  return 2 * BS + (BS - 2) + t1 - 1;
}

template <typename T, int BS>
__global__ void __launch_bounds__(SlabSmem<T, BS>::NT, SlabSmem<T, BS>::MINB)
k_coarse_slabs(const T* reg, T* slab, const int4* tasks, const int32_t* ntasks, const int32_t* nbh_all, uint32_t* offc,
               int use_cache) {
  using L = Lay<T, BS>;
  using S = SlabSmem<T, BS>;
  constexpr int M = L::M, NT = S::NT, NC = S::NC, NN = S::NN;
  constexpr int NP3 = NN * NC * NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);
  T* A = P + S::P;
  T* B = A + S::A;
  int* nbh = reinterpret_cast<int*>(B + S::B);
  const int tid = threadIdx.x;
  const int nt = *ntasks;
  for (int task = blockIdx.x; task < nt; task += gridDim.x) {
  const int4 tk = tasks[task];
  uint32_t* oc = offc ? offc + (size_t)tk.z * S::NOFF : nullptr;
  const bool cached = oc && use_cache;
  __syncthreads();                                  // previous task done with shared memory
  if (!cached) {
    for (int i = tid; i < kNbhStride; i += NT) nbh[i] = nbh_all[(size_t)tk.x * kNbhStride + i];
    __syncthreads();
  }
  const int F = tk.y, ax = F >> 1;
  const bool plus = F & 1;
  const int n0 = plus ? M - 2 : -6;                 // first coarse plane (even local coordinate)
  auto place = [&](int nl, int t0, int t1, int* x, int* y, int* z) {
    if (ax == 0) { *x = nl; *y = t0; *z = t1; }
    else if (ax == 1) { *x = t0; *y = nl; *z = t1; }
    else { *x = t0; *y = t1; *z = nl; }
  };
  // leaf lookups of the halo column (t0, t1) on the face's boundary lines (component 0
  // offsets; component f is FS further), and its values
  auto edge_values = [&](int t0, int t1, long long (&eo)[3], T (&ev)[3][4]) {
    eo[0] = eo[1] = eo[2] = -1;
    if (t0 == 0 || t0 == M || t1 == 0 || t1 == M) {
      const int ei = edge_index<BS>(t0, t1);
#pragma unroll
      for (int l = 1; l <= 3; ++l) {
        if (cached) {
          const uint32_t v = oc[NP3 + 3 * ei + l - 1];
          eo[l - 1] = v == 0xffffffffu ? -1 : (long long)v;
        } else {
          int x, y, z;
          place(plus ? M + l : -l, t0, t1, &x, &y, &z);
          eo[l - 1] = direct_offset<T, BS>(nbh, x, y, z, 0);
          if (oc) oc[NP3 + 3 * ei + l - 1] = eo[l - 1] < 0 ? 0xffffffffu : (uint32_t)eo[l - 1];
        }
      }
    }
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int f = 0; f < 4; ++f) ev[l][f] = eo[l] >= 0 ? reg[eo[l] + (long long)f * L::FS] : T(0);
  };
  // with one column per thread its edge values are loaded with the patch, before the passes
  const bool col = tid < BS * BS;
  long long eo[3];
  T ev[3][4];
  if (S::ONE && col) edge_values(tid % BS, tid / BS, eo, ev);
  constexpr int U = (NP3 + NT - 1) / NT;
  long long off[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int i = tid + k * NT;
    off[k] = -2;
    if (i < NP3) {
      if (cached) {
        const uint32_t v = oc[i];
        off[k] = v == 0xffffffffu ? -1 : (long long)v;
      } else {
        const int a0 = i % NC, a1 = (i / NC) % NC, an = i / (NC * NC);
        int x, y, z;
        place(n0 + 2 * an, 2 * a0 - 2, 2 * a1 - 2, &x, &y, &z);
        off[k] = direct_offset<T, BS>(nbh, x, y, z, 0);
        if (oc) oc[i] = off[k] < 0 ? 0xffffffffu : (uint32_t)off[k];
      }
    }
  }
  T pv[U][4];
#pragma unroll
  for (int k = 0; k < U; ++k)
#pragma unroll
    for (int f = 0; f < 4; ++f)
      pv[k][f] = off[k] >= 0 ? reg[off[k] + (long long)f * L::FS] : T(__longlong_as_double(0x7ff8000000000000ll));
#pragma unroll
  for (int k = 0; k < U; ++k)
    if (off[k] != -2)
#pragma unroll
      for (int f = 0; f < 4; ++f) P[f * NP3 + tid + k * NT] = pv[k][f];
  __syncthreads();
  for (int it = tid; it < 4 * NN * NC; it += NT) {  // along t0: line (f, n, a1)
    T cv[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) cv[k] = P[it * NC + k];
#pragma unroll
    for (int i = 0; i < BS; ++i) A[it * BS + i] = dd4_line<T, BS>(cv, i);
  }
  __syncthreads();
  for (int it = tid; it < 4 * NN * BS; it += NT) {  // along t1: line (f, n, t0)
    const int l0 = it % BS, fn = it / BS;
    T cv[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) cv[k] = A[(fn * NC + k) * BS + l0];
#pragma unroll
    for (int i = 0; i < BS; ++i) B[(fn * BS + i) * BS + l0] = dd4_line<T, BS>(cv, i);
  }
  __syncthreads();
  // across the face: column (t0, t1)
  auto column_out = [&](int t0, int t1, const long long (&eo)[3], const T (&ev)[3][4]) {
    const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      T cn[NN];
#pragma unroll
      for (int n = 0; n < NN; ++n) cn[n] = B[((f * NN + n) * BS + t1) * BS + t0];
#pragma unroll
      for (int l = 1; l <= 3; ++l) {
        T v;
        if (eo[l - 1] >= 0) {
          v = ev[l - 1][f];
        } else {
          const int c = (plus ? M + l : -l) - n0;   // fine offset from the first coarse plane
          if (c & 1) {
            const int k0 = (c - 3) >> 1;            // 0 or 1
            v = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) v = v + w[k] * (k0 == 0 ? cn[k] : cn[k + 1]);
          } else {
            v = cn[c >> 1];
          }
        }
        slab[((((size_t)tk.z * 4 + f) * 3 + (l - 1)) * BS + t1) * BS + t0] = v;
      }
    }
  };
  if (S::ONE) {
    if (col) column_out(tid % BS, tid / BS, eo, ev);
  } else {
    for (int c = tid; c < BS * BS; c += NT) {
      edge_values(c % BS, c / BS, eo, ev);
      column_out(c % BS, c / BS, eo, ev);
    }
  }
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
// One CTA per block.  The coarse samples are the block's even points, local coordinates -2..M+2
// (those outside the block are held directly by a neighbour leaf; each is looked up once for
// all four components); they are predicted back to every point separably (x, then y, then z:
// the tensor DD-4 sum in that nesting) and subtracted.  In every pass a thread owns one whole
// line: it reads the line's coarse samples once and produces its Bs values.  Components run one
// after another through the passes; the block's own values of a component, compared in its last
// pass, are loaded one z-column per thread when its first pass starts.  The z-pass of one
// component and the x-pass of the next share a phase (they touch different buffers).
// Dynamic shared memory: c [4][NC^3], px [NC][NC][Bs], py [NC][Bs][Bs] in T, then the
// neighbourhood.
template <typename T, int BS>
struct DetSmem {
  static constexpr int NT = ((BS * BS + 31) / 32) * 32;
  static constexpr int NC = (BS - 1) / 2 + 3;   // coarse samples per axis, -1..M/2+1
  static constexpr int NC3 = NC * NC * NC;
  static constexpr int PX = NC * NC * BS, PY = NC * BS * BS;
  static constexpr size_t bytes = (size_t)(4 * NC3 + PX + PY) * sizeof(T) + kNbhStride * sizeof(int);
};

template <typename T, int BS>
__global__ void __launch_bounds__(DetSmem<T, BS>::NT) k_details(const T* reg, const T* chi, const int32_t* blist,
                                                                 const int32_t* ranks, const int32_t* nbh_all,
                                                                 const unsigned long long* norm_bits, double* ind,
                                                                 double* chirange) {
  using L = Lay<T, BS>;
  using S = DetSmem<T, BS>;
  constexpr int M = L::M;
  constexpr int NT = S::NT, NC = S::NC, NC3 = S::NC3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);       // c[f][zc][yc][xc]
  T* px = cs + 4 * NC3;                         // px[zc][yc][x]
  T* py = px + S::PX;                           // py[zc][y][x]
  int* nbh = reinterpret_cast<int*>(py + S::PY);
  __shared__ T red[6][NT / 32];
  const int tid = threadIdx.x;
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  const bool col = tid < BS * BS;
  const int x = col ? tid % BS : 0, y = col ? tid / BS : 0;
  const int wid = tid >> 5, lane = tid & 31;
  const T* bb = reg + (size_t)slot * L::BLK;

  // mask range from one z-column per thread
  T tmin = T(1e30), tmax = T(-1e30);
  if (chi && col) {
    const T* cb = chi + (size_t)slot * L::FS;
    T v[BS];
#pragma unroll
    for (int z = 0; z < BS; ++z) v[z] = cb[L::idx(x, y, z)];
#pragma unroll
    for (int z = 0; z < BS; ++z) {
      tmin = v[z] < tmin ? v[z] : tmin;
      tmax = v[z] > tmax ? v[z] : tmax;
    }
  }
  for (int i = tid; i < kNbhStride; i += NT) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  __syncthreads();
  {
    // coarse samples: offsets (component 0) first, then the loads of all components at once
    constexpr int U = (NC3 + NT - 1) / NT;
    long long off[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int i = tid + k * NT;
      off[k] = -2;
      if (i < NC3) {
        const int cx = 2 * (i % NC) - 2, cy = 2 * ((i / NC) % NC) - 2, cz = 2 * (i / (NC * NC)) - 2;
        if (cx >= 0 && cx <= M && cy >= 0 && cy <= M && cz >= 0 && cz <= M)
          off[k] = (long long)slot * L::BLK + L::idx(cx, cy, cz);
        else
          off[k] = direct_offset<T, BS>(nbh, cx, cy, cz, 0);
      }
    }
    T v[U][4];
#pragma unroll
    for (int k = 0; k < U; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f)
        v[k][f] = off[k] >= 0 ? reg[off[k] + (long long)f * L::FS] : T(__longlong_as_double(0x7ff8000000000000ll));
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (off[k] != -2)
#pragma unroll
        for (int f = 0; f < 4; ++f) cs[f * NC3 + tid + k * NT] = v[k][f];
  }
  __syncthreads();
  auto xpass = [&](int f) {
    if (tid < NC * NC) {                        // line (yc, zc) = tid
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = cs[f * NC3 + tid * NC + k];
#pragma unroll
      for (int i = 0; i < BS; ++i) px[tid * BS + i] = dd4_line<T, BS>(cv, i);
    }
  };
  double best = 0.0;
  T u[BS];
  xpass(0);
  for (int f = 0; f < 4; ++f) {
    if (col) {
#pragma unroll
      for (int z = 0; z < BS; ++z) u[z] = bb[(size_t)f * L::FS + L::idx(x, y, z)];
    }
    __syncthreads();                            // px of component f complete
    if (tid < NC * BS) {                        // y-pass: line (x, zc)
      const int lx = tid % BS, zc = tid / BS;
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = px[(zc * NC + k) * BS + lx];
#pragma unroll
      for (int i = 0; i < BS; ++i) py[(zc * BS + i) * BS + lx] = dd4_line<T, BS>(cv, i);
    }
    __syncthreads();                            // py complete, px free
    T dmax = T(0);    // max |detail| in the field precision; max(|d| inv) = max|d| inv exactly
    if (col) {                                  // z-pass: column (x, y), compared with the block
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = py[(k * BS + y) * BS + x];
#pragma unroll
      for (int z = 0; z < BS; ++z) {
        const T dv = tabs(u[z] - dd4_line<T, BS>(cv, z));
        dmax = dv > dmax ? dv : dmax;
      }
    }
    if (f < 3) xpass(f + 1);
    for (int o = 16; o > 0; o >>= 1) {
      const T t = __shfl_xor_sync(0xffffffffu, dmax, o);
      dmax = t > dmax ? t : dmax;
    }
    if (lane == 0) red[f][wid] = dmax;
    // the barrier at the top of the next component (or the one below) orders py's reuse
  }
  for (int o = 16; o > 0; o >>= 1) {
    const T a = __shfl_xor_sync(0xffffffffu, tmin, o), b = __shfl_xor_sync(0xffffffffu, tmax, o);
    tmin = a < tmin ? a : tmin;
    tmax = b > tmax ? b : tmax;
  }
  if (lane == 0) { red[4][wid] = tmin; red[5][wid] = tmax; }
  __syncthreads();
  if (tid == 0) {
    for (int f = 0; f < 4; ++f) {
      // global max norm of component f, as left by the max-norm reduction (non-negative bits)
      const double nf = __longlong_as_double((long long)norm_bits[f]);
      const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
      if (inv == 0.0) continue;
      T m = red[f][0];
      for (int k = 1; k < NT / 32; ++k) m = red[f][k] > m ? red[f][k] : m;
      const double r = (double)m * inv;
      best = r > best ? r : best;
    }
    T mn = red[4][0], mx = red[5][0];
    for (int k = 1; k < NT / 32; ++k) {
      mn = red[4][k] < mn ? red[4][k] : mn;
      mx = red[5][k] > mx ? red[5][k] : mx;
    }
    ind[rank] = best;
    chirange[rank] = chi ? (double)mx - (double)mn : 0.0;
  }
}

// Block indicators of Bs = 33 blocks: the same passes with one component's coarse samples in
// shared memory at a time (four would not fit beside px and py); the leaf lookups are done once
// and kept in shared memory as 32-bit offsets (the pool's element offsets fit 32 bits, checked at
// forest creation).  A thread owns up to two columns in the mask range and the z-pass, and reads
// the block's values there as it compares them.  Same values as k_details.
template <typename T, int BS>
struct DetBigSmem {
  static constexpr int NT = 1024;
  static constexpr int NC = (BS - 1) / 2 + 3;
  static constexpr int NC3 = NC * NC * NC;
  static constexpr int PX = NC * NC * BS, PY = NC * BS * BS;
  static constexpr size_t bytes = (size_t)(NC3 + PX + PY) * sizeof(T) + (size_t)NC3 * sizeof(uint32_t) +
                                  kNbhStride * sizeof(int);
};

template <typename T, int BS>
__global__ void __launch_bounds__(DetBigSmem<T, BS>::NT, 1)
k_details_big(const T* reg, const T* chi, const int32_t* blist, const int32_t* ranks, const int32_t* nbh_all,
              const unsigned long long* norm_bits, double* ind, double* chirange) {
  using L = Lay<T, BS>;
  using S = DetBigSmem<T, BS>;
  constexpr int M = L::M;
  constexpr int NT = S::NT, NC = S::NC, NC3 = S::NC3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);       // c[zc][yc][xc] of one component
  T* px = cs + NC3;                             // px[zc][yc][x]
  T* py = px + S::PX;                           // py[zc][y][x]
  uint32_t* offs = reinterpret_cast<uint32_t*>(py + S::PY);
  int* nbh = reinterpret_cast<int*>(offs + NC3);
  __shared__ T red[6][NT / 32];
  const int tid = threadIdx.x;
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  const int wid = tid >> 5, lane = tid & 31;
  const T* bb = reg + (size_t)slot * L::BLK;
  T tmin = T(1e30), tmax = T(-1e30);
  if (chi) {
    const T* cb = chi + (size_t)slot * L::FS;
    for (int c = tid; c < BS * BS; c += NT) {
      for (int z = 0; z < BS; ++z) {
        const T v = cb[L::idx(c % BS, c / BS, z)];
        tmin = v < tmin ? v : tmin;
        tmax = v > tmax ? v : tmax;
      }
    }
  }
  for (int i = tid; i < kNbhStride; i += NT) nbh[i] = nbh_all[(size_t)rank * kNbhStride + i];
  __syncthreads();
  for (int i = tid; i < NC3; i += NT) {
    const int cx = 2 * (i % NC) - 2, cy = 2 * ((i / NC) % NC) - 2, cz = 2 * (i / (NC * NC)) - 2;
    long long off;
    if (cx >= 0 && cx <= M && cy >= 0 && cy <= M && cz >= 0 && cz <= M)
      off = (long long)slot * L::BLK + L::idx(cx, cy, cz);
    else
      off = direct_offset<T, BS>(nbh, cx, cy, cz, 0);
    offs[i] = off < 0 ? 0xffffffffu : (uint32_t)off;
  }
  __syncthreads();
  for (int f = 0; f < 4; ++f) {
    for (int i = tid; i < NC3; i += NT) {
      const uint32_t o = offs[i];
      cs[i] = o == 0xffffffffu ? T(__longlong_as_double(0x7ff8000000000000ll)) : reg[(size_t)o + (size_t)f * L::FS];
    }
    __syncthreads();                            // cs complete (py free: the last z-pass is done)
    if (tid < NC * NC) {                        // x-pass: line (yc, zc)
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = cs[tid * NC + k];
#pragma unroll
      for (int i = 0; i < BS; ++i) px[tid * BS + i] = dd4_line<T, BS>(cv, i);
    }
    __syncthreads();
    if (tid < NC * BS) {                        // y-pass: line (x, zc)
      const int lx = tid % BS, zc = tid / BS;
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = px[(zc * NC + k) * BS + lx];
#pragma unroll
      for (int i = 0; i < BS; ++i) py[(zc * BS + i) * BS + lx] = dd4_line<T, BS>(cv, i);
    }
    __syncthreads();
    T dmax = T(0);
    for (int c = tid; c < BS * BS; c += NT) {   // z-pass: column (x, y), compared with the block
      const int x = c % BS, y = c / BS;
      T cv[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) cv[k] = py[(k * BS + y) * BS + x];
#pragma unroll
      for (int z = 0; z < BS; ++z) {
        const T dv = tabs(bb[(size_t)f * L::FS + L::idx(x, y, z)] - dd4_line<T, BS>(cv, z));
        dmax = dv > dmax ? dv : dmax;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T t = __shfl_xor_sync(0xffffffffu, dmax, o);
      dmax = t > dmax ? t : dmax;
    }
    if (lane == 0) red[f][wid] = dmax;
    __syncthreads();                            // the z-pass is done with py before the next x-pass
  }
  for (int o = 16; o > 0; o >>= 1) {
    const T a = __shfl_xor_sync(0xffffffffu, tmin, o), b = __shfl_xor_sync(0xffffffffu, tmax, o);
    tmin = a < tmin ? a : tmin;
    tmax = b > tmax ? b : tmax;
  }
  if (lane == 0) { red[4][wid] = tmin; red[5][wid] = tmax; }
  __syncthreads();
  if (tid == 0) {
    double best = 0.0;
    for (int f = 0; f < 4; ++f) {
      const double nf = __longlong_as_double((long long)norm_bits[f]);
      const double inv = nf > 0.0 ? 1.0 / nf : 0.0;
      if (inv == 0.0) continue;
      T m = red[f][0];
      for (int k = 1; k < NT / 32; ++k) m = red[f][k] > m ? red[f][k] : m;
      const double r = (double)m * inv;
      best = r > best ? r : best;
    }
    T mn = red[4][0], mx = red[5][0];
    for (int k = 1; k < NT / 32; ++k) {
      mn = red[4][k] < mn ? red[4][k] : mn;
      mx = red[5][k] > mx ? red[5][k] : mx;
    }
    ind[rank] = best;
    chirange[rank] = chi ? (double)mx - (double)mn : 0.0;
  }
}

// ---- (5) max norms (Sec. 2.3 u_max, Sec. 3.4 normalisation) ------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_maxnorm(const T* reg, const int32_t* blist, unsigned long long* out) {
  using L = Lay<T, BS>;
  const int slot = blist[blockIdx.x];
  const T* b = reg + (size_t)slot * L::BLK;
  // arithmetic in the field precision (an FP32 field gives an FP32 norm, stored as double);
  // m[4] holds the squared magnitude, its root is taken once at the end.  The maxima propagate
  // NaN (a comparison with NaN is false, so a plain maximum would drop it): a non-finite state
  // reaches the host as a non-finite norm.
  T m[5] = {T(0), T(0), T(0), T(0), T(0)};
  auto keep = [](T a, T m) { return (a > m || a != a) ? a : m; };
  constexpr int N = BS * BS * BS, U = 4;
  for (int base = threadIdx.x; base < N; base += kNT * U) {
    T v[U][4];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int i = base + k * kNT;
      const int pi = i < N ? L::idx(i % BS, (i / BS) % BS, i / (BS * BS)) : 0;
#pragma unroll
      for (int f = 0; f < 4; ++f) v[k][f] = i < N ? b[(size_t)f * L::FS + pi] : T(0);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        m[f] = keep(tabs(v[k][f]), m[f]);
      }
      m[4] = keep(mag2(v[k][0], v[k][1], v[k][2]), m[4]);
    }
  }
  __shared__ T red[5][kNT / 32];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    T mk = m[k];
    for (int o = 16; o > 0; o >>= 1) mk = keep(__shfl_xor_sync(0xffffffffu, mk, o), mk);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = mk;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    T mk = T(0);
    for (int w = 0; w < kNT / 32; ++w) mk = keep(red[threadIdx.x][w], mk);
    const double d = threadIdx.x == 4 ? (double)tsqrt(mk) : (double)mk;
    atomicMax(out + threadIdx.x, (unsigned long long)__double_as_longlong(d));
  }
}

// ---- (6) refinement: 8 children predicted from the synchronised parent (Sec. 3.5 step 1) -------
// One CTA per (parent, component); task = [parent rank in the old grid, new slots of children
// 0..7].  src is a copy of the state taken before any child is written (children may reuse the
// parent's slot).  Per component the parent's samples over local [-1, M+1]^3 are put in shared
// memory once: the interior one z-column per thread, the ghost shell from the finest leaf
// holding each point, else by the tensor DD-4 prediction from the even lattice [-4, M+4] (only
// gathered when a neighbour box is coarser).  Each child is then predicted separably (x, then
// y, then z), a thread producing one whole line per pass; the z-pass writes the child, and the
// next child's x-pass runs in the same phase (it writes qx while the z-pass reads qy).
// Dynamic shared memory: pp (M+3)^3, ev/qx, qy in T, then the neighbourhood.
template <typename T, int BS>
struct RefSmem {
  static constexpr int NT = ((BS * BS + 31) / 32) * 32;
  static constexpr int M = BS - 1;
  static constexpr int NPP = M + 3;                 // parent samples per axis: -1..M+1
  static constexpr int NEV = M / 2 + 5;             // even lattice per axis: -4..M+4
  static constexpr int NP = M / 2 + 3;              // samples per axis one child uses
  static constexpr int PP = NPP * NPP * NPP;
  static constexpr int EQ = (NEV * NEV * NEV > NP * NP * BS) ? NEV * NEV * NEV : NP * NP * BS;
  static constexpr int QY = NP * BS * BS;
  static constexpr int NSHELL = PP - BS * BS * BS;  // ghost-shell points
  static constexpr size_t bytes = (size_t)(PP + EQ + QY) * sizeof(T) + kNbhStride * sizeof(int);
};

// Tensor DD-4 prediction at local point (gx, gy, gz) from the even lattice -4..M+4 in ev
// (NEV points per axis; or a window of it starting at even index (bx, by, bz)): z outer, then
// y, then x.
template <typename T, int NEV>
__device__ __forceinline__ T predict_from_even(const T* ev, int gx, int gy, int gz, int bx = 0, int by = 0,
                                               int bz = 0) {
  const int p[3] = {gx, gy, gz};
  const T w[4] = {T(-1) / T(16), T(9) / T(16), T(9) / T(16), T(-1) / T(16)};
  const int o4[4] = {-3, -1, 1, 3};
  int cnt[3];
  for (int a = 0; a < 3; ++a) cnt[a] = (p[a] & 1) ? 4 : 1;
  T accz = T(0);
  for (int kz = 0; kz < cnt[2]; ++kz) {
    const int zz = (((cnt[2] == 4 ? gz + o4[kz] : gz) + 4) >> 1) - bz;
    T accy = T(0);
    for (int ky = 0; ky < cnt[1]; ++ky) {
      const int yy = (((cnt[1] == 4 ? gy + o4[ky] : gy) + 4) >> 1) - by;
      T accx = T(0);
      for (int kx = 0; kx < cnt[0]; ++kx) {
        const int xx = (((cnt[0] == 4 ? gx + o4[kx] : gx) + 4) >> 1) - bx;
        accx = accx + (cnt[0] == 4 ? w[kx] : T(1)) * ev[(zz * NEV + yy) * NEV + xx];
      }
      accy = accy + (cnt[1] == 4 ? w[ky] : T(1)) * accx;
    }
    accz = accz + (cnt[2] == 4 ? w[kz] : T(1)) * accy;
  }
  return accz;
}

template <typename T, int BS>
__global__ void __launch_bounds__(RefSmem<T, BS>::NT, sizeof(T) == 4 ? 3 : 2)
k_refine(const T* src, T* dst, const int32_t* tasks, const int32_t* blist, const int32_t* nbh_all) {
  using L = Lay<T, BS>;
  using S = RefSmem<T, BS>;
  constexpr int M = L::M, NPP = S::NPP, NEV = S::NEV, NP = S::NP, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pp = reinterpret_cast<T*>(smem_raw);
  T* eq = pp + S::PP;                           // even lattice ev, later the x-pass qx
  T* qy = eq + S::EQ;
  int* nbh = reinterpret_cast<int*>(qy + S::QY);
  const int tid = threadIdx.x;
  const int32_t* tk = tasks + (size_t)(blockIdx.x >> 2) * 9;
  const int f = blockIdx.x & 3;
  const int prank = tk[0];
  const int pslot = blist[prank];
  const bool col = tid < BS * BS;
  const int x = col ? tid % BS : 0, y = col ? tid / BS : 0;
  const T NaN = T(__longlong_as_double(0x7ff8000000000000ll));
  auto PPI = [&](int px, int py, int pz) { return ((pz + 1) * NPP + (py + 1)) * NPP + (px + 1); };

  // the parent's interior, one z-column per thread (stored once the loads have arrived)
  const T* pb = src + (size_t)pslot * L::BLK + (size_t)f * L::FS;
  T u[BS];
  if (col) {
#pragma unroll
    for (int z = 0; z < BS; ++z) u[z] = pb[L::idx(x, y, z)];
  }
  for (int i = tid; i < kNbhStride; i += NT) nbh[i] = nbh_all[(size_t)prank * kNbhStride + i];
  __syncthreads();
  const int coarser = __syncthreads_or(tid < 27 && tid != 13 && (nbh[kNbhType + tid] & 15) == kTypeCoarser);
  if (coarser) {
    // even-lattice points -4..M+4 (each held directly by some leaf)
    constexpr int NE3 = NEV * NEV * NEV;
    constexpr int U = (NE3 + NT - 1) / NT;
    long long off[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int i = tid + k * NT;
      off[k] = -2;
      if (i < NE3) {
        const int ex = 2 * (i % NEV) - 4, ey = 2 * ((i / NEV) % NEV) - 4, ez = 2 * (i / (NEV * NEV)) - 4;
        if (ex >= 0 && ex <= M && ey >= 0 && ey <= M && ez >= 0 && ez <= M)
          off[k] = (long long)pslot * L::BLK + (long long)f * L::FS + L::idx(ex, ey, ez);
        else
          off[k] = direct_offset<T, BS>(nbh, ex, ey, ez, f);
      }
    }
    T v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) v[k] = off[k] >= 0 ? src[off[k]] : NaN;
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (off[k] != -2) eq[tid + k * NT] = v[k];
  }
  {
    // ghost shell of [-1, M+1]^3: the z = -1, M+1 planes, then y = -1, M+1 rows (z in 0..M),
    // then x = -1, M+1 (y, z in 0..M)
    constexpr int U = (S::NSHELL + NT - 1) / NT;
    constexpr int NZ = 2 * NPP * NPP, NY = 2 * NPP * BS;
    int gi[U];
    long long off[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      int i = tid + k * NT;
      gi[k] = -1;
      off[k] = -1;
      if (i < S::NSHELL) {
        int gx, gy, gz;
        if (i < NZ) {
          const int r = i % (NPP * NPP);
          gx = r % NPP - 1; gy = r / NPP - 1; gz = i < NZ / 2 ? -1 : M + 1;
        } else if ((i -= NZ) < NY) {
          const int r = i % (NPP * BS);
          gx = r % NPP - 1; gz = r / NPP; gy = i < NY / 2 ? -1 : M + 1;
        } else {
          i -= NY;
          const int r = i % (BS * BS);
          gy = r % BS; gz = r / BS; gx = i < BS * BS ? -1 : M + 1;
        }
        gi[k] = PPI(gx, gy, gz);
        off[k] = direct_offset<T, BS>(nbh, gx, gy, gz, f);
      }
    }
    T v[U];
#pragma unroll
    for (int k = 0; k < U; ++k) v[k] = off[k] >= 0 ? src[off[k]] : T(0);
    if (col) {
#pragma unroll
      for (int z = 0; z < BS; ++z) pp[PPI(x, y, z)] = u[z];
    }
    __syncthreads();                          // ev complete
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (gi[k] < 0) continue;
      if (off[k] < 0) {
        const int i = gi[k];
        v[k] = predict_from_even<T, NEV>(eq, i % NPP - 1, (i / NPP) % NPP - 1, i / (NPP * NPP) - 1);
      }
      pp[gi[k]] = v[k];
    }
  }
  T* qx = eq;
  // x-pass of child c: line (yy, zz) = item; the threads from the top of the CTA take these
  // lines, so that in the phase shared with the previous child's z-pass few threads do both
  auto xpass = [&](int c, int item) {
    const int o0 = (c & 1) * (M / 2) - 1, o1 = ((c >> 1) & 1) * (M / 2) - 1, o2 = ((c >> 2) & 1) * (M / 2) - 1;
    const int yy = item % NP, zz = item / NP;
    T cv[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) cv[k] = pp[PPI(o0 + k, o1 + yy, o2 + zz)];
#pragma unroll
    for (int i = 0; i < BS; ++i) qx[(zz * NP + yy) * BS + i] = dd4_line<T, BS>(cv, i);
  };
  const int xitem = NT - 1 - tid;             // x-pass line of this thread, if < NP^2
  __syncthreads();                            // pp complete
  if (xitem < NP * NP) xpass(0, xitem);
  for (int c = 0; c < 8; ++c) {
    __syncthreads();                          // qx of child c complete, qy free
    if (tid < NP * BS) {                      // y-pass: line (ix, zz)
      const int ix = tid % BS, zz = tid / BS;
      T cv[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) cv[k] = qx[(zz * NP + k) * BS + ix];
#pragma unroll
      for (int i = 0; i < BS; ++i) qy[(zz * BS + i) * BS + ix] = dd4_line<T, BS>(cv, i);
    }
    __syncthreads();                          // qy complete, qx free
    if (col) {                                // z-pass: column (x, y), written to the child
      T cv[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) cv[k] = qy[(k * BS + y) * BS + x];
      T* out = dst + (size_t)tk[1 + c] * L::BLK + (size_t)f * L::FS;
#pragma unroll
      for (int z = 0; z < BS; ++z) out[L::idx(x, y, z)] = dd4_line<T, BS>(cv, z);
    }
    if (c < 7 && xitem < NP * NP) xpass(c + 1, xitem);   // the next child's x-pass alongside
  }
}

// Refinement of Bs = 33 blocks: the parent with its shell, 35^3 values of one component, does
// not fit beside the passes' buffers, so a CTA predicts one child of one component from the
// parent samples that child uses (local [o, o + M/2 + 2]^3, o = -1 or M/2 - 1 per axis): the
// parent's points where it has them, a shell point from the finest leaf holding it, else the
// tensor DD-4 prediction from the even lattice.  Same values as k_refine (the same expressions
// in the same order).  One CTA per (parent, component, child).
template <typename T, int BS>
struct RefBigSmem {
  static constexpr int NT = 1024;
  static constexpr int M = BS - 1;
  static constexpr int NEV = M / 2 + 5;             // even lattice per axis: -4..M+4
  static constexpr int NP = M / 2 + 3;              // samples per axis one child uses
  static constexpr int NW = M / 4 + 5;              // the even points one child's predictions read
  static constexpr int SUB = NP * NP * NP;
  static constexpr int EQ = (NEV * NEV * NEV > NP * NP * BS) ? NEV * NEV * NEV : NP * NP * BS;
  static constexpr int QY = NP * BS * BS;
  static constexpr size_t bytes = (size_t)(SUB + EQ + QY) * sizeof(T) + kNbhStride * sizeof(int);
};

template <typename T, int BS>
__global__ void __launch_bounds__(RefBigSmem<T, BS>::NT, 1)
k_refine_child(const T* src, T* dst, const int32_t* tasks, const int32_t* blist, const int32_t* nbh_all) {
  using L = Lay<T, BS>;
  using S = RefBigSmem<T, BS>;
  constexpr int M = L::M, NW = S::NW, NP = S::NP, NT = S::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sub = reinterpret_cast<T*>(smem_raw);
  T* eq = sub + S::SUB;                         // the child's window of the even lattice, later qx
  T* qy = eq + S::EQ;
  int* nbh = reinterpret_cast<int*>(qy + S::QY);
  const int tid = threadIdx.x;
  const int32_t* tk = tasks + (size_t)(blockIdx.x >> 5) * 9;
  const int f = (blockIdx.x >> 3) & 3, c = blockIdx.x & 7;
  const int prank = tk[0];
  const int pslot = blist[prank];
  const int o[3] = {(c & 1) * (M / 2) - 1, ((c >> 1) & 1) * (M / 2) - 1, ((c >> 2) & 1) * (M / 2) - 1};
  const T NaN = T(__longlong_as_double(0x7ff8000000000000ll));
  const T* pb = src + (size_t)pslot * L::BLK + (size_t)f * L::FS;
  for (int i = tid; i < kNbhStride; i += NT) nbh[i] = nbh_all[(size_t)prank * kNbhStride + i];
  __syncthreads();
  const int coarser = __syncthreads_or(tid < 27 && tid != 13 && (nbh[kNbhType + tid] & 15) == kTypeCoarser);
  // the even points within 3 of the child's samples: local o - 3 .. o + NP + 2, even index
  // b .. b + NW - 1 with b = (o - 3 + 4) / 2 (0 or M/4)
  const int bw[3] = {(o[0] + 1) >> 1, (o[1] + 1) >> 1, (o[2] + 1) >> 1};
  if (coarser) {
    for (int i = tid; i < NW * NW * NW; i += NT) {
      const int ex = 2 * (bw[0] + i % NW) - 4, ey = 2 * (bw[1] + (i / NW) % NW) - 4,
                ez = 2 * (bw[2] + i / (NW * NW)) - 4;
      long long off;
      if (ex >= 0 && ex <= M && ey >= 0 && ey <= M && ez >= 0 && ez <= M)
        off = (long long)pslot * L::BLK + (long long)f * L::FS + L::idx(ex, ey, ez);
      else
        off = direct_offset<T, BS>(nbh, ex, ey, ez, f);
      eq[i] = off >= 0 ? src[off] : NaN;
    }
    __syncthreads();
  }
  for (int i = tid; i < S::SUB; i += NT) {
    const int gx = o[0] + i % NP, gy = o[1] + (i / NP) % NP, gz = o[2] + i / (NP * NP);
    T v;
    if (gx >= 0 && gx <= M && gy >= 0 && gy <= M && gz >= 0 && gz <= M) {
      v = pb[L::idx(gx, gy, gz)];
    } else {
      const long long off = direct_offset<T, BS>(nbh, gx, gy, gz, f);
      v = off >= 0 ? src[off] : predict_from_even<T, NW>(eq, gx, gy, gz, bw[0], bw[1], bw[2]);
    }
    sub[i] = v;
  }
  __syncthreads();
  T* qx = eq;
  if (tid < NP * NP) {                          // x-pass: line (yy, zz)
    const int yy = tid % NP, zz = tid / NP;
    T cv[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) cv[k] = sub[(zz * NP + yy) * NP + k];
#pragma unroll
    for (int i = 0; i < BS; ++i) qx[(zz * NP + yy) * BS + i] = dd4_line<T, BS>(cv, i);
  }
  __syncthreads();
  if (tid < NP * BS) {                          // y-pass: line (ix, zz)
    const int ix = tid % BS, zz = tid / BS;
    T cv[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) cv[k] = qx[(zz * NP + k) * BS + ix];
#pragma unroll
    for (int i = 0; i < BS; ++i) qy[(zz * BS + i) * BS + ix] = dd4_line<T, BS>(cv, i);
  }
  __syncthreads();
  T* out = dst + (size_t)tk[1 + c] * L::BLK + (size_t)f * L::FS;
  for (int col = tid; col < BS * BS; col += NT) {   // z-pass: column (x, y), written to the child
    const int x = col % BS, y = col / BS;
    T cv[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) cv[k] = qy[(k * BS + y) * BS + x];
#pragma unroll
    for (int z = 0; z < BS; ++z) out[L::idx(x, y, z)] = dd4_line<T, BS>(cv, z);
  }
}

// ---- (7) coarsening: parent by decimation of its 8 children (Sec. 3.1 R, Sec. 3.5 step 3) ----
// task = [new parent slot, old child slots 0..7]; dst is a register other than src (a parent
// may take a slot freed by a child that another CTA is still reading): the parents are copied
// into the state afterwards.
// One CTA per (task, component); a thread owns one z-column of the parent (two for Bs = 33)
// and has all its loads in flight before it stores.
template <int BS>
struct ColCfg {
  // a thread per (x, y) column; above 1024 columns (Bs = 33) a thread takes two
  static constexpr int NT = BS * BS <= 1024 ? ((BS * BS + 31) / 32) * 32 : ((BS * BS / 2 + 32) / 32) * 32;
};

template <typename T, int BS>
__global__ void __launch_bounds__(ColCfg<BS>::NT) k_coarsen(const T* src, T* dst, const int32_t* tasks) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int32_t* tk = tasks + (size_t)(blockIdx.x >> 2) * 9;
  const int f = blockIdx.x & 3;
  for (int col = threadIdx.x; col < BS * BS; col += ColCfg<BS>::NT) {
    const int x = col % BS, y = col / BS;
    const int cx = x > M / 2, cy = y > M / 2;
    const int lx = 2 * x - cx * M, ly = 2 * y - cy * M;
    const T* c0 = src + (size_t)tk[1 + (cx | (cy << 1))] * L::BLK + (size_t)f * L::FS;       // cz = 0
    const T* c1 = src + (size_t)tk[1 + (cx | (cy << 1) | 4)] * L::BLK + (size_t)f * L::FS;   // cz = 1
    T v[BS];
#pragma unroll
    for (int z = 0; z < BS; ++z) v[z] = z <= M / 2 ? c0[L::idx(lx, ly, 2 * z)] : c1[L::idx(lx, ly, 2 * z - M)];
    T* out = dst + (size_t)tk[0] * L::BLK + (size_t)f * L::FS;
#pragma unroll
    for (int z = 0; z < BS; ++z) out[L::idx(x, y, z)] = v[z];
  }
}

// ---- (7b) CDF 4/4 coarsening (Sec. 3.2.1 lifted wavelet, Sec. 3.5 step 3) ------------------------
// The parent's interior points (1..M-1 per axis) take the CDF 4/4 analysis low-pass of the
// level-(J+1) point values around the sister group; its boundary points keep the decimated
// child values, so a redundant point that the parent shares with a same-level leaf not merged
// in this pass keeps the value that leaf holds.  The low-pass is the primal lifting of the cubic
// interpolating transform: details d_j = f_{2j+1} - (-f_{2j-2} + 9 f_{2j} + 9 f_{2j+2} - f_{2j+4})/16,
// then c_i = f_{2i} + (-d_{i-2} + 9 d_{i-1} + 9 d_i - d_{i+1})/32 (the update weights that give
// the lifted wavelet 4 vanishing moments).  Expanded, c_i is the symmetric 13-tap filter
// (348; 144, -63, -16, 18, 0, -1)/512 on f_{2i}, f_{2i+-1}, ..., f_{2i+-6}, applied here along
// x, then y, then z.  It reaches 6 fine points past the parent's points 1 and M-1, i.e. 4 past
// the group: the fine values there are the children's ghost values (finest leaf holding the
// point, else the tensor DD-4 prediction from the coarse lattice).
// task = [new parent slot, old child slots 0..7, rank of child 0] (the children are 8
// consecutive blocks of the old order); dst is a register other than src.
//
// One CTA per task, all four components together (each point is looked up once).  The 64
// child-sized boxes around and inside the group (-1..2 per axis, in units of a child) are read
// once from the children's neighbourhoods into a box table, so a lookup is a few shifts and one
// shared-memory read.  If a box is coarser than the children, the offsets of the even fine points
// -6..2M+6 (the coarse lattice, held directly by some leaf) are tabled as well and the points
// that must be predicted take the tensor DD-4 sum of their stencil from there.  The fine lattice
// -4..2M+4 of the group is streamed one z-plane at a time: the loads of the next plane are in
// flight while the current one is filtered along x, then y; the x-y filtered values of each
// (component, parent column) are kept for the last 13 planes, and a parent point's z-pass runs as
// soon as its 13th plane has arrived.
template <typename T, int BS>
struct C44Smem {
  static constexpr int M = BS - 1;
  static constexpr int LM = M == 16 ? 4 : 3;  // log2 M
  static constexpr int NF = 2 * M + 9;        // fine points per axis: -4..2M+4
  static constexpr int NI = M - 1;            // filtered parent points per axis: 1..M-1
  static constexpr int NEV = M + 7;           // even fine points per axis: -6..2M+6
  static constexpr int RING = 13;             // planes one z-output reads
  static constexpr int NT = BS == 17 ? 512 : 128;
  static constexpr int UP = (NF * NF + NT - 1) / NT;   // plane points per thread
  static constexpr int NCOL = 4 * NI * NI;             // (component, parent column) items
  static constexpr int PL = 4 * NF * NF, TX = 4 * NF * NI, RG = RING * NCOL, EV = NEV * NEV * NEV;
  static constexpr size_t bytes = 64 * sizeof(int4) + (size_t)(PL + TX + RG) * sizeof(T) + (size_t)EV * sizeof(uint32_t);
};
static_assert(C44Smem<double, 17>::bytes <= 227 * 1024, "CDF 4/4 coarsening: shared memory");

// The expanded lifting filter at p[0] = f_{2i}, neighbours s elements apart.
template <typename T>
__device__ __forceinline__ T cdf44_lowpass(const T* p, int s) {
  T acc = T(348) * p[0];
  acc = fma(T(144), p[-s] + p[s], acc);
  acc = fma(T(-63), p[-2 * s] + p[2 * s], acc);
  acc = fma(T(-16), p[-3 * s] + p[3 * s], acc);
  acc = fma(T(18), p[-4 * s] + p[4 * s], acc);
  acc = acc - (p[-6 * s] + p[6 * s]);
  return acc * (T(1) / T(512));
}

constexpr uint32_t kOffPred = 0xFFFFFFFEu;    // the point must be predicted
constexpr uint32_t kOffBad = 0xFFFFFFFFu;     // no leaf holds the point (not a graded grid)

template <typename T, int BS>
__global__ void __launch_bounds__(C44Smem<T, BS>::NT, 1) k_coarsen44(const T* src, T* dst, const int32_t* tasks,
                                                                     const int32_t* nbh_all) {
  using L = Lay<T, BS>;
  using S = C44Smem<T, BS>;
  constexpr int M = L::M, LM = S::LM, NF = S::NF, NI = S::NI, NEV = S::NEV, NT = S::NT, UP = S::UP;
  constexpr int RING = S::RING, NCOL = S::NCOL, NF2 = NF * NF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 16-byte box table first, then the T arrays (8-byte aligned), the 4-byte offsets last
  int4* gb = reinterpret_cast<int4*>(smem_raw);              // box table [bz+1][by+1][bx+1]
  T* pl = reinterpret_cast<T*>(gb + 64);                     // pl[f][Y][X]: one fine plane
  T* tx = pl + S::PL;                                        // tx[f][Y][i]: filtered along x
  T* rg = tx + S::TX;                                        // rg[plane % 13][item]: along x and y
  uint32_t* ev = reinterpret_cast<uint32_t*>(rg + S::RG);    // ev[Z][Y][X]: offsets of even points
  __shared__ int cslot[8];
  const int tid = threadIdx.x;
  const int32_t* tk = tasks + (size_t)blockIdx.x * 10;
  const int r0 = tk[9];
  const T NaN = T(__longlong_as_double(0x7ff8000000000000ll));
  if (tid < 8) cslot[tid] = tk[1 + tid];
  int mine = 0;
  if (tid < 64) {
    // box (bx, by, bz) seen from the child next to it; children see themselves as box 13
    const int bx = tid % 4 - 1, by = (tid / 4) % 4 - 1, bz = tid / 16 - 1;
    const int cx = bx < 0 ? 0 : (bx > 1 ? 1 : bx), cy = by < 0 ? 0 : (by > 1 ? 1 : by),
              cz = bz < 0 ? 0 : (bz > 1 ? 1 : bz);
    const int d = box_index(bx - cx, by - cy, bz - cz);
    const size_t rowi = (size_t)(r0 + (cx | (cy << 1) | (cz << 2))) * kNbhStride;
    const int tw = nbh_all[rowi + kNbhType + d];
    int4 g = make_int4(tw, nbh_all[rowi + 8 * d], 0, 0);
    if ((tw & 15) == kTypeRefined) g.y = (int)(rowi + 8 * d);   // where its children's slots are
    gb[tid] = g;
    mine = (tw & 15) == kTypeCoarser;
  }
  const int coarser = __syncthreads_or(mine);
  // Element offset (component 0) of fine point P of the group's lattice (-6..2M+6 per axis) in the
  // finest leaf holding it: candidate boxes b = floor(P/M), and b - 1 if P is on their face.
  auto group_offset = [&](int X, int Y, int Z) -> uint32_t {
    const int P[3] = {X, Y, Z};
    int b[3], nc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      b[a] = ((P[a] + M) >> LM) - 1;
      nc[a] = (P[a] & (M - 1)) == 0 ? 2 : 1;
    }
    int best = 0, bestp = 0, bb[3] = {0, 0, 0};
    for (int kz = 0; kz < nc[2]; ++kz)
      for (int ky = 0; ky < nc[1]; ++ky)
        for (int kx = 0; kx < nc[0]; ++kx) {
          const int e = ((b[2] - kz + 1) * 4 + (b[1] - ky + 1)) * 4 + (b[0] - kx + 1);
          const int t = gb[e].x & 15;
          const int pr = t == kTypeRefined ? 3 : (t == kTypeLeaf ? 2 : (t == kTypeCoarser ? 1 : 0));
          if (pr > bestp) {
            bestp = pr;
            best = e;
            bb[0] = b[0] - kx; bb[1] = b[1] - ky; bb[2] = b[2] - kz;
          }
        }
    if (bestp == 0) return kOffBad;
    const int4 g = gb[best];
    int q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = P[a] - bb[a] * M;   // 0..M inside the box
    if (bestp == 2) return (uint32_t)g.y * (uint32_t)L::BLK + (uint32_t)L::idx(q[0], q[1], q[2]);
    if (bestp == 1) {
      const int oct = g.x >> 4;
      int r[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] = ((oct >> a) & 1) * M + q[a];
      if ((r[0] | r[1] | r[2]) & 1) return kOffPred;
      return (uint32_t)g.y * (uint32_t)L::BLK + (uint32_t)L::idx(r[0] >> 1, r[1] >> 1, r[2] >> 1);
    }
    int c = 0, l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ca = q[a] > M / 2;
      c |= ca << a;
      l[a] = 2 * q[a] - ca * M;
    }
    const int sl = nbh_all[(size_t)g.y + c];
    return sl < 0 ? kOffBad : (uint32_t)sl * (uint32_t)L::BLK + (uint32_t)L::idx(l[0], l[1], l[2]);
  };
  if (coarser) {
    for (int i = tid; i < S::EV; i += NT) {
      const uint32_t o = group_offset(2 * (i % NEV) - 6, 2 * ((i / NEV) % NEV) - 6, 2 * (i / (NEV * NEV)) - 6);
      ev[i] = o == kOffPred ? kOffBad : o;
    }
  }
  auto load = [&](uint32_t o, int f) -> T { return o < kOffPred ? src[(size_t)o + (size_t)f * L::FS] : NaN; };
  // tensor DD-4 prediction of the 4 components at fine point (X, Y, Z): x innermost, then y, z
  auto predict = [&](int X, int Y, int Z, T (&v)[4]) {
    const bool ox = X & 1, oy = Y & 1, oz = Z & 1;
    T az[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
      if (!oz && kz) continue;
      const int zz = ((oz ? Z + 2 * kz - 3 : Z) + 6) >> 1;
      const T wz = oz ? ((kz == 0 || kz == 3) ? T(-1) / T(16) : T(9) / T(16)) : T(1);
      T ay[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        if (!oy && ky) continue;
        const int yy = ((oy ? Y + 2 * ky - 3 : Y) + 6) >> 1;
        const T wy = oy ? ((ky == 0 || ky == 3) ? T(-1) / T(16) : T(9) / T(16)) : T(1);
        T ax[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
          if (!ox && kx) continue;
          const int xx = ((ox ? X + 2 * kx - 3 : X) + 6) >> 1;
          const T wx = ox ? ((kx == 0 || kx == 3) ? T(-1) / T(16) : T(9) / T(16)) : T(1);
          const uint32_t o = ev[(zz * NEV + yy) * NEV + xx];
#pragma unroll
          for (int f = 0; f < 4; ++f) ax[f] = ax[f] + wx * load(o, f);
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) ay[f] = ay[f] + wy * ax[f];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) az[f] = az[f] + wz * ay[f];
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) v[f] = az[f];
  };
  // Per-thread geometry, the same in every plane.  Plane points are enumerated so that warps
  // meet one kind of point: in a plane that cuts the group, first its (2M+1)^2 points inside the
  // group, then the ring around them (4 rows below, 4 rows above, then 4 + 4 points on each side
  // of the rows in between); a plane outside the group row by row.
  constexpr int UX = (4 * NF * NI + NT - 1) / NT, UY = (NCOL + NT - 1) / NT;
  constexpr int NG = 2 * M + 1, NGI = NG * NG;
  int gx[UP], gy[UP], sx[UP], sy[UP];               // -1000: no point
#pragma unroll
  for (int k = 0; k < UP; ++k) {
    const int p = tid + k * NT;
    if (p < NGI) {
      gx[k] = p % NG; gy[k] = p / NG;
    } else if (p < NF2) {
      const int q = p - NGI;
      if (q < 4 * NF) { gx[k] = q % NF - 4; gy[k] = q / NF - 4; }
      else if (q < 8 * NF) { gx[k] = (q - 4 * NF) % NF - 4; gy[k] = 2 * M + 1 + (q - 4 * NF) / NF; }
      else { const int r = q - 8 * NF, e = r % 8; gy[k] = r / 8; gx[k] = e < 4 ? e - 4 : 2 * M + 1 + (e - 4); }
    } else {
      gx[k] = -1000; gy[k] = 0;
    }
    sx[k] = p < NF2 ? p % NF - 4 : -1000;
    sy[k] = p / NF - 4;
  }
  int xs[UX];                                       // x-pass: pl offset of f_{2i} (-1: none)
#pragma unroll
  for (int u = 0; u < UX; ++u) {
    const int it = tid + u * NT;
    const int f = it / (NF * NI), r = it % (NF * NI);
    xs[u] = it < 4 * NF * NI ? f * NF2 + (r / NI) * NF + 2 * (r % NI + 1) + 4 : -1;
  }
  int ys[UY], yo[UY];                               // y-pass: tx offset; parent offset at z = 0
#pragma unroll
  for (int u = 0; u < UY; ++u) {
    const int it = tid + u * NT;
    const int f = it / (NI * NI), r = it % (NI * NI);
    const int j = r / NI + 1, i = r % NI;
    ys[u] = it < NCOL ? f * NF * NI + (2 * j + 4) * NI + i : -1;
    yo[u] = f * L::FS + L::idx(i + 1, j, 0);
  }
  uint32_t poff[UP];
  T pv[UP][4];
  int px[UP], py[UP];                               // the points of the plane in flight
  auto issue = [&](int Z) {                         // offsets and loads of plane Z
    const int cz = Z > M, lz = Z - cz * M;
    const bool zin = Z >= 0 && Z <= 2 * M;
#pragma unroll
    for (int k = 0; k < UP; ++k) {
      const int X = zin ? gx[k] : sx[k], Y = zin ? gy[k] : sy[k];
      px[k] = X;
      py[k] = Y;
      uint32_t o = kOffBad;
      if (X != -1000) {
        if (zin && X >= 0 && X <= 2 * M && Y >= 0 && Y <= 2 * M) {
          const int cx = X > M, cy = Y > M;
          o = (uint32_t)cslot[cx | (cy << 1) | (cz << 2)] * (uint32_t)L::BLK +
              (uint32_t)L::idx(X - cx * M, Y - cy * M, lz);
        } else {
          o = group_offset(X, Y, Z);
        }
      }
      poff[k] = o;
    }
#pragma unroll
    for (int k = 0; k < UP; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) pv[k][f] = load(poff[k], f);
  };
  auto finish = [&](int Z) {                        // plane Z into pl, predicted points filled in
#pragma unroll
    for (int k = 0; k < UP; ++k) {
      if (px[k] == -1000) continue;
      if (poff[k] == kOffPred && coarser) predict(px[k], py[k], Z, pv[k]);
      const int i = (py[k] + 4) * NF + (px[k] + 4);
#pragma unroll
      for (int f = 0; f < 4; ++f) pl[f * NF2 + i] = pv[k][f];
    }
  };
  T* out = dst + (size_t)tk[0] * L::BLK;
  __syncthreads();                                  // ev complete
  issue(-4);
  int slot = 0;                                     // ring slot of the current plane
  for (int Z = -4; Z <= 2 * M + 4; ++Z) {
    finish(Z);
    __syncthreads();                                // pl complete; tx free
    if (Z < 2 * M + 4) issue(Z + 1);
#pragma unroll
    for (int u = 0; u < UX; ++u)                    // x-pass: component, row Y, parent index
      if (xs[u] >= 0) tx[tid + u * NT] = cdf44_lowpass(pl + xs[u], 1);
    __syncthreads();                                // tx complete; pl free
    const int zi = Z + 4;
    const bool zpass = zi >= 12 && !(zi & 1);       // plane 2k + 6 arrived: z-pass of point k
#pragma unroll
    for (int u = 0; u < UY; ++u) {                  // y-pass, then the z-pass once complete
      if (ys[u] < 0) continue;
      const int it = tid + u * NT;
      rg[slot * NCOL + it] = cdf44_lowpass(tx + ys[u], NI);
      if (zpass) {
        T a[RING];
#pragma unroll
        for (int n = 0; n < RING; ++n) {            // plane zi - 12 + n sits in slot + 1 + n (mod 13)
          int sn = slot + 1 + n;
          sn -= sn >= RING ? RING : 0;
          a[n] = rg[sn * NCOL + it];
        }
        out[yo[u] + ((Z - 6) >> 1) * L::PP] = cdf44_lowpass(a + 6, 1);
      }
    }
    slot = slot + 1 == RING ? 0 : slot + 1;
  }
  for (int p = tid; p < BS * BS * BS; p += NT) {   // boundary points: decimated children
    const int x = p % BS, y = (p / BS) % BS, z = p / (BS * BS);
    if (x > 0 && x < M && y > 0 && y < M && z > 0 && z < M) continue;
    const int cx = x > M / 2, cy = y > M / 2, cz = z > M / 2;
    const size_t o = (size_t)cslot[cx | (cy << 1) | (cz << 2)] * L::BLK +
                     L::idx(2 * x - cx * M, 2 * y - cy * M, 2 * z - cz * M);
#pragma unroll
    for (int f = 0; f < 4; ++f) out[(size_t)f * L::FS + L::idx(x, y, z)] = src[o + (size_t)f * L::FS];
  }
}

// ---- copy of whole blocks (same slots) between two registers --------------------------------------
// Slots list[i * stride], i = 0..n-1.
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_copy_blocks(const T* src, T* dst, const int32_t* list, int stride) {
  using L = Lay<T, BS>;
  const size_t base = (size_t)list[(size_t)blockIdx.x * stride] * L::BLK;
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
  const double h = ph.h[bi.x];
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
    } else if (ic.kind == 4) {   // pulse + vortex ring (curl of an azimuthal vector potential)
      const double c[3] = {ic.p[0], ic.p[1], ic.p[2]}, Lb[3] = {ic.p[5], ic.p[6], ic.p[7]};
      const double P[3] = {X, Y, Z};
      double r2 = 0.0, d[3];
      for (int a = 0; a < 3; ++a) {
        double e = P[a] - c[a];
        e = e - Lb[a] * rint(e / Lb[a]);
        r2 += e * e;
        double g = P[a] - ic.p[8 + a];
        d[a] = g - Lb[a] * rint(g / Lb[a]);
      }
      v[3] = ic.p[4] * exp(-r2 / (ic.p[3] * ic.p[3]));
      const double nn = sqrt(ic.p[11] * ic.p[11] + ic.p[12] * ic.p[12] + ic.p[13] * ic.p[13]);
      const double n[3] = {ic.p[11] / nn, ic.p[12] / nn, ic.p[13] / nn};
      const double R = ic.p[14], gam = ic.p[15], sg = ic.p[16];
      const double zeta = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
      double rp[3], rho2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        rp[a] = d[a] - zeta * n[a];
        rho2 += rp[a] * rp[a];
      }
      const double rho = sqrt(rho2);
      const double E = exp(-((rho - R) * (rho - R) + zeta * zeta) / (sg * sg));
      const double K = gam * E / (2.0 * 3.14159265358979323846 * R);
      const double ar = K * 2.0 * zeta / (sg * sg), an = K * (2.0 - 2.0 * rho * (rho - R) / (sg * sg));
      for (int a = 0; a < 3; ++a) v[a] = ar * rp[a] + an * n[a];
    }
    const int pi = L::idx(ix, iy, iz);
#pragma unroll
    for (int f = 0; f < 4; ++f) reg[(size_t)slot * L::BLK + (size_t)f * L::FS + pi] = T(v[f]);
  }
}

// chi along the z-column (ix, iy) of one block (out: the block's mask component).
template <typename T, int BS>
__device__ __forceinline__ void mask_column(T* out, const int ix, const int iy, const int uniform, const int4 bi,
                                            const PhysK& ph, const MaskK& m, const double h) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  if (uniform >= 0) {
#pragma unroll
    for (int iz = 0; iz < BS; ++iz) out[L::idx(ix, iy, iz)] = T(uniform);
    return;
  }
  if (m.kind == 2) {
    // signed distance to the box in the body frame, in the field precision
    const T hT = T(h);
    T Rm[9], x0[3], cb[3], hb[3];
    for (int k = 0; k < 9; ++k) Rm[k] = T(m.p[k]);
    for (int a = 0; a < 3; ++a) {
      x0[a] = T(m.p[9 + a]);
      cb[a] = T(m.p[12 + a]);
      hb[a] = T(m.p[15 + a]);
    }
    const T dl = T(m.p[18]);
    const T cut = T(sizeof(T) == 4 ? 10.0 : 20.0) * dl;
    const T rx = T(lattice(ph, bi, 0, ix, M)) * hT - x0[0], ry = T(lattice(ph, bi, 1, iy, M)) * hT - x0[1];
    for (int iz = 0; iz < BS; ++iz) {
      const T rz = T(lattice(ph, bi, 2, iz, M)) * hT - x0[2];
      T out2 = T(0), qmax = T(-1e30);
      for (int k = 0; k < 3; ++k) {
        const T xb = Rm[k] * rx + Rm[3 + k] * ry + Rm[6 + k] * rz;     // (R^T r)_k
        const T q = (xb - cb[k] < T(0) ? cb[k] - xb : xb - cb[k]) - hb[k];
        if (q > T(0)) out2 += q * q;
        qmax = q > qmax ? q : qmax;
      }
      const T d = tsqrt(out2) + (qmax < T(0) ? qmax : T(0));
      T c;
      if (d > cut) c = T(0);
      else if (d < -cut) c = T(1);
      else c = T(0.5) * (T(1) - ttanh(d / dl));
      out[L::idx(ix, iy, iz)] = c;
    }
    return;
  }
  // evaluated in the field precision: FP64 fields in double, FP32 fields in float; the
  // conversions of the constants are done once, outside the point loop
  const T hT = T(h);
  const T c0 = T(m.p[0]), c1 = T(m.p[1]), c2 = T(m.p[2]), R = T(m.p[3]), dl = T(m.p[4]);
  // beyond 10 delta (FP32) / 20 delta (FP64) tanh(d/delta) rounds to exactly +-1
  const T cut = T(sizeof(T) == 4 ? 10.0 : 20.0) * dl;
  // coordinates i h with i the wrapped lattice index (exact when h is dyadic, as for
  // power-of-two root sides)
  const T dx = T(lattice(ph, bi, 0, ix, M)) * hT - c0, dy = T(lattice(ph, bi, 1, iy, M)) * hT - c1;
#pragma unroll
  for (int iz = 0; iz < BS; ++iz) {
    const T dz = T(lattice(ph, bi, 2, iz, M)) * hT - c2;
    const T d = tsqrt(dx * dx + dy * dy + dz * dz) - R;
    T c;
    if (d > cut) c = T(0);
    else if (d < -cut) c = T(1);
    else c = T(0.5) * (T(1) - ttanh(d / dl));
    out[L::idx(ix, iy, iz)] = c;
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(ColCfg<BS>::NT) k_mask(T* chi, const int32_t* blist, const int32_t* ranks,
                                                         const int4* binfo, const PhysK ph, const MaskK m) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int rank = ranks ? ranks[blockIdx.x] : (int)blockIdx.x;
  const int slot = blist[rank];
  const int4 bi = binfo[rank];
  const double h = ph.h[bi.x];
  // A block that lies entirely farther than 40 delta from the sphere surface has tanh(d/delta)
  // = +-1 exactly in double precision at all its points (1 - tanh(40) < 1e-34): chi is exactly
  // 0 or 1 there and needs no transcendental.  Blocks on the periodic seam are evaluated fully.
  // One thread decides (FP64), the block reads the answer.
  __shared__ int s_uniform;
  if (threadIdx.x == 0) {
    int uniform = 0;
    if (m.kind == 1) {
      uniform = -1;
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
    } else if (m.kind == 2) {
      // rigid box: outside the sphere of radius p[22] around the pivot by more than 40 delta
      uniform = -1;
      const double lo[3] = {(double)bi.y * M * h, (double)bi.z * M * h, (double)bi.w * M * h};
      const double L[3] = {ph.nroot[0] * ph.root_len, ph.nroot[1] * ph.root_len, ph.nroot[2] * ph.root_len};
      bool seam = false;
      double dmin2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double hi = lo[a] + M * h;
        if (hi >= L[a]) seam = true;
        const double c = m.p[9 + a];
        const double near = c < lo[a] ? lo[a] - c : (c > hi ? c - hi : 0.0);
        dmin2 += near * near;
      }
      if (!seam && sqrt(dmin2) - m.p[22] > 40.0 * m.p[18]) uniform = 0;
    }
    s_uniform = uniform;
  }
  __syncthreads();
  const int uniform = s_uniform;
  for (int col = threadIdx.x; col < BS * BS; col += ColCfg<BS>::NT)
    mask_column<T, BS>(chi + (size_t)slot * L::FS, col % BS, col / BS, uniform, bi, ph, m, h);
}

// ---- (9) diagnostics: raw per-block sums over the half-open points [0, M-1]^3 -----------------
// Penalization source of a rotating rigid body (mask kind 2): S = chi (omega x (x - x_0)) / C_eta,
// added to the stage outputs (out += c_out S, acc += c_acc S).  FP64 arithmetic per point is
// avoided for FP32 fields: the pose arrives in double and is converted once.
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_solid_source(T* out, T* acc, const T* chi, const int32_t* blist,
                                                      const int4* binfo, const PhysK ph, const MaskK m, double c_out,
                                                      double c_acc, int acc_too) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const T hT = T(ph.h[bi.x]);
  const T w0 = T(m.p[19]), w1 = T(m.p[20]), w2 = T(m.p[21]);
  const T x0 = T(m.p[9]), y0 = T(m.p[10]), z0 = T(m.p[11]);
  const T ci = T(ph.inv_ceta), co = T(c_out), ca = T(c_acc);
  const size_t base = (size_t)slot * L::BLK;
  for (int t = threadIdx.x; t < BS * BS * BS; t += kNT) {
    const int x = t % BS, y = (t / BS) % BS, z = t / (BS * BS);
    const int pi = L::idx(x, y, z);
    const T c = chi[(size_t)slot * L::FS + pi];
    if (c == T(0)) continue;
    const T rx = T(lattice(ph, bi, 0, x, M)) * hT - x0;
    const T ry = T(lattice(ph, bi, 1, y, M)) * hT - y0;
    const T rz = T(lattice(ph, bi, 2, z, M)) * hT - z0;
    const T s[3] = {c * ci * (w1 * rz - w2 * ry), c * ci * (w2 * rx - w0 * rz), c * ci * (w0 * ry - w1 * rx)};
    for (int a = 0; a < 3; ++a) {
      out[base + (size_t)a * L::FS + pi] += co * s[a];
      if (acc_too) acc[base + (size_t)a * L::FS + pi] += ca * s[a];
    }
  }
}

// Per block sums over the half-open points of chi u_s (force of a moving body, Sec. 2.2).
template <typename T, int BS>
__global__ void __launch_bounds__(kNT) k_solid_moment(const T* chi, const int32_t* blist, const int4* binfo,
                                                      const PhysK ph, const MaskK m, double* out) {
  using L = Lay<T, BS>;
  constexpr int M = L::M;
  const int slot = blist[blockIdx.x];
  const int4 bi = binfo[blockIdx.x];
  const double h = ph.h[bi.x];
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < M * M * M; i += kNT) {
    const int x = i % M, y = (i / M) % M, z = i / (M * M);
    const double c = chi[(size_t)slot * L::FS + L::idx(x, y, z)];
    if (c == 0.0) continue;
    const double rx = lattice(ph, bi, 0, x, M) * h - m.p[9];
    const double ry = lattice(ph, bi, 1, y, M) * h - m.p[10];
    const double rz = lattice(ph, bi, 2, z, M) * h - m.p[11];
    s[0] += c * (m.p[20] * rz - m.p[21] * ry);
    s[1] += c * (m.p[21] * rx - m.p[19] * rz);
    s[2] += c * (m.p[19] * ry - m.p[20] * rx);
  }
  __shared__ double red[3][kNT / 32];
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
  if ((threadIdx.x & 31) == 0)
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x >> 5] = s[k];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    if (threadIdx.x < 3)
      for (int w = 0; w < kNT / 32; ++w) t += red[threadIdx.x][w];
    out[(size_t)blockIdx.x * 4 + threadIdx.x] = t;
  }
}

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

// Objective terms on the device: acc += wF C_eta^-1 sum_r h_r^3 part[4r] + wE sum_r h_r^3 part[4r+3] / 2
// over the per-block sums of k_diag (or, with wE = 0, of k_solid_moment), one CTA, each thread's
// blocks in a fixed order and a fixed reduction tree, so the sum is the same on every call.
__global__ void __launch_bounds__(1024) k_diag_sum(const double* part, const int4* binfo, int64_t n, const PhysK ph,
                                                   double wF, double wE, double* acc) {
  __shared__ double red[1024];
  double v = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
    const double h = ph.h[binfo[r].x];
    const double h3 = h * h * h;
    v += wF * part[4 * r] * h3 * ph.inv_ceta + wE * 0.5 * part[4 * r + 3] * h3;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += red[0];
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
__global__ void __launch_bounds__(kNT) k_scatter(const T* dense, T* reg, const int32_t* blist, int ncomp, int comp_stride_blk) {
  using L = Lay<T, BS>;
  const int slot = blist[blockIdx.x];
  const int n = ncomp * BS * BS * BS;
  for (int i = threadIdx.x; i < n; i += kNT) {
    const int f = i / (BS * BS * BS), r = i % (BS * BS * BS);
    const int x = r % BS, y = (r / BS) % BS, z = r / (BS * BS);
    reg[(size_t)slot * comp_stride_blk + (size_t)f * L::FS + L::idx(x, y, z)] = dense[(size_t)blockIdx.x * n + i];
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
    if (Bs == 33) { ACM_FILL(double, 33) } else if (Bs == 17) { ACM_FILL(double, 17) } else { ACM_FILL(double, 9) }
  } else {
    if (Bs == 33) { ACM_FILL(float, 33) } else if (Bs == 17) { ACM_FILL(float, 17) } else { ACM_FILL(float, 9) }
  }
#undef ACM_FILL
  return li;
}

// Bs = 33 blocks are FP32 only (the forest refuses FP64 with them).
#define ACM_BS_DISPATCH(Bs, KERNEL, ...)                                      \
  do {                                                                        \
    if ((Bs) == 33) {                                                         \
      if constexpr (sizeof(T) == 4) { KERNEL<T, 33> __VA_ARGS__; }            \
    } else if ((Bs) == 17) { KERNEL<T, 17> __VA_ARGS__; }                     \
    else { KERNEL<T, 9> __VA_ARGS__; }                                        \
  } while (0)

template <typename T>
void launch_fine_wins(int Bs, T* reg, const int2* tasks, const int32_t* ntasks, int64_t max_tasks,
                      const int32_t* nbh, const int32_t* blist, int ctas_per_sm, cudaStream_t st) {
  if (max_tasks <= 0) return;
  const int64_t g = std::min<int64_t>(max_tasks, (int64_t)std::max(1, ctas_per_sm) * sm_count());
  ACM_BS_DISPATCH(Bs, k_fine_wins, <<<grid1(g), kNT, 0, st>>>(reg, tasks, ntasks, nbh, blist));
}
template <typename T, int BS>
void launch_coarse_slabs_bs(const T* reg, T* slab, const int4* tasks, const int32_t* ntasks, int64_t max_tasks,
                            const int32_t* nbh, uint32_t* offc, int use_cache, int ctas_per_sm, cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0};   // devices whose context has the opt-in
  smem_opt_in(k_coarse_slabs<T, BS>, SlabSmem<T, BS>::bytes, opted);
  // CTAs walking the task list: ctas_per_sm per SM (at most 3 are resident for Bs = 17)
  const int64_t g = std::min<int64_t>(max_tasks, (int64_t)std::max(1, ctas_per_sm) * sm_count());
  k_coarse_slabs<T, BS><<<grid1(g), SlabSmem<T, BS>::NT, SlabSmem<T, BS>::bytes, st>>>(reg, slab, tasks, ntasks, nbh,
                                                                                       offc, use_cache);
}
template <typename T>
void launch_coarse_slabs(int Bs, const T* reg, T* slab, const int4* tasks, const int32_t* ntasks, int64_t max_tasks,
                         const int32_t* nbh, uint32_t* offc, int use_cache, int ctas_per_sm, cudaStream_t st) {
  if (max_tasks <= 0) return;
  if (Bs == 33) {
    // one CTA per SM is resident (166 KB of shared memory)
    if constexpr (sizeof(T) == 4)
      launch_coarse_slabs_bs<T, 33>(reg, slab, tasks, ntasks, max_tasks, nbh, offc, use_cache, 1, st);
  } else if (Bs == 17) {
    launch_coarse_slabs_bs<T, 17>(reg, slab, tasks, ntasks, max_tasks, nbh, offc, use_cache, ctas_per_sm, st);
  } else {
    launch_coarse_slabs_bs<T, 9>(reg, slab, tasks, ntasks, max_tasks, nbh, offc, use_cache, ctas_per_sm, st);
  }
}
size_t slab_offset_words(int Bs) {
  return Bs == 33 ? SlabSmem<float, 33>::NOFF : (Bs == 17 ? SlabSmem<float, 17>::NOFF : SlabSmem<float, 9>::NOFF);
}
template <typename T>
void launch_sync_ext(int Bs, const T* reg, T* out, int g, const int32_t* list, int64_t n, const int32_t* nbh, int by_rank, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_sync_ext, <<<grid1(n), kNT, 0, st>>>(reg, out, g, list, nbh, by_rank));
}
template <typename T, int BS>
void launch_details_bs(const T* reg, const T* chi, const int32_t* blist, const int32_t* ranks, const int32_t* nbh,
                       int64_t n, const unsigned long long* norm_bits, double* ind, double* chirange, cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0};   // devices whose context has the opt-in
  smem_opt_in(k_details<T, BS>, DetSmem<T, BS>::bytes, opted);
  k_details<T, BS><<<grid1(n), DetSmem<T, BS>::NT, DetSmem<T, BS>::bytes, st>>>(reg, chi, blist, ranks, nbh,
                                                                              norm_bits, ind, chirange);
}
template <typename T>
void launch_details(int Bs, const T* reg, const T* chi, const int32_t* blist, const int32_t* ranks,
                    const int32_t* nbh, int64_t n, const unsigned long long* norm_bits, double* ind,
                    double* chirange, cudaStream_t st) {
  if (n <= 0) return;
  if (Bs == 33) {
    if constexpr (sizeof(T) == 4) {
      static std::atomic<unsigned long long> opted{0};
      smem_opt_in(k_details_big<T, 33>, DetBigSmem<T, 33>::bytes, opted);
      k_details_big<T, 33><<<grid1(n), DetBigSmem<T, 33>::NT, DetBigSmem<T, 33>::bytes, st>>>(
          reg, chi, blist, ranks, nbh, norm_bits, ind, chirange);
    }
  } else if (Bs == 17) {
    launch_details_bs<T, 17>(reg, chi, blist, ranks, nbh, n, norm_bits, ind, chirange, st);
  } else {
    launch_details_bs<T, 9>(reg, chi, blist, ranks, nbh, n, norm_bits, ind, chirange, st);
  }
}
template <typename T>
void launch_maxnorm(int Bs, const T* reg, const int32_t* blist, int64_t n, unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_maxnorm, <<<grid1(n), kNT, 0, st>>>(reg, blist, out));
}
template <typename T, int BS>
void launch_refine_bs(const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* blist,
                      const int32_t* nbh, cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0};   // devices whose context has the opt-in
  smem_opt_in(k_refine<T, BS>, RefSmem<T, BS>::bytes, opted);
  k_refine<T, BS><<<grid1(4 * n), RefSmem<T, BS>::NT, RefSmem<T, BS>::bytes, st>>>(src, dst, tasks, blist, nbh);
}
template <typename T>
void launch_refine(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* blist,
                   const int32_t* nbh, cudaStream_t st) {
  if (n <= 0) return;
  if (Bs == 33) {
    if constexpr (sizeof(T) == 4) {
      static std::atomic<unsigned long long> opted{0};
      smem_opt_in(k_refine_child<T, 33>, RefBigSmem<T, 33>::bytes, opted);
      k_refine_child<T, 33><<<grid1(32 * n), RefBigSmem<T, 33>::NT, RefBigSmem<T, 33>::bytes, st>>>(src, dst, tasks,
                                                                                                    blist, nbh);
    }
  } else if (Bs == 17) {
    launch_refine_bs<T, 17>(src, dst, tasks, n, blist, nbh, st);
  } else {
    launch_refine_bs<T, 9>(src, dst, tasks, n, blist, nbh, st);
  }
}
template <typename T>
void launch_coarsen(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  if (Bs == 33) {
    if constexpr (sizeof(T) == 4) k_coarsen<T, 33><<<grid1(4 * n), ColCfg<33>::NT, 0, st>>>(src, dst, tasks);
  } else if (Bs == 17) {
    k_coarsen<T, 17><<<grid1(4 * n), ColCfg<17>::NT, 0, st>>>(src, dst, tasks);
  } else {
    k_coarsen<T, 9><<<grid1(4 * n), ColCfg<9>::NT, 0, st>>>(src, dst, tasks);
  }
}
template <typename T, int BS>
void launch_coarsen44_bs(const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* nbh, cudaStream_t st) {
  static std::atomic<unsigned long long> opted{0};   // devices whose context has the opt-in
  smem_opt_in(k_coarsen44<T, BS>, C44Smem<T, BS>::bytes, opted);
  k_coarsen44<T, BS><<<grid1(n), C44Smem<T, BS>::NT, C44Smem<T, BS>::bytes, st>>>(src, dst, tasks, nbh);
}
template <typename T>
void launch_coarsen44(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t n, const int32_t* nbh, cudaStream_t st) {
  if (n <= 0 || Bs == 33) return;     // CDF 4/4 merging is built for Bs 9 and 17 (refused above)
  if (Bs == 17) launch_coarsen44_bs<T, 17>(src, dst, tasks, n, nbh, st);
  else launch_coarsen44_bs<T, 9>(src, dst, tasks, n, nbh, st);
}
template <typename T>
void launch_copy_blocks(int Bs, const T* src, T* dst, const int32_t* list, int stride, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_copy_blocks, <<<grid1(n), kNT, 0, st>>>(src, dst, list, stride));
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
  if (Bs == 33) {
    if constexpr (sizeof(T) == 4) k_mask<T, 33><<<grid1(n), ColCfg<33>::NT, 0, st>>>(chi, blist, ranks, binfo, p, m);
  } else if (Bs == 17) {
    k_mask<T, 17><<<grid1(n), ColCfg<17>::NT, 0, st>>>(chi, blist, ranks, binfo, p, m);
  } else {
    k_mask<T, 9><<<grid1(n), ColCfg<9>::NT, 0, st>>>(chi, blist, ranks, binfo, p, m);
  }
}
template <typename T>
void launch_solid_source(int Bs, T* out, T* acc, const T* chi, const int32_t* blist, const int4* binfo, int64_t n,
                         const PhysK& p, const MaskK& m, double c_out, double c_acc, int acc_too, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_solid_source, <<<grid1(n), kNT, 0, st>>>(out, acc, chi, blist, binfo, p, m, c_out, c_acc, acc_too));
}
template <typename T>
void launch_solid_moment(int Bs, const T* chi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& p,
                         const MaskK& m, double* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_solid_moment, <<<grid1(n), kNT, 0, st>>>(chi, blist, binfo, p, m, out));
}
template <typename T>
void launch_diag(int Bs, const T* reg, const T* chi, const int32_t* blist, int64_t n, double* out, cudaStream_t st) {
  if (n <= 0) return;
  ACM_BS_DISPATCH(Bs, k_diag, <<<grid1(n), kNT, 0, st>>>(reg, chi, blist, out));
}
void launch_diag_sum(const double* part, const int4* binfo, int64_t n, const PhysK& p, double wF, double wE,
                     double* acc, cudaStream_t st) {
  k_diag_sum<<<1, 1024, 0, st>>>(part, binfo, n, p, wF, wE, acc);
}
template <typename T>
void launch_gather(int Bs, const T* reg, T* dense, const int32_t* blist, int64_t n, int ncomp, cudaStream_t st) {
  if (n <= 0) return;
  const int stride = (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).BLK;
  const int cstride = ncomp == 1 ? (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).FS : stride;
  ACM_BS_DISPATCH(Bs, k_gather, <<<grid1(n), kNT, 0, st>>>(reg, dense, blist, ncomp, cstride));
}
template <typename T>
void launch_scatter(int Bs, const T* dense, T* reg, const int32_t* blist, int64_t n, int ncomp, cudaStream_t st) {
  if (n <= 0) return;
  // a one-component register (the mask) has one component per slot, like launch_gather's
  const int stride = (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).BLK;
  const int cstride = ncomp == 1 ? (int)layout_info(sizeof(T) == 8 ? 64 : 32, Bs).FS : stride;
  ACM_BS_DISPATCH(Bs, k_scatter, <<<grid1(n), kNT, 0, st>>>(dense, reg, blist, ncomp, cstride));
}

#define ACM_INST(T)                                                                                        \
  template void launch_fine_wins<T>(int, T*, const int2*, const int32_t*, int64_t, const int32_t*, const int32_t*, int, cudaStream_t); \
  template void launch_coarse_slabs<T>(int, const T*, T*, const int4*, const int32_t*, int64_t, const int32_t*, uint32_t*, int, int, cudaStream_t); \
  template void launch_sync_ext<T>(int, const T*, T*, int, const int32_t*, int64_t, const int32_t*, int, cudaStream_t); \
  template void launch_details<T>(int, const T*, const T*, const int32_t*, const int32_t*, const int32_t*, int64_t, const unsigned long long*, double*, double*, cudaStream_t); \
  template void launch_maxnorm<T>(int, const T*, const int32_t*, int64_t, unsigned long long*, cudaStream_t); \
  template void launch_refine<T>(int, const T*, T*, const int32_t*, int64_t, const int32_t*, const int32_t*, cudaStream_t); \
  template void launch_coarsen<T>(int, const T*, T*, const int32_t*, int64_t, cudaStream_t);               \
  template void launch_coarsen44<T>(int, const T*, T*, const int32_t*, int64_t, const int32_t*, cudaStream_t); \
  template void launch_copy_blocks<T>(int, const T*, T*, const int32_t*, int, int64_t, cudaStream_t);          \
  template void launch_ic<T>(int, T*, const int32_t*, const int32_t*, int64_t, const int4*, const PhysK&, const IcK&, cudaStream_t); \
  template void launch_mask<T>(int, T*, const int32_t*, const int32_t*, int64_t, const int4*, const PhysK&, const MaskK&, cudaStream_t); \
  template void launch_diag<T>(int, const T*, const T*, const int32_t*, int64_t, double*, cudaStream_t);   \
  template void launch_solid_source<T>(int, T*, T*, const T*, const int32_t*, const int4*, int64_t, const PhysK&, const MaskK&, double, double, int, cudaStream_t); \
  template void launch_solid_moment<T>(int, const T*, const int32_t*, const int4*, int64_t, const PhysK&, const MaskK&, double*, cudaStream_t); \
  template void launch_gather<T>(int, const T*, T*, const int32_t*, int64_t, int, cudaStream_t);          \
  template void launch_scatter<T>(int, const T*, T*, const int32_t*, int64_t, int, cudaStream_t);
ACM_INST(float)
ACM_INST(double)

}  // namespace acm
