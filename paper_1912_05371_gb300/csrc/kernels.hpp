// Internal launch interface of the libacm kernels (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "leafhash.hpp"

namespace acm {

constexpr int kMaxLevel = 18;   // finest level a grid may use

// Per-launch model constants (Sec. 2.1-2.3), in double; kernels convert to their precision.
struct PhysK {
  double nu, c0sq, inv_ceta, cgamma, inv_csp;
  double uinf[3], pinf;
  int mask, sponge;
  double sp_L[3], sp_width, sp_delta;
  double root_len;
  int nroot[3];
  double a1, a2, a3;        // first-derivative coefficients
  double h[kMaxLevel + 1];  // grid spacing of each level, root_len / (2^J (Bs-1))
};

// Device leaf table: open addressing on leaf_hash(box) over `mask + 1` slot words (-1 empty);
// the box of a slot is box[slot] = (J, x, y, z).
struct TreeK {
  const int* tab;
  const int4* box;
  unsigned long long mask;   // capacity - 1 (capacity a power of two, >= 2 x max_blocks)
  int nroot[3];
};

// Rebuild the device leaf table (tab, box) from the blocks binfo/blist[0..n) of the current order,
// then the neighbourhood rows (nbh, rank-indexed), the per-block flag "a neighbour box is
// refined" (finer), and the fine-wins task list (fw) and coarse-face slab list (slabt, slabidx);
// counts[0], counts[1] receive the two list lengths.  fwmask/slabmask/fw_off/slab_off: per-block
// scratch.  err |= 2 if the grid is not graded, |= 4 if the table overflowed.
void launch_topology(const TreeK& t, int* tab, int4* box, const int4* binfo, const int32_t* blist, int64_t n,
                     int32_t* nbh, uint8_t* finer, uint32_t* fwmask, uint32_t* slabmask, int32_t* fw_off,
                     int32_t* slab_off, int32_t* counts, int2* fw, int4* slabt, int32_t* slabidx, int* err,
                     cudaStream_t st);

// Device topology: pointers into the pool, all indexed by rank (position in block order).
struct TopoK {
  const int32_t* nbh;       // [n][kNbhStride] neighbourhood tables
  const int4* binfo;        // [n] (J, gx, gy, gz)
  const int32_t* blist;     // [n] slot of each block
  const int32_t* slabidx;   // [n][8]: coarse-face halo slab per face (-1: none)
  int64_t n;
};

// Model and RK constants of one stage in the field precision (kernel parameters, so the
// stage kernel reads them from the constant bank).
template <typename T>
struct StageConst {
  T a1, a2, a3;             // first-derivative coefficients
  T nu, c0sq, cgam, inv_ceta, inv_csp;
  T uinf[3], pinf;
  T c_acc, c_out;           // RK coefficients of the stage
  T ih[kMaxLevel + 1];      // 1 / h_J
  T ih2[kMaxLevel + 1];     // 1 / (12 h_J^2)
};

// Stage of the fused RK4 update (Sec. 2.3).  in: the stage state (synchronised); U: the
// state at t^n; acc: the RK accumulator; out: next stage state (or U^{n+1} in stage 4).
template <typename T>
struct StageK {
  const T* in;
  const T* U;
  T* acc;
  T* out;
  const T* chi;
  const T* slab;
  double c_acc, c_out;      // stage coefficients (see stage.cu)
  StageConst<T> kc;         // the constants above in the field precision (filled by launch_stage)
  // stage 4 only, if set: the max norms of U^{n+1} (layout and zeroing as for launch_maxnorm)
  unsigned long long* norms;
  // if set, the stage reads its (c_acc, c_out) from coefp[2 (stage-1)], written on the device by
  // launch_rk_coefs, instead of c_acc/c_out
  const double* coefp;
};

// The arrays one stage update of one block reads and writes (see StageK).
template <typename T>
struct StagePtrs {
  const T* in;
  const T* U;
  T* acc;
  T* out;
  const T* chi;
  const T* slab;
  unsigned long long* norms;
  const double* coefp;
};

// One instance of the persistent multi-instance stage launch: its arrays and its topology.
template <typename T>
struct StageInst {
  StagePtrs<T> p;
  TopoK tp;
};

// One RK stage of several independent instances in one persistent launch (ctas CTAs walking the
// nwork (instance, rank) pairs of work); the instances share PhysK and take their stage
// coefficients from their own p.coefp (the time step on the device).  desc and work are device
// arrays.
template <typename T>
void launch_stage_multi(int stage, int Bs, const PhysK& p, const StageInst<T>* desc, const int2* work, int64_t nwork,
                        int ctas, int* err, cudaStream_t st);

// Parameters of the device time step (Sec. 2.3): CFL rule as on the host; h = finest spacing.
struct RkK {
  double dt_fixed;          // > 0: use it
  double h, c0, cfl, cfl_eta, C_eta, cfl_nu, nu;
  int mask;
};
void launch_rk_coefs(const unsigned long long* maxbits, const RkK& p, double* rk, cudaStream_t st);

// err: device int set to 1 if a bounded wait inside the kernel expired (never cleared here).
// variant kStagePair: FP32 fields take the two-points-per-thread kernel (stage_pair.cu);
// kStagePointTMA: FP32 fields take the one-point kernel with U, the accumulator and chi staged
// by bulk copies; kStagePointRows: FP32 blocks of 17^3 and 33^3 take the one-point kernel with a
// block's rows over CTAs of 9 rows; otherwise, and always for FP64 fields, the one-point kernel
// (stage.cu; 33^3 blocks over three CTAs of 11 rows).
constexpr int kStagePair = 0, kStagePoint = 1, kStagePointTMA = 2, kStagePointRows = 3;
template <typename T>
void launch_stage(int stage, int Bs, const StageK<T>& s, const TopoK& t, const PhysK& p, int* err,
                  cudaStream_t st, int variant = kStagePair);

// Constants of the FP32 pair kernel (kernel parameters, read from the constant bank): equal
// pairs (v, v) for the packed operations, plain floats for the rest.
struct PairConst {
  float2 a1, a2, a3, k16, km90, mcgam, minv_ceta, minv_csp, uinf0, uinf1, uinf2, pinf;
  float nu, c0sq, c_acc, c_out;
  float ih[kMaxLevel + 1];     // 1 / h_J
  float ih2[kMaxLevel + 1];    // 1 / (12 h_J^2)
};
void launch_stage_pair(int stage, int Bs, const StageK<float>& s, const TopoK& t, const PhysK& p,
                       cudaStream_t st);

// The per-stage synchronisation kernels walk a task list whose length the device holds
// (*ntasks, written by launch_topology); max_tasks bounds it and sizes the grid, with
// ctas_per_sm CTAs per SM.
template <typename T>
void launch_fine_wins(int Bs, T* reg, const int2* tasks, const int32_t* ntasks, int64_t max_tasks,
                      const int32_t* nbh, const int32_t* blist, int ctas_per_sm, cudaStream_t st);

// offc: per-slab cache of the leaf lookups (slab_offset_words(Bs) words per slab) or nullptr;
// use_cache = 0 fills it, 1 reads it (valid while the grid is unchanged).
// ctas_per_sm: resident CTAs per SM the grid is sized for (1..3 for Bs = 17).
template <typename T>
void launch_coarse_slabs(int Bs, const T* reg, T* slab, const int4* tasks, const int32_t* ntasks,
                         int64_t max_tasks, const int32_t* nbh, uint32_t* offc, int use_cache, int ctas_per_sm,
                         cudaStream_t st);
size_t slab_offset_words(int Bs);

// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// Extended arrays (interior + g ghost layers) of all n blocks: out index = rank if by_rank,
// else slot.
template <typename T>
void launch_sync_ext(int Bs, const T* reg, T* out, int g, const int32_t* blist, int64_t n,
                     const int32_t* nbh, int by_rank, cudaStream_t st);

// Block indicators from the state itself (fine-wins applied): ind[rank], chirange[rank].
// (ranks: the blocks to evaluate, nullptr = all n; results are written at their ranks;
// norm_bits: the 4 component max norms as left by launch_maxnorm, read on the device)
template <typename T>
void launch_details(int Bs, const T* reg, const T* chi, const int32_t* blist, const int32_t* ranks,
                    const int32_t* nbh, int64_t n, const unsigned long long* norm_bits, double* ind,
                    double* chirange, cudaStream_t st);

// Max norms: out[0..3] = max |u|,|v|,|w|,|p|, out[4] = max |(u,v,w)|, as ordered bit patterns
// (non-negative doubles) combined with atomicMax; out must be zeroed before.
template <typename T>
void launch_maxnorm(int Bs, const T* reg, const int32_t* blist, int64_t n,
                    unsigned long long* out, cudaStream_t st);

// Children from a copy `src` of the synchronised state, old-grid tables (blist, nbh);
// one task per parent: [parent rank, new slots of children 0..7].
template <typename T>
void launch_refine(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t nparents,
                   const int32_t* blist, const int32_t* nbh, cudaStream_t st);

template <typename T>
void launch_coarsen(int Bs, const T* src, T* dst, const int32_t* tasks /*[n][9]*/, int64_t ntasks,
                    cudaStream_t st);

// CDF 4/4 coarsening: tasks [n][10] = [new parent slot, old child slots 0..7, rank of child 0]
// (the children are consecutive in the old block order; nbh is the old grid's table).
template <typename T>
void launch_coarsen44(int Bs, const T* src, T* dst, const int32_t* tasks, int64_t ntasks, const int32_t* nbh,
                      cudaStream_t st);

template <typename T>
void launch_copy_blocks(int Bs, const T* src, T* dst, const int32_t* list, int stride, int64_t n, cudaStream_t st);

struct IcK {
  int kind;
  double p[24];
};
// Initial condition on the blocks of rank list `ranks` (nullptr: all n blocks).
template <typename T>
void launch_ic(int Bs, T* reg, const int32_t* blist, const int32_t* ranks, int64_t n, const int4* binfo,
               const PhysK& p, const IcK& ic, cudaStream_t st);

// kind 1 (sphere): p = cx, cy, cz, R, delta.  kind 2 (rigid box, e.g. the moving plate, at one
// time): p[0..8] = R (body to world, row-major), p[9..11] = pivot x_0, p[12..14] = box centre and
// p[15..17] = half extents in the body frame, p[18] = delta, p[19..21] = angular velocity omega,
// p[22] = radius around x_0 that contains the box, p[24..32] = dR/dtheta and p[33..35] =
// d omega/dtheta for the parameter theta whose gradient the adjoint takes (the plate's pitch
// amplitude).  Body coordinates x_b = R^T (x - x_0).
struct MaskK {
  int kind;
  double p[40];
};
template <typename T>
void launch_mask(int Bs, T* chi, const int32_t* blist, const int32_t* ranks, int64_t n, const int4* binfo,
                 const PhysK& p, const MaskK& m, cudaStream_t st);

// Solid velocity of a rotating rigid body (mask kind 2), u_s = omega x (x - x_0): adds the
// penalization's source chi u_s / C_eta of the stage to the stage outputs, out += c_out S and,
// if acc_too, acc += c_acc S (the stage kernel has applied -chi u / C_eta).
template <typename T>
void launch_solid_source(int Bs, T* out, T* acc, const T* chi, const int32_t* blist, const int4* binfo, int64_t n,
                         const PhysK& p, const MaskK& m, double c_out, double c_acc, int acc_too, cudaStream_t st);
// Per block sums over the half-open points of chi u_s (3 components): out[n][4].
template <typename T>
void launch_solid_moment(int Bs, const T* chi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& p,
                         const MaskK& m, double* out, cudaStream_t st);

// Per block raw sums over the half-open points: [sum chi u, sum chi v, sum chi w, sum |u|^2].
template <typename T>
void launch_diag(int Bs, const T* reg, const T* chi, const int32_t* blist, int64_t n,
                 double* out, cudaStream_t st);
// acc += wF C_eta^-1 sum_r h_r^3 part[4r] + wE sum_r h_r^3 part[4r+3] / 2 over n blocks (part: the
// per-block sums of launch_diag or launch_solid_moment), on the device, in a fixed order.
void launch_diag_sum(const double* part, const int4* binfo, int64_t n, const PhysK& p, double wF, double wE,
                     double* acc, cudaStream_t st);

// Block-order gather/scatter of interiors between the pool and a dense array.
template <typename T>
void launch_gather(int Bs, const T* reg, T* dense, const int32_t* blist, int64_t n, int ncomp,
                   cudaStream_t st);
template <typename T>
void launch_scatter(int Bs, const T* dense, T* reg, const int32_t* blist, int64_t n, int ncomp,
                    cudaStream_t st);

// ---- discrete adjoint (adjoint.cu): state, mask and adjoint variables in T; the sums onto the
// mask parameters and the U_0 gradient handed out in FP64 ------------------------------------------
// One RK stage's adjoint: nu = W^T E^T loc(E W Y)^T kappa, kappa = c_lam lam + c_nu nup (nup may be
// null: kappa = c_lam lam).  Y: the stage's synchronised state; slab: its coarse-face halo slabs.
// sum_mode 1: sum = nup; 2: sum += nup (at interior points).  The stage's mask sensitivity is added
// to gchi (sphere; null: none), or for a moving box (m.kind 2, the stage's pose) its parameter's
// sensitivity to *dtheta.
template <typename T>
struct AdjStageK {
  const T* Y;
  const T* slab;
  const T* chi;
  const T* lam;
  const T* nup;
  double c_lam, c_nu;
  T* nu;
  T* sum;
  int sum_mode;
  T* gchi;
  double* dtheta;
};
// The forward's fine-wins task list (rank, refined box), its device-held length and its bound.
struct FwTasks {
  const int2* tasks;
  const int32_t* ntasks;
  int64_t max_tasks;
};
// err |= 8 if a ghost point's source is missing.
template <typename T>
void launch_adj_stage(int Bs, const AdjStageK<T>& a, const TopoK& t, const PhysK& ph, const MaskK& m,
                      const FwTasks& fw, int* err, cudaStream_t st);
// W^T applied to register r in place (n: blocks of the grid).
template <typename T>
void launch_adj_fw_T(int Bs, T* r, const FwTasks& fw, const int32_t* blist, const int32_t* nbh, int64_t n,
                     cudaStream_t st);
// out = x + y + z over every element of the listed blocks.
template <typename T>
void launch_adj_sum3(int Bs, T* out, const T* x, const T* y, const T* z, const int32_t* blist, int64_t n,
                     cudaStream_t st);
// Direct terms of wN (F_x(U) + wE E(U)) into lam and gchi (a moving box: its parameter's direct
// term into *dtheta, F_x integrating chi (u - u_s) at the pose of m).
template <typename T>
void launch_adj_objective(int Bs, const T* U, const T* chi, T* lam, T* gchi, const int32_t* blist,
                          const int4* binfo, int64_t n, const PhysK& ph, double wN, double wE, const MaskK& m,
                          double* dtheta, cudaStream_t st);
// out[0..3] += sum gchi d chi / d (centre, radius) for the sphere mask m.
template <typename T>
void launch_adj_theta(int Bs, const T* gchi, const int32_t* blist, const int4* binfo, int64_t n, const PhysK& ph,
                      const MaskK& m, double* out, cudaStream_t st);
// Block-order copy (n, 4, Bs^3, FP64) of an adjoint register, and its inverse (interior points only).
template <typename T>
void launch_adj_gather(int Bs, const T* r, double* dense, const int32_t* blist, int64_t n, cudaStream_t st);
template <typename T>
void launch_adj_put(int Bs, const double* dense, T* r, const int32_t* blist, int64_t n, cudaStream_t st);

}  // namespace acm
