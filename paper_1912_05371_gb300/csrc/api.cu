// C-ABI entry points of libacm (declared in include/acm.h).
//
// The host side keeps the block tree (forest.hpp) and drives the kernels (kernels.hpp) on the
// caller's stream; all device memory is carved out of the caller's pool at creation
// (Sec. 4.1: one allocation at start-up, released only at the end).
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/acm.h"
#include "checkpoint.hpp"
#include "common.cuh"
#include "forest.hpp"
#include "kernels.hpp"

using acm::BoxKey;
using acm::BoxStatus;

namespace {
// Tam & Webb's free coefficient of the 4th-order 7-point first derivative: the minimiser of
// the integrated dispersion error over kh in [0, pi/2] (published as 0.02651995).
constexpr double kTamWebbA3 = 0.0265199520614978;
}  // namespace

struct acm_forest {
  acm_grid_params gp;
  acm_phys_params pp;
  cudaStream_t st = nullptr;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  acm::LayoutInfo lay{};
  size_t esz = 8;
  std::unique_ptr<acm::Forest> fo;

  // heavy data (slot-indexed)
  void* U = nullptr;
  void* ACC = nullptr;
  void* YA = nullptr;
  void* YB = nullptr;
  void* CHI = nullptr;
  void* DENSE = nullptr;   // staging for block-order copies (n_blocks x 4 x Bs^3)
  void* SLAB = nullptr;
  // metadata (rank-indexed)
  int32_t* d_nbh = nullptr;
  int4* d_binfo = nullptr;
  int32_t* d_blist = nullptr;
  int32_t* d_slabidx = nullptr;
  int2* d_fw = nullptr;
  int4* d_slabt = nullptr;
  int4* d_reft = nullptr;
  int32_t* d_crst = nullptr;
  int32_t* d_ranks = nullptr;
  double* d_norms = nullptr;
  unsigned long long* d_maxbits = nullptr;
  double* d_ind = nullptr;
  double* d_chir = nullptr;
  double* d_diag = nullptr;
  int* d_err = nullptr;            // error bits set by kernels (see device_error)
  int* h_err = nullptr;            // pinned copy, refreshed after every RK4 step and every
                                   // indicator evaluation
  int* d_ltab = nullptr;            // device leaf table (slot words) and box per slot, rebuilt
  int4* d_bslot = nullptr;          // by the topology kernels after every grid change
  size_t leaf_cap = 0;
  uint8_t* d_finer = nullptr;      // per rank: a neighbour box is refined
  uint32_t* d_fwmask = nullptr;    // per rank scratch of the topology build
  uint32_t* d_slabmask = nullptr;
  int32_t* d_fwoff = nullptr;
  int32_t* d_slaboff = nullptr;
  int32_t* d_counts = nullptr;     // [0] fine-wins tasks, [1] coarse-face slabs
  uint32_t* d_slaboffc = nullptr;  // slab leaf-lookup cache (filled by RK stage 1)
  double* d_rk = nullptr;          // device time step: [0] dt, [1] time, [2..9] stage coefficients
  // RK4 steps captured as a CUDA graph (acm_rk4_steps), valid for one grid and one dt mode
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_gen = -1;
  double graph_dt = 0.0;
  int64_t graph_launches = 0;
  int64_t topo_gen = 0;            // incremented by every topology upload
  double* h_scal = nullptr;        // pinned scalars (time in / out of the device)
  // launch knobs chosen by acm_autotune (defaults until it runs)
  int tune_fw_ctas = 8;            // fine-wins kernel: CTAs per SM walking the task list
  int tune_slab_ctas = 3;          // coarse-face slab kernel: CTAs per SM walking the task list
  int stage_variant = acm::kStagePoint;  // FP32 stage kernel: one point per thread, or two
  float tune_stage_ms[4] = {0.f, 0.f, 0.f, 0.f};   // the autotuner's times of the forms (FP32)

  // host side of the current topology (the neighbourhood tables are built on the device from
  // the block list; the host leaf map is brought up to date only when a host query needs it)
  std::vector<BoxKey> order;
  std::vector<int32_t> blist;
  std::vector<int32_t> slot_rank;     // slot -> rank (-1: free)
  std::vector<double> ind_slot, chr_slot;   // indicators of the current coarsening, by slot
  bool leaves_stale = false;          // fo->leaves lags behind (order, blist)
  // parents refined by the last acm_refine_all (tags of the coarsen-everywhere cycle)
  std::unordered_set<BoxKey, acm::BoxKeyHash> last_refined;
  int4* h_binfo = nullptr;
  int32_t* h_blist = nullptr;
  uint8_t* h_finer = nullptr;
  void* h_pinned = nullptr;
  cudaEvent_t ev_topo = nullptr;      // after the copies of the last topology upload
  bool topo_pending = false;
  int Jtop = 0;

  bool mask_on = false;
  acm::MaskK mask{};
  // moving rigid plate (mask kind 2): chord, span, thickness, stroke and pitch amplitudes (rad),
  // frequency, pivot x, y, z, delta; its pose follows the simulated time
  bool moving = false;
  double plate[10] = {};
  acm::PhysK phk{};
  double time = 0.0;
  std::string err;
  int64_t launches = 0;
  bool timing = false;
  acm_step_stats stats{};
  bool stats_pending = false;
  // d_maxbits holds the max norms of U as the last RK4 stage left it (nothing changed U since)
  bool norms_fresh = false;
  double host_topology_ms = 0, host_tree_ms = 0;   // cumulative host time of the tree logic
  double host_sort_ms = 0, host_rows_ms = 0, host_wait_ms = 0;   // parts of host_topology_ms
  cudaEvent_t ev[12] = {};          // per stage: before sync, after sync, after the stage kernel
};

namespace {

acm_status fail(acm_forest* f, acm_status s, const std::string& msg) {
  if (f) f->err = msg;
  return s;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(f, ACM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

#define CK_F(g, call)                                                                          \
  do {                                                                                         \
    const cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail((g), ACM_ECUDA, cudaGetErrorString(e_));                 \
  } while (0)
#define CKL()                                                                                  \
  do {                                                                                         \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess)                                                                     \
      return fail(f, ACM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_));      \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// After a stream synchronisation that refreshed h_err: bit 0 a kernel's bounded wait expired,
// bit 1 the device topology build met an ungraded grid, bit 2 the leaf table was full.
acm_status device_error(acm_forest* f) {
  if (!f->h_err || !*f->h_err) return ACM_OK;
  if (*f->h_err & 1) return fail(f, ACM_ETIMEOUT, "a bounded wait inside a kernel expired");
  if (*f->h_err & 2) return fail(f, ACM_EGRADING, "grid is not 2:1 graded");
  if (*f->h_err & 8) return fail(f, ACM_EGRADING, "adjoint: a ghost point's source leaf is missing");
  return fail(f, ACM_ECUDA, "leaf table probe exceeded its capacity");
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Carve {
  size_t off = 0;
  char* base = nullptr;
  template <typename P>
  P* take(size_t bytes) {
    P* p = reinterpret_cast<P*>(base ? base + off : nullptr);
    off = align256(off + bytes);
    return p;
  }
};

bool valid_grid(const acm_grid_params* g) {
  if (!g) return false;
  if (g->Bs != 9 && g->Bs != 17 && g->Bs != 33) return false;
  if (g->precision != 32 && g->precision != 64) return false;
  if (g->g < 1 || g->g > 4) return false;
  if (g->wavelet != 0 && g->wavelet != 40 && g->wavelet != 44) return false;
  // Bs = 33 blocks: FP32 fields and the CDF 4/0 merge (the kernels built for that size)
  if (g->Bs == 33 && (g->precision != 32 || g->wavelet == 44)) return false;
  if (g->Jmin < 0 || g->Jmax < g->Jmin || g->Jmax > 18) return false;
  if (g->max_blocks < 1 || g->max_blocks > (int64_t)1 << 30) return false;
  if (!(g->root_len > 0)) return false;
  for (int a = 0; a < 3; ++a)
    if (g->nroot[a] < 1 || g->nroot[a] > 64) return false;
  if ((int64_t)g->nroot[0] * g->nroot[1] * g->nroot[2] > 255) return false;
  // the stage kernel addresses the block pool and the coarse-face slab buffer with 32-bit
  // element offsets
  const acm::LayoutInfo L = acm::layout_info(g->precision, g->Bs);
  const int64_t slab_per_block = 6 * 4 * 3 * (int64_t)g->Bs * g->Bs;
  if (g->max_blocks * std::max<int64_t>(L.BLK, slab_per_block) >= ((int64_t)1 << 32)) return false;
  return true;
}

// Lay out (or just size, when base == nullptr) every device region of a forest.
size_t carve(acm_forest* f, const acm_grid_params* g, char* base) {
  const acm::LayoutInfo L = acm::layout_info(g->precision, g->Bs);
  const size_t es = g->precision == 64 ? 8 : 4;
  const size_t nb = (size_t)g->max_blocks;
  const size_t bs2 = (size_t)g->Bs * g->Bs;
  Carve c;
  c.base = base;
  void* U = c.take<char>(nb * L.BLK * es);
  void* ACC = c.take<char>(nb * L.BLK * es);
  void* YA = c.take<char>(nb * L.BLK * es);
  void* YB = c.take<char>(nb * L.BLK * es);
  void* CHI = c.take<char>(nb * L.FS * es);
  void* DENSE = c.take<char>(nb * 4 * (size_t)g->Bs * g->Bs * g->Bs * es);
  void* SLAB = c.take<char>(nb * 6 * 4 * 3 * bs2 * es);
  int32_t* nbh = c.take<int32_t>(nb * acm::kNbhStride * 4);
  int4* binfo = c.take<int4>(nb * 16);
  int32_t* blist = c.take<int32_t>(nb * 4);
  int32_t* slabidx = c.take<int32_t>(nb * 8 * 4);
  int2* fw = c.take<int2>(nb * 26 * 8);
  int4* slabt = c.take<int4>(nb * 6 * 16);
  int4* reft = c.take<int4>(nb * 16);   // refinement tasks: 9 int32 per parent fit in 16 B per block
  int32_t* crst = c.take<int32_t>(nb * 9 * 4);
  int32_t* ranks = c.take<int32_t>(nb * 4);
  double* norms = c.take<double>(16 * 8);
  unsigned long long* maxbits = c.take<unsigned long long>(16 * 8);
  double* ind = c.take<double>(nb * 8);
  double* chir = c.take<double>(nb * 8);
  double* diag = c.take<double>(nb * 4 * 8);
  int* errf = c.take<int>(16);
  int* ltab = c.take<int>(acm::LeafMap::capacity_for(g->max_blocks) * sizeof(int));
  int4* bslot = c.take<int4>(nb * sizeof(int4));
  uint8_t* finer = c.take<uint8_t>(nb);
  uint32_t* fwmask = c.take<uint32_t>(nb * 4);
  uint32_t* slabmask = c.take<uint32_t>(nb * 4);
  int32_t* fwoff = c.take<int32_t>(nb * 4);
  int32_t* slaboff = c.take<int32_t>(nb * 4);
  int32_t* counts = c.take<int32_t>(16);
  uint32_t* slaboffc = c.take<uint32_t>(nb * 6 * acm::slab_offset_words(g->Bs) * 4);
  double* rk = c.take<double>(32 * 8);
  if (f) {
    f->U = U; f->ACC = ACC; f->YA = YA; f->YB = YB; f->CHI = CHI; f->DENSE = DENSE; f->SLAB = SLAB;
    f->d_nbh = nbh; f->d_binfo = binfo; f->d_blist = blist; f->d_slabidx = slabidx;
    f->d_fw = fw; f->d_slabt = slabt; f->d_reft = reft; f->d_crst = crst; f->d_ranks = ranks;
    f->d_norms = norms; f->d_maxbits = maxbits; f->d_ind = ind; f->d_chir = chir; f->d_diag = diag;
    f->d_err = errf;
    f->d_ltab = ltab; f->d_bslot = bslot; f->d_finer = finer; f->d_fwmask = fwmask; f->d_slabmask = slabmask;
    f->d_fwoff = fwoff; f->d_slaboff = slaboff; f->d_counts = counts; f->d_slaboffc = slaboffc;
    f->d_rk = rk;
  }
  return c.off;
}

acm::TopoK topo(const acm_forest* f) {
  acm::TopoK t;
  t.nbh = f->d_nbh;
  t.binfo = f->d_binfo;
  t.blist = f->d_blist;
  t.slabidx = f->d_slabidx;
  t.n = (int64_t)f->order.size();
  return t;
}

// The host may rewrite the pinned staging arrays only once the copies of the previous topology
// upload have been consumed.
acm_status topo_copies_done(acm_forest* f) {
  if (f->topo_pending) {
    const double t0 = now_ms();
    CK(cudaEventSynchronize(f->ev_topo));
    f->host_wait_ms += now_ms() - t0;
    f->topo_pending = false;
  }
  return ACM_OK;
}

// Bring the host leaf map up to date with (order, blist) when a host query needs it.
void sync_leaf_map(acm_forest* f) {
  if (!f->leaves_stale) return;
  f->fo->leaves.clear();
  for (size_t r = 0; r < f->order.size(); ++r) f->fo->leaves.put(f->order[r], f->blist[r]);
  f->leaves_stale = false;
}

// Install the block order after a grid change (new_order / new_blist: the order and its slots
// when the caller knows them, else sorted from the leaf map) and rebuild the rank-indexed
// device metadata: block info and slots are copied from pinned staging, and the device leaf
// table, the neighbourhood rows and the task lists are built by the topology kernels.
// Nothing here waits for the device.
acm_status upload_topology(acm_forest* f, std::vector<BoxKey>* new_order = nullptr,
                           std::vector<int32_t>* new_blist = nullptr) {
  const double t0 = now_ms();
  const acm::Forest& fo = *f->fo;
  for (int32_t sl : f->blist) f->slot_rank[sl] = -1;
  if (new_order) f->order.swap(*new_order);
  else f->order = fo.sorted();
  const int64_t n = (int64_t)f->order.size();
  if (new_blist) {
    f->blist.swap(*new_blist);
  } else {
    f->blist.resize(n);
    for (int64_t r = 0; r < n; ++r) f->blist[r] = fo.leaves.get(f->order[r]);
  }
  const double t1 = now_ms();
  f->host_sort_ms += t1 - t0;
  acm_status s = topo_copies_done(f);
  if (s) return s;
  int jtop = 0;
  for (int64_t r = 0; r < n; ++r) {
    const BoxKey& b = f->order[r];
    f->h_blist[r] = f->blist[r];
    f->h_binfo[r] = make_int4(b.J, b.x, b.y, b.z);
    f->slot_rank[f->blist[r]] = (int32_t)r;
    jtop = std::max(jtop, b.J);
  }
  f->Jtop = jtop;
  if (n) {
    CK(cudaMemcpyAsync(f->d_binfo, f->h_binfo, n * sizeof(int4), cudaMemcpyHostToDevice, f->st));
    CK(cudaMemcpyAsync(f->d_blist, f->h_blist, n * 4, cudaMemcpyHostToDevice, f->st));
  }
  CK(cudaEventRecord(f->ev_topo, f->st));
  f->topo_pending = true;
  ++f->topo_gen;
  acm::TreeK tk;
  tk.tab = f->d_ltab;
  tk.box = f->d_bslot;
  tk.mask = (unsigned long long)(f->leaf_cap - 1);
  for (int a = 0; a < 3; ++a) tk.nroot[a] = f->gp.nroot[a];
  acm::launch_topology(tk, f->d_ltab, f->d_bslot, f->d_binfo, f->d_blist, n, f->d_nbh, f->d_finer, f->d_fwmask,
                       f->d_slabmask, f->d_fwoff, f->d_slaboff, f->d_counts, f->d_fw, f->d_slabt, f->d_slabidx,
                       f->d_err, f->st);
  CKL();
  f->launches += 4;
  f->host_rows_ms += now_ms() - t1;
  f->host_topology_ms += now_ms() - t0;
  return ACM_OK;
}

template <typename T>
T* reg_ptr(acm_forest* f, void* r) { return reinterpret_cast<T*>(r); }

// Fine wins + coarse-face slabs on a register (the per-stage synchronisation).
template <typename T>
acm_status sync_stage(acm_forest* f, T* reg, int use_slab_cache = 0) {
  const int Bs = f->gp.Bs;
  const int64_t n = (int64_t)f->order.size();
  acm::launch_fine_wins<T>(Bs, reg, f->d_fw, f->d_counts, 26 * n, f->d_nbh, f->d_blist, f->tune_fw_ctas, f->st);
  CKL();
  acm::launch_coarse_slabs<T>(Bs, reg, reinterpret_cast<T*>(f->SLAB), f->d_slabt, f->d_counts + 1, 6 * n, f->d_nbh,
                              f->d_slaboffc, use_slab_cache, f->tune_slab_ctas, f->st);
  CKL();
  f->launches += 2;
  return ACM_OK;
}

template <typename T>
acm_status fine_wins(acm_forest* f, T* reg) {
  acm::launch_fine_wins<T>(f->gp.Bs, reg, f->d_fw, f->d_counts, 26 * (int64_t)f->order.size(), f->d_nbh, f->d_blist,
                           f->tune_fw_ctas, f->st);
  CKL();
  ++f->launches;
  return ACM_OK;
}

// Copy every block of U to YA (same slots): the source of refinement and coarsening moves.
template <typename T>
acm_status snapshot_state(acm_forest* f) {
  acm::launch_copy_blocks<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U), reinterpret_cast<T*>(f->YA), f->d_blist, 1,
                             (int64_t)f->order.size(), f->st);
  CKL();
  ++f->launches;
  return ACM_OK;
}

// Enqueue the max-norm reduction into d_maxbits without waiting for it.
template <typename T>
acm_status max_norms_async(acm_forest* f) {
  CK(cudaMemsetAsync(f->d_maxbits, 0, 8 * sizeof(unsigned long long), f->st));
  acm::launch_maxnorm<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U), f->d_blist, (int64_t)f->order.size(),
                         f->d_maxbits, f->st);
  CKL();
  ++f->launches;
  return ACM_OK;
}

template <typename T>
acm_status max_norms(acm_forest* f, double out[5]) {
  CK(cudaMemsetAsync(f->d_maxbits, 0, 8 * sizeof(unsigned long long), f->st));
  acm::launch_maxnorm<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U), f->d_blist, (int64_t)f->order.size(),
                         f->d_maxbits, f->st);
  CKL();
  ++f->launches;
  unsigned long long bits[5];
  CK(cudaMemcpyAsync(bits, f->d_maxbits, sizeof(bits), cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  if (acm_status e = device_error(f)) return e;
  for (int k = 0; k < 5; ++k) {
    double v;
    std::memcpy(&v, &bits[k], 8);
    out[k] = v;
  }
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(out[k])) return fail(f, ACM_ENUMERIC, "non-finite value in the state");
  return ACM_OK;
}

double h_of(const acm_forest* f, int J) { return f->gp.root_len / ((double)(1 << J) * (f->gp.Bs - 1)); }

double cfl_dt(const acm_forest* f, double u_max) {
  const acm_phys_params& p = f->pp;
  const double h = h_of(f, f->Jtop);
  const double ueig = std::fabs(u_max) + std::sqrt(u_max * u_max + p.c0 * p.c0);
  double dt = p.cfl * h / ueig;
  if (f->mask_on) dt = std::min(dt, p.cfl_eta * p.C_eta);
  if (p.nu > 0) dt = std::min(dt, p.cfl_nu * h * h / p.nu);
  return dt;
}

// Pose of the moving plate at time t into the mask parameters (kind 2): the plate is the box
// |x_b| <= c/2, 0 <= y_b <= b, |z_b| <= thickness/2 of its body frame, x = x_0 + R(t) x_b with
// R = R_z(phi) R_y(alpha), phi = phi_m sin(2 pi f t) (stroke about the vertical), alpha =
// alpha_m cos(2 pi f t) (pitch about the span axis), and u_s = omega x (x - x_0) with
// omega = phi' e_z + alpha' R_z(phi) e_y (Sec. 2.2 mask and solid velocity of a rigid body).
void plate_pose(acm_forest* f, double t) {
  const double* q = f->plate;
  const double w = 2.0 * 3.14159265358979323846 * q[5];
  const double phi = q[3] * std::sin(w * t), alpha = q[4] * std::cos(w * t);
  const double dphi = q[3] * w * std::cos(w * t), dalpha = -q[4] * w * std::sin(w * t);
  const double cp = std::cos(phi), sp = std::sin(phi), ca = std::cos(alpha), sa = std::sin(alpha);
  // R_z(phi) R_y(alpha), row-major
  const double R[9] = {cp * ca, -sp, cp * sa, sp * ca, cp, sp * sa, -sa, 0.0, ca};
  acm::MaskK& m = f->mask;
  m.kind = 2;
  for (int k = 0; k < 9; ++k) m.p[k] = R[k];
  for (int a = 0; a < 3; ++a) m.p[9 + a] = q[6 + a];
  m.p[12] = 0.0;
  m.p[13] = 0.5 * q[1];
  m.p[14] = 0.0;
  m.p[15] = 0.5 * q[0];
  m.p[16] = 0.5 * q[1];
  m.p[17] = 0.5 * q[2];
  m.p[18] = q[9];
  // omega = phi' e_z + alpha' R_z(phi) e_y, R_z(phi) e_y = (-sin phi, cos phi, 0)
  m.p[19] = -dalpha * sp;
  m.p[20] = dalpha * cp;
  m.p[21] = dphi;
  m.p[22] = std::sqrt(0.25 * q[0] * q[0] + q[1] * q[1] + 0.25 * q[2] * q[2]);
  // derivatives with respect to the pitch amplitude alpha_m (alpha = alpha_m cos(w t)):
  // dR = R_z(phi) dR_y/dalpha cos(w t), d omega = -w sin(w t) R_z(phi) e_y
  const double cw = std::cos(w * t);
  const double dRy[9] = {-sa, 0.0, ca, 0.0, 0.0, 0.0, -ca, 0.0, -sa};
  const double Rz[9] = {cp, -sp, 0.0, sp, cp, 0.0, 0.0, 0.0, 1.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += Rz[3 * i + k] * dRy[3 * k + j];
      m.p[24 + 3 * i + j] = v * cw;
    }
  const double dw = -w * std::sin(w * t);
  m.p[33] = -dw * sp;
  m.p[34] = dw * cp;
  m.p[35] = 0.0;
}

// Mask on every block, or only on the blocks whose slots are in `fresh` (new blocks).
template <typename T>
acm_status eval_mask(acm_forest* f, const std::vector<int32_t>* fresh = nullptr) {
  if (!f->mask_on || f->mask.kind == 3) return ACM_OK;   // a field mask is the caller's
  if (f->moving) plate_pose(f, f->time);
  const int32_t* ranks = nullptr;
  int64_t n = (int64_t)f->order.size();
  std::vector<int32_t> rl;
  if (fresh) {
    rl.reserve(fresh->size());
    for (int32_t s : *fresh) rl.push_back(f->slot_rank[s]);
    if (rl.empty()) return ACM_OK;
    CK(cudaMemcpyAsync(f->d_ranks, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice, f->st));
    ranks = f->d_ranks;
    n = (int64_t)rl.size();
  }
  acm::launch_mask<T>(f->gp.Bs, reinterpret_cast<T*>(f->CHI), f->d_blist, ranks, n, f->d_binfo, f->phk, f->mask,
                      f->st);
  CKL();
  ++f->launches;
  return ACM_OK;
}

// save (optional, 4 registers): receives each stage's synchronised input Y_s (the adjoint
// recomputes a step with it).
template <typename T>
acm_status rk4(acm_forest* f, double dt, double* dt_used, T* const* save = nullptr) {
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  if (!(dt > 0)) {
    double m[5];
    acm_status s = max_norms<T>(f, m);
    if (s) return s;
    dt = cfl_dt(f, m[4]);
  }
  if (dt_used) *dt_used = dt;
  T* U = reinterpret_cast<T*>(f->U);
  T* ACC = reinterpret_cast<T*>(f->ACC);
  T* YA = reinterpret_cast<T*>(f->YA);
  T* YB = reinterpret_cast<T*>(f->YB);
  const acm::TopoK t = topo(f);
  const int64_t l0 = f->launches;
  for (int s = 1; s <= 4; ++s) {
    // with `save` the stages write their outputs (the next stages' inputs) into save[1..3]
    // themselves, so only U (the first stage's input) is copied
    T* in = s == 1 ? U : (save ? save[s - 1] : (s == 2 ? YA : (s == 3 ? YB : YA)));
    T* out = s == 4 ? U : (save ? save[s] : (s == 1 ? YA : (s == 2 ? YB : YA)));
    if (f->timing) CK(cudaEventRecord(f->ev[3 * (s - 1)], f->st));
    // stage 1 looks up the slabs' source points and caches them for stages 2-4 (same grid)
    acm_status st = sync_stage<T>(f, in, s > 1);
    if (st) return st;
    const double cs_out = s == 1 || s == 2 ? dt / 2.0 : (s == 3 ? dt : dt / 6.0);
    const double cs_acc = s == 1 ? dt / 6.0 : dt / 3.0;
    if (f->moving) {
      // the plate's mask at the stage time (RK4 nodes t, t + dt/2, t + dt/2, t + dt)
      plate_pose(f, f->time + (s == 1 ? 0.0 : (s == 4 ? dt : 0.5 * dt)));
      acm::launch_mask<T>(f->gp.Bs, reinterpret_cast<T*>(f->CHI), f->d_blist, nullptr, (int64_t)f->order.size(),
                          f->d_binfo, f->phk, f->mask, f->st);
      CKL();
      ++f->launches;
    }
    if (save && s == 1) {
      acm::launch_copy_blocks<T>(f->gp.Bs, in, save[0], f->d_blist, 1, (int64_t)f->order.size(), f->st);
      CKL();
      ++f->launches;
    }
    if (f->timing) CK(cudaEventRecord(f->ev[3 * (s - 1) + 1], f->st));
    acm::StageK<T> a{};
    a.in = in;
    a.U = U;
    a.acc = ACC;
    a.out = out;
    a.chi = f->mask_on ? reinterpret_cast<const T*>(f->CHI) : nullptr;
    a.slab = reinterpret_cast<const T*>(f->SLAB);
    a.c_acc = s == 1 ? dt / 6.0 : dt / 3.0;
    a.c_out = s == 1 || s == 2 ? dt / 2.0 : (s == 3 ? dt : dt / 6.0);
    a.norms = nullptr;
    if (s == 4) {
      // the last stage also reduces the max norms of U^{n+1} (read by the next coarsening)
      CK(cudaMemsetAsync(f->d_maxbits, 0, 8 * sizeof(unsigned long long), f->st));
      a.norms = f->d_maxbits;
    }
    acm::launch_stage<T>(s, f->gp.Bs, a, t, f->phk, f->d_err, f->st, f->stage_variant);
    CKL();
    ++f->launches;
    if (f->moving) {
      // + chi u_s / C_eta, the part of the penalization the stage kernel leaves out (u_s = 0 there)
      acm::launch_solid_source<T>(f->gp.Bs, out, ACC, reinterpret_cast<const T*>(f->CHI), f->d_blist, f->d_binfo,
                                  (int64_t)f->order.size(), f->phk, f->mask, cs_out, cs_acc, s < 4, f->st);
      CKL();
      ++f->launches;
    }
    if (f->timing) CK(cudaEventRecord(f->ev[3 * (s - 1) + 2], f->st));
  }
  CK(cudaMemcpyAsync(f->h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, f->st));
  f->norms_fresh = !f->moving;
  f->time += dt;
  if (f->moving) {
    acm_status st = eval_mask<T>(f);
    if (st) return st;
  }
  // algorithmic bytes of the four stage kernels: per point 64 words (registers Y, U, acc in and
  // out, see stage.cu) plus one word of mask per stage when a mask is set
  const double npts = (double)f->order.size() * f->gp.Bs * f->gp.Bs * f->gp.Bs;
  const double words = 64.0 + (f->mask_on ? 4.0 : 0.0);
  f->stats.stage_ms = 0;
  f->stats.sync_ms = 0;
  f->stats.stage_bytes = npts * words * (double)f->esz;
  f->stats.n_launches = f->launches - l0;
  f->stats_pending = f->timing;
  return ACM_OK;
}

// One RK4 step with the time step computed on the device (no host synchronisation): the
// time-step kernel, then 4 x (synchronisation, stage kernel reading its coefficients from device
// memory); stage 4 reduces the max norms of U^{n+1}, which the next step's time step reads.
acm::RkK rk_params(const acm_forest* f, double dt) {
  acm::RkK rp;
  rp.dt_fixed = dt;
  rp.h = h_of(f, f->Jtop);
  rp.c0 = f->pp.c0;
  rp.cfl = f->pp.cfl;
  rp.cfl_eta = f->pp.cfl_eta;
  rp.C_eta = f->pp.C_eta;
  rp.cfl_nu = f->pp.cfl_nu;
  rp.nu = f->pp.nu;
  rp.mask = f->mask_on ? 1 : 0;
  return rp;
}

template <typename T>
acm_status enqueue_rk4_device_dt(acm_forest* f, double dt) {
  acm::launch_rk_coefs(f->d_maxbits, rk_params(f, dt), f->d_rk, f->st);
  CKL();
  ++f->launches;
  T* U = reinterpret_cast<T*>(f->U);
  T* ACC = reinterpret_cast<T*>(f->ACC);
  T* YA = reinterpret_cast<T*>(f->YA);
  T* YB = reinterpret_cast<T*>(f->YB);
  const acm::TopoK t = topo(f);
  for (int s = 1; s <= 4; ++s) {
    T* in = s == 1 ? U : (s == 2 ? YA : (s == 3 ? YB : YA));
    T* out = s == 1 ? YA : (s == 2 ? YB : (s == 3 ? YA : U));
    acm_status st = sync_stage<T>(f, in, s > 1);
    if (st) return st;
    acm::StageK<T> a{};
    a.in = in;
    a.U = U;
    a.acc = ACC;
    a.out = out;
    a.chi = f->mask_on ? reinterpret_cast<const T*>(f->CHI) : nullptr;
    a.slab = reinterpret_cast<const T*>(f->SLAB);
    a.c_acc = 0.0;
    a.c_out = 0.0;
    a.coefp = f->d_rk + 2;
    a.norms = nullptr;
    if (s == 4) {
      CK(cudaMemsetAsync(f->d_maxbits, 0, 8 * sizeof(unsigned long long), f->st));
      a.norms = f->d_maxbits;
    }
    acm::launch_stage<T>(s, f->gp.Bs, a, t, f->phk, f->d_err, f->st, f->stage_variant);
    CKL();
    ++f->launches;
  }
  return ACM_OK;
}

// nsteps RK4 steps on the current grid.  With use_graph the first step runs as plain launches
// and the second is captured into a CUDA graph that the remaining steps replay (the grid, and so
// every launch, stays the same; the time step lives in device memory).  A stream that cannot be
// captured (the legacy default stream) runs every step as plain launches.
template <typename T>
acm_status rk4_steps(acm_forest* f, int nsteps, double dt, int use_graph, int* graph_used) {
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  if (nsteps < 0) return fail(f, ACM_EINVAL, "negative step count");
  if (graph_used) *graph_used = 0;
  if (nsteps == 0) return ACM_OK;
  // the device clock starts from the host's; the first time step needs the norms of U
  *f->h_scal = f->time;
  CK(cudaMemcpyAsync(f->d_rk + 1, f->h_scal, sizeof(double), cudaMemcpyHostToDevice, f->st));
  if (!(dt > 0) && !f->norms_fresh) {
    acm_status s = max_norms_async<T>(f);
    if (s) return s;
  }
  const bool can_graph = use_graph && f->st != nullptr;
  for (int k = 0; k < nsteps; ++k) {
    const bool reuse = can_graph && f->gexec && f->graph_gen == f->topo_gen && f->graph_dt == dt;
    if (reuse) {
      CK(cudaGraphLaunch(f->gexec, f->st));
      f->launches += f->graph_launches;
      if (graph_used) *graph_used = 1;
    } else if (can_graph && k >= 1) {
      // capture one step (every launch attribute was set by the plain step before)
      if (f->gexec) { cudaGraphExecDestroy(f->gexec); f->gexec = nullptr; }
      if (f->graph) { cudaGraphDestroy(f->graph); f->graph = nullptr; }
      const int64_t l0 = f->launches;
      CK(cudaStreamBeginCapture(f->st, cudaStreamCaptureModeThreadLocal));
      acm_status s = enqueue_rk4_device_dt<T>(f, dt);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(f->st, &g);
      if (s) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (ec != cudaSuccess) return fail(f, ACM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      f->graph = g;
      CK(cudaGraphInstantiate(&f->gexec, f->graph, 0));
      f->graph_gen = f->topo_gen;
      f->graph_dt = dt;
      f->graph_launches = f->launches - l0;
      CK(cudaGraphLaunch(f->gexec, f->st));
      if (graph_used) *graph_used = 1;
    } else {
      acm_status s = enqueue_rk4_device_dt<T>(f, dt);
      if (s) return s;
    }
  }
  CK(cudaMemcpyAsync(f->h_scal, f->d_rk, 2 * sizeof(double), cudaMemcpyDeviceToHost, f->st));
  CK(cudaMemcpyAsync(f->h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  f->time = f->h_scal[1];
  f->norms_fresh = true;
  if (acm_status e = device_error(f)) return e;
  // a non-finite state is reported here: the last stage's fused norms pass NaN over, the
  // reduction of max_norms does not (for a finite state it leaves the same norms)
  double m[5];
  return max_norms<T>(f, m);
}

template <typename T>
acm_status refine_all(acm_forest* f) {
  f->norms_fresh = false;
  acm::Forest& fo = *f->fo;
  const double t0 = now_ms();
  std::vector<int32_t> prank, pslot;
  for (size_t r = 0; r < f->order.size(); ++r)
    if (f->order[r].J < fo.Jmax) {
      prank.push_back((int32_t)r);
      pslot.push_back(f->blist[r]);
    }
  f->last_refined.clear();
  if (prank.empty()) return ACM_OK;
  // children in ascending key order (each parent's children 0..7 in turn) take the lowest free
  // slots once the parents' slots are released
  std::vector<int32_t> new_slot;
  if (!fo.take_slots(pslot, prank.size() * 8, &new_slot))
    return fail(f, ACM_ECAPACITY, "block pool too small to refine");
  for (int32_t r : prank) f->last_refined.insert(f->order[(size_t)r]);
  std::vector<int32_t> tasks(prank.size() * 9);
  for (size_t i = 0; i < prank.size(); ++i) {
    tasks[9 * i] = prank[i];
    for (int c = 0; c < 8; ++c) tasks[9 * i + 1 + c] = new_slot[8 * i + c];
  }
  f->host_tree_ms += now_ms() - t0;
  // synchronise U (fine wins), keep a copy of it as the source of the predictions, refine; the
  // old-grid tables are still on the device (the upload below is ordered after these kernels)
  acm_status s = fine_wins<T>(f, reinterpret_cast<T*>(f->U));
  if (s) return s;
  s = snapshot_state<T>(f);
  if (s) return s;
  CK(cudaMemcpyAsync(f->d_reft, tasks.data(), tasks.size() * sizeof(int32_t), cudaMemcpyHostToDevice, f->st));
  acm::launch_refine<T>(f->gp.Bs, reinterpret_cast<const T*>(f->YA), reinterpret_cast<T*>(f->U),
                        reinterpret_cast<const int32_t*>(f->d_reft), (int64_t)prank.size(), f->d_blist, f->d_nbh,
                        f->st);
  CKL();
  ++f->launches;
  // the block order of the refined grid, while the GPU refines: every parent replaced in place
  // by its children 0..7
  const double t1 = now_ms();
  std::vector<BoxKey> order2;
  std::vector<int32_t> blist2;
  order2.reserve(f->order.size() + 7 * prank.size());
  blist2.reserve(f->order.size() + 7 * prank.size());
  for (size_t r = 0, i = 0; r < f->order.size(); ++r) {
    const BoxKey& b = f->order[r];
    if (b.J < fo.Jmax) {
      for (int c = 0; c < 8; ++c) {
        order2.push_back(acm::Forest::child(b, c));
        blist2.push_back(new_slot[8 * i + c]);
      }
      ++i;
    } else {
      order2.push_back(b);
      blist2.push_back(f->blist[r]);
    }
  }
  f->leaves_stale = true;
  f->host_tree_ms += now_ms() - t1;
  s = upload_topology(f, &order2, &blist2);
  if (s) return s;
  return eval_mask<T>(f, &new_slot);
}

// Block indicators (details + mask range) of every block, or of the blocks whose slots are
// in `only`, copied to ind/chr (host, by rank); the component norms are read on the device from
// the last max-norm reduction.  One stream synchronisation.
template <typename T>
acm_status indicators(acm_forest* f, std::vector<double>& ind, std::vector<double>& chr,
                      const std::vector<int32_t>* only = nullptr) {
  acm_status s = fine_wins<T>(f, reinterpret_cast<T*>(f->U));
  if (s) return s;
  const int32_t* ranks = nullptr;
  int64_t n = (int64_t)f->order.size();
  std::vector<int32_t> rl;
  if (only) {
    for (int32_t sl : *only) rl.push_back(f->slot_rank[sl]);
    n = (int64_t)rl.size();
    if (n) {
      CK(cudaMemcpyAsync(f->d_ranks, rl.data(), rl.size() * 4, cudaMemcpyHostToDevice, f->st));
      ranks = f->d_ranks;
    }
  }
  acm::launch_details<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U),
                         f->mask_on ? reinterpret_cast<const T*>(f->CHI) : nullptr, f->d_blist, ranks, f->d_nbh, n,
                         f->d_maxbits, f->d_ind, f->d_chir, f->st);
  CKL();
  ++f->launches;
  const size_t nb = f->order.size();
  ind.resize(nb);
  chr.resize(nb);
  CK(cudaMemcpyAsync(ind.data(), f->d_ind, nb * 8, cudaMemcpyDeviceToHost, f->st));
  CK(cudaMemcpyAsync(chr.data(), f->d_chir, nb * 8, cudaMemcpyDeviceToHost, f->st));
  CK(cudaMemcpyAsync(f->h_finer, f->d_finer, nb, cudaMemcpyDeviceToHost, f->st));
  CK(cudaMemcpyAsync(f->h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  return device_error(f);
}

template <typename T>
acm_status coarsen(acm_forest* f, int64_t* n_blocks, int* n_passes) {
  acm::Forest& fo = *f->fo;
  // component norms of the state before the first pass stay on the device (d_maxbits): left
  // there by the last RK4 stage when nothing has changed the state since, else reduced here
  acm_status s = ACM_OK;
  if (!f->norms_fresh) s = max_norms_async<T>(f);
  f->norms_fresh = false;
  if (s) return s;
  int passes = 0;
  // With CDF 4/0 a merge leaves every other block's indicator unchanged: its even samples keep
  // their values (decimation preserves coincident points), so later passes evaluate the new
  // parents only.  The CDF 4/4 low-pass changes the parents' interior points, which the details
  // of their neighbours read: every pass evaluates every block.
  const bool c44 = f->gp.wavelet == 44;
  const int tstride = c44 ? 10 : 9;
  std::vector<double>& ind_slot = f->ind_slot;
  std::vector<double>& chr_slot = f->chr_slot;
  std::vector<int32_t> fresh;
  std::vector<double> ind, chr;
  for (int it = 0; it < 64; ++it) {
    s = indicators<T>(f, ind, chr, it == 0 || c44 ? nullptr : &fresh);
    if (s) return s;
    const size_t n = f->order.size();
    if (it == 0 || c44) {
      for (size_t r = 0; r < n; ++r) {
        ind_slot[f->blist[r]] = ind[r];
        chr_slot[f->blist[r]] = chr[r];
      }
    } else {
      for (int32_t sl : fresh) {
        ind_slot[sl] = ind[f->slot_rank[sl]];
        chr_slot[sl] = chr[f->slot_rank[sl]];
      }
    }
    for (size_t r = 0; r < n; ++r) {
      ind[r] = ind_slot[f->blist[r]];
      chr[r] = chr_slot[f->blist[r]];
    }
    const double th = now_ms();
    std::vector<uint8_t> tag(n, 0);
    for (size_t r = 0; r < n; ++r) {
      const BoxKey& b = f->order[r];
      bool t = false;
      if (f->pp.coarsen_everywhere) {
        t = b.J > 0 && f->last_refined.count(BoxKey{b.J - 1, b.x >> 1, b.y >> 1, b.z >> 1}) > 0;
      } else if (b.J > fo.Jmin) {
        if (f->pp.dealias && b.J == fo.Jmax) t = true;
        else t = (ind[r] < f->pp.eps) && !(chr[r] > f->pp.mask_range_thr);
      }
      tag[r] = t;
    }
    // sister groups: the 8 children of a parent are 8 consecutive blocks (children 0..7) in block
    // order; a group merges if all are tagged and none has a finer neighbour (grading)
    std::vector<BoxKey> groups;
    std::vector<size_t> gstart;
    for (size_t r = 0; r + 7 < n;) {
      const BoxKey& b = f->order[r];
      bool grp = b.J > 0 && (b.x & 1) == 0 && (b.y & 1) == 0 && (b.z & 1) == 0;
      const BoxKey p{b.J - 1, b.x >> 1, b.y >> 1, b.z >> 1};
      for (int c = 1; c < 8 && grp; ++c) grp = f->order[r + c] == acm::Forest::child(p, c);
      if (!grp) { ++r; continue; }
      bool ok = true;
      for (int c = 0; c < 8 && ok; ++c)
        if (!tag[r + c] || f->h_finer[r + c]) ok = false;
      if (ok) {
        groups.push_back(p);
        gstart.push_back(r);
      }
      r += 8;
    }
    if (groups.empty()) {
      f->host_tree_ms += now_ms() - th;
      break;
    }
    // parents (ascending keys) take the lowest free slots once the children's are released
    std::vector<int32_t> freed(groups.size() * 8);
    for (size_t g = 0; g < groups.size(); ++g)
      for (int c = 0; c < 8; ++c) freed[8 * g + c] = f->blist[gstart[g] + c];
    std::vector<int32_t> new_slot;
    if (!fo.take_slots(freed, groups.size(), &new_slot)) return fail(f, ACM_ECAPACITY, "block pool exhausted");
    std::vector<int32_t> tasks(groups.size() * tstride);
    for (size_t g = 0; g < groups.size(); ++g) {
      tasks[tstride * g] = new_slot[g];
      for (int c = 0; c < 8; ++c) tasks[tstride * g + 1 + c] = freed[8 * g + c];
      if (c44) tasks[tstride * g + 9] = (int32_t)gstart[g];
    }
    // the parents are made in YA (a parent may take a slot freed by a child that is still being
    // read), then copied into U; the CDF 4/4 low-pass reads the old grid's neighbourhoods, which
    // the topology upload below replaces only after it (stream order)
    CK(cudaMemcpyAsync(f->d_crst, tasks.data(), tasks.size() * 4, cudaMemcpyHostToDevice, f->st));
    if (c44)
      acm::launch_coarsen44<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U), reinterpret_cast<T*>(f->YA), f->d_crst,
                               (int64_t)groups.size(), f->d_nbh, f->st);
    else
      acm::launch_coarsen<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U), reinterpret_cast<T*>(f->YA), f->d_crst,
                             (int64_t)groups.size(), f->st);
    CKL();
    acm::launch_copy_blocks<T>(f->gp.Bs, reinterpret_cast<const T*>(f->YA), reinterpret_cast<T*>(f->U), f->d_crst,
                               tstride, (int64_t)groups.size(), f->st);
    CKL();
    f->launches += 2;
    // the host side of the merged grid while the GPU merges
    f->leaves_stale = true;
    // block order of the merged grid: each group's 8 consecutive children replaced by the parent
    std::vector<BoxKey> order2;
    std::vector<int32_t> blist2;
    order2.reserve(n);
    blist2.reserve(n);
    for (size_t r = 0, g = 0; r < n;) {
      if (g < gstart.size() && r == gstart[g]) {
        order2.push_back(groups[g]);
        blist2.push_back(new_slot[g]);
        r += 8;
        ++g;
      } else {
        blist2.push_back(f->blist[r]);
        order2.push_back(f->order[r++]);
      }
    }
    f->host_tree_ms += now_ms() - th;
    s = upload_topology(f, &order2, &blist2);
    if (s) return s;
    s = eval_mask<T>(f, &new_slot);
    if (s) return s;
    fresh = new_slot;
    ++passes;
    // With CDF 4/0 the next pass can only merge a sister group whose members are all new parents
    // or tagged already (the other blocks' indicators are unchanged): when there is none, that
    // pass would merge nothing, and its indicator evaluation (a launch and a read-back) is skipped.
    if (!c44) {
      const double tc = now_ms();
      std::vector<uint8_t> is_new(ind_slot.size(), 0);
      for (int32_t sl : fresh) is_new[sl] = 1;
      auto tagged = [&](size_t r) -> bool {
        const BoxKey& b = f->order[r];
        if (f->pp.coarsen_everywhere)
          return b.J > 0 && f->last_refined.count(BoxKey{b.J - 1, b.x >> 1, b.y >> 1, b.z >> 1}) > 0;
        if (b.J <= fo.Jmin) return false;
        if (f->pp.dealias && b.J == fo.Jmax) return true;
        const int32_t sl = f->blist[r];
        return ind_slot[sl] < f->pp.eps && !(chr_slot[sl] > f->pp.mask_range_thr);
      };
      bool possible = false;
      const size_t n2 = f->order.size();
      for (size_t r = 0; r + 7 < n2 && !possible;) {
        const BoxKey& b = f->order[r];
        bool grp = b.J > 0 && (b.x & 1) == 0 && (b.y & 1) == 0 && (b.z & 1) == 0;
        const BoxKey p{b.J - 1, b.x >> 1, b.y >> 1, b.z >> 1};
        for (int c = 1; c < 8 && grp; ++c) grp = f->order[r + c] == acm::Forest::child(p, c);
        if (!grp) { ++r; continue; }
        bool ok = true;
        for (int c = 0; c < 8 && ok; ++c) ok = is_new[f->blist[r + c]] || tagged(r + c);
        possible = ok;
        r += 8;
      }
      f->host_tree_ms += now_ms() - tc;
      if (!possible) break;
    }
  }
  if (n_blocks) *n_blocks = (int64_t)f->order.size();
  if (n_passes) *n_passes = passes;
  return ACM_OK;
}

template <typename T>
acm_status set_ic(acm_forest* f, int kind, const double* params, int n) {
  f->norms_fresh = false;
  acm::IcK ic{};
  ic.kind = kind;
  for (int i = 0; i < n && i < 24; ++i) ic.p[i] = params[i];
  acm::launch_ic<T>(f->gp.Bs, reinterpret_cast<T*>(f->U), f->d_blist, nullptr, (int64_t)f->order.size(),
                    f->d_binfo, f->phk, ic, f->st);
  CKL();
  ++f->launches;
  return ACM_OK;
}

template <typename T>
acm_status diagnostics(acm_forest* f, acm_diag* out) {
  std::memset(out, 0, sizeof(*out));
  double m[5];
  acm_status s = max_norms<T>(f, m);
  if (s) return s;
  const size_t n = f->order.size();
  acm::launch_diag<T>(f->gp.Bs, reinterpret_cast<const T*>(f->U),
                      f->mask_on ? reinterpret_cast<const T*>(f->CHI) : nullptr, f->d_blist, (int64_t)n,
                      f->d_diag, f->st);
  CKL();
  ++f->launches;
  std::vector<double> part(n * 4);
  CK(cudaMemcpyAsync(part.data(), f->d_diag, n * 4 * 8, cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  for (size_t r = 0; r < n; ++r) {
    const double h = h_of(f, f->order[r].J);
    const double h3 = h * h * h;
    for (int i = 0; i < 3; ++i) out->force[i] += part[4 * r + i] * h3 / f->pp.C_eta;
    out->energy += 0.5 * part[4 * r + 3] * h3;
    out->blocks_per_level[f->order[r].J]++;
  }
  if (f->moving) {
    // the force of a moving body integrates chi (u - u_s): subtract the sums of chi u_s
    plate_pose(f, f->time);
    acm::launch_solid_moment<T>(f->gp.Bs, reinterpret_cast<const T*>(f->CHI), f->d_blist, f->d_binfo, (int64_t)n,
                                f->phk, f->mask, f->d_diag, f->st);
    CKL();
    ++f->launches;
    CK(cudaMemcpyAsync(part.data(), f->d_diag, n * 4 * 8, cudaMemcpyDeviceToHost, f->st));
    CK(cudaStreamSynchronize(f->st));
    for (size_t r = 0; r < n; ++r) {
      const double h = h_of(f, f->order[r].J);
      for (int i = 0; i < 3; ++i) out->force[i] -= part[4 * r + i] * h * h * h / f->pp.C_eta;
    }
  }
  out->u_max = m[4];
  for (int k = 0; k < 4; ++k) out->norms[k] = m[k];
  out->n_blocks = (int64_t)n;
  out->time = f->time;
  return ACM_OK;
}

void fill_phys(acm_forest* f) {
  const acm_phys_params& p = f->pp;
  acm::PhysK& k = f->phk;
  k.nu = p.nu;
  k.c0sq = p.c0 * p.c0;
  k.inv_ceta = p.C_eta > 0 ? 1.0 / p.C_eta : 0.0;
  k.cgamma = p.C_gamma;
  k.sponge = (p.sponge && p.C_sp > 0) ? 1 : 0;
  k.inv_csp = k.sponge ? 1.0 / p.C_sp : 0.0;
  for (int a = 0; a < 3; ++a) k.uinf[a] = p.u_inf[a];
  k.pinf = p.p_inf;
  for (int a = 0; a < 3; ++a) k.sp_L[a] = p.sponge_L[a];
  k.sp_width = p.sponge_width;
  k.sp_delta = p.sponge_delta > 0 ? p.sponge_delta : 1.0;
  k.root_len = f->gp.root_len;
  for (int a = 0; a < 3; ++a) k.nroot[a] = f->gp.nroot[a];
  const double a3 = f->gp.fd_scheme == 1 ? kTamWebbA3 : 0.0;
  k.a1 = 2.0 / 3.0 + 5.0 * a3;
  k.a2 = -1.0 / 12.0 - 4.0 * a3;
  k.a3 = a3;
  k.mask = f->mask_on ? 1 : 0;
  for (int J = 0; J <= acm::kMaxLevel; ++J) k.h[J] = h_of(f, J);
}

#define DISPATCH(f, fn, ...) ((f)->gp.precision == 64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

}  // namespace

namespace {

// Time `launch` (reps times after one warm-up) on the forest's stream; median milliseconds.
template <typename F>
acm_status time_launches(acm_forest* f, F&& launch, int reps, float* ms_out) {
  std::vector<float> v;
  launch();
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(f->ev[0], f->st));
    launch();
    CK(cudaEventRecord(f->ev[1], f->st));
    CK(cudaEventSynchronize(f->ev[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, f->ev[0], f->ev[1]));
    v.push_back(ms);
  }
  CKL();
  std::sort(v.begin(), v.end());
  *ms_out = v[v.size() / 2];
  return ACM_OK;
}

// The autotuner: on the current grid, time the two task-list kernels of the per-stage
// synchronisation for each number of CTAs per SM walking the list (fine wins: 2, 4, 8, 16; coarse
// faces: 1, 2, 3 -- at most 3 are resident) and keep the fastest of each.  Fine wins rewrites
// stored boundary points with the values of finer leaves (what every synchronisation does first);
// the slab kernel writes only the slab buffer.  FP32 forests also time the three forms of the
// fused stage kernel (two points per thread with packed arithmetic, one point per thread, one
// point per thread with U, the accumulator and chi staged by bulk copies)
// on RK stage 2 of the live grid (reading U, the first stage register and the accumulator,
// writing the accumulator and the second stage register: registers a step rewrites before it
// reads them) and keep the faster.
template <typename T>
acm_status autotune(acm_forest* f, int* fw_ctas, int* slab_ctas) {
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  const int64_t n = (int64_t)f->order.size();
  T* U = reinterpret_cast<T*>(f->U);
  float best = 1e30f;
  int best_fw = f->tune_fw_ctas;
  for (int c : {2, 4, 8, 16}) {
    float ms = 0.f;
    acm_status s = time_launches(f, [&]() {
      acm::launch_fine_wins<T>(f->gp.Bs, U, f->d_fw, f->d_counts, 26 * n, f->d_nbh, f->d_blist, c, f->st);
    }, 5, &ms);
    if (s) return s;
    f->launches += 6;
    if (ms < best) { best = ms; best_fw = c; }
  }
  best = 1e30f;
  int best_sc = f->tune_slab_ctas;
  for (int c = 1; c <= 3; ++c) {
    float ms = 0.f;
    acm_status s = time_launches(f, [&]() {
      acm::launch_coarse_slabs<T>(f->gp.Bs, U, reinterpret_cast<T*>(f->SLAB), f->d_slabt, f->d_counts + 1, 6 * n,
                                  f->d_nbh, f->d_slaboffc, 0, c, f->st);
    }, 5, &ms);
    if (s) return s;
    f->launches += 6;
    if (ms < best) { best = ms; best_sc = c; }
  }
  if constexpr (sizeof(T) == 4) {
    const acm::TopoK t = topo(f);
    acm::StageK<T> a{};
    a.in = reinterpret_cast<const T*>(f->YA);
    a.U = U;
    a.acc = reinterpret_cast<T*>(f->ACC);
    a.out = reinterpret_cast<T*>(f->YB);
    a.chi = f->mask_on ? reinterpret_cast<const T*>(f->CHI) : nullptr;
    a.slab = reinterpret_cast<const T*>(f->SLAB);
    a.c_acc = 0.0;
    a.c_out = 0.0;
    best = 1e30f;
    int best_v = f->stage_variant;
    for (int v : {acm::kStagePair, acm::kStagePoint, acm::kStagePointTMA, acm::kStagePointRows}) {
      // 33^3 blocks: the row-split point form, three CTAs of 11 rows or four of 9
      if (f->gp.Bs == 33 && v != acm::kStagePoint && v != acm::kStagePointRows) continue;
      if (v == acm::kStagePointRows && f->gp.Bs == 9) continue;
      float ms = 0.f;
      acm_status s = time_launches(f, [&]() {
        acm::launch_stage<T>(2, f->gp.Bs, a, t, f->phk, f->d_err, f->st, v);
      }, 5, &ms);
      if (s) return s;
      f->launches += 6;
      f->tune_stage_ms[v] = ms;
      if (ms < best) { best = ms; best_v = v; }
    }
    f->stage_variant = best_v;
  }
  f->tune_fw_ctas = best_fw;
  f->tune_slab_ctas = best_sc;
  f->norms_fresh = false;
  // a captured graph holds the old launch knobs
  if (f->gexec) { cudaGraphExecDestroy(f->gexec); f->gexec = nullptr; }
  if (f->graph) { cudaGraphDestroy(f->graph); f->graph = nullptr; }
  if (fw_ctas) *fw_ctas = best_fw;
  if (slab_ctas) *slab_ctas = best_sc;
  return ACM_OK;
}

// ---- discrete adjoint of RK4 steps on the frozen grid (FP32 and FP64 forests) --------------------
// Workspace (caller-provided, 256-byte aligned regions), all adjoint registers in the forest's
// precision and indexed like its registers: lam, the nu of two consecutive RK stages, the running
// sum of the stage nus, the 4 stage states of the step being differentiated, the step's starting
// state, the snapshots of the checkpoint schedule, the 4 stage states of each recomputed step of
// an equidistant segment (kept for its turn), the mask sensitivity (one component), a dense
// FP64 array (n_blocks x 4 x Bs^3: the caller's dL/dU_N coming in, dJ/dU_0 going out) and the 4
// parameter sums (FP64).
struct AdjLayout {
  size_t lam, nu[2], sum, y[4], tape, ck, ys, gchi, dense, theta, total;
  size_t reg;    // bytes of a register in the forest's precision
  int64_t nslots;   // snapshots of the checkpoint schedule (ck: snapshot 0, 1, ...)
  int64_t nys;      // steps whose four stage states can be kept between an advance and its turn
};

// policy > 0: equidistant checkpoints every policy steps; policy < 0: binomial checkpointing with
// -policy snapshots.  total = 0 for an invalid policy or step count.
AdjLayout adj_layout(const acm_forest* f, int nsteps, int policy) {
  AdjLayout L{};
  L.nslots = acm::ckpt::snapshots_needed(nsteps, policy);
  if (L.nslots < 1) return L;
  L.reg = (size_t)f->gp.max_blocks * (size_t)f->lay.BLK * f->esz;
  size_t o = 0;
  auto take = [&](size_t b) { const size_t r = o; o = (o + b + 255) & ~(size_t)255; return r; };
  L.lam = take(L.reg);
  L.nu[0] = take(L.reg);
  L.nu[1] = take(L.reg);
  L.sum = take(L.reg);
  for (int s = 0; s < 4; ++s) L.y[s] = take(L.reg);
  L.tape = take(L.reg);
  L.ck = take(L.reg * (size_t)L.nslots);
  // equidistant checkpoints every c steps: a segment's recomputed steps (at most c - 1) keep
  // their stage states for their turns; binomial schedules never advance a step before its turn
  const int64_t c = policy > 0 ? std::min<int64_t>(policy, nsteps) : 1;
  L.nys = c - 1;
  L.ys = take(L.reg * 4 * (size_t)L.nys);
  L.gchi = take((size_t)f->gp.max_blocks * (size_t)f->lay.FS * f->esz);
  L.dense = take((size_t)f->gp.max_blocks * 4 * (size_t)f->gp.Bs * f->gp.Bs * f->gp.Bs * 8);
  L.theta = take(64);
  L.total = o + 256;
  return L;
}

template <typename T>
acm_status adjoint_sweep(acm_forest* f, int nsteps, double dt, int c, double wE, void* ws, size_t ws_bytes,
                         double* J_out, double* dtheta, void* dU0, int64_t n_elems, int on_device, const void* lamN,
                         bool* saved) {
  // the sphere's centre and radius (static mask), or the moving plate's pitch amplitude
  const bool plate = f->moving;
  // with lamN (dL/dU_N, block order, FP64, on the device if on_device) the sweep is the
  // vector-Jacobian product of the N-step map: lam starts from lamN, no objective terms
  const bool vjp = lamN != nullptr;
  // the objective's force needs a body; the vector-Jacobian product also runs without a mask
  if ((!vjp && !f->mask_on) || (f->mask_on && !plate && f->mask.kind != 1 && !(vjp && f->mask.kind == 3)))
    return fail(f, ACM_EINVAL, "the adjoint needs a sphere or plate mask");
  // the mask the adjoint kernels see: the forest's current one (a moving plate's pose changes at
  // every stage time), with kind 0 when no body is set (no mask parameter to differentiate)
  auto cur_mask = [&]() {
    acm::MaskK m = f->mask;
    if (!f->mask_on) m.kind = 0;
    return m;
  };
  if (nsteps < 1 || c == 0 || !(dt > 0) || !ws || !dtheta || (!vjp && !J_out) || (vjp && !dU0))
    return fail(f, ACM_EINVAL, "bad arguments");
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  const AdjLayout L = adj_layout(f, nsteps, c);
  if (L.total == 0) return fail(f, ACM_EINVAL, "bad checkpoint policy");
  if (ws_bytes < L.total) return fail(f, ACM_ENOMEM, "adjoint workspace too small");
  const int64_t nb = (int64_t)f->order.size();
  if ((dU0 || vjp) && n_elems != nb * 4 * (int64_t)f->gp.Bs * f->gp.Bs * f->gp.Bs)
    return fail(f, ACM_EINVAL, "element count does not match n_blocks*4*Bs^3");
  char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  auto S = [&](size_t off) { return reinterpret_cast<T*>(base + off); };
  T* LAM = S(L.lam);
  T* NUR[2] = {S(L.nu[0]), S(L.nu[1])};
  T* SUM = S(L.sum);
  T* Y[4] = {S(L.y[0]), S(L.y[1]), S(L.y[2]), S(L.y[3])};
  T* GCHI = S(L.gchi);
  double* DENSE = reinterpret_cast<double*>(base + L.dense);
  double* TH = reinterpret_cast<double*>(base + L.theta);
  auto CKP = [&](int k) { return S(L.ck + (size_t)k * L.reg); };
  const int Bs = f->gp.Bs;
  T* U = reinterpret_cast<T*>(f->U);
  const T* CHI = reinterpret_cast<const T*>(f->CHI);
  T* SLAB = reinterpret_cast<T*>(f->SLAB);
  const double t0 = f->time;
  auto copy = [&](const T* src, T* dst) {
    acm::launch_copy_blocks<T>(Bs, src, dst, f->d_blist, 1, nb, f->st);
    ++f->launches;
    return cudaGetLastError();
  };
  // the moving plate's pose and mask at time t (a static mask needs nothing)
  auto pose_at = [&](double t) {
    if (!plate) return;
    plate_pose(f, t);
    acm::launch_mask<T>(Bs, reinterpret_cast<T*>(f->CHI), f->d_blist, nullptr, nb, f->d_binfo, f->phk, f->mask, f->st);
    ++f->launches;
  };
  // one RK stage's adjoint: nu_out = J_G(Y_s)^T kappa with kappa = c_lam lam + c_nu nup, the
  // running sum of the stage nus updated from nup (sum_mode), the stage's mask sensitivity into
  // gchi (or for the plate straight into its parameter's sum).  The stage state's halo slabs
  // toward coarser neighbours are predicted first, as the forward's synchronisation does (the
  // slab kernel's source lookups were cached by the forward's first stage on this grid).
  const acm::TopoK tk_topo = topo(f);
  const acm::FwTasks fwt{f->d_fw, f->d_counts, 26 * nb};
  auto astage = [&](const T* Ys, double ts, const T* nup, double c_lam, double c_nu, T* nu_out, int sum_mode) {
    pose_at(ts);
    acm::launch_coarse_slabs<T>(Bs, Ys, SLAB, f->d_slabt, f->d_counts + 1, 6 * nb, f->d_nbh, f->d_slaboffc, 1,
                                f->tune_slab_ctas, f->st);
    acm::AdjStageK<T> a{};
    a.Y = Ys;
    a.slab = SLAB;
    a.chi = CHI;
    a.lam = LAM;
    a.nup = nup;
    a.c_lam = c_lam;
    a.c_nu = c_nu;
    a.nu = nu_out;
    a.sum = SUM;
    a.sum_mode = sum_mode;
    a.gchi = GCHI;
    a.dtheta = TH;
    acm::launch_adj_stage<T>(Bs, a, tk_topo, f->phk, cur_mask(), fwt, f->d_err, f->st);
    f->launches += 5;
    return cudaGetLastError() == cudaSuccess ? ACM_OK : fail(f, ACM_ECUDA, "adjoint kernel launch failed");
  };
  auto objective = [&](const T* Us, double tn) {
    pose_at(tn);
    acm::launch_adj_objective<T>(Bs, Us, CHI, LAM, GCHI, f->d_blist, f->d_binfo, nb, f->phk, 1.0 / nsteps, wE,
                                 cur_mask(), TH, f->st);
    ++f->launches;
  };
  acm::ckpt::Schedule sched;
  if (!acm::ckpt::build(nsteps, c, &sched) || sched.slots > L.nslots)
    return fail(f, ACM_EINVAL, "bad checkpoint policy");
  T* TAPE = S(L.tape);
  CK(cudaMemsetAsync(LAM, 0, L.reg, f->st));
  CK(cudaMemsetAsync(NUR[0], 0, L.reg, f->st));
  CK(cudaMemsetAsync(NUR[1], 0, L.reg, f->st));
  CK(cudaMemsetAsync(SUM, 0, L.reg, f->st));
  CK(cudaMemsetAsync(GCHI, 0, (size_t)f->gp.max_blocks * f->lay.FS * f->esz, f->st));
  CK(cudaMemsetAsync(TH, 0, 64, f->st));
  if (vjp) {
    // lam_N into LAM's interior points (a host array is staged in the dense region)
    const double* src = on_device ? reinterpret_cast<const double*>(lamN) : DENSE;
    if (!on_device) CK(cudaMemcpyAsync(DENSE, lamN, (size_t)n_elems * 8, cudaMemcpyHostToDevice, f->st));
    acm::launch_adj_put<T>(Bs, src, LAM, f->d_blist, nb, f->st);
    CKL();
    ++f->launches;
  }
  acm_status s;
  // J's terms are summed on the device when a state is first reached (U_1, ..., U_N in that
  // order), the force and energy as acm_diagnostics sums them (Sec. 2.2), into TH[7]; no host
  // round trip per step
  double* JDEV = TH + 7;
  int hi = 0;
  auto reached = [&](int k) -> acm_status {
    if (vjp || k <= hi) return ACM_OK;
    acm::launch_diag<T>(Bs, U, f->mask_on ? CHI : nullptr, f->d_blist, nb, f->d_diag, f->st);
    acm::launch_diag_sum(f->d_diag, f->d_binfo, nb, f->phk, 1.0 / nsteps, wE / nsteps, JDEV, f->st);
    f->launches += 2;
    if (f->moving) {
      // a moving body's force integrates chi (u - u_s) (pose and mask at the state's time)
      acm::launch_solid_moment<T>(Bs, CHI, f->d_blist, f->d_binfo, nb, f->phk, f->mask, f->d_diag, f->st);
      acm::launch_diag_sum(f->d_diag, f->d_binfo, nb, f->phk, -1.0 / nsteps, 0.0, JDEV, f->st);
      f->launches += 2;
    }
    hi = k;
    return cudaGetLastError() == cudaSuccess ? ACM_OK : fail(f, ACM_ECUDA, "objective kernel launch failed");
  };
  // An advance of step k whose next appearance in the schedule is its turn keeps the step's
  // stage states in a free slot of the stage-state tape (a segment's recomputation, equidistant
  // checkpoints), and the turn then takes its adjoint without running the step again.
  std::vector<uint8_t> keep_stages(sched.act.size(), 0);
  {
    std::vector<int8_t> next_op((size_t)nsteps, -1);
    for (size_t i = sched.act.size(); i-- > 0;) {
      const acm::ckpt::Action& a = sched.act[i];
      if (a.op != acm::ckpt::ADVANCE && a.op != acm::ckpt::TURN) continue;
      if (a.arg < 0 || a.arg >= nsteps) continue;
      if (a.op == acm::ckpt::ADVANCE) keep_stages[i] = next_op[(size_t)a.arg] == acm::ckpt::TURN;
      next_op[(size_t)a.arg] = a.op;
    }
  }
  std::vector<int64_t> ys_free;
  for (int64_t q = L.nys - 1; q >= 0; --q) ys_free.push_back(q);
  std::vector<int64_t> ys_of((size_t)nsteps, -1);
  auto ys_reg = [&](int64_t q, int st) { return S(L.ys + ((size_t)q * 4 + (size_t)st) * L.reg); };
  // the schedule's actions: snapshots are copies of U; a turn takes step k from U_k with its
  // stage inputs kept (or finds them kept by the step's advance) and then the step's adjoint
  // (lam' -> lam)
  for (size_t ai = 0; ai < sched.act.size(); ++ai) {
    const acm::ckpt::Action& act = sched.act[ai];
    const int k = act.arg;
    if (act.op == acm::ckpt::STORE || act.op == acm::ckpt::RESTORE) {
      if (k < 0 || k >= L.nslots) return fail(f, ACM_EINVAL, "snapshot index outside the workspace");
      T* snap = CKP(k);
      CK(act.op == acm::ckpt::STORE ? copy(U, snap) : copy(snap, U));
      if (k == 0) *saved = true;                   // snapshot 0 holds U_0 from here on
      continue;
    }
    if (k < 0 || k >= nsteps) return fail(f, ACM_EINVAL, "step index outside the sweep");
    const double tk = t0 + k * dt;
    if (act.op == acm::ckpt::ADVANCE) {
      f->time = tk;                                // a moving mask follows the step's clock
      T* kept[4] = {nullptr, nullptr, nullptr, nullptr};
      if (keep_stages[ai] && !ys_free.empty()) {
        const int64_t q = ys_free.back();
        ys_free.pop_back();
        ys_of[(size_t)k] = q;
        for (int st = 0; st < 4; ++st) kept[st] = ys_reg(q, st);
      }
      if ((s = rk4<T>(f, dt, nullptr, kept[0] ? kept : nullptr))) return s;
      if ((s = reached(k + 1))) return s;
      continue;
    }
    const int64_t q = ys_of[(size_t)k];
    T* Ys[4] = {Y[0], Y[1], Y[2], Y[3]};
    const T* Uk = U;                               // U_k (restored) when the stages were kept
    if (q >= 0) {
      for (int st = 0; st < 4; ++st) Ys[st] = ys_reg(q, st);
    } else {
      CK(copy(U, TAPE));
      Uk = TAPE;
      f->time = tk;
      if ((s = rk4<T>(f, dt, nullptr, Y))) return s;
      if ((s = reached(k + 1))) return s;
      if (k == nsteps - 1 && !vjp) objective(U, t0 + nsteps * dt);
    }
    // the step's adjoint, RK stages 4, 3, 2, 1 (kappa_4 = dt/6 lam, kappa_3 = dt/3 lam + dt nu_4,
    // kappa_2 = dt/3 lam + dt/2 nu_3, kappa_1 = dt/6 lam + dt/2 nu_2), then
    // lam <- W^T (lam + nu_4 + nu_3 + nu_2 + nu_1)
    if ((s = astage(Ys[3], tk + dt, nullptr, dt / 6.0, 0.0, NUR[0], 0))) return s;
    if ((s = astage(Ys[2], tk + 0.5 * dt, NUR[0], dt / 3.0, dt, NUR[1], 1))) return s;
    if ((s = astage(Ys[1], tk + 0.5 * dt, NUR[1], dt / 3.0, dt / 2.0, NUR[0], 2))) return s;
    if ((s = astage(Ys[0], tk, NUR[0], dt / 6.0, dt / 2.0, NUR[1], 2))) return s;
    acm::launch_adj_sum3<T>(Bs, LAM, LAM, SUM, NUR[1], f->d_blist, nb, f->st);
    acm::launch_adj_fw_T<T>(Bs, LAM, fwt, f->d_blist, f->d_nbh, nb, f->st);
    f->launches += 2;
    if (k >= 1 && !vjp) objective(Uk, tk);
    if (q >= 0) {
      ys_free.push_back(q);
      ys_of[(size_t)k] = -1;
    }
  }
  if (!plate && f->mask_on && f->mask.kind == 1) {
    acm::launch_adj_theta<T>(Bs, GCHI, f->d_blist, f->d_binfo, nb, f->phk, cur_mask(), TH, f->st);
    ++f->launches;
  }
  CKL();
  CK(cudaMemcpyAsync(dtheta, TH, (plate ? 1 : 4) * sizeof(double), cudaMemcpyDeviceToHost, f->st));
  double J = 0.0;
  CK(cudaMemcpyAsync(&J, JDEV, sizeof(double), cudaMemcpyDeviceToHost, f->st));
  // the forest keeps its state, time and mask
  CK(copy(CKP(0), U));
  f->time = t0;
  f->norms_fresh = false;
  if (plate) {
    if ((s = eval_mask<T>(f))) return s;
  }
  CK(cudaMemcpyAsync(f->h_err, f->d_err, sizeof(int), cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  if ((s = device_error(f))) return s;
  if (J_out) *J_out = J;
  if (dU0) {
    // FP64 gradient in block order; a host copy goes through the dense region
    void* dense = on_device ? dU0 : reinterpret_cast<void*>(DENSE);
    acm::launch_adj_gather<T>(Bs, LAM, reinterpret_cast<double*>(dense), f->d_blist, nb, f->st);
    CKL();
    ++f->launches;
    if (!on_device) CK(cudaMemcpyAsync(dU0, dense, (size_t)n_elems * 8, cudaMemcpyDeviceToHost, f->st));
    CK(cudaStreamSynchronize(f->st));
  }
  return ACM_OK;
}

// The sweep above, with the forest's state and time put back if it stops on an error once
// U_0 is in snapshot 0 (the first action of every schedule; no step runs before it).
acm_status adjoint_sphere(acm_forest* f, int nsteps, double dt, int c, double wE, void* ws, size_t ws_bytes,
                          double* J_out, double* dtheta, void* dU0, int64_t n_elems, int on_device,
                          const void* lamN = nullptr) {
  const double t0 = f->time;
  bool saved = false;
  const acm_status s = DISPATCH(f, adjoint_sweep, f, nsteps, dt, c, wE, ws, ws_bytes, J_out, dtheta, dU0, n_elems,
                                on_device, lamN, &saved);
  if (s != ACM_OK && saved) {
    const AdjLayout L = adj_layout(f, nsteps, c);
    char* base = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    if (f->gp.precision == 64)
      acm::launch_copy_blocks<double>(f->gp.Bs, reinterpret_cast<const double*>(base + L.ck),
                                      reinterpret_cast<double*>(f->U), f->d_blist, 1, (int64_t)f->order.size(), f->st);
    else
      acm::launch_copy_blocks<float>(f->gp.Bs, reinterpret_cast<const float*>(base + L.ck),
                                     reinterpret_cast<float*>(f->U), f->d_blist, 1, (int64_t)f->order.size(), f->st);
    cudaStreamSynchronize(f->st);
    f->time = t0;
    f->norms_fresh = false;
    if (f->moving) DISPATCH(f, eval_mask, f);
    cudaStreamSynchronize(f->st);
  }
  return s;
}

}  // namespace

extern "C" {

size_t acm_pool_bytes(const acm_grid_params* grid) {
  if (!valid_grid(grid)) return 0;
  return carve(nullptr, grid, nullptr) + 256;
}

acm_status acm_create_forest(const acm_grid_params* grid, const acm_phys_params* phys, void* stream,
                             void* device_pool, size_t pool_bytes, acm_forest** out) {
  if (!out) return ACM_EINVAL;
  *out = nullptr;
  if (!valid_grid(grid) || !phys || !device_pool) return ACM_EINVAL;
  const size_t need = acm_pool_bytes(grid);
  if (pool_bytes < need) return ACM_ENOMEM;
  if (((uintptr_t)device_pool) & 255) return ACM_EINVAL;
  std::unique_ptr<acm_forest> f(new acm_forest());
  f->gp = *grid;
  if (f->gp.wavelet == 0) f->gp.wavelet = 40;
  f->pp = *phys;
  f->st = reinterpret_cast<cudaStream_t>(stream);
  f->pool = reinterpret_cast<char*>(device_pool);
  f->pool_bytes = pool_bytes;
  f->lay = acm::layout_info(grid->precision, grid->Bs);
  f->esz = grid->precision == 64 ? 8 : 4;
  carve(f.get(), grid, f->pool);
  fill_phys(f.get());
  acm_forest* fp = f.get();
  fp->slot_rank.assign((size_t)grid->max_blocks, -1);
  fp->ind_slot.assign((size_t)grid->max_blocks, 0.0);
  fp->chr_slot.assign((size_t)grid->max_blocks, 0.0);
  {
    acm_forest* f = fp;   // for CK
    const size_t nb = (size_t)grid->max_blocks;
    f->leaf_cap = acm::LeafMap::capacity_for(grid->max_blocks);
    const size_t bytes = nb * sizeof(int4) + nb * 4 + nb + 9 * 256;
    CK(cudaMallocHost(&f->h_pinned, bytes));
    char* p = (char*)f->h_pinned;
    auto take = [&](size_t b) { char* q = p; p += (b + 255) & ~(size_t)255; return q; };
    f->h_binfo = (int4*)take(nb * sizeof(int4));
    f->h_blist = (int32_t*)take(nb * 4);
    f->h_finer = (uint8_t*)take(nb);
    f->h_err = (int*)take(16);
    *f->h_err = 0;
    f->h_scal = (double*)take(8 * sizeof(double));
    f->fo.reset(new acm::Forest(grid->nroot, grid->Bs, grid->Jmin, grid->Jmax, grid->max_blocks));
    CK(cudaMemset(f->d_err, 0, 16 * sizeof(int)));
    CK(cudaMemset(f->d_counts, 0, 16 * sizeof(int32_t)));
    for (auto& e : f->ev) CK(cudaEventCreate(&e));
    CK(cudaEventCreateWithFlags(&f->ev_topo, cudaEventDisableTiming));
  }
  *out = f.release();
  return ACM_OK;
}

acm_status acm_destroy_forest(acm_forest* f) {
  if (!f) return ACM_OK;
  cudaStreamSynchronize(f->st);   // no copy may still read the pinned memory
  for (auto& e : f->ev)
    if (e) cudaEventDestroy(e);
  if (f->ev_topo) cudaEventDestroy(f->ev_topo);
  if (f->gexec) cudaGraphExecDestroy(f->gexec);
  if (f->graph) cudaGraphDestroy(f->graph);
  f->fo.reset();
  if (f->h_pinned) cudaFreeHost(f->h_pinned);
  delete f;
  return ACM_OK;
}

acm_status acm_init_uniform(acm_forest* f, int J) {
  if (!f) return ACM_EINVAL;
  if (J < f->gp.Jmin || J > f->gp.Jmax) return fail(f, ACM_EINVAL, "level outside [Jmin, Jmax]");
  std::vector<int32_t> lv, gx, gy, gz;
  const int64_t nx = (int64_t)f->gp.nroot[0] << J, ny = (int64_t)f->gp.nroot[1] << J, nz = (int64_t)f->gp.nroot[2] << J;
  if (nx * ny * nz > f->gp.max_blocks) return fail(f, ACM_ECAPACITY, "uniform grid exceeds max_blocks");
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        lv.push_back(J);
        gx.push_back((int32_t)x);
        gy.push_back((int32_t)y);
        gz.push_back((int32_t)z);
      }
  return acm_set_leaves(f, lv.data(), gx.data(), gy.data(), gz.data(), (int64_t)lv.size());
}

acm_status acm_set_leaves(acm_forest* f, const int32_t* level, const int32_t* gx, const int32_t* gy,
                          const int32_t* gz, int64_t n) {
  if (f && f->mask_on && f->mask.kind == 3) return fail(f, ACM_EINVAL, "a field mask belongs to its grid: set another mask first");
  if (!f || !level || !gx || !gy || !gz || n <= 0) return fail(f, ACM_EINVAL, "bad leaves");
  if (n > f->gp.max_blocks) return fail(f, ACM_ECAPACITY, "more leaves than max_blocks");
  f->norms_fresh = false;
  f->last_refined.clear();
  acm::Forest trial(f->gp.nroot, f->gp.Bs, f->gp.Jmin, f->gp.Jmax, f->gp.max_blocks);
  std::vector<BoxKey> created((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    if (level[i] < 0 || level[i] > 18) return fail(f, ACM_EINVAL, "level out of range");
    for (int a = 0; a < 3; ++a) {
      const int32_t v = a == 0 ? gx[i] : (a == 1 ? gy[i] : gz[i]);
      if (v < 0 || v >= trial.nblocks_axis(level[i], a)) return fail(f, ACM_EINVAL, "block coordinate out of range");
    }
    created[i] = BoxKey{level[i], gx[i], gy[i], gz[i]};
  }
  trial.apply_pass({}, created, nullptr);
  if ((int64_t)trial.leaves.size() != n) return fail(f, ACM_EGRADING, "duplicate leaves");
  if (!trial.tiles_domain()) return fail(f, ACM_EGRADING, "leaves do not tile the domain");
  if (!trial.is_graded()) return fail(f, ACM_EGRADING, "leaves are not 2:1 graded");
  acm_status s = topo_copies_done(f);
  if (s) return s;
  f->fo->clear();
  f->leaves_stale = false;
  f->fo->apply_pass({}, created, nullptr);
  s = upload_topology(f);
  if (s) return s;
  const size_t blk = (size_t)f->lay.BLK * f->esz;
  for (int32_t sl : f->blist) CK(cudaMemsetAsync((char*)f->U + (size_t)sl * blk, 0, blk, f->st));
  f->time = 0.0;
  s = DISPATCH(f, eval_mask, f);
  if (s) return s;
  CK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_set_ic(acm_forest* f, int kind, const double* params, int n) {
  if (!f) return ACM_EINVAL;
  static const int need[5] = {0, 2, 4, 8, 17};   // parameters each kind reads
  if (kind < 1 || kind > 4 || n < need[kind] || n > 24 || !params) return fail(f, ACM_EINVAL, "bad initial condition");
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  acm_status s = DISPATCH(f, set_ic, f, kind, params, n);
  if (s) return s;
  CK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_set_mask(acm_forest* f, int kind, const double* params, int n, double t) {
  (void)t;
  if (!f) return ACM_EINVAL;
  if (kind == ACM_MASK_NONE) {
    f->mask_on = false;
    f->moving = false;
  } else if (kind == ACM_MASK_SPHERE) {
    if (!params || n < 5 || !(params[4] > 0)) return fail(f, ACM_EINVAL, "sphere mask needs cx, cy, cz, R, delta>0");
    f->mask_on = true;
    f->moving = false;
    f->mask.kind = 1;
    for (int i = 0; i < 5; ++i) f->mask.p[i] = params[i];
  } else if (kind == ACM_MASK_FIELD) {
    f->mask_on = true;
    f->moving = false;
    f->mask.kind = 3;
    CK(cudaMemsetAsync(f->CHI, 0, (size_t)f->gp.max_blocks * f->lay.FS * f->esz, f->st));
  } else if (kind == ACM_MASK_PLATE) {
    if (!params || n < 10 || !(params[0] > 0) || !(params[1] > 0) || !(params[2] > 0) || !(params[9] > 0))
      return fail(f, ACM_EINVAL, "plate mask needs chord, span, thickness > 0, phi_m, alpha_m, f, x0, y0, z0, delta > 0");
    f->mask_on = true;
    f->moving = true;
    for (int i = 0; i < 10; ++i) f->plate[i] = params[i];
    plate_pose(f, f->time);
  } else {
    return fail(f, ACM_EINVAL, "unknown mask kind");
  }
  fill_phys(f);
  if (!f->order.empty()) {
    acm_status s = DISPATCH(f, eval_mask, f);
    if (s) return s;
    CK(cudaStreamSynchronize(f->st));
  }
  return ACM_OK;
}

acm_status acm_sync_ghosts(acm_forest* f, int reg, void* out, int on_device) {
  if (!f || !out || reg != ACM_REG_U) return fail(f, ACM_EINVAL, "bad arguments");
  f->norms_fresh = false;
  const int g = f->gp.g;
  const int ne = f->gp.Bs + 2 * g;
  const size_t per = (size_t)4 * ne * ne * ne * f->esz;
  const size_t n = f->order.size();
  // fine wins on U, then the extended arrays in chunks that fit the adaptation buffer
  {
    acm_status s = f->gp.precision == 64 ? fine_wins<double>(f, (double*)f->U) : fine_wins<float>(f, (float*)f->U);
    if (s) return s;
  }
  const size_t cap = std::max<size_t>(1, (size_t)f->gp.max_blocks * 4 * f->gp.Bs * f->gp.Bs * f->gp.Bs * f->esz / per);
  for (size_t r0 = 0; r0 < n; r0 += cap) {
    const size_t m = std::min(cap, n - r0);
    char* dst = on_device ? (char*)out + r0 * per : (char*)f->DENSE;
    if (f->gp.precision == 64)
      acm::launch_sync_ext<double>(f->gp.Bs, (const double*)f->U, (double*)dst, g, f->d_blist + r0, (int64_t)m,
                                   f->d_nbh + r0 * acm::kNbhStride, 1, f->st);
    else
      acm::launch_sync_ext<float>(f->gp.Bs, (const float*)f->U, (float*)dst, g, f->d_blist + r0, (int64_t)m,
                                  f->d_nbh + r0 * acm::kNbhStride, 1, f->st);
    CKL();
    ++f->launches;
    if (!on_device) {
      CK(cudaMemcpyAsync((char*)out + r0 * per, f->DENSE, m * per, cudaMemcpyDeviceToHost, f->st));
      CK(cudaStreamSynchronize(f->st));
    }
  }
  CK(cudaStreamSynchronize(f->st));
  return ACM_OK;
}

acm_status acm_rk4_step(acm_forest* f, double dt, double* dt_used) {
  if (!f) return ACM_EINVAL;
  return DISPATCH(f, rk4, f, dt, dt_used);
}

acm_status acm_rk4_steps(acm_forest* f, int nsteps, double dt, int use_graph, double* t_end, int* graph_used) {
  if (f && f->moving) return fail(f, ACM_EINVAL, "a moving mask needs acm_rk4_step (its pose changes per stage)");
  if (!f) return ACM_EINVAL;
  acm_status s = DISPATCH(f, rk4_steps, f, nsteps, dt, use_graph, graph_used);
  if (s) return s;
  if (t_end) *t_end = f->time;
  return ACM_OK;
}

extern "C++" {
namespace {

// The persistent form of the batched steps: per RK stage, every instance's synchronisation (and
// at the first stage its time step on the device) on its own stream, joined into the origin
// stream, then one launch of the stage kernel whose CTAs walk the (instance, rank) pairs of all
// instances.  The per-stage instance descriptors and the work list live in forests[0]'s dense
// staging buffer (free during steps).
template <typename T>
struct BatchPersistent {
  acm_forest* const* forests = nullptr;
  int n = 0;
  int64_t nwork = 0;
  const acm::StageInst<T>* desc = nullptr;   // [4][n] on the device
  const int2* work = nullptr;                // [nwork] on the device
  std::vector<cudaEvent_t> ev;               // fork, then one join event per instance

  // ACM_EINVAL (nothing changed) if the instances cannot share one launch
  acm_status setup(acm_forest* const* fs, int nn) {
    forests = fs;
    n = nn;
    acm_forest* f0 = fs[0];
    for (int i = 0; i < n; ++i) {
      const acm_forest* g = fs[i];
      if (g->gp.precision != f0->gp.precision || g->gp.Bs != f0->gp.Bs || g->gp.Bs == 33 || !g->st ||
          std::memcmp(&g->phk, &f0->phk, sizeof(acm::PhysK)) != 0)
        return ACM_EINVAL;
      nwork += (int64_t)g->order.size();
    }
    const size_t dbytes = (size_t)4 * n * sizeof(acm::StageInst<T>);
    const size_t wofs = (dbytes + 255) & ~(size_t)255;
    const size_t need = wofs + (size_t)nwork * sizeof(int2);
    const size_t cap = (size_t)f0->gp.max_blocks * 4 * f0->gp.Bs * f0->gp.Bs * f0->gp.Bs * f0->esz;
    if (need > cap) return ACM_EINVAL;
    std::vector<acm::StageInst<T>> hd((size_t)4 * n);
    std::vector<int2> hw;
    hw.reserve((size_t)nwork);
    for (int i = 0; i < n; ++i) {
      acm_forest* g = fs[i];
      T* U = reinterpret_cast<T*>(g->U);
      T* YA = reinterpret_cast<T*>(g->YA);
      T* YB = reinterpret_cast<T*>(g->YB);
      for (int st = 1; st <= 4; ++st) {
        acm::StageInst<T>& d = hd[(size_t)(st - 1) * n + i];
        d.p.in = st == 1 ? U : (st == 2 ? YA : (st == 3 ? YB : YA));
        d.p.out = st == 1 ? YA : (st == 2 ? YB : (st == 3 ? YA : U));
        d.p.U = U;
        d.p.acc = reinterpret_cast<T*>(g->ACC);
        d.p.chi = g->mask_on ? reinterpret_cast<const T*>(g->CHI) : nullptr;
        d.p.slab = reinterpret_cast<const T*>(g->SLAB);
        d.p.norms = st == 4 ? g->d_maxbits : nullptr;
        d.p.coefp = g->d_rk + 2;
        d.tp = topo(g);
      }
      for (int64_t r = 0; r < (int64_t)g->order.size(); ++r) hw.push_back(make_int2(i, (int)r));
    }
    char* base = reinterpret_cast<char*>(f0->DENSE);
    if (cudaMemcpyAsync(base, hd.data(), dbytes, cudaMemcpyHostToDevice, f0->st) != cudaSuccess ||
        cudaMemcpyAsync(base + wofs, hw.data(), hw.size() * sizeof(int2), cudaMemcpyHostToDevice, f0->st) != cudaSuccess ||
        cudaStreamSynchronize(f0->st) != cudaSuccess)
      return fail(f0, ACM_ECUDA, "persistent batch: descriptor upload");
    desc = reinterpret_cast<const acm::StageInst<T>*>(base);
    work = reinterpret_cast<const int2*>(base + wofs);
    ev.assign((size_t)n + 1, nullptr);
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(f0, ACM_ECUDA, "event");
    return ACM_OK;
  }
  ~BatchPersistent() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }

  // one RK4 step of every instance, ordered after the origin stream's work and before its later work
  acm_status enqueue(double dt) {
    acm_forest* f0 = forests[0];
    cudaStream_t origin = f0->st;
    for (int st = 1; st <= 4; ++st) {
      CK_F(f0, cudaEventRecord(ev[0], origin));
      for (int i = 1; i < n; ++i) CK_F(f0, cudaStreamWaitEvent(forests[i]->st, ev[0], 0));
      for (int i = 0; i < n; ++i) {
        acm_forest* g = forests[i];
        if (st == 1) {
          acm::launch_rk_coefs(g->d_maxbits, rk_params(g, dt), g->d_rk, g->st);
          ++g->launches;
        }
        T* in = reinterpret_cast<T*>(st == 1 ? g->U : (st == 2 ? g->YA : (st == 3 ? g->YB : g->YA)));
        acm_status s = sync_stage<T>(g, in, st > 1);
        if (s) return s;
        if (st == 4) CK_F(g, cudaMemsetAsync(g->d_maxbits, 0, 8 * sizeof(unsigned long long), g->st));
      }
      for (int i = 1; i < n; ++i) {
        CK_F(f0, cudaEventRecord(ev[i], forests[i]->st));
        CK_F(f0, cudaStreamWaitEvent(origin, ev[i], 0));
      }
      acm::launch_stage_multi<T>(st, f0->gp.Bs, f0->phk, desc + (size_t)(st - 1) * n, work, nwork,
                                 acm::sm_count() * 3, f0->d_err, origin);
      CK_F(f0, cudaGetLastError());
      ++f0->launches;
    }
    return ACM_OK;
  }
};

}  // namespace
}  // extern "C++"

acm_status acm_rk4_steps_batch(acm_forest* const* forests, int n, int nsteps, double dt, int use_graph,
                               double* t_end, int* graph_used) {
  if (!forests || n <= 0 || nsteps < 0) return ACM_EINVAL;
  if (graph_used) *graph_used = 0;
  for (int i = 0; i < n; ++i) {
    if (!forests[i]) return ACM_EINVAL;
    if (forests[i]->order.empty()) return fail(forests[i], ACM_EINVAL, "empty forest");
    if (forests[i]->moving) return fail(forests[i], ACM_EINVAL, "a moving mask needs acm_rk4_step");
    for (int j = 0; j < i; ++j)
      if (forests[j] == forests[i]) return fail(forests[i], ACM_EINVAL, "forest listed twice");
  }
  if (nsteps == 0) return ACM_OK;
  auto step = [&](acm_forest* f) {
    return f->gp.precision == 64 ? enqueue_rk4_device_dt<double>(f, dt) : enqueue_rk4_device_dt<float>(f, dt);
  };
  // the device clocks start from the host's; the first time step needs the norms of each U
  for (int i = 0; i < n; ++i) {
    acm_forest* f = forests[i];
    *f->h_scal = f->time;
    CK(cudaMemcpyAsync(f->d_rk + 1, f->h_scal, sizeof(double), cudaMemcpyHostToDevice, f->st));
    if (!(dt > 0) && !f->norms_fresh) {
      acm_status s = f->gp.precision == 64 ? max_norms_async<double>(f) : max_norms_async<float>(f);
      if (s) return s;
    }
  }
  bool can_graph = use_graph != 0;
  for (int i = 0; i < n; ++i)
    if (!forests[i]->st) can_graph = false;
  acm_forest* f = forests[0];             // for CK: errors are reported on the first forest
  cudaStream_t origin = f->st;
  // use_graph = 2: the persistent form (falls back to the graph of per-instance launches if the
  // instances cannot share one stage launch)
  BatchPersistent<float> pf;
  BatchPersistent<double> pd;
  bool persistent = false;
  if (use_graph == 2 && can_graph) {
    const acm_status ps = f->gp.precision == 64 ? pd.setup(forests, n) : pf.setup(forests, n);
    if (ps == ACM_OK) persistent = true;
    else if (ps != ACM_EINVAL) return ps;
  }
  auto combined = [&]() { return f->gp.precision == 64 ? pd.enqueue(dt) : pf.enqueue(dt); };
  std::vector<cudaEvent_t> ev((size_t)n + 1, nullptr);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<int64_t> per_step((size_t)n, 0);
  auto cleanup = [&]() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  };
  acm_status rs = ACM_OK;
  if (can_graph)
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cleanup(); return fail(f, ACM_ECUDA, "event"); }
  for (int k = 0; k < nsteps && !rs; ++k) {
    if (!can_graph || k == 0) {
      // plain launches, every instance on its own stream (they run side by side)
      if (persistent) rs = combined();
      else
        for (int i = 0; i < n && !rs; ++i) rs = step(forests[i]);
      continue;
    }
    if (persistent && !gexec) {
      // capture one combined step (its fork and join events tie the instances' streams in)
      for (int i = 1; i < n; ++i) {
        cudaEventRecord(ev[i], forests[i]->st);
        cudaStreamWaitEvent(origin, ev[i], 0);
      }
      if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cleanup();
        return fail(f, ACM_ECUDA, "graph capture could not start");
      }
      for (int i = 0; i < n; ++i) per_step[i] = forests[i]->launches;
      rs = combined();
      for (int i = 0; i < n; ++i) per_step[i] = forests[i]->launches - per_step[i];
      const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
      if (rs) break;
      if (ec != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
        cleanup();
        return fail(f, ACM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      }
      if (graph_used) *graph_used = 2;
      if (cudaGraphLaunch(gexec, origin) != cudaSuccess) { cleanup(); return fail(f, ACM_ECUDA, "graph launch"); }
      continue;
    }
    if (!gexec) {
      // the graph reads what the instances' streams wrote: order the origin after them
      for (int i = 1; i < n; ++i) {
        cudaEventRecord(ev[i], forests[i]->st);
        cudaStreamWaitEvent(origin, ev[i], 0);
      }
      // capture one step of every instance as parallel branches forked from the origin stream
      if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cleanup();
        return fail(f, ACM_ECUDA, "graph capture could not start");
      }
      cudaEventRecord(ev[0], origin);
      for (int i = 1; i < n; ++i) cudaStreamWaitEvent(forests[i]->st, ev[0], 0);
      for (int i = 0; i < n && !rs; ++i) {
        const int64_t l0 = forests[i]->launches;
        rs = step(forests[i]);
        per_step[i] = forests[i]->launches - l0;
      }
      for (int i = 1; i < n; ++i) {
        cudaEventRecord(ev[i], forests[i]->st);
        cudaStreamWaitEvent(origin, ev[i], 0);
      }
      const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
      if (rs) break;
      if (ec != cudaSuccess || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
        cleanup();
        return fail(f, ACM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      }
      if (graph_used) *graph_used = 1;
    } else {
      for (int i = 0; i < n; ++i) forests[i]->launches += per_step[i];
    }
    if (cudaGraphLaunch(gexec, origin) != cudaSuccess) { cleanup(); return fail(f, ACM_ECUDA, "graph launch"); }
  }
  if (gexec || persistent) {
    // the instances' streams continue after the last replay (or the last combined step)
    cudaEventRecord(ev[n], origin);
    for (int i = 1; i < n; ++i) cudaStreamWaitEvent(forests[i]->st, ev[n], 0);
  }
  if (rs) {
    cleanup();
    return rs;
  }
  for (int i = 0; i < n; ++i) {
    acm_forest* g = forests[i];
    if (cudaMemcpyAsync(g->h_scal, g->d_rk, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->st) != cudaSuccess ||
        cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->st) != cudaSuccess) {
      cleanup();
      return fail(g, ACM_ECUDA, "copy");
    }
  }
  for (int i = 0; i < n; ++i) {
    acm_forest* g = forests[i];
    if (cudaStreamSynchronize(g->st) != cudaSuccess) { cleanup(); return fail(g, ACM_ECUDA, "synchronise"); }
    g->time = g->h_scal[1];
    g->norms_fresh = true;
    if (t_end) t_end[i] = g->time;
    if (acm_status e = device_error(g)) { cleanup(); return e; }
  }
  cleanup();
  return ACM_OK;
}

size_t acm_adjoint_bytes(const acm_forest* f, int nsteps, int ckpt) {
  if (!f) return 0;
  return adj_layout(f, nsteps, ckpt).total;
}

acm_status acm_adjoint_vjp(acm_forest* f, int nsteps, double dt, int ckpt, void* ws, size_t ws_bytes,
                           const void* dL_dUN, void* dL_dU0, int64_t n_elems, int on_device, double* dL_dtheta) {
  if (!f) return ACM_EINVAL;
  if (!dL_dUN || !dL_dU0) return fail(f, ACM_EINVAL, "bad arguments");
  double th[4] = {0.0, 0.0, 0.0, 0.0};
  const acm_status s = adjoint_sphere(f, nsteps, dt, ckpt, 0.0, ws, ws_bytes, nullptr, th, dL_dU0, n_elems,
                                      on_device, dL_dUN);
  if (s == ACM_OK && dL_dtheta)
    for (int i = 0; i < (f->moving ? 1 : 4); ++i) dL_dtheta[i] = f->mask_on ? th[i] : 0.0;
  return s;
}

acm_status acm_set_time(acm_forest* f, double t) {
  if (!f || !std::isfinite(t)) return fail(f, ACM_EINVAL, "bad time");
  f->time = t;
  if (f->moving && !f->order.empty()) {
    f->norms_fresh = false;
    acm_status s = DISPATCH(f, eval_mask, f);
    if (s) return s;
    CK(cudaStreamSynchronize(f->st));
  }
  return ACM_OK;
}

acm_status acm_checkpoint_schedule(int nsteps, int ckpt, int32_t* snapshots, int64_t* advances, int8_t* ops,
                                   int32_t* args, int64_t cap, int64_t* n_actions) {
  acm::ckpt::Schedule sched;
  if (!acm::ckpt::build(nsteps, ckpt, &sched)) return ACM_EINVAL;
  if (snapshots) *snapshots = sched.slots;
  if (advances) *advances = sched.advances;
  const int64_t n = (int64_t)sched.act.size();
  if (n_actions) *n_actions = n;
  if (!ops && !args) return ACM_OK;
  if (!ops || !args || cap < n) return ACM_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    ops[i] = sched.act[(size_t)i].op;
    args[i] = sched.act[(size_t)i].arg;
  }
  return ACM_OK;
}

acm_status acm_adjoint_sphere(acm_forest* f, int nsteps, double dt, int ckpt, double w_energy, void* ws,
                              size_t ws_bytes, double* J, double* dJ_dtheta, void* dJ_dU0, int64_t n_elems,
                              int on_device) {
  if (!f) return ACM_EINVAL;
  if (f->moving || !f->mask_on || f->mask.kind != 1) return fail(f, ACM_EINVAL, "acm_adjoint_sphere needs the sphere mask");
  return adjoint_sphere(f, nsteps, dt, ckpt, w_energy, ws, ws_bytes, J, dJ_dtheta, dJ_dU0, n_elems, on_device);
}

acm_status acm_adjoint_plate_pitch(acm_forest* f, int nsteps, double dt, int ckpt, double w_energy, void* ws,
                                   size_t ws_bytes, double* J, double* dJ_dalpha, void* dJ_dU0, int64_t n_elems,
                                   int on_device) {
  if (!f) return ACM_EINVAL;
  if (!f->moving) return fail(f, ACM_EINVAL, "acm_adjoint_plate_pitch needs the moving plate mask");
  return adjoint_sphere(f, nsteps, dt, ckpt, w_energy, ws, ws_bytes, J, dJ_dalpha, dJ_dU0, n_elems, on_device);
}

acm_status acm_autotune(acm_forest* f, int* fw_ctas, int* slab_ctas) {
  if (!f) return ACM_EINVAL;
  return DISPATCH(f, autotune, f, fw_ctas, slab_ctas);
}

acm_status acm_set_stage_variant(acm_forest* f, int variant) {
  if (!f) return ACM_EINVAL;
  if (variant != ACM_STAGE_PAIR && variant != ACM_STAGE_POINT && variant != ACM_STAGE_POINT_TMA &&
      variant != ACM_STAGE_POINT_ROWS)
    return fail(f, ACM_EINVAL, "unknown stage kernel");
  f->stage_variant = variant == ACM_STAGE_PAIR ? acm::kStagePair
                     : (variant == ACM_STAGE_POINT ? acm::kStagePoint
                        : (variant == ACM_STAGE_POINT_TMA ? acm::kStagePointTMA : acm::kStagePointRows));
  // a captured graph holds the old kernel
  if (f->gexec) { cudaGraphExecDestroy(f->gexec); f->gexec = nullptr; }
  if (f->graph) { cudaGraphDestroy(f->graph); f->graph = nullptr; }
  return ACM_OK;
}

acm_status acm_get_tuning(const acm_forest* f, acm_tuning* out) {
  if (!f || !out) return ACM_EINVAL;
  out->fw_ctas_per_sm = f->tune_fw_ctas;
  out->slab_ctas_per_sm = f->tune_slab_ctas;
  out->stage_variant = f->gp.precision == 64 ||
                               (f->gp.Bs == 33 && f->stage_variant != acm::kStagePointRows) ||
                               (f->stage_variant == acm::kStagePointRows && f->gp.Bs == 9)
                           ? ACM_STAGE_POINT
                       : (f->stage_variant == acm::kStagePair ? ACM_STAGE_PAIR
                          : (f->stage_variant == acm::kStagePoint ? ACM_STAGE_POINT
                             : (f->stage_variant == acm::kStagePointTMA ? ACM_STAGE_POINT_TMA
                                                                         : ACM_STAGE_POINT_ROWS)));
  out->stage_ms[ACM_STAGE_PAIR] = f->tune_stage_ms[acm::kStagePair];
  out->stage_ms[ACM_STAGE_POINT] = f->tune_stage_ms[acm::kStagePoint];
  out->stage_ms[ACM_STAGE_POINT_TMA] = f->tune_stage_ms[acm::kStagePointTMA];
  out->stage_ms[ACM_STAGE_POINT_ROWS] = f->tune_stage_ms[acm::kStagePointRows];
  return ACM_OK;
}

acm_status acm_refine_all(acm_forest* f) {
  if (!f) return ACM_EINVAL;
  if (f->mask_on && f->mask.kind == 3) return fail(f, ACM_EINVAL, "a field mask belongs to its grid: no refinement");
  return DISPATCH(f, refine_all, f);
}

acm_status acm_coarsen(acm_forest* f, int64_t* n_blocks, int* n_passes) {
  if (!f) return ACM_EINVAL;
  if (f->mask_on && f->mask.kind == 3) return fail(f, ACM_EINVAL, "a field mask belongs to its grid: no coarsening");
  return DISPATCH(f, coarsen, f, n_blocks, n_passes);
}

acm_status acm_adapt(acm_forest* f, int* n_blocks) {
  int64_t n = 0;
  const acm_status st = acm_coarsen(f, &n, nullptr);
  if (st == ACM_OK && n_blocks) *n_blocks = (int)n;
  return st;
}

acm_status acm_step(acm_forest* f, double dt, double* dt_used, int64_t* n_blocks) {
  if (!f) return ACM_EINVAL;
  acm_status s = acm_refine_all(f);
  if (s) return s;
  s = acm_rk4_step(f, dt, dt_used);
  if (s) return s;
  return acm_coarsen(f, n_blocks, nullptr);
}

static acm_status init_grid_thresholded(acm_forest* f, int ic_kind, const double* params, int n,
                                        int64_t* n_blocks) {
  acm_status s = acm_init_uniform(f, f->gp.Jmin);
  if (s) return s;
  s = acm_set_ic(f, ic_kind, params, n);
  if (s) return s;
  for (int it = 0; it < 64; ++it) {
    std::vector<BoxKey> before = f->order;
    // refine all, then evaluate the initial condition analytically on the new grid
    s = acm_refine_all(f);
    if (s) return s;
    s = acm_set_ic(f, ic_kind, params, n);
    if (s) return s;
    s = acm_coarsen(f, nullptr, nullptr);
    if (s) return s;
    if (f->order == before) {
      if (n_blocks) *n_blocks = (int64_t)f->order.size();
      f->time = 0.0;
      return ACM_OK;
    }
  }
  return fail(f, ACM_EINVAL, "initial grid did not converge");
}

acm_status acm_init_grid(acm_forest* f, int ic_kind, const double* params, int n, int64_t* n_blocks) {
  if (!f) return ACM_EINVAL;
  // the initial grid follows the thresholds whatever the coarsening mode
  const int everywhere = f->pp.coarsen_everywhere;
  f->pp.coarsen_everywhere = 0;
  const acm_status s = init_grid_thresholded(f, ic_kind, params, n, n_blocks);
  f->pp.coarsen_everywhere = everywhere;
  return s;
}

acm_status acm_block_indicators(acm_forest* f, double* ind, double* chirange, int64_t n) {
  if (!f) return ACM_EINVAL;
  if (n < (int64_t)f->order.size()) return fail(f, ACM_EINVAL, "output arrays too small");
  f->norms_fresh = false;
  acm_status s = f->gp.precision == 64 ? max_norms_async<double>(f) : max_norms_async<float>(f);
  if (s) return s;
  std::vector<double> iv, cv;
  s = f->gp.precision == 64 ? indicators<double>(f, iv, cv) : indicators<float>(f, iv, cv);
  if (s) return s;
  if (ind) std::memcpy(ind, iv.data(), iv.size() * 8);
  if (chirange) std::memcpy(chirange, cv.data(), cv.size() * 8);
  return ACM_OK;
}

acm_status acm_diagnostics(acm_forest* f, acm_diag* out) {
  if (!f || !out) return ACM_EINVAL;
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  return DISPATCH(f, diagnostics, f, out);
}

int64_t acm_n_blocks(const acm_forest* f) { return f ? (int64_t)f->order.size() : 0; }

acm_status acm_get_topology(acm_forest* f, uint64_t* treecode, uint8_t* level, int32_t* slot, int32_t* gx,
                            int32_t* gy, int32_t* gz, int32_t* nbr, int8_t* rel, int64_t n) {
  if (!f) return ACM_EINVAL;
  const size_t nb = f->order.size();
  if (n < (int64_t)nb) return fail(f, ACM_EINVAL, "output arrays too small");
  for (size_t r = 0; r < nb; ++r) {
    const BoxKey& b = f->order[r];
    if (treecode) treecode[r] = f->fo->treecode(b);
    if (level) level[r] = (uint8_t)b.J;
    if (slot) slot[r] = f->blist[r];
    if (gx) gx[r] = b.x;
    if (gy) gy[r] = b.y;
    if (gz) gz[r] = b.z;
  }
  if (nbr || rel) {
    sync_leaf_map(f);
    std::vector<int32_t> nb56(nb * 56);
    std::vector<int8_t> r26(nb * 26);
    f->fo->neighbour_table(f->order, nb56.data(), r26.data());
    if (nbr) std::memcpy(nbr, nb56.data(), nb56.size() * 4);
    if (rel) std::memcpy(rel, r26.data(), r26.size());
  }
  return ACM_OK;
}

static acm_status copy_fields(acm_forest* f, void* buf, int64_t n_elems, int on_device, bool to_pool, int ncomp,
                              void* reg) {
  const int64_t nb = (int64_t)f->order.size();
  const int64_t need = nb * ncomp * (int64_t)f->gp.Bs * f->gp.Bs * f->gp.Bs;
  if (n_elems != need) return fail(f, ACM_EINVAL, "element count does not match n_blocks*comp*Bs^3");
  const size_t bytes = (size_t)need * f->esz;
  void* dense = on_device ? buf : f->DENSE;
  if (to_pool) {
    f->norms_fresh = false;
    if (!on_device) CK(cudaMemcpyAsync(dense, buf, bytes, cudaMemcpyHostToDevice, f->st));
    if (f->gp.precision == 64)
      acm::launch_scatter<double>(f->gp.Bs, (const double*)dense, (double*)reg, f->d_blist, nb, ncomp, f->st);
    else
      acm::launch_scatter<float>(f->gp.Bs, (const float*)dense, (float*)reg, f->d_blist, nb, ncomp, f->st);
  } else {
    if (f->gp.precision == 64)
      acm::launch_gather<double>(f->gp.Bs, (const double*)reg, (double*)dense, f->d_blist, nb, ncomp, f->st);
    else
      acm::launch_gather<float>(f->gp.Bs, (const float*)reg, (float*)dense, f->d_blist, nb, ncomp, f->st);
  }
  CKL();
  ++f->launches;
  if (!to_pool && !on_device) CK(cudaMemcpyAsync(buf, dense, bytes, cudaMemcpyDeviceToHost, f->st));
  CK(cudaStreamSynchronize(f->st));
  return device_error(f);
}

// ---- restart files -------------------------------------------------------------------------------
// Header, then acm_grid_params, acm_phys_params, the leaves' level, x, y, z (int32, block order)
// and the interior fields of U (block order, the forest's precision).  Host byte order.
namespace {

struct StateHeader {
  char magic[8];
  int32_t version;
  int32_t precision;
  int32_t grid_bytes;
  int32_t phys_bytes;
  int32_t mask_kind;
  int32_t reserved;
  double mask_params[10];
  double time;
  int64_t n_blocks;
};
constexpr char kStateMagic[8] = {'A', 'C', 'M', 'S', 'T', 'A', 'T', 'E'};
constexpr int32_t kStateVersion = 1;

struct File {
  FILE* p = nullptr;
  explicit File(FILE* q) : p(q) {}
  ~File() {
    if (p) fclose(p);
  }
};

// Reads and checks the header and both parameter blocks.
acm_status read_state_head(acm_forest* f, FILE* in, StateHeader* h, acm_grid_params* g, acm_phys_params* ph) {
  if (fread(h, sizeof(*h), 1, in) != 1 || std::memcmp(h->magic, kStateMagic, 8) != 0)
    return fail(f, ACM_EINVAL, "not a restart file");
  if (h->version != kStateVersion || h->grid_bytes != (int32_t)sizeof(acm_grid_params) ||
      h->phys_bytes != (int32_t)sizeof(acm_phys_params))
    return fail(f, ACM_EINVAL, "restart file of another version or build");
  if (fread(g, sizeof(*g), 1, in) != 1 || fread(ph, sizeof(*ph), 1, in) != 1)
    return fail(f, ACM_EINVAL, "truncated restart file");
  if (h->n_blocks < 1 || h->n_blocks > g->max_blocks || (h->precision != 32 && h->precision != 64) ||
      h->precision != g->precision || h->mask_kind < ACM_MASK_NONE || h->mask_kind > ACM_MASK_FIELD)
    return fail(f, ACM_EINVAL, "inconsistent restart file header");
  return ACM_OK;
}

}  // namespace

acm_status acm_save_state(acm_forest* f, const char* path) {
  if (!f || !path) return fail(f, ACM_EINVAL, "bad arguments");
  const int64_t n = (int64_t)f->order.size();
  if (n < 1) return fail(f, ACM_EINVAL, "empty forest");
  StateHeader h{};
  std::memcpy(h.magic, kStateMagic, 8);
  h.version = kStateVersion;
  h.precision = f->gp.precision;
  h.grid_bytes = (int32_t)sizeof(acm_grid_params);
  h.phys_bytes = (int32_t)sizeof(acm_phys_params);
  if (f->mask_on && f->moving) {
    h.mask_kind = ACM_MASK_PLATE;
    for (int i = 0; i < 10; ++i) h.mask_params[i] = f->plate[i];
  } else if (f->mask_on && f->mask.kind == 3) {
    h.mask_kind = ACM_MASK_FIELD;
  } else if (f->mask_on) {
    h.mask_kind = ACM_MASK_SPHERE;
    for (int i = 0; i < 5; ++i) h.mask_params[i] = f->mask.p[i];
  }
  h.time = f->time;
  h.n_blocks = n;
  std::vector<int32_t> leaves((size_t)(4 * n));
  for (int64_t r = 0; r < n; ++r) {
    const BoxKey& b = f->order[(size_t)r];
    leaves[(size_t)r] = b.J;
    leaves[(size_t)(n + r)] = b.x;
    leaves[(size_t)(2 * n + r)] = b.y;
    leaves[(size_t)(3 * n + r)] = b.z;
  }
  const int64_t ne = n * 4 * (int64_t)f->gp.Bs * f->gp.Bs * f->gp.Bs;
  std::vector<char> fields((size_t)ne * f->esz);
  acm_status s = copy_fields(f, fields.data(), ne, 0, false, 4, f->U);
  if (s) return s;
  std::vector<char> chi;
  if (h.mask_kind == ACM_MASK_FIELD) {
    chi.resize((size_t)(ne / 4) * f->esz);
    if ((s = copy_fields(f, chi.data(), ne / 4, 0, false, 1, f->CHI))) return s;
  }
  File out(fopen(path, "wb"));
  if (!out.p) return fail(f, ACM_EINVAL, std::string("cannot open ") + path);
  if (fwrite(&h, sizeof(h), 1, out.p) != 1 || fwrite(&f->gp, sizeof(f->gp), 1, out.p) != 1 ||
      fwrite(&f->pp, sizeof(f->pp), 1, out.p) != 1 ||
      fwrite(leaves.data(), sizeof(int32_t), leaves.size(), out.p) != leaves.size() ||
      fwrite(fields.data(), 1, fields.size(), out.p) != fields.size() ||
      fwrite(chi.data(), 1, chi.size(), out.p) != chi.size())
    return fail(f, ACM_EINVAL, std::string("cannot write ") + path);
  if (fclose(out.p) != 0) {
    out.p = nullptr;
    return fail(f, ACM_EINVAL, std::string("cannot write ") + path);
  }
  out.p = nullptr;
  return ACM_OK;
}

acm_status acm_read_state_header(const char* path, acm_grid_params* grid, acm_phys_params* phys, int64_t* n_blocks,
                                 double* time) {
  if (!path) return ACM_EINVAL;
  File in(fopen(path, "rb"));
  if (!in.p) return ACM_EINVAL;
  StateHeader h{};
  acm_grid_params g{};
  acm_phys_params ph{};
  if (read_state_head(nullptr, in.p, &h, &g, &ph)) return ACM_EINVAL;
  if (grid) *grid = g;
  if (phys) *phys = ph;
  if (n_blocks) *n_blocks = h.n_blocks;
  if (time) *time = h.time;
  return ACM_OK;
}

acm_status acm_load_state(acm_forest* f, const char* path) {
  if (!f || !path) return fail(f, ACM_EINVAL, "bad arguments");
  File in(fopen(path, "rb"));
  if (!in.p) return fail(f, ACM_EINVAL, std::string("cannot open ") + path);
  StateHeader h{};
  acm_grid_params g{};
  acm_phys_params ph{};
  acm_status s = read_state_head(f, in.p, &h, &g, &ph);
  if (s) return s;
  const acm_grid_params& me = f->gp;
  if (g.wavelet == 0) g.wavelet = 40;
  if (g.nroot[0] != me.nroot[0] || g.nroot[1] != me.nroot[1] || g.nroot[2] != me.nroot[2] ||
      g.root_len != me.root_len || g.Bs != me.Bs || g.g != me.g || g.Jmin != me.Jmin || g.Jmax != me.Jmax ||
      g.precision != me.precision || g.fd_scheme != me.fd_scheme || g.wavelet != me.wavelet)
    return fail(f, ACM_EINVAL, "restart file of a different grid");
  if (h.n_blocks > me.max_blocks) return fail(f, ACM_ECAPACITY, "restart file has more blocks than max_blocks");
  // everything is read before the forest changes
  const int64_t n = h.n_blocks;
  std::vector<int32_t> leaves((size_t)(4 * n));
  const int64_t ne = n * 4 * (int64_t)me.Bs * me.Bs * me.Bs;
  std::vector<char> fields((size_t)ne * f->esz);
  std::vector<char> chi(h.mask_kind == ACM_MASK_FIELD ? (size_t)(ne / 4) * f->esz : 0);
  if (fread(leaves.data(), sizeof(int32_t), leaves.size(), in.p) != leaves.size() ||
      fread(fields.data(), 1, fields.size(), in.p) != fields.size() ||
      fread(chi.data(), 1, chi.size(), in.p) != chi.size())
    return fail(f, ACM_EINVAL, "truncated restart file");
  // the file's mask replaces a field mask below; a field mask would make acm_set_leaves refuse
  // the grid change, so it is switched off for that call and back on if the call fails (the
  // forest is then unchanged)
  const bool had_field_mask = f->mask_on && f->mask.kind == 3;
  if (had_field_mask) f->mask_on = false;
  s = acm_set_leaves(f, leaves.data(), leaves.data() + n, leaves.data() + 2 * n, leaves.data() + 3 * n, n);
  if (s) {
    if (had_field_mask) f->mask_on = true;
    return s;
  }
  s = copy_fields(f, fields.data(), ne, 0, true, 4, f->U);
  if (s) return s;
  f->pp = ph;
  f->time = h.time;
  f->norms_fresh = false;
  const int np = h.mask_kind == ACM_MASK_PLATE ? 10 : (h.mask_kind == ACM_MASK_SPHERE ? 5 : 0);
  s = acm_set_mask(f, h.mask_kind, np ? h.mask_params : nullptr, np, h.time);
  if (s || h.mask_kind != ACM_MASK_FIELD) return s;
  return copy_fields(f, chi.data(), ne / 4, 0, true, 1, f->CHI);
}

acm_status acm_read_fields(acm_forest* f, int reg, void* out, int64_t n_elems, int on_device) {
  if (!f || !out || reg != ACM_REG_U) return fail(f, ACM_EINVAL, "bad arguments");
  return copy_fields(f, out, n_elems, on_device, false, 4, f->U);
}

acm_status acm_write_fields(acm_forest* f, const void* in, int64_t n_elems, int on_device) {
  if (!f || !in) return fail(f, ACM_EINVAL, "bad arguments");
  return copy_fields(f, const_cast<void*>(in), n_elems, on_device, true, 4, f->U);
}

acm_status acm_write_mask(acm_forest* f, const void* chi, int64_t n_elems, int on_device) {
  if (!f || !chi) return fail(f, ACM_EINVAL, "bad arguments");
  if (!f->mask_on || f->mask.kind != 3) return fail(f, ACM_EINVAL, "acm_write_mask needs the field mask");
  f->norms_fresh = false;
  return copy_fields(f, const_cast<void*>(chi), n_elems, on_device, true, 1, f->CHI);
}

acm_status acm_read_mask(acm_forest* f, void* out, int64_t n_elems, int on_device) {
  if (!f || !out) return fail(f, ACM_EINVAL, "bad arguments");
  if (!f->mask_on) return fail(f, ACM_EINVAL, "no mask set");
  return copy_fields(f, out, n_elems, on_device, false, 1, f->CHI);
}

acm_status acm_rhs(acm_forest* f, void* out, int64_t n_elems, int on_device) {
  if (!f || !out) return fail(f, ACM_EINVAL, "bad arguments");
  f->norms_fresh = false;
  if (f->order.empty()) return fail(f, ACM_EINVAL, "empty forest");
  acm::TopoK t = topo(f);
  if (f->gp.precision == 64) {
    acm_status s = sync_stage<double>(f, (double*)f->U);
    if (s) return s;
    acm::StageK<double> a{(const double*)f->U, (const double*)f->U, (double*)f->ACC, (double*)f->YA,
                          f->mask_on ? (const double*)f->CHI : nullptr, (const double*)f->SLAB, 0.0, 0.0};
    acm::launch_stage<double>(0, f->gp.Bs, a, t, f->phk, f->d_err, f->st, f->stage_variant);
  } else {
    acm_status s = sync_stage<float>(f, (float*)f->U);
    if (s) return s;
    acm::StageK<float> a{(const float*)f->U, (const float*)f->U, (float*)f->ACC, (float*)f->YA,
                         f->mask_on ? (const float*)f->CHI : nullptr, (const float*)f->SLAB, 0.0, 0.0};
    acm::launch_stage<float>(0, f->gp.Bs, a, t, f->phk, f->d_err, f->st, f->stage_variant);
  }
  CKL();
  ++f->launches;
  return copy_fields(f, out, n_elems, on_device, false, 4, f->ACC);
}

acm_status acm_enable_timing(acm_forest* f, int on) {
  if (!f) return ACM_EINVAL;
  f->timing = on != 0;
  return ACM_OK;
}

acm_status acm_last_step_stats(acm_forest* f, acm_step_stats* out) {
  if (!f || !out) return ACM_EINVAL;
  if (f->stats_pending) {
    CK(cudaEventSynchronize(f->ev[11]));
    double st = 0, sy = 0;
    for (int s = 0; s < 4; ++s) {
      float a = 0, b = 0;
      CK(cudaEventElapsedTime(&a, f->ev[3 * s], f->ev[3 * s + 1]));
      CK(cudaEventElapsedTime(&b, f->ev[3 * s + 1], f->ev[3 * s + 2]));
      sy += a;
      st += b;
    }
    f->stats.sync_ms = sy;
    f->stats.stage_ms = st;
    f->stats_pending = false;
  }
  f->stats.host_topology_ms = f->host_topology_ms;
  f->stats.host_tree_ms = f->host_tree_ms;
  f->stats.host_sort_ms = f->host_sort_ms;
  f->stats.host_rows_ms = f->host_rows_ms;
  f->stats.host_wait_ms = f->host_wait_ms;
  *out = f->stats;
  return ACM_OK;
}

int64_t acm_launch_count(const acm_forest* f) { return f ? f->launches : 0; }

const char* acm_last_error(const acm_forest* f) { return f ? f->err.c_str() : "null forest"; }

const char* acm_status_string(acm_status s) {
  switch (s) {
    case ACM_OK: return "ok";
    case ACM_EINVAL: return "invalid argument";
    case ACM_ENOMEM: return "pool too small";
    case ACM_ECAPACITY: return "block pool exhausted";
    case ACM_ECUDA: return "CUDA error";
    case ACM_ETIMEOUT: return "device wait timed out";
    case ACM_ENUMERIC: return "non-finite value";
    case ACM_EGRADING: return "layout not graded or not tiling";
  }
  return "unknown";
}

}  // extern "C"
