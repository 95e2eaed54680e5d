/*
 * libacm -- wavelet-adaptive artificial-compressibility solver on one GB300 (sm_103a).
 *
 * C ABI of the hot path of Engels, Schneider, Reiss, Farge, "A wavelet-adaptive method for
 * multiscale simulation of turbulent flows in flying insects" (arXiv:1912.05371): the
 * per-RK4-stage update over all cubic blocks of an adaptive block grid (ghost synchronisation,
 * fused ACM right-hand side, RK4 combination) and the per-step wavelet detail thresholding
 * that refines and coarsens the grid.  Beyond that path: RK4 steps replayed from CUDA graphs and
 * many instances per graph (acm_rk4_steps, acm_rk4_steps_batch), an autotuner (acm_autotune),
 * the lifted CDF 4/4 wavelet for coarsening (acm_grid_params.wavelet), a moving rigid plate
 * (ACM_MASK_PLATE), a discrete adjoint on a frozen grid (acm_adjoint_*, with equidistant or
 * binomial checkpointing, acm_checkpoint_schedule, and a vector-Jacobian product of the step
 * map) and restart files (acm_save_state, acm_load_state).
 *
 * Conventions (all entry points):
 *  - Every call returns an acm_status; nothing throws across the ABI.  On an error the forest
 *    is left as it was before the call unless the description says otherwise, and
 *    acm_last_error() returns a one-line message.
 *  - Device memory: the caller hands acm_create_forest ONE device buffer (the "pool") of at
 *    least acm_pool_bytes() bytes; all heavy data and device metadata live in it for the
 *    lifetime of the forest (the paper allocates its block array once at start-up, Sec. 4.1).
 *    The library makes no device allocation of its own.  The pool stays owned by the caller
 *    and must outlive the forest.
 *  - Streams: every device operation is enqueued on the cudaStream_t given at creation.  Calls
 *    that return host-visible results (dt, diagnostics, topology, indicators) synchronise
 *    that stream before returning; the others may return while their kernels still run, and
 *    a device error then surfaces at the next synchronising call.
 *  - Devices: a forest belongs to the CUDA device current when it is created (its pool and
 *    stream must be on that device); every call on it must be made with that device current.
 *    The library never switches devices.  Forests on several devices may coexist in one
 *    process.
 *  - Pointers passed in are borrowed for the duration of the call only.
 *  - Layouts: "block order" is ascending (treecode, level); a field array is block-major,
 *    then component (u, v, w, p), then z, y, x with x fastest, Bs^3 points per block, in the
 *    forest's precision (float for precision 32, double for 64).
 *  - Grids are periodic in all three directions; blocks are "redundant": neighbouring blocks
 *    share their face points (Sec. 3.1: x_{2i}^{J+1} = x_i^J, odd point count per block).
 */
#ifndef ACM_H
#define ACM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acm_forest acm_forest;

typedef enum {
  ACM_OK = 0,
  ACM_EINVAL = 1,     /* bad argument or inconsistent parameters                          */
  ACM_ENOMEM = 2,     /* pool too small for the requested layout                          */
  ACM_ECAPACITY = 3,  /* block pool (max_blocks) exhausted; forest unchanged               */
  ACM_ECUDA = 4,      /* a CUDA call failed; message in acm_last_error                      */
  ACM_ETIMEOUT = 5,   /* reserved for bounded device waits                                  */
  ACM_ENUMERIC = 6,   /* non-finite value met (e.g. NaN in the state)                        */
  ACM_EGRADING = 7    /* a supplied layout is not 2:1 graded / does not tile the domain     */
} acm_status;

/* ACM_ENUMERIC comes from the max-norm reduction, which propagates NaN and infinity: acm_rk4_step
 * with dt <= 0 and acm_diagnostics report a non-finite state before changing anything, acm_step
 * with dt <= 0 after its refinement, acm_rk4_steps after its steps (the state and time are then
 * those the steps left).  The batched steps (acm_rk4_steps_batch) do not check. */

/* Grid of cubic blocks (Sec. 4.1).  nroot[3] roots of side root_len tile the periodic box
 * [0, nroot*root_len]; a block at level J has side root_len/2^J and spacing
 * h_J = root_len / (2^J (Bs-1)).  Bs is 9, 17 or 33; Bs = 33 takes precision 32 and the CDF 4/0
 * wavelet (ACM_EINVAL otherwise), and its forests have no adjoint (acm_adjoint_* return
 * ACM_EINVAL) and no persistent batched form (acm_rk4_steps_batch falls back to the graph of
 * per-instance launches).  g is the ghost depth reported by
 * acm_sync_ghosts (1..4).  precision is 32 or 64.  fd_scheme: 1 = Tam-Webb optimised first
 * derivative (Sec. 2.3, the paper's choice), 0 = classical (8,-1)/12.  Levels obey
 * 0 <= Jmin <= Jmax <= 18 (Sec. 3.5).  max_blocks (the block pool) is below 2^32 divided by
 * the larger of a block's padded element count and 72 Bs^2 (about 206,000 blocks at Bs = 17,
 * 29,700 at Bs = 33): device offsets into the pool are 32-bit.
 * wavelet (Sec. 3.2): 40 = CDF 4/0, the interpolating wavelet (a merged parent is the decimated
 * children); 44 = CDF 4/4, its lifted form (Sec. 3.2.1): a merged parent's interior points take
 * the lifted analysis low-pass of the children's level and the 4 fine points around them, its
 * boundary points the decimated value.  Details, thresholds and refinement are the same for
 * both.  0 is read as 40; other values are ACM_EINVAL. */
typedef struct {
  int nroot[3];
  double root_len;
  int Bs;
  int g;
  int Jmin, Jmax;
  int precision;
  int64_t max_blocks;
  int fd_scheme;
  int wavelet;
} acm_grid_params;

/* Model parameters of eqs. (u_eqn-1, p_eqn-1), Sec. 2.1-2.2, and the adaptation controls of
 * Sec. 3.3-3.5.  C_sp <= 0 or sponge == 0 disables the sponge term.  eps is C_eps (strict
 * "<" test on the normalised details); dealias = 1 always tags blocks at Jmax; a block whose
 * mask range max(chi)-min(chi) exceeds mask_range_thr is not coarsened unless dealiasing
 * tags it. */
typedef struct {
  double nu, c0, C_eta, C_gamma, C_sp;
  double u_inf[3], p_inf;
  double cfl, cfl_eta, cfl_nu;
  double eps;
  int dealias;
  double mask_range_thr;
  int sponge;
  double sponge_L[3];     /* periodic box lengths used by the sponge profile               */
  double sponge_width;    /* L_sp: sponge thickness at each box face                        */
  double sponge_delta;    /* smoothing length of the sponge profile                         */
  int coarsen_everywhere; /* 0: tags by thresholds (Sec. 3.3); 1: the performance cycle of
                             Sec. 5.4 ("coarsen everywhere" on random data): every block made by
                             the last acm_refine_all is tagged and the thresholds are ignored,
                             so acm_coarsen restores the grid the step started from (the
                             indicators are still computed; acm_init_grid always thresholds) */
} acm_phys_params;

/* Per-step diagnostics (Sec. 2.2 force by midpoint rule; every physical point counted once:
 * the half-open points [0, Bs-2]^3 of each block, weight h_J^3).  FP64 accumulation. */
typedef struct {
  double force[3];        /* C_eta^{-1} sum chi (u - u_s) h^3                               */
  double energy;          /* 1/2 sum |u|^2 h^3                                              */
  double u_max;           /* max |u| (vector magnitude) over all stored points              */
  double norms[4];        /* max |u|, |v|, |w|, |p| over all stored points                  */
  int64_t n_blocks;
  int64_t blocks_per_level[19];
  double time;
} acm_diag;

/* Initial conditions for acm_set_ic (params in order):
 *  ACM_IC_TAYLOR_GREEN: k, amp     u = amp sin kx cos ky cos kz, v = -amp cos kx sin ky cos kz, w = p = 0
 *  ACM_IC_UNIFORM:      u0, v0, w0, p0
 *  ACM_IC_PULSE:        cx, cy, cz, width, amp, Lx, Ly, Lz   (Gaussian p, u = 0, nearest periodic image)
 *  ACM_IC_PULSE_RING:   the pulse's 8 parameters, then ring cx, cy, cz, axis nx, ny, nz, R, gamma,
 *                       sigma (17 in all): the pulse's p plus a vortex ring's velocity
 *                       u = curl(psi e_theta), psi = gamma/(2 pi) (rho/R) exp(-((rho-R)^2 + zeta^2)/sigma^2)
 *                       in ring coordinates (zeta along the unit axis, rho from it), nearest
 *                       periodic image of the centre -- the synthetic input of the batched
 *                       workload (no counterpart in the paper). */
enum { ACM_IC_TAYLOR_GREEN = 1, ACM_IC_UNIFORM = 2, ACM_IC_PULSE = 3, ACM_IC_PULSE_RING = 4 };

/* Masks for acm_set_mask: ACM_MASK_NONE; ACM_MASK_SPHERE: cx, cy, cz, R, delta with
 * chi = (1 - tanh(d/delta))/2, d the signed distance to the sphere (Sec. 2.2 smoothed mask);
 * ACM_MASK_PLATE: a rigid plate flapping about a pivot (Sec. 2.2 with a moving body; no
 * counterpart workload in the paper): chord, span, thickness, stroke amplitude phi_m, pitch
 * amplitude alpha_m (radians), frequency f, pivot x0, y0, z0, delta.  The plate is the box
 * |x_b| <= chord/2, 0 <= y_b <= span, |z_b| <= thickness/2 of its body frame; x = x0 + R(t) x_b
 * with R = R_z(phi) R_y(alpha), phi = phi_m sin(2 pi f t), alpha = alpha_m cos(2 pi f t); chi is
 * the same tanh profile of the box's signed distance and u_s = omega x (x - x0).  Its pose
 * follows the forest's simulated time: chi is evaluated at every RK4 stage time and the
 * penalization uses u_s; acm_rk4_steps and acm_rk4_steps_batch refuse a moving mask
 * (ACM_EINVAL); the force of acm_diagnostics integrates chi (u - u_s).
 * ACM_MASK_FIELD (no parameters): chi is the caller's field (any geometry, e.g. a mask made
 * from a surface), written with acm_write_mask and 0 until then; u_s = 0.  It belongs to the
 * grid it was written for: acm_set_leaves, acm_init_uniform, acm_init_grid, acm_refine_all,
 * acm_coarsen and acm_step return ACM_EINVAL while it is set (set another mask first).  The
 * vector-Jacobian product (acm_adjoint_vjp) accepts it, with no parameter gradient. */
enum { ACM_MASK_NONE = 0, ACM_MASK_SPHERE = 1, ACM_MASK_PLATE = 2, ACM_MASK_FIELD = 3 };

/* Register ids for acm_sync_ghosts / acm_read_fields (U is the solution). */
enum { ACM_REG_U = 0 };

/* Bytes of device pool needed for these grid parameters (0 on invalid parameters). */
size_t acm_pool_bytes(const acm_grid_params* grid);

/* Create a forest.  stream: a cudaStream_t (borrowed; NULL = legacy default stream).
 * device_pool/pool_bytes: caller-owned device buffer, >= acm_pool_bytes(grid), 256-byte
 * aligned.  The forest starts empty (no blocks).  Returns ACM_EINVAL on bad parameters,
 * ACM_ENOMEM if the pool is too small, ACM_ECUDA if the device is not usable. */
acm_status acm_create_forest(const acm_grid_params* grid, const acm_phys_params* phys,
                             void* stream, void* device_pool, size_t pool_bytes,
                             acm_forest** out);

/* Release host state (the pool is the caller's).  NULL is accepted. */
acm_status acm_destroy_forest(acm_forest* f);

/* Replace the grid by the uniform level-J grid (Jmin <= J <= Jmax); fields are zeroed. */
acm_status acm_init_uniform(acm_forest* f, int J);

/* Replace the grid by the given leaves (level[i], gx[i], gy[i], gz[i]: global block
 * coordinates at that level), created in one pass in block order (Sec. 4.1 slot rule:
 * lowest free slot in ascending key order).  ACM_EGRADING if the leaves do not tile the
 * domain exactly or are not 26-neighbour 2:1 graded.  Fields are zeroed. */
acm_status acm_set_leaves(acm_forest* f, const int32_t* level, const int32_t* gx,
                          const int32_t* gy, const int32_t* gz, int64_t n);

/* Evaluate an initial condition (see ACM_IC_*) at every point of every block, in FP64,
 * stored in the forest precision.  n_params must be at least the kind's count (2, 4, 8, 17)
 * and at most 24; ACM_EINVAL otherwise. */
acm_status acm_set_ic(acm_forest* f, int ic_kind, const double* params, int n_params);

/* Set the obstacle mask chi (Sec. 2.2), evaluated analytically on every block now and after
 * every grid change; u_s = 0 except for the moving plate (see ACM_MASK_PLATE, whose pose
 * follows the forest's time).  kind ACM_MASK_NONE removes it.  t is unused. */
acm_status acm_set_mask(acm_forest* f, int kind, const double* params, int n_params, double t);

/* Initial grid (Sec. 3.5, last paragraph): start from the uniform Jmin grid and repeat
 * {refine all, evaluate the initial condition and the mask, coarsen} until the grid is
 * unchanged.  ic as in acm_set_ic.  On return *n_blocks holds the block count. */
acm_status acm_init_grid(acm_forest* f, int ic_kind, const double* params, int n_params,
                         int64_t* n_blocks);

/* Synchronise register reg (ACM_REG_U) and copy every block's extended array -- interior
 * plus g ghost layers, (Bs+2g)^3 points per component, block order, layout as fields -- to
 * out (device pointer if out_on_device, else host).  Redundant points shared with a finer
 * leaf first take the finer value ("fine wins", modifies the register); ghost points take
 * the value of the finest leaf holding them, else the tensor DD-4 prediction (Sec. 3.1) from
 * the coarser neighbour (Sec. 4.2).  For tests and debugging; acm_rk4_step synchronises by
 * itself. */
acm_status acm_sync_ghosts(acm_forest* f, int reg, void* out, int out_on_device);

/* One classical RK4 step (Sec. 2.3) of eqs. (u_eqn-1, p_eqn-1) on the current grid, each
 * stage = ghost synchronisation + fused right-hand side + RK combination.  dt > 0: use it;
 * dt <= 0: use the CFL rule of Sec. 2.3.  *dt_used (may be NULL) receives the step. */
acm_status acm_rk4_step(acm_forest* f, double dt, double* dt_used);

/* nsteps classical RK4 steps (Sec. 2.3) on the current grid, without adaptation, with the time
 * step computed on the device (dt > 0: fixed; dt <= 0: the CFL rule of Sec. 2.3 from the
 * velocity max norm of the state, each step), so no step waits for the host.  use_graph = 1: the
 * first step runs as plain launches, the second is captured into a CUDA graph and the remaining
 * steps replay it (the graph is kept while the grid and the dt mode stay the same); the legacy
 * default stream cannot be captured and always runs plain launches.  Bitwise the same result as
 * nsteps calls of acm_rk4_step with the same dt rule.  Synchronises the stream at the end;
 * *t_end (may be NULL) receives the simulated time, *graph_used (may be NULL) whether a graph
 * ran.  No counterpart in the paper (a GPU execution form of its time loop). */
acm_status acm_rk4_steps(acm_forest* f, int nsteps, double dt, int use_graph, double* t_end, int* graph_used);

/* acm_rk4_steps for n distinct forests on one device (independent instances, each on its own
 * stream): every step enqueues each instance's step on its stream, so the instances run side by
 * side.  use_graph = 1: the second step of all instances is captured into ONE CUDA graph (each
 * instance a parallel branch forked from forests[0]'s stream) and replayed for the remaining
 * steps.  use_graph = 2, the persistent form: per RK stage every instance's synchronisation (and
 * its time step) runs as a parallel branch, then ONE launch of the fused stage kernel whose CTAs
 * walk the (instance, block) pairs of all instances; the first step runs as plain launches, the
 * second is captured into one CUDA graph and replayed.  It needs forests of one precision and
 * block size with identical physics and grid spacings, and uses forests[0]'s staging buffer
 * (the one acm_read_fields/acm_write_fields use) for its instance table and work list; otherwise
 * the call takes use_graph = 1.  *graph_used receives 0 (plain launches), 1 or 2.  The persistent
 * form computes every block's update bitwise as the other forms do.  Synchronises every stream at
 * the end; t_end (may be NULL) receives n simulated times.  Errors are reported on the forest
 * concerned (forests[0] for capture errors and the persistent stage launches).  No counterpart in
 * the paper. */
acm_status acm_rk4_steps_batch(acm_forest* const* forests, int n, int nsteps, double dt, int use_graph,
                               double* t_end, int* graph_used);

/* Autotuner: on the current grid, time the two task-list kernels of the per-stage ghost
 * synchronisation -- fine wins and the coarse-face halo slabs -- for each number of CTAs per SM
 * walking the list (fine wins 2, 4, 8, 16; slabs 1, 2, 3) and keep the fastest of each for this
 * forest (either output may be NULL).  FP32 forests also time the forms of the fused stage
 * kernel (ACM_STAGE_* below; blocks of 33^3 have one) on one RK stage of the live grid and keep
 * the fastest.  Like every synchronisation it first lets finer leaves' values win on shared
 * boundary points of U; nothing else of the state changes (the stage timing writes only the
 * accumulator and a stage register, which every step rewrites before reading).  Synchronises
 * the stream.  No counterpart in the paper. */
acm_status acm_autotune(acm_forest* f, int* fw_ctas, int* slab_ctas);

/* Forms of the fused right-hand side + RK4 stage kernel (Sec. 2.1-2.3): ACM_STAGE_POINT, one
 * point per thread (the default); ACM_STAGE_PAIR, two x-adjacent points per thread with packed
 * FP32x2 arithmetic (FP32 forests only: fewer instructions, half the resident threads);
 * ACM_STAGE_POINT_TMA, one point per thread with the planes of U, the RK accumulator and the mask
 * brought into a shared-memory ring by mbarrier-tracked bulk copies one plane ahead (FP32 forests
 * only); ACM_STAGE_POINT_ROWS, one point per thread with a block's rows split over CTAs of 9 rows (FP32,
 * Bs = 17: two CTAs of 9 and 8 rows; Bs = 33: four of 9, 9, 9 and 6 rows; smaller CTAs, more of
 * them per SM, each reading the rows next to its own like a halo).  All compute every point by
 * the same formula; ACM_STAGE_POINT, ACM_STAGE_POINT_TMA and ACM_STAGE_POINT_ROWS give bitwise
 * equal results, ACM_STAGE_PAIR differs in FP32 rounding order.  FP64 forests always use
 * ACM_STAGE_POINT; forests of 33^3 blocks use ACM_STAGE_POINT_ROWS or else their three-CTA
 * form (11 rows each) for ACM_STAGE_POINT, ACM_STAGE_PAIR and ACM_STAGE_POINT_TMA. */
#define ACM_STAGE_PAIR 0
#define ACM_STAGE_POINT 1
#define ACM_STAGE_POINT_TMA 2
#define ACM_STAGE_POINT_ROWS 3
/* Force the stage kernel's form (until the next acm_autotune); drops a captured graph.
 * ACM_EINVAL for another value. */
acm_status acm_set_stage_variant(acm_forest* f, int variant);

/* The launch knobs in use: CTAs per SM of the fine-wins and slab kernels, the stage kernel's
 * form, and the autotuner's median times (ms) of one stage launch in each form (indexed by
 * ACM_STAGE_*; 0 until it has timed them). */
typedef struct {
  int fw_ctas_per_sm, slab_ctas_per_sm, stage_variant;
  float stage_ms[4];
} acm_tuning;
acm_status acm_get_tuning(const acm_forest* f, acm_tuning* out);

/* Discrete adjoint (an extension; the paper has none).  For nsteps RK4 steps of fixed dt from
 * the current state on the current grid, frozen (no adaptation: adaptation is not
 * differentiable), the objective J = (1/N) sum_{n=1..N} [F_x(U_n) + w_energy E(U_n)] with the
 * force and energy of Sec. 2.2, and its gradient with respect to the sphere mask's centre and
 * radius (dJ_dtheta[0..3] = d/dcx, d/dcy, d/dcz, d/dR, host) and the initial state (dJ_dU0,
 * FP64 values whatever the forest's precision, block order, fields layout of acm_read_fields,
 * n_elems = n_blocks*4*Bs^3; device pointer if on_device, else host; may be NULL).  FP32 or
 * FP64 forests with the sphere mask (ACM_EINVAL otherwise): the forward steps and the adjoint
 * variables are in the forest's precision, the sums onto the mask parameters (and the returned
 * gradients) in FP64.  States are recomputed from
 * snapshots by the schedule of acm_checkpoint_schedule(nsteps, ckpt): ckpt > 0 keeps the state
 * at every ckpt-th step and recomputes each segment with its states stored; ckpt < 0 is binomial
 * checkpointing with -ckpt snapshots (the fewest recomputed steps for that memory).  Every
 * schedule takes the same steps in the same arithmetic, so the result does not depend on it
 * (up to the order of floating-point atomic sums).  ws: caller device buffer of at least
 * acm_adjoint_bytes(f, nsteps, ckpt) bytes (ACM_ENOMEM if smaller): nine registers and the
 * snapshots in the forest's precision, with ckpt > 0 also the four RK stage states of each of a
 * segment's min(ckpt, nsteps) - 1 recomputed steps (a recomputed step keeps them for its
 * adjoint, which then runs without repeating the step), the mask's sensitivity and one FP64
 * array of n_blocks x 4 x Bs^3 values (all sized for max_blocks).
 * acm_adjoint_bytes returns 0 for an invalid ckpt (0), nsteps outside [1, 2^20] or a refused
 * binomial schedule (see acm_checkpoint_schedule).  The
 * forest's state and time are unchanged on return, also when the sweep stops on an error; the
 * call synchronises the stream.  ACM_EGRADING if a ghost point's source is missing.  The
 * gradient with respect to U_0 is that of the forward map as computed: a point shared by
 * several blocks carries its sensitivity in the copy the forward map reads. */
size_t acm_adjoint_bytes(const acm_forest* f, int nsteps, int ckpt);
acm_status acm_adjoint_sphere(acm_forest* f, int nsteps, double dt, int ckpt, double w_energy, void* ws,
                              size_t ws_bytes, double* J, double* dJ_dtheta, void* dJ_dU0, int64_t n_elems,
                              int on_device);

/* The same for the moving plate (ACM_MASK_PLATE; ACM_EINVAL otherwise), from the forest's time:
 * the mask and the solid velocity follow the RK4 stage times, F_x integrates chi (u - u_s), and
 * *dJ_dalpha (host) receives the derivative with respect to the pitch amplitude alpha_m (the
 * plate's drag sensitivity of the full-scale configuration).  Workspace as acm_adjoint_bytes. */
acm_status acm_adjoint_plate_pitch(acm_forest* f, int nsteps, double dt, int ckpt, double w_energy, void* ws,
                                   size_t ws_bytes, double* J, double* dJ_dalpha, void* dJ_dU0, int64_t n_elems,
                                   int on_device);

/* Vector-Jacobian product of the N-step map U_0 -> U_N (nsteps RK4 steps of fixed dt from the
 * current state and time on the frozen grid, the forward map and checkpointing of
 * acm_adjoint_sphere; a sphere, a moving plate, a field mask or none): for any L with dL_dUN = dL/dU_N
 * (FP64, block order, layout of acm_read_fields, n_elems = n_blocks*4*Bs^3, one value per copy
 * of a redundant point), writes dL_dU0 = dL/dU_0 (same layout; both arrays on the device if
 * on_device, else host) and, if dL_dtheta is not NULL, dL/d(cx, cy, cz, R) of the sphere (4
 * values), dL/d alpha_m of the plate (1 value) or 4 zeros without a mask or with a field mask.  Workspace, restoration of the forest's state
 * and time, and errors as acm_adjoint_sphere.  With it a caller composes the solver with any
 * loss of the final state (the Python binding's step_map_function does so for torch.autograd). */
acm_status acm_adjoint_vjp(acm_forest* f, int nsteps, double dt, int ckpt, void* ws, size_t ws_bytes,
                           const void* dL_dUN, void* dL_dU0, int64_t n_elems, int on_device, double* dL_dtheta);

/* Set the simulated time (a moving mask is evaluated at it).  ACM_EINVAL for a non-finite t. */
acm_status acm_set_time(acm_forest* f, double t);

/* Write the field mask chi (ACM_MASK_FIELD only, ACM_EINVAL otherwise): block order, Bs^3 values
 * per block (layout of acm_read_mask), forest precision, n_elems = n_blocks*Bs^3, device
 * pointer if on_device, else host.  Synchronises the stream. */
acm_status acm_write_mask(acm_forest* f, const void* chi, int64_t n_elems, int on_device);

/* Restart files (the paper's runs resume from saved states across job limits, Sec. 4).
 * acm_save_state writes to path: a header (8 bytes "ACMSTATE", int32 version 1, precision,
 * sizeof(acm_grid_params), sizeof(acm_phys_params), mask kind, 0, the mask's 10 parameters as
 * acm_set_mask takes them (unused ones 0), the time, int64 n_blocks), the forest's
 * acm_grid_params and acm_phys_params, the leaves' level, x, y and z (int32 arrays of n_blocks,
 * block order), the interior fields of U as acm_read_fields returns them and, for a field mask,
 * chi as acm_read_mask returns it; host byte order.
 * acm_read_state_header (host only, no forest) returns a file's parameters, block count and
 * time, so a caller can create a matching forest.  acm_load_state replaces a forest's grid,
 * state, physics parameters, mask and time with the file's; the forest's acm_grid_params must
 * equal the file's except max_blocks, which must hold its blocks (ACM_ECAPACITY), and the file is
 * read whole before anything changes.  ACM_EINVAL for a missing, foreign, truncated or
 * inconsistent file, or a different grid.  Save and load synchronise the stream. */
acm_status acm_save_state(acm_forest* f, const char* path);
acm_status acm_read_state_header(const char* path, acm_grid_params* grid, acm_phys_params* phys, int64_t* n_blocks,
                                 double* time);
acm_status acm_load_state(acm_forest* f, const char* path);

/* The adjoint's checkpoint schedule (host only: no forest, no device work).  The reverse sweep
 * over nsteps steps takes the steps' adjoints in the order nsteps-1, ..., 0, each from its own
 * state, recomputed from snapshots.  ckpt > 0: equidistant, U_k kept for every multiple k of
 * ckpt, ceil(nsteps/ckpt) + max(ckpt - 2, 0) snapshots (ckpt capped at nsteps).  ckpt < 0: binomial
 * checkpointing (Griewank's revolve) with S = -ckpt snapshots (capped at nsteps): the fewest
 * recomputed steps for S stored states, r n - C(S + r, r - 1) with r the least integer with
 * C(S + r, S) >= n.  Writes the snapshots used and the recomputed (plain forward) steps, the n
 * steps taken with their adjoint not counted (either pointer may be NULL) and the number of
 * actions.  With ops and args (both non-NULL, cap entries) it also writes the actions in order:
 * op 0 STORE j (current state into snapshot j), 1 RESTORE j (snapshot j becomes current),
 * 2 ADVANCE k (plain step k -> k+1 from U_k), 3 TURN k (step k with its adjoint, from U_k; the
 * current state is used up); args holds j or k.  The first action stores U_0 in snapshot 0,
 * which is never written again.  ACM_EINVAL for nsteps outside [1, 2^20], ckpt = 0, a binomial
 * schedule of more than 2^26 recomputed steps, or cap below the number of actions (which is
 * still written). */
acm_status acm_checkpoint_schedule(int nsteps, int ckpt, int32_t* snapshots, int64_t* advances, int8_t* ops,
                                   int32_t* args, int64_t cap, int64_t* n_actions);

/* Right-hand side K = F(U) of eqs. (u_eqn-1, p_eqn-1) at every point of every block, after
 * the same synchronisation as an RK4 stage, written in block order (fields layout) to out
 * (device pointer if on_device, else host; n_elems = n_blocks*4*Bs^3).  For checks: the
 * fused stage kernel computes exactly this K inside acm_rk4_step. */
acm_status acm_rhs(acm_forest* f, void* out, int64_t n_elems, int on_device);

/* Refine every block below Jmax by one level (Sec. 3.5 step 1); children are the DD-4
 * prediction of the synchronised parent.  ACM_ECAPACITY (forest unchanged) if the pool of
 * max_blocks slots is too small. */
acm_status acm_refine_all(acm_forest* f);

/* Coarsening (Sec. 3.5 step 3): details of every block, normalised per component by its
 * global max norm (taken once, before the first pass); tag if below eps (and J > Jmin, and
 * the mask range <= thr), or always at Jmax with dealiasing; merge tagged sister groups that
 * keep the grid graded; repeat until nothing changes.  A merged parent is made as the grid's
 * wavelet says (decimation for CDF 4/0, the lifted low-pass inside for CDF 4/4).  *n_blocks (may
 * be NULL) receives the block count, *n_passes (may be NULL) the number of merging passes. */
acm_status acm_coarsen(acm_forest* f, int64_t* n_blocks, int* n_passes);

/* The grid adaptation after a time step (Sec. 3.5 step 3: details -> tags -> tree -> data
 * moves): acm_coarsen, with the block count as an int (n_blocks may be NULL).  Errors as
 * acm_coarsen. */
acm_status acm_adapt(acm_forest* f, int* n_blocks);

/* The paper's time step (Sec. 3.5): refine all, RK4 (dt as in acm_rk4_step), coarsen. */
acm_status acm_step(acm_forest* f, double dt, double* dt_used, int64_t* n_blocks);

/* Per-block indicators of the current (synchronised) state, block order:
 * ind[i] = max over components of max |detail| / ||component||_inf (components with zero norm
 * skipped), chi_range[i] = max chi - min chi (0 without mask).  Either pointer may be NULL. */
acm_status acm_block_indicators(acm_forest* f, double* ind, double* chi_range, int64_t n);

/* Diagnostics of the current state (see acm_diag). */
acm_status acm_diagnostics(acm_forest* f, acm_diag* out);

/* Number of blocks. */
int64_t acm_n_blocks(const acm_forest* f);

/* Topology in block order, for bit-exact checks.  Any pointer may be NULL; each non-NULL
 * array must hold n entries (nbr: n*56, rel: n*26) with n >= acm_n_blocks.
 *  treecode: root number << 56 | per-level octal digit (bx + 2by + 4bz) of level l at bits
 *            3*(18-l) .. +2 (Sec. 4.1, Gargantini)
 *  level, slot (position in the block pool)
 *  nbr[56]: 26 directions ordered by iterating dz, dy, dx over -1,0,1 (x fastest), faces
 *           first, then edges, then corners; face k -> entries 4k..4k+3, edge k -> 24+2k..,
 *           corner k -> 48+k; same-level or coarser neighbour: its slot in the first entry;
 *           finer: the touching children's slots in ascending child number; unused: -1
 *  rel[26]: 0 same level, -1 coarser, +1 finer. */
acm_status acm_get_topology(acm_forest* f, uint64_t* treecode, uint8_t* level, int32_t* slot,
                            int32_t* gx, int32_t* gy, int32_t* gz, int32_t* nbr, int8_t* rel,
                            int64_t n);

/* Copy the fields of register reg in block order to/from host or device memory (layout in
 * the header conventions; n_elems must equal n_blocks*4*Bs^3). */
acm_status acm_read_fields(acm_forest* f, int reg, void* out, int64_t n_elems, int on_device);
acm_status acm_write_fields(acm_forest* f, const void* in, int64_t n_elems, int on_device);

/* Copy the mask chi in block order (n_blocks*Bs^3 elements, forest precision). */
acm_status acm_read_mask(acm_forest* f, void* out, int64_t n_elems, int on_device);

/* Per-kernel timing of the last acm_rk4_step with timing enabled (CUDA events recorded on the
 * forest's stream around each stage's synchronisation kernels and fused stage kernel; read
 * when this is called, which waits for the last of them), milliseconds summed over the four
 * stages, and the algorithmic bytes of the four fused stage kernels (per point 64 words of
 * register traffic, plus 4 words of mask when a mask is set). */
typedef struct {
  double stage_ms;        /* fused RHS+RK4 stage kernels                                    */
  double sync_ms;         /* fine-wins and coarse-face prediction kernels                    */
  double stage_bytes;     /* algorithmic bytes of the stage kernels                          */
  int64_t n_launches;     /* kernels launched by the step                                    */
  double host_topology_ms;/* cumulative host time rebuilding block tables since creation     */
  double host_tree_ms;    /* cumulative host time of refine/coarsen tree logic since creation */
  double host_sort_ms;    /* part of host_topology_ms: ordering the blocks                     */
  double host_rows_ms;    /* part of host_topology_ms: building the neighbourhood rows          */
  double host_wait_ms;    /* part of host_topology_ms: waiting for the stream after the copies  */
} acm_step_stats;
acm_status acm_enable_timing(acm_forest* f, int on);
acm_status acm_last_step_stats(acm_forest* f, acm_step_stats* out);

/* Fused multiply-add rate of the current device in flop/s (2 per FMA), measured by a kernel of
 * this library: independent chains of dependent FMAs in FP64 (precision 64) or FP32 (32) on every
 * SM, the median CUDA-event time of five launches after a warm-up, on `stream` (cudaStream_t,
 * NULL = legacy default); synchronises the stream.  The FP64 stage kernel's roofline denominator
 * (GB300's FP64 pipe, not HBM, bounds FP64 fields).  ACM_EINVAL for another precision or a NULL
 * output, ACM_ECUDA if a launch fails.  No counterpart in the paper. */
acm_status acm_fma_rate(int precision, double* flops_out, void* stream);

/* Total kernel launches since creation (every launch of this library). */
int64_t acm_launch_count(const acm_forest* f);

/* Largest block count acm_max_norms_noalloc accepts (its scratch holds 5 doubles per block,
 * 640 KiB, resident on every device that loads the library until the process exits). */
#define ACM_NOALLOC_MAX_BLOCKS 16384

/* Max norms of a field array without any device allocation.  (The paper has no counterpart:
 * this serves callers of the library, not the method.)
 *
 * Some callers cannot allocate device memory at the point of the call: a process whose device
 * memory is owned and budgeted by another allocator (a framework's caching pool), a time-critical
 * host loop that must not trigger the device-wide synchronisation cudaMalloc/cudaFree can imply,
 * or a caller that holds only a field array and no forest (whose pool would otherwise provide the
 * scratch).  This call needs nothing from them but the input and the output.
 *
 * fields: device array in block order as written by acm_read_fields (n_blocks x 4 components
 * x Bs^3, x fastest), float for precision 32, double for 64.  norms_out: device array of 5
 * doubles receiving max|u|, max|v|, max|w|, max|p| and max |(u,v,w)| (arithmetic in the field
 * precision, as inside acm_diagnostics; a NaN or an infinity in a component is carried into its
 * norm, NaN before infinity, as acm_diagnostics reports a non-finite state).  stream:
 * cudaStream_t (NULL = legacy default stream);
 * the call is asynchronous on it.
 * Returns ACM_EINVAL for bad arguments (Bs other than 9, 17 or 33, precision other than 32 or 64,
 * NULL pointers, n_blocks < 1), ACM_ECAPACITY if n_blocks > ACM_NOALLOC_MAX_BLOCKS (nothing is
 * launched), ACM_ECUDA if a launch or the set-up fails.
 * Scratch: a fixed array compiled into the library (per-block partial maxima).  The first call
 * on each device looks up that array's device address (with the device current); make that
 * first call before any stream capture.  Every call shares the one array and writes the entries
 * it reads, so nothing needs clearing; calls that overlap on the GPU (different streams, or
 * different host threads on one device) race on it and must be serialised by the caller. */
acm_status acm_max_norms_noalloc(const void* fields, int64_t n_blocks, int Bs, int precision,
                                 double* norms_out, void* stream);

const char* acm_last_error(const acm_forest* f);
const char* acm_status_string(acm_status s);

#ifdef __cplusplus
}
#endif
#endif /* ACM_H */
