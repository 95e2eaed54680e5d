"""Python binding of libacm (include/acm.h): argument marshalling only.

Every operation runs in the CUDA library; this module converts arguments and raises on a
non-zero status.  PyTorch supplies the device pool and the stream.  There is no fallback: if
the compiled library is missing, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libacm.so")

ACM_IC_TAYLOR_GREEN, ACM_IC_UNIFORM, ACM_IC_PULSE, ACM_IC_PULSE_RING = 1, 2, 3, 4
ACM_MASK_NONE, ACM_MASK_SPHERE, ACM_MASK_PLATE, ACM_MASK_FIELD = 0, 1, 2, 3
ACM_STAGE_PAIR, ACM_STAGE_POINT, ACM_STAGE_POINT_TMA, ACM_STAGE_POINT_ROWS = 0, 1, 2, 3
ACM_REG_U = 0


class GridParams(C.Structure):
    _fields_ = [("nroot", C.c_int * 3), ("root_len", C.c_double), ("Bs", C.c_int), ("g", C.c_int),
                ("Jmin", C.c_int), ("Jmax", C.c_int), ("precision", C.c_int),
                ("max_blocks", C.c_int64), ("fd_scheme", C.c_int), ("wavelet", C.c_int)]


class PhysParams(C.Structure):
    _fields_ = [("nu", C.c_double), ("c0", C.c_double), ("C_eta", C.c_double), ("C_gamma", C.c_double),
                ("C_sp", C.c_double), ("u_inf", C.c_double * 3), ("p_inf", C.c_double),
                ("cfl", C.c_double), ("cfl_eta", C.c_double), ("cfl_nu", C.c_double), ("eps", C.c_double),
                ("dealias", C.c_int), ("mask_range_thr", C.c_double), ("sponge", C.c_int),
                ("sponge_L", C.c_double * 3), ("sponge_width", C.c_double), ("sponge_delta", C.c_double),
                ("coarsen_everywhere", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("force", C.c_double * 3), ("energy", C.c_double), ("u_max", C.c_double),
                ("norms", C.c_double * 4), ("n_blocks", C.c_int64), ("blocks_per_level", C.c_int64 * 19),
                ("time", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("fw_ctas_per_sm", C.c_int), ("slab_ctas_per_sm", C.c_int), ("stage_variant", C.c_int),
                ("stage_ms", C.c_float * 4)]


class StepStats(C.Structure):
    _fields_ = [("stage_ms", C.c_double), ("sync_ms", C.c_double), ("stage_bytes", C.c_double),
                ("n_launches", C.c_int64), ("host_topology_ms", C.c_double), ("host_tree_ms", C.c_double),
                ("host_sort_ms", C.c_double), ("host_rows_ms", C.c_double), ("host_wait_ms", C.c_double)]


EXPORTS = {
    "acm_pool_bytes": (C.c_size_t, [C.POINTER(GridParams)]),
    "acm_create_forest": (C.c_int, [C.POINTER(GridParams), C.POINTER(PhysParams), C.c_void_p, C.c_void_p,
                                    C.c_size_t, C.POINTER(C.c_void_p)]),
    "acm_destroy_forest": (C.c_int, [C.c_void_p]),
    "acm_init_uniform": (C.c_int, [C.c_void_p, C.c_int]),
    "acm_set_leaves": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "acm_set_ic": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "acm_set_mask": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_double]),
    "acm_init_grid": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(C.c_int64)]),
    "acm_sync_ghosts": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "acm_rk4_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "acm_rk4_steps": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                C.POINTER(C.c_int)]),
    "acm_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "acm_set_stage_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "acm_fma_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "acm_get_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "acm_adjoint_bytes": (C.c_size_t, [C.c_void_p, C.c_int, C.c_int]),
    "acm_adjoint_sphere": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double, C.c_void_p, C.c_size_t,
                                     C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "acm_adjoint_plate_pitch": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double, C.c_void_p,
                                          C.c_size_t, C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_int64,
                                          C.c_int]),
    "acm_checkpoint_schedule": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_void_p,
                                          C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "acm_adjoint_vjp": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                  C.c_void_p, C.c_int64, C.c_int, C.c_void_p]),
    "acm_set_time": (C.c_int, [C.c_void_p, C.c_double]),
    "acm_save_state": (C.c_int, [C.c_void_p, C.c_char_p]),
    "acm_read_state_header": (C.c_int, [C.c_char_p, C.POINTER(GridParams), C.POINTER(PhysParams),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "acm_load_state": (C.c_int, [C.c_void_p, C.c_char_p]),
    "acm_rk4_steps_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "acm_refine_all": (C.c_int, [C.c_void_p]),
    "acm_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "acm_coarsen": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "acm_adapt": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "acm_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "acm_block_indicators": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "acm_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(Diag)]),
    "acm_n_blocks": (C.c_int64, [C.c_void_p]),
    "acm_get_topology": (C.c_int, [C.c_void_p] + [C.c_void_p] * 8 + [C.c_int64]),
    "acm_read_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_int]),
    "acm_write_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "acm_read_mask": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "acm_write_mask": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int]),
    "acm_enable_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "acm_last_step_stats": (C.c_int, [C.c_void_p, C.POINTER(StepStats)]),
    "acm_launch_count": (C.c_int64, [C.c_void_p]),
    "acm_last_error": (C.c_char_p, [C.c_void_p]),
    "acm_status_string": (C.c_char_p, [C.c_int]),
    "acm_max_norms_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """The loaded libacm; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libacm is not built ({LIB_PATH}); run paper_1912_05371_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class AcmError(RuntimeError):
    pass


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


NOALLOC_MAX_BLOCKS = 16384


def rk4_steps_batch(forests, nsteps, dt=0.0, graph=True):
    """nsteps RK4 steps of several independent forests (each on its own stream), optionally as
    one CUDA graph per step (graph=True or 1) or in the persistent form (graph=2: one stage launch
    walking the blocks of all instances, inside one graph per step); returns (list of simulated
    times, the form that ran: 0 plain launches, 1 graph, 2 persistent)."""
    n = len(forests)
    hs = (C.c_void_p * n)(*[f.h for f in forests])
    t = (C.c_double * n)()
    g = C.c_int()
    mode = graph if (isinstance(graph, int) and not isinstance(graph, bool)) else int(bool(graph))
    st = lib().acm_rk4_steps_batch(hs, n, int(nsteps), float(dt), int(mode), t, C.byref(g))
    if st != 0:
        msg = lib().acm_status_string(st).decode()
        raise AcmError(f"libacm status {st}: {msg}")
    return list(t), int(g.value)


def fma_rate(precision, stream=None):
    """Fused multiply-add rate of the current GPU in flop/s, measured by the library's own kernel
    (acm_fma_rate)."""
    v = C.c_double()
    st = lib().acm_fma_rate(int(precision), C.byref(v), C.c_void_p(0 if stream is None else stream.cuda_stream))
    if st != 0:
        raise AcmError(f"libacm status {st}: {lib().acm_status_string(st).decode()}")
    return v.value


def max_norms_noalloc(fields, n_blocks, Bs, precision, norms_out, stream=None):
    """Max norms of a device field array through the allocation-free entry point
    (acm_max_norms_noalloc): ``fields`` and ``norms_out`` are CUDA tensors (the latter 5
    doubles); returns the status code (0 on success)."""
    st = 0 if stream is None else stream.cuda_stream
    return lib().acm_max_norms_noalloc(C.c_void_p(fields.data_ptr()), int(n_blocks), int(Bs), int(precision),
                                       C.c_void_p(norms_out.data_ptr()), C.c_void_p(st))


class Forest:
    """One forest of the C library.  ``pool`` is a torch uint8 CUDA tensor (allocated here from
    the size the library asks for) kept alive for the forest's lifetime.  The forest belongs to
    ``device`` (default: the current one); call its methods with that device current
    (``torch.cuda.device(...)``), as the library uses the current device."""

    def __init__(self, grid: dict, phys: dict, stream=None, device=None):
        import torch
        self.L = lib()
        g = GridParams()
        g.nroot = (C.c_int * 3)(*grid.get("nroot", (1, 1, 1)))
        g.root_len = grid.get("root_len", 1.0)
        g.Bs = grid.get("Bs", 17)
        g.g = grid.get("g", 4)
        g.Jmin = grid.get("Jmin", 0)
        g.Jmax = grid.get("Jmax", 18)
        g.precision = grid.get("precision", 64)
        g.max_blocks = grid.get("max_blocks", 4096)
        g.fd_scheme = grid.get("fd_scheme", 1)
        g.wavelet = grid.get("wavelet", 40)
        p = PhysParams()
        p.nu = phys.get("nu", 0.0)
        p.c0 = phys.get("c0", 1.0)
        p.C_eta = phys.get("C_eta", 1.0)
        p.C_gamma = phys.get("C_gamma", 0.0)
        p.C_sp = phys.get("C_sp", 0.0)
        p.u_inf = (C.c_double * 3)(*phys.get("u_inf", (0.0, 0.0, 0.0)))
        p.p_inf = phys.get("p_inf", 0.0)
        p.cfl = phys.get("cfl", 0.5)
        p.cfl_eta = phys.get("cfl_eta", 1.0)
        p.cfl_nu = phys.get("cfl_nu", 0.25)
        p.eps = phys.get("eps", 1e-3)
        p.dealias = int(phys.get("dealias", 0))
        p.mask_range_thr = phys.get("mask_range_thr", 1e-5)
        p.sponge = int(phys.get("sponge", 0))
        p.sponge_L = (C.c_double * 3)(*phys.get("sponge_L", (1.0, 1.0, 1.0)))
        p.sponge_width = phys.get("sponge_width", 0.0)
        p.sponge_delta = phys.get("sponge_delta", 1.0)
        p.coarsen_everywhere = int(phys.get("coarsen_everywhere", 0))
        self.grid, self.phys = g, p
        self.Bs = g.Bs
        self.dtype = np.float64 if g.precision == 64 else np.float32
        nbytes = self.L.acm_pool_bytes(C.byref(g))
        if nbytes == 0:
            raise AcmError("invalid grid parameters")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.pool = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        with torch.cuda.device(dev):
            self._check(self.L.acm_create_forest(C.byref(g), C.byref(p), C.c_void_p(self.stream.cuda_stream),
                                                 C.c_void_p(self.pool.data_ptr()), nbytes, C.byref(h)), None)
        self.h = h

    def _after_producer(self, t):
        """Make the forest's stream wait for the caller's current stream, which made the device
        tensor t (torch's convention); the library's calls synchronise their own stream before
        returning, so outputs need no wait."""
        import torch
        cur = torch.cuda.current_stream(t.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)

    def _check(self, st, h="self"):
        if st != 0:
            msg = self.L.acm_status_string(st).decode()
            if h is not None and getattr(self, "h", None):
                msg += ": " + self.L.acm_last_error(self.h).decode()
            raise AcmError(f"libacm status {st}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.L.acm_destroy_forest(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- grid ------------------------------------------------------------------------------------
    def init_uniform(self, J):
        self._check(self.L.acm_init_uniform(self.h, J))

    def set_leaves(self, leaves):
        a = np.asarray(leaves, dtype=np.int32).reshape(-1, 4)
        cols = [np.ascontiguousarray(a[:, i]) for i in range(4)]
        self._check(self.L.acm_set_leaves(self.h, *[_ptr(c) for c in cols], a.shape[0]))

    def set_ic(self, kind, params):
        pr = np.asarray(params, dtype=np.float64)
        self._check(self.L.acm_set_ic(self.h, kind, _ptr(pr), pr.size))

    def set_mask(self, kind, params=(), t=0.0):
        pr = np.asarray(params, dtype=np.float64)
        self._check(self.L.acm_set_mask(self.h, kind, _ptr(pr) if pr.size else None, pr.size, t))

    def init_grid(self, ic_kind, params):
        pr = np.asarray(params, dtype=np.float64)
        n = C.c_int64()
        self._check(self.L.acm_init_grid(self.h, ic_kind, _ptr(pr), pr.size, C.byref(n)))
        return n.value

    def n_blocks(self):
        return self.L.acm_n_blocks(self.h)

    # ---- time stepping -----------------------------------------------------------------------
    def rk4_step(self, dt=0.0):
        d = C.c_double()
        self._check(self.L.acm_rk4_step(self.h, dt, C.byref(d)))
        return d.value

    def rk4_steps(self, nsteps, dt=0.0, graph=True):
        """nsteps RK4 steps on the current grid with the time step on the device; returns
        (simulated time, whether a CUDA graph ran)."""
        t = C.c_double()
        g = C.c_int()
        self._check(self.L.acm_rk4_steps(self.h, int(nsteps), float(dt), int(bool(graph)), C.byref(t), C.byref(g)))
        return t.value, bool(g.value)

    def autotune(self):
        """Choose this forest's launch knobs by timing them on the current grid; returns the CTAs
        per SM of the fine-wins and of the coarse-face slab kernels."""
        a, b = C.c_int(), C.c_int()
        self._check(self.L.acm_autotune(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_stage_variant(self, variant):
        """Force the stage kernel's form: ACM_STAGE_POINT (one point per thread), ACM_STAGE_PAIR
        (two points per thread, FP32), ACM_STAGE_POINT_TMA (one point per thread, bulk-copy
        staging, FP32) or ACM_STAGE_POINT_ROWS (one point per thread, a 17^3 block's rows over
        two CTAs, FP32)."""
        self._check(self.L.acm_set_stage_variant(self.h, int(variant)))

    def tuning(self):
        """The launch knobs in use (see acm_get_tuning)."""
        t = Tuning()
        self._check(self.L.acm_get_tuning(self.h, C.byref(t)))
        return dict(fw_ctas_per_sm=t.fw_ctas_per_sm, slab_ctas_per_sm=t.slab_ctas_per_sm,
                    stage_variant=t.stage_variant, stage_ms=tuple(t.stage_ms))

    def _adjoint_workspace(self, nsteps, policy):
        import torch
        nbytes = int(self.L.acm_adjoint_bytes(self.h, int(nsteps), policy))
        if nbytes == 0:
            raise ValueError(f"invalid checkpointing ({policy}) or step count ({nsteps})")
        return torch.empty(nbytes, dtype=torch.uint8, device=self.pool.device), nbytes

    def adjoint_sphere(self, nsteps, dt, ckpt_every=10, w_energy=0.1, snapshots=None):
        """J = (1/N) sum_n [F_x(U_n) + w_energy E(U_n)] over nsteps fixed-dt RK4 steps on the frozen
        grid, and its gradient: returns (J, dJ/d(cx, cy, cz, R) (4,), dJ/dU_0 in the layout of
        read_fields, float64).  The forward runs in the forest's precision, the adjoint in FP64;
        the sphere mask must be set; the forest's state is unchanged.  States are recomputed from
        a checkpoint every ckpt_every steps, or with snapshots=S by binomial checkpointing with S
        stored states (see checkpoint_schedule)."""
        policy = checkpoint_policy(ckpt_every, snapshots)
        ws, nbytes = self._adjoint_workspace(nsteps, policy)
        n = self.n_blocks()
        g = np.empty((n, 4, self.Bs, self.Bs, self.Bs), dtype=np.float64)
        J = C.c_double()
        th = np.zeros(4)
        self._check(self.L.acm_adjoint_sphere(self.h, int(nsteps), float(dt), policy, float(w_energy),
                                              C.c_void_p(ws.data_ptr()), nbytes, C.byref(J), _ptr(th), _ptr(g),
                                              g.size, 0))
        return J.value, th, g

    def adjoint_plate_pitch(self, nsteps, dt, ckpt_every=10, w_energy=0.1, snapshots=None):
        """As adjoint_sphere for the moving plate, from the forest's time: returns (J, dJ/d alpha_m,
        dJ/dU_0)."""
        policy = checkpoint_policy(ckpt_every, snapshots)
        ws, nbytes = self._adjoint_workspace(nsteps, policy)
        n = self.n_blocks()
        g = np.empty((n, 4, self.Bs, self.Bs, self.Bs), dtype=np.float64)
        J = C.c_double()
        da = np.zeros(1)
        self._check(self.L.acm_adjoint_plate_pitch(self.h, int(nsteps), float(dt), policy, float(w_energy),
                                                   C.c_void_p(ws.data_ptr()), nbytes, C.byref(J), _ptr(da),
                                                   _ptr(g), g.size, 0))
        return J.value, float(da[0]), g

    def adjoint_vjp(self, nsteps, dt, dL_dUN, ckpt_every=10, snapshots=None):
        """Vector-Jacobian product of nsteps fixed-dt RK4 steps from the current state and time:
        dL_dUN (n_blocks, 4, Bs, Bs, Bs) float64, numpy or a CUDA tensor -> (dL/dU_0 of the same
        kind, dL/d(cx, cy, cz, R) for the sphere; for the plate element 0 is dL/d alpha_m)."""
        import torch
        policy = checkpoint_policy(ckpt_every, snapshots)
        ws, nbytes = self._adjoint_workspace(nsteps, policy)
        n = self.n_blocks()
        shape = (n, 4, self.Bs, self.Bs, self.Bs)
        on_dev = int(hasattr(dL_dUN, "data_ptr") and dL_dUN.is_cuda)
        if on_dev:
            src = dL_dUN.detach().to(torch.float64).contiguous()
            out = torch.empty(shape, dtype=torch.float64, device=src.device)
            self._after_producer(src)
        else:
            src = np.ascontiguousarray(dL_dUN, dtype=np.float64)
            out = np.empty(shape, dtype=np.float64)
        if tuple(src.shape) != shape:
            raise ValueError(f"dL_dUN must have shape {shape}")
        th = np.zeros(4)
        self._check(self.L.acm_adjoint_vjp(self.h, int(nsteps), float(dt), policy, C.c_void_p(ws.data_ptr()), nbytes,
                                           _ptr(src), _ptr(out), int(np.prod(shape)), on_dev, _ptr(th)))
        return out, th

    def set_time(self, t):
        self._check(self.L.acm_set_time(self.h, float(t)))

    def rhs(self):
        n = self.n_blocks()
        out = np.empty((n, 4, self.Bs, self.Bs, self.Bs), dtype=self.dtype)
        self._check(self.L.acm_rhs(self.h, _ptr(out), out.size, 0))
        return out

    def refine_all(self):
        self._check(self.L.acm_refine_all(self.h))

    # ---- restart files --------------------------------------------------------------------------
    def save(self, path):
        """Write the grid, state, parameters, mask and time to a restart file."""
        self._check(self.L.acm_save_state(self.h, os.fsencode(path)))

    def load(self, path):
        """Replace this forest's grid, state, parameters, mask and time with a restart file's
        (its grid parameters must equal this forest's, max_blocks large enough)."""
        self._check(self.L.acm_load_state(self.h, os.fsencode(path)))

    @classmethod
    def from_file(cls, path, max_blocks=None, stream=None, device=None):
        """A new forest resumed from a restart file (max_blocks defaults to the saving forest's)."""
        grid, phys, _, _ = read_state_header(path)
        if max_blocks is not None:
            grid["max_blocks"] = int(max_blocks)
        f = cls(grid, phys, stream=stream, device=device)
        f.load(path)
        return f

    def coarsen(self):
        n, p = C.c_int64(), C.c_int()
        self._check(self.L.acm_coarsen(self.h, C.byref(n), C.byref(p)))
        return n.value, p.value

    def adapt(self):
        """The grid adaptation after a step (acm_adapt: coarsening); returns the block count."""
        n = C.c_int()
        self._check(self.L.acm_adapt(self.h, C.byref(n)))
        return n.value

    def step(self, dt=0.0):
        d, n = C.c_double(), C.c_int64()
        self._check(self.L.acm_step(self.h, dt, C.byref(d), C.byref(n)))
        return d.value, n.value

    # ---- data ---------------------------------------------------------------------------------------
    def read_fields(self, out=None):
        n = self.n_blocks()
        shape = (n, 4, self.Bs, self.Bs, self.Bs)
        if out is None:
            out = np.empty(shape, dtype=self.dtype)
        on_dev = int(hasattr(out, "data_ptr") and out.is_cuda)
        self._check(self.L.acm_read_fields(self.h, ACM_REG_U, _ptr(out), int(np.prod(shape)), on_dev))
        return out

    def write_fields(self, arr):
        n = self.n_blocks()
        on_dev = int(hasattr(arr, "data_ptr") and arr.is_cuda)
        if on_dev:
            self._after_producer(arr)
        if not hasattr(arr, "data_ptr"):
            arr = np.ascontiguousarray(arr, dtype=self.dtype)
        self._check(self.L.acm_write_fields(self.h, _ptr(arr), n * 4 * self.Bs ** 3, on_dev))

    def write_mask(self, chi):
        """The field mask's chi (ACM_MASK_FIELD): (n_blocks, Bs, Bs, Bs), numpy or a CUDA tensor."""
        n = self.n_blocks()
        on_dev = int(hasattr(chi, "data_ptr") and chi.is_cuda)
        if on_dev:
            self._after_producer(chi)
        else:
            chi = np.ascontiguousarray(chi, dtype=self.dtype)
        self._check(self.L.acm_write_mask(self.h, _ptr(chi), n * self.Bs ** 3, on_dev))

    def read_mask(self):
        n = self.n_blocks()
        out = np.empty((n, self.Bs, self.Bs, self.Bs), dtype=self.dtype)
        self._check(self.L.acm_read_mask(self.h, _ptr(out), out.size, 0))
        return out

    def sync_ghosts(self):
        n = self.n_blocks()
        ne = self.Bs + 2 * self.grid.g
        out = np.empty((n, 4, ne, ne, ne), dtype=self.dtype)
        self._check(self.L.acm_sync_ghosts(self.h, ACM_REG_U, _ptr(out), 0))
        return out

    def block_indicators(self):
        n = self.n_blocks()
        ind = np.empty(n)
        rng = np.empty(n)
        self._check(self.L.acm_block_indicators(self.h, _ptr(ind), _ptr(rng), n))
        return ind, rng

    def diagnostics(self):
        d = Diag()
        self._check(self.L.acm_diagnostics(self.h, C.byref(d)))
        return dict(force=tuple(d.force), energy=d.energy, u_max=d.u_max, norms=tuple(d.norms),
                    n_blocks=d.n_blocks, blocks_per_level=tuple(d.blocks_per_level), time=d.time)

    def topology(self):
        n = self.n_blocks()
        tc = np.empty(n, np.uint64)
        lv = np.empty(n, np.uint8)
        sl = np.empty(n, np.int32)
        gx, gy, gz = np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n, np.int32)
        nbr = np.empty((n, 56), np.int32)
        rel = np.empty((n, 26), np.int8)
        self._check(self.L.acm_get_topology(self.h, _ptr(tc), _ptr(lv), _ptr(sl), _ptr(gx), _ptr(gy), _ptr(gz),
                                            _ptr(nbr), _ptr(rel), n))
        return dict(treecode=tc, level=lv, slot=sl, gx=gx, gy=gy, gz=gz, nbr=nbr, rel=rel)

    def enable_timing(self, on=True):
        self._check(self.L.acm_enable_timing(self.h, int(on)))

    def last_step_stats(self):
        s = StepStats()
        self._check(self.L.acm_last_step_stats(self.h, C.byref(s)))
        return dict(stage_ms=s.stage_ms, sync_ms=s.sync_ms, stage_bytes=s.stage_bytes, n_launches=s.n_launches,
                    host_topology_ms=s.host_topology_ms, host_tree_ms=s.host_tree_ms, host_sort_ms=s.host_sort_ms,
                    host_rows_ms=s.host_rows_ms, host_wait_ms=s.host_wait_ms)

    def launch_count(self):
        return self.L.acm_launch_count(self.h)


def _fields_dict(st):
    out = {}
    for name, _ in st._fields_:
        v = getattr(st, name)
        out[name] = tuple(v) if isinstance(v, C.Array) else v
    return out


def read_state_header(path):
    """(grid dict, phys dict, n_blocks, time) of a restart file (host only); the dicts are what
    Forest takes."""
    L = lib()
    g, p = GridParams(), PhysParams()
    n, t = C.c_int64(), C.c_double()
    st = L.acm_read_state_header(os.fsencode(path), C.byref(g), C.byref(p), C.byref(n), C.byref(t))
    if st != 0:
        raise AcmError(f"acm_read_state_header: {L.acm_status_string(st).decode()} ({path})")
    return _fields_dict(g), _fields_dict(p), n.value, t.value


def step_map_function():
    """A torch.autograd.Function for the N-step map: forward(forest, U0, theta, nsteps, dt,
    ckpt_every=10, snapshots=None) writes U0 (block order, read_fields layout, float64) and the
    sphere mask theta = (cx, cy, cz, R, delta) into the forest, takes nsteps fixed-dt RK4 steps on
    its frozen grid and returns U_N (float64), leaving the forest at U0 and its start time;
    backward returns dL/dU0 and dL/d(cx, cy, cz, R) (none for delta) from the library's
    vector-Jacobian product, so any loss of U_N can be differentiated."""
    import torch

    class StepMap(torch.autograd.Function):
        @staticmethod
        def forward(ctx, forest, U0, theta, nsteps, dt, ckpt_every=10, snapshots=None):
            u0 = U0.detach().cpu().numpy()
            t0 = forest.diagnostics()["time"] if forest.n_blocks() else 0.0
            forest.write_fields(u0)
            forest.set_mask(ACM_MASK_SPHERE, [float(v) for v in theta.detach().cpu()])
            for _ in range(int(nsteps)):
                forest.rk4_step(float(dt))
            UN = forest.read_fields().astype(np.float64)
            forest.write_fields(u0)
            forest.set_time(t0)
            ctx.forest, ctx.u0 = forest, u0
            ctx.args = (int(nsteps), float(dt), ckpt_every, snapshots)
            ctx.devices = (U0.device, theta.device)
            return torch.from_numpy(UN).to(U0.device)

        @staticmethod
        def backward(ctx, gUN):
            nsteps, dt, ckpt_every, snapshots = ctx.args
            ctx.forest.write_fields(ctx.u0)
            gU0, gth = ctx.forest.adjoint_vjp(nsteps, dt, gUN.detach().cpu().numpy(), ckpt_every, snapshots)
            gtheta = torch.tensor(list(gth[:4]) + [0.0], dtype=torch.float64, device=ctx.devices[1])
            return None, torch.from_numpy(gU0).to(ctx.devices[0]), gtheta, None, None, None, None

    return StepMap


CKPT_OPS = ("store", "restore", "advance", "turn")


def checkpoint_policy(ckpt_every=10, snapshots=None):
    """The library's checkpointing argument: ckpt_every > 0, or -snapshots for binomial."""
    if snapshots is not None:
        if int(snapshots) < 1:
            raise ValueError("binomial checkpointing needs at least one snapshot")
        return -int(snapshots)
    if int(ckpt_every) < 1:
        raise ValueError("ckpt_every must be positive")
    return int(ckpt_every)


def checkpoint_schedule(nsteps, ckpt_every=10, snapshots=None):
    """The adjoint's checkpoint schedule as the library runs it (host only): a dict with the
    snapshots used, the recomputed (plain forward) steps and the actions, a list of (op, arg)
    with op in CKPT_OPS."""
    L = lib()
    policy = checkpoint_policy(ckpt_every, snapshots)
    ns, adv, na = C.c_int32(), C.c_int64(), C.c_int64()
    st = L.acm_checkpoint_schedule(int(nsteps), policy, C.byref(ns), C.byref(adv), None, None, 0, C.byref(na))
    if st != 0:
        raise AcmError(f"acm_checkpoint_schedule: {L.acm_status_string(st).decode()}")
    ops = np.empty(na.value, dtype=np.int8)
    args = np.empty(na.value, dtype=np.int32)
    st = L.acm_checkpoint_schedule(int(nsteps), policy, None, None, _ptr(ops), _ptr(args), na.value, C.byref(na))
    if st != 0:
        raise AcmError(f"acm_checkpoint_schedule: {L.acm_status_string(st).decode()}")
    return dict(snapshots=ns.value, advances=adv.value,
                actions=[(CKPT_OPS[o], int(a)) for o, a in zip(ops.tolist(), args.tolist())])


def sphere_objective_function():
    """A torch.autograd.Function over a forest: forward(forest, U0, theta, nsteps, dt, ckpt_every,
    w_energy) writes U0 (block order, read_fields layout, float64) and the sphere mask theta =
    (cx, cy, cz, R, delta) into the forest and returns J; backward returns dJ/dU0 and
    dJ/d(cx, cy, cz, R) (no gradient for delta), both computed by the hand-written adjoint."""
    import torch

    class SphereObjective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, forest, U0, theta, nsteps, dt, ckpt_every=10, w_energy=0.1):
            forest.write_fields(U0.detach().cpu().numpy())
            forest.set_mask(ACM_MASK_SPHERE, [float(v) for v in theta.detach().cpu()])
            J, gth, gU = forest.adjoint_sphere(nsteps, dt, ckpt_every, w_energy)
            ctx.save_for_backward(torch.from_numpy(gU).to(U0.device),
                                  torch.tensor(list(gth) + [0.0], dtype=torch.float64, device=theta.device))
            return torch.tensor(J, dtype=torch.float64, device=U0.device)

        @staticmethod
        def backward(ctx, gJ):
            gU, gth = ctx.saved_tensors
            return None, gJ * gU, gJ * gth, None, None, None, None

    return SphereObjective
