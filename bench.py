"""Benchmark of the wavelet-adaptive ACM hot path on GB300.

One step = the paper's time step (Sec. 3.5) through the C-ABI: refine every block by one
level, one RK4 step (4 x [ghost sync + fused RHS + RK combination]), wavelet-detail
thresholding and coarsening.  Workload: the penalised sphere case (periodic box 4x2x2, sphere
R = 0.25, C_eta = 1e-3, nu = 1e-3, c0 = 20, Bs = 17, levels 2..5, C_eps = 1e-3, dealiasing,
sponge), FP32 fields, synthetic (analytic) initial data.

value = point-updates/s = sum over timed steps of N_b(evolved) * Bs^3 * 4 RHS evaluations,
divided by the device time of the timed steps (CUDA events on the forest's stream), whole job.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK4 point-updates/s (adaptive grid)"
UNIT = "point-updates/s"


def sphere_setup(Jmax=5, precision=32, max_blocks=40000):
    from paper_1912_05371_gb300 import workloads as W
    cfg = W.sphere(Jmax=Jmax)
    g, p = cfg["grid"], cfg["phys"]
    grid = dict(g, precision=precision, max_blocks=max_blocks, fd_scheme=1)
    sp = cfg["sponge"]
    phys = dict(p, eps=cfg["eps"], dealias=int(cfg["dealias"]), mask_range_thr=cfg["mask_thr"], sponge=1,
                sponge_L=sp["L"], sponge_width=sp["L_sp"], sponge_delta=sp["delta"])
    m = cfg["mask"][1]
    mask = (*m["centre"], m["R"], m["delta"])
    ic = [*cfg["ic"][1]["u0"], cfg["ic"][1]["p0"]]
    return grid, phys, mask, ic, cfg


def workload_name(grid):
    return (f"sphere: periodic box 4x2x2, R=0.25 tanh mask, C_eta=1e-3, nu=1e-3, c0=20, sponge, "
            f"Bs={grid['Bs']}, levels {grid['Jmin']}..{grid['Jmax']}, C_eps=1e-3, dealiasing, "
            f"refine-RK4-coarsen per step")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic():
    """dram bytes per launch of the stage kernel from the committed ncu summary, or None if the
    kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "stage_kernel_traffic.txt")
    src = os.path.join(ROOT, "paper_1912_05371_gb300", "csrc", "stage.cu")
    try:
        kv = {}
        for line in open(p):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if kv.get("stage_cu_sha256_16") != h:
            return None, None
        return float(kv["dram_bytes_per_point_per_launch"]), kv.get("capture", "")
    except (OSError, KeyError, ValueError):
        return None, None


def oracle_rhs_sample(leaves, U_blocks, grid, phys, mask):
    """Time the FP64 oracle's right-hand side (ghost sync + RHS of every block) on the given
    grid and state.  Returns (point-updates/s, seconds, blocks)."""
    import numpy as np

    from oracle import acm as oacm
    from oracle.adapt import Solver
    from oracle.forest import Forest as OForest
    fo = OForest(nroot=grid["nroot"], root_len=grid["root_len"], Bs=grid["Bs"], Jmin=grid["Jmin"],
                 Jmax=grid["Jmax"], max_blocks=len(leaves) + 8)
    fo.set_leaves(leaves)
    ph = oacm.Physics(nu=phys["nu"], c0=phys["c0"], C_eta=phys["C_eta"], C_gamma=phys["C_gamma"],
                      C_sp=phys["C_sp"], u_inf=phys["u_inf"], p_inf=phys["p_inf"])
    cx, cy, cz, R, d = mask
    S = Solver(fo, ph, mask=lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, (cx, cy, cz), R, d),
               sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, phys["sponge_L"], phys["sponge_width"],
                                                       phys["sponge_delta"]))
    for i, l in enumerate(fo.sorted_leaves()):
        S.U[fo.leaves[l]] = np.asarray(U_blocks[i], dtype=np.float64)
    S.eval_mask()
    t0 = time.perf_counter()
    S.rhs(S.U)
    dt = time.perf_counter() - t0
    n = len(leaves)
    return n * grid["Bs"] ** 3 / dt, dt, n


def _oracle_worker(path, grid, phys, mask, steps, warmup, barrier):
    """One host process of the all-core oracle timing: builds the oracle solver on the sample
    saved at `path`, waits for every worker, then times `steps` RHS evaluations."""
    import numpy as np

    from oracle import acm as oacm
    from oracle.adapt import Solver
    from oracle.forest import Forest as OForest
    d = np.load(path, allow_pickle=False)
    leaves = [tuple(int(v) for v in r) for r in d["leaves"]]
    fo = OForest(nroot=grid["nroot"], root_len=grid["root_len"], Bs=grid["Bs"], Jmin=grid["Jmin"],
                 Jmax=grid["Jmax"], max_blocks=len(leaves) + 8)
    fo.set_leaves(leaves)
    ph = oacm.Physics(nu=phys["nu"], c0=phys["c0"], C_eta=phys["C_eta"], C_gamma=phys["C_gamma"],
                      C_sp=phys["C_sp"], u_inf=phys["u_inf"], p_inf=phys["p_inf"])
    cx, cy, cz, R, dl = mask
    S = Solver(fo, ph, mask=lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, (cx, cy, cz), R, dl),
               sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, phys["sponge_L"], phys["sponge_width"],
                                                       phys["sponge_delta"]))
    for i, l in enumerate(fo.sorted_leaves()):
        S.U[fo.leaves[l]] = d["U"][i]
    S.eval_mask()
    for _ in range(warmup):
        S.rhs(S.U)
    barrier.wait()
    t0 = time.perf_counter()
    for _ in range(steps):
        S.rhs(S.U)
    return time.perf_counter() - t0


def oracle_all_cores(leaves, U_blocks, grid, phys, mask, cores, steps=1, warmup=0):
    """The oracle as it stands on `cores` host processes at once, each evaluating the RHS of its
    own copy of the sample (processes started with spawn, after the GPU work; they never touch
    the GPU).  Returns (point-updates/s of all processes together, seconds of the slowest)."""
    import multiprocessing as mp
    import tempfile

    import numpy as np
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "sample.npz")
        np.savez(path, leaves=np.asarray(leaves, dtype=np.int64), U=np.asarray(U_blocks, dtype=np.float64))
        with ctx.Manager() as mgr:
            bar = mgr.Barrier(cores)
            with ctx.Pool(cores) as pool:
                secs = pool.starmap(_oracle_worker, [(path, grid, phys, mask, steps, warmup, bar)] * cores)
    n = len(leaves)
    slowest = max(secs)
    return cores * steps * n * grid["Bs"] ** 3 / slowest, slowest


def adaptive_run(A, stream, precision, Jmax, max_blocks, nsteps=200):
    """Config 2 as stated: the sphere workload from its initial grid through 200 adaptive steps
    (refine, RK4 at the CFL time step, coarsen), the block count after every step (N_b(t)), the
    share of the step time spent refining, evolving and coarsening (events between the three
    calls, as the paper splits its step, Sec. 5.4), and the clocks sampled during the run."""
    import torch
    grid, phys, mask, ic, _ = sphere_setup(Jmax=Jmax, precision=precision, max_blocks=max_blocks)
    f = A.Forest(grid, phys, stream=stream)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    n0 = f.init_grid(A.ACM_IC_UNIFORM, ic)
    Bs3 = grid["Bs"] ** 3
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * nsteps + 1)]
    nev, nst, t = [], [], 0.0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(nsteps):
        f.refine_all()
        ev[3 * k + 1].record(stream)
        nev.append(f.n_blocks())
        t += f.rk4_step(0.0)
        ev[3 * k + 2].record(stream)
        n_after, _ = f.coarsen()
        nst.append(n_after)
        ev[3 * k + 3].record(stream)
    ev[-1].synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[-1])
    phase = [sum(ev[3 * k + q].elapsed_time(ev[3 * k + q + 1]) for k in range(nsteps)) for q in range(3)]
    f.close()
    tot = sum(phase)
    pu = 4 * Bs3 * sum(nev)
    return {"workload": "the sphere workload from its initial grid, 200 adaptive steps at the CFL time step",
            "precision": f"fp{precision}", "steps": nsteps, "t_end": t, "ms_per_step": ms / nsteps,
            "value": pu / (ms * 1e-3), "unit": UNIT, "blocks_initial": n0,
            "n_blocks": {"evolved": nev, "after_coarsening": nst},
            "phase_fractions": {"refine": phase[0] / tot, "evolve": phase[1] / tot, "coarsen": phase[2] / tot},
            "clocks": clk}


def fp64_measurement(A, stream, Jmax, max_blocks, nsteps=20, warmup=3):
    """The sphere workload with FP64 fields (config 2 asks for both precisions): whole steps
    timed by CUDA events as in the main line, the stage kernel's launch time, and its roofline
    against both bounds -- HBM (136 B per point-update) and the FP64 pipe (224 flops per
    point-update, counted from the kernel: 12 first derivatives at 8, 3 Laplacians at 20, the
    right-hand side 52, the RK combination 16 -- over the FMA rate of this GPU measured by the
    library's own kernel)."""
    import numpy as np
    import torch
    grid, phys, mask, ic, _ = sphere_setup(Jmax=Jmax, precision=64, max_blocks=max_blocks)
    f = A.Forest(grid, phys, stream=stream)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.init_grid(A.ACM_IC_UNIFORM, ic)
    for _ in range(warmup):
        f.step(0.0)
    Bs3 = grid["Bs"] ** 3
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f.enable_timing(True)
    pu, nev, st_ms, st_b = 0, [], 0.0, 0.0
    e0.record(stream)
    for _ in range(nsteps):
        f.refine_all()
        n_ev = f.n_blocks()
        f.rk4_step(0.0)
        st = f.last_step_stats()
        st_ms += st["stage_ms"]
        st_b += st["stage_bytes"]
        f.coarsen()
        pu += 4 * n_ev * Bs3
        nev.append(n_ev)
    e1.record(stream)
    e1.synchronize()
    f.enable_timing(False)
    ms = e0.elapsed_time(e1)
    f.close()
    fma64 = A.fma_rate(64, stream)
    fma32 = A.fma_rate(32, stream)
    peak, kind = measured_peaks()
    pts_per_launch = float(np.mean(nev)) * Bs3
    launch_s = st_ms * 1e-3 / (4 * nsteps)
    flops = 224.0 * pts_per_launch / launch_s
    gbs = st_b / (st_ms * 1e-3) / 1e9
    return {"workload": "the sphere workload above with FP64 fields", "precision": "fp64", "steps": nsteps,
            "ms_per_step": ms / nsteps, "value": pu / (ms * 1e-3), "unit": UNIT,
            "blocks_evolved_mean": float(np.mean(nev)),
            "stage_ms_per_launch": launch_s * 1e3,
            "fma_rate_tflops": {"fp64": fma64 / 1e12, "fp32": fma32 / 1e12,
                                "how": "acm_fma_rate: 8 independent FMA chains per thread, 8 CTAs of 256 "
                                       "threads per SM, median of 5 launches"},
            "roofline": {"alu": {"bound": "alu", "achieved": flops / 1e12, "peak": fma64 / 1e12,
                                 "unit": "TFLOP/s", "frac": flops / fma64,
                                 "flops_per_point_update": 224},
                         "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                                 "bytes_per_point_update": 136, "peak_kind": kind}},
            "ceilings_point_updates_per_s": {"fp64_pipe": fma64 / 224.0, "hbm": peak * 1e9 / 136.0}}


def graph_comparison(A, stream, precision, nsteps=200):
    """RK4 steps on config 1's grid (periodic unit cube, 4x4x4 blocks of 17^3, Taylor-Green,
    nu = 1e-2, c0 = 10, CFL 0.5), three ways: one C-ABI call per step with the time step on the
    host (a stream synchronisation per step), the same steps with the time step on the device
    (plain launches, no synchronisation), and replayed from one captured CUDA graph."""
    import torch
    grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=17, g=4, Jmin=2, Jmax=2, precision=precision, max_blocks=64,
                fd_scheme=1)
    phys = dict(nu=1e-2, c0=10.0, C_gamma=1.0, cfl=0.5)
    out = {}
    for mode in ("host_dt_calls", "device_dt", "graph"):
        f = A.Forest(grid, phys, stream=stream)
        f.init_uniform(2)
        f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])

        def run(n):
            if mode == "host_dt_calls":
                for _ in range(n):
                    f.rk4_step(0.0)
            else:
                f.rk4_steps(n, 0.0, graph=(mode == "graph"))
        run(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run(nsteps)
        e1.record(stream)
        e1.synchronize()
        out[mode] = e0.elapsed_time(e1) / nsteps
        f.close()
    pts = 64 * 17 ** 3 * 4
    return {"workload": "Taylor-Green, periodic unit cube, 4x4x4 blocks of 17^3 (config 1 grid)",
            "precision": f"fp{precision}", "steps": nsteps,
            "ms_per_step": {k: round(v, 5) for k, v in out.items()},
            "point_updates_per_s": {k: pts / (v * 1e-3) for k, v in out.items()},
            "graph_speedup_vs_host_dt_calls": out["host_dt_calls"] / out["graph"]}


def uniform_roofline(A, stream, precision, J=5, nsteps=5):
    """The fused stage kernel on a uniform periodic grid (unit cube at level J: 8^J blocks of
    17^3, Taylor-Green, the config-1 physics): its CUDA-event time per launch over nsteps RK4
    steps and the algorithmic bandwidth (64 words per point and RK4 step without a mask)."""
    import torch
    nb = 8 ** J
    grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=17, g=4, Jmin=J, Jmax=J, precision=precision, max_blocks=nb,
                fd_scheme=1)
    phys = dict(nu=1e-2, c0=10.0, C_gamma=1.0, cfl=0.5)
    f = A.Forest(grid, phys, stream=stream)
    f.init_uniform(J)
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    for _ in range(2):
        f.rk4_step(1e-5)
    f.enable_timing(True)
    ms = byt = 0.0
    for _ in range(nsteps):
        f.rk4_step(1e-5)
        st = f.last_step_stats()
        ms += st["stage_ms"]
        byt += st["stage_bytes"]
    f.enable_timing(False)
    f.close()
    torch.cuda.synchronize()
    peak, kind = measured_peaks()
    gbs = byt / (ms * 1e-3) / 1e9
    return {"workload": f"Taylor-Green, periodic unit cube, uniform level {J}: {nb} blocks of 17^3",
            "precision": f"fp{precision}", "stage_ms_per_launch": ms / (4 * nsteps), "achieved_gbs": gbs,
            "frac": gbs / peak, "peak_kind": kind}


def wavelet_comparison(A, stream, precision, Jmax, max_blocks, nsteps=10, warmup=3):
    """The sphere workload with the CDF 4/4 wavelet (Sec. 3.2.1: merged parents take the lifted
    low-pass): whole steps (refine, RK4, coarsen) timed by CUDA events, as in the main line."""
    import numpy as np
    import torch
    grid, phys, mask, ic, _ = sphere_setup(Jmax=Jmax, precision=precision, max_blocks=max_blocks)
    grid = dict(grid, wavelet=44)
    f = A.Forest(grid, phys, stream=stream)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.init_grid(A.ACM_IC_UNIFORM, ic)
    for _ in range(warmup):
        f.step(0.0)
    Bs3 = grid["Bs"] ** 3
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pu, nev = 0, []
    e0.record(stream)
    for _ in range(nsteps):
        f.refine_all()
        n_ev = f.n_blocks()
        f.rk4_step(0.0)
        f.coarsen()
        pu += 4 * n_ev * Bs3
        nev.append(n_ev)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    nb = f.n_blocks()
    f.close()
    return {"workload": "the sphere workload above with the CDF 4/4 wavelet", "precision": f"fp{precision}",
            "steps": nsteps, "ms_per_step": ms / nsteps, "value": pu / (ms * 1e-3), "unit": UNIT,
            "blocks_evolved_mean": float(np.mean(nev)), "blocks_after_coarsening": nb}


def adjoint_measurement(A, stream, nsteps=100, ckpt_every=10, w_energy=0.1, binomial_snapshots=4):
    """The adjoint workload: the sphere case at levels 2..4, FP32 fields and adjoint, on its
    initial grid (frozen), nsteps RK4 steps of one fixed dt; CUDA-event time of the forward steps
    alone and of the whole adjoint call (forward with checkpoints every ckpt_every steps,
    recomputation, backward sweep), then of the same call with binomial checkpointing in
    binomial_snapshots stored states."""
    import numpy as np
    import torch
    grid, phys, mask, ic, _ = sphere_setup(Jmax=4, precision=32, max_blocks=2048)
    f = A.Forest(grid, phys, stream=stream)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.init_grid(A.ACM_IC_UNIFORM, ic)
    dt = f.rk4_step(0.0)
    U0 = f.read_fields().copy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nsteps):
        f.rk4_step(dt)
    e1.record(stream)
    e1.synchronize()
    fwd = e0.elapsed_time(e1)
    f.write_fields(U0)
    torch.cuda.synchronize()
    e0.record(stream)
    J, gth, _ = f.adjoint_sphere(nsteps, dt, ckpt_every, w_energy)
    e1.record(stream)
    e1.synchronize()
    adj = e0.elapsed_time(e1)
    # the same gradient with binomial checkpointing in 4 snapshots: less memory, more recomputation
    e0.record(stream)
    J4, gth4, _ = f.adjoint_sphere(nsteps, dt, w_energy=w_energy, snapshots=binomial_snapshots)
    e1.record(stream)
    e1.synchronize()
    adj4 = e0.elapsed_time(e1)
    nb = f.n_blocks()
    f.close()
    eq = A.checkpoint_schedule(nsteps, ckpt_every=ckpt_every)
    bi = A.checkpoint_schedule(nsteps, snapshots=binomial_snapshots)
    return {"workload": f"sphere, levels 2..4, frozen grid of {nb} blocks of 17^3, FP32 forward and adjoint, "
                        f"{nsteps} steps, checkpoints every {ckpt_every}", "forward_ms_per_step": fwd / nsteps,
            "adjoint_ms_per_step": adj / nsteps, "adjoint_over_forward": adj / fwd, "J": J,
            "dJ_dtheta": [float(v) for v in gth], "snapshots": eq["snapshots"],
            "recomputed_steps": eq["advances"],
            "binomial": {"snapshots": bi["snapshots"], "recomputed_steps": bi["advances"],
                         "adjoint_ms_per_step": adj4 / nsteps, "adjoint_over_forward": adj4 / fwd,
                         "rel_diff_J": abs(J4 - J) / abs(J),
                         "rel_diff_dJ_dtheta": float(np.abs(gth4 - gth).max() / np.abs(gth).max())}}


def adjoint_at_scale(A, stream, nsteps=10, ckpt_every=5, w_energy=0.1):
    """The adjoint on the main line's grid: the sphere workload refined to its evolved grid
    (levels 2..5, 4608 blocks of 17^3), frozen, FP32; forward and adjoint time per step as in the
    adjoint workload (which has 184 blocks, too few to fill the GPU)."""
    import torch
    grid, phys, mask, ic, _ = sphere_setup(Jmax=5, precision=32, max_blocks=6000)
    f = A.Forest(grid, phys, stream=stream)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.init_grid(A.ACM_IC_UNIFORM, ic)
    f.step(0.0)
    f.refine_all()
    dt = f.rk4_step(0.0)
    U0 = f.read_fields().copy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(nsteps):
        f.rk4_step(dt)
    e1.record(stream)
    e1.synchronize()
    fwd = e0.elapsed_time(e1)
    f.write_fields(U0)
    torch.cuda.synchronize()
    e0.record(stream)
    J, gth, _ = f.adjoint_sphere(nsteps, dt, ckpt_every, w_energy)
    e1.record(stream)
    e1.synchronize()
    adj = e0.elapsed_time(e1)
    nb = f.n_blocks()
    f.close()
    return {"workload": f"sphere, the evolved grid of {nb} blocks of 17^3 (levels 2..5), frozen, FP32, {nsteps} "
                        f"steps, checkpoints every {ckpt_every}", "forward_ms_per_step": fwd / nsteps,
            "adjoint_ms_per_step": adj / nsteps, "adjoint_over_forward": adj / fwd, "J": J,
            "dJ_dtheta": [float(v) for v in gth]}


def fullscale_plate(A, stream, Bs=33, Jmax=7, max_blocks=29000, nsteps=20, adj_Bs=33, adj_Jmax=7, adj_steps=10,
                    adj_ckpt=5):
    """The full-scale case: the flapping plate (chord 1, span 3, thickness 0.05; stroke +-60 deg,
    pitch +-45 deg, frequency 1) in the periodic box 8^3, fluid at rest, nu = 1/2000, C_eta = 1e-4,
    c0 = 30, C_eps = 1e-3, blocks of Bs^3 at levels 2..Jmax, FP32 (the pool sized at max_blocks, at
    Bs = 33 the most that 32-bit element offsets address): its initial grid by the paper's
    procedure, then nsteps adaptive steps (refine, RK4 at the CFL time step with the mask and solid
    velocity at every stage time, coarsen) timed by CUDA events, with the block count after every
    step and the device memory the forest holds.  Then the adjoint workload of this case -- the
    gradient of J = (1/N) sum [F_x + 0.1 E] with respect to the pitch amplitude on the frozen
    initial grid of the case at levels 2..adj_Jmax with blocks of adj_Bs^3 (a forest of its own,
    made after the adaptive run's pool is freed) -- forward and adjoint time per step."""
    import numpy as np
    import torch
    from paper_1912_05371_gb300 import workloads as W

    def make(J, mb, bs, leaves=None):
        """The case's forest: its initial grid by the paper's procedure, or the given leaves
        with the fluid at rest."""
        cfg = W.plate_fullscale(Jmax=J, Bs=bs)
        pl = cfg["plate"]
        grid = dict(cfg["grid"], precision=32, max_blocks=mb, fd_scheme=1)
        phys = dict(cfg["phys"], eps=cfg["eps"], dealias=1, mask_range_thr=cfg["mask_thr"])
        f = A.Forest(grid, phys, stream=stream)
        params = [pl["chord"], pl["span"], pl["thickness"], pl["phi_m"], pl["alpha_m"], pl["freq"], *pl["root"],
                  pl["delta"]]
        f.set_mask(A.ACM_MASK_PLATE, params)
        if leaves is None:
            n0 = f.init_grid(A.ACM_IC_UNIFORM, [0.0, 0.0, 0.0, 0.0])
        else:
            f.set_leaves(leaves)
            f.set_ic(A.ACM_IC_UNIFORM, [0.0, 0.0, 0.0, 0.0])
            f.set_mask(A.ACM_MASK_PLATE, params)
            n0 = len(leaves)
        return f, n0, grid

    def leaves_of(f):
        t = f.topology()
        return list(zip(t["level"].tolist(), t["gx"].tolist(), t["gy"].tolist(), t["gz"].tolist()))

    f, n0, grid = make(Jmax, max_blocks, Bs)
    leaves0 = leaves_of(f)
    # the launch knobs timed on this case's refined grid, then that step finished (untimed)
    f.refine_all()
    f.autotune()
    tuning = f.tuning()
    t = f.rk4_step(0.0)
    f.coarsen()
    Bs3 = Bs ** 3
    gb = f.pool.numel() / 1e9
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps + 1)]
    nev, nst = [], []
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(nsteps):
        f.refine_all()
        nev.append(f.n_blocks())
        t += f.rk4_step(0.0)
        n_after, _ = f.coarsen()
        nst.append(n_after)
        ev[k + 1].record(stream)
    ev[-1].synchronize()
    ms = ev[0].elapsed_time(ev[-1])
    # one more step with the library's own event timing: the stage kernel on this grid
    f.enable_timing(True)
    f.refine_all()
    f.rk4_step(0.0)
    f.coarsen()
    st = f.last_step_stats()
    f.enable_timing(False)
    peak, peak_kind = measured_peaks()
    stage_gbs = st["stage_bytes"] / (st["stage_ms"] * 1e-3) / 1e9 if st["stage_ms"] > 0 else None
    f.close()
    del f
    torch.cuda.empty_cache()
    out = {"workload": f"flapping plate in the box 8^3, Bs = {Bs}, levels 2..{Jmax}, FP32, {nsteps} adaptive steps",
           # the events around each stage also hold the plate's solid-velocity source kernel
           "autotune": {"stage_variant": tuning["stage_variant"], "stage_ms": tuning["stage_ms"]},
           "stage_kernel": {"ms_per_launch_with_solid_source": st["stage_ms"] / 4,
                            "achieved_gbs": stage_gbs, "frac": stage_gbs / peak if stage_gbs else None,
                            "peak_kind": peak_kind, "bytes_per_launch": st["stage_bytes"] / 4},
           "blocks_initial": n0, "n_blocks": {"evolved": nev, "after_coarsening": nst},
           "points_evolved_max": max(nev) * Bs3, "pool_gb": gb, "t_end": t, "ms_per_step": ms / nsteps,
           "value": 4 * Bs3 * sum(nev) / (ms * 1e-3), "unit": UNIT,
           "note": f"pool sized for {max_blocks} blocks; 32-bit element offsets bound a register at 2^32 "
                   "elements (29,700 blocks of 33^3, 206,000 of 17^3)"}
    # adjoint of the pitch amplitude on a frozen initial grid, in a forest sized for it (the
    # adjoint's workspace is some twelve registers of the pool's size)
    Bs3 = adj_Bs ** 3
    if (adj_Jmax, adj_Bs) == (Jmax, Bs):
        leaves_a = leaves0
    else:
        g0, _, _ = make(adj_Jmax, max_blocks, adj_Bs)
        leaves_a = leaves_of(g0)
        g0.close()
        del g0
        torch.cuda.empty_cache()
    f, n0a, _ = make(adj_Jmax, len(leaves_a) + 64, adj_Bs, leaves=leaves_a)
    dt = f.rk4_step(0.0)
    f.set_time(0.0)
    U0 = f.read_fields().copy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(adj_steps):
        f.rk4_step(dt)
    e1.record(stream)
    e1.synchronize()
    fwd = e0.elapsed_time(e1)
    f.write_fields(U0)
    f.set_time(0.0)
    torch.cuda.synchronize()
    e0.record(stream)
    J, dJ, _ = f.adjoint_plate_pitch(adj_steps, dt, ckpt_every=adj_ckpt, w_energy=0.1)
    e1.record(stream)
    e1.synchronize()
    adj = e0.elapsed_time(e1)
    f.close()
    out["adjoint"] = {"workload": f"the plate case at levels 2..{adj_Jmax}: {n0a} blocks of {adj_Bs}^3 frozen, FP32, "
                                 f"{adj_steps} steps of dt = {dt:.3e}, checkpoints every {adj_ckpt}",
                      "forward_ms_per_step": fwd / adj_steps, "adjoint_ms_per_step": adj / adj_steps,
                      "adjoint_over_forward": adj / fwd, "J": J, "dJ_dalpha_m": float(dJ),
                      "point_updates_per_s_adjoint": 4 * Bs3 * n0a * adj_steps / (adj * 1e-3)}
    return out


def batched_comparison(A, precision, seed=0, n=64, nsteps=10):
    """The batched workload: n independent instances (periodic unit cubes, N_b ~ U{8..512} blocks
    of 17^3 on random graded layouts over levels 2..5, pulse + vortex ring, seeded), nsteps RK4
    steps each, four ways: one C-ABI call per instance and step (time step on the host), all
    instances' steps as plain launches on their own streams (time step on the device), one CUDA
    graph per step holding every instance as a parallel branch, and the persistent form (per RK
    stage the instances' synchronisation as parallel branches and one stage launch whose CTAs walk
    the blocks of all instances, in one graph per step)."""
    import torch
    from paper_1912_05371_gb300 import workloads as W
    insts = W.batched_instances(seed=seed, n=n)
    phys = dict(nu=1e-3, c0=10.0, C_gamma=0.0, cfl=0.5)
    streams = [torch.cuda.Stream() for _ in insts]
    forests = []
    for inst, s in zip(insts, streams):
        grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=17, g=4, Jmin=1, Jmax=5, precision=precision,
                    max_blocks=len(inst["leaves"]) + 8, fd_scheme=1)
        f = A.Forest(grid, phys, stream=s)
        f.set_leaves(inst["leaves"])
        f.set_ic(A.ACM_IC_PULSE_RING, inst["ic"])
        forests.append(f)
    nb = sum(len(i["leaves"]) for i in insts)
    pts = nb * 17 ** 3 * 4 * nsteps
    out = {}
    for mode in ("per_instance_calls", "streams", "graph", "persistent"):
        def run(k):
            if mode == "per_instance_calls":
                for _ in range(k):
                    for f in forests:
                        f.rk4_step(0.0)
            else:
                A.rk4_steps_batch(forests, k, 0.0, graph={"streams": 0, "graph": 1, "persistent": 2}[mode])
        run(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(nsteps)
        torch.cuda.synchronize()
        out[mode] = time.perf_counter() - t0
    for f in forests:
        f.close()
    return {"workload": f"{n} independent instances, {nb} blocks of 17^3 in all (N_b ~ U{{8..512}}, levels 1..5), "
                        f"pulse + vortex ring, seed {seed}", "precision": f"fp{precision}", "steps": nsteps,
            "ms_per_step": {k: round(1e3 * v / nsteps, 4) for k, v in out.items()},
            "point_updates_per_s": {k: pts / v for k, v in out.items()},
            "graph_speedup_vs_per_instance_calls": out["per_instance_calls"] / out["graph"],
            "persistent_speedup_vs_per_instance_calls": out["per_instance_calls"] / out["persistent"]}


def reduce_over_ranks(ms, point_updates, dist=None, device="cpu"):
    """Whole-job figures over the ranks of a replica run: the slowest rank's time and the sum of
    all ranks' point-updates (each rank runs its own replica: weak scaling)."""
    if dist is None:
        return float(ms), float(point_updates)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(point_updates)], dtype=torch.float64, device=device)
    dist.all_reduce(p)
    return float(t.item()), float(p.item())


def random_grid_sweep(args):
    """The paper's performance study (Sec. 5.4) on one GPU: for each N_b a random 2:1-graded grid
    of about N_b blocks of 17^3 (periodic unit cube, levels 3..Jmax), Taylor-Green data, `steps`
    refine-evolve-coarsen steps with the coarsening forced everywhere (every block the step's
    refinement made merges back, so the grid is the same at every step), FP32.  Per N_b: device
    time per step (CUDA events on the forest's stream) and per evolved point and RHS evaluation,
    the paper's unit.  Grids grow until the 32-bit element offsets (2^32 / (72 Bs^2) blocks after
    refinement) or the memory cap would be exceeded.  The fractions of the step spent refining,
    evolving and coarsening (Fig. 5D) come from events between the three calls.  Prints one JSON
    line."""
    import numpy as np
    import torch

    from paper_1912_05371_gb300 import acm as A
    from paper_1912_05371_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    Bs, steps, warm = 17, args.steps, args.warmup
    limit = (1 << 32) // (72 * Bs * Bs)
    rows = []
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    for nb in (int(v) for v in args.sweep_blocks.split(",")):
        J = 5 if nb <= 2000 else (6 if nb <= 16000 else 7)
        leaves = W.random_graded_leaves(nb, nroot=(1, 1, 1), J0=2, Jmax=J, n_target=nb)
        evolved = sum(8 if l[0] < J + 1 else 1 for l in leaves)
        grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=Bs, g=4, Jmin=2, Jmax=J + 1, precision=args.precision,
                    max_blocks=evolved + 64, fd_scheme=1)
        if grid["max_blocks"] > limit:
            break
        phys = dict(nu=1e-3, c0=10.0, C_gamma=1.0, cfl=0.5, eps=1e-3, dealias=0, coarsen_everywhere=1)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            f = A.Forest(grid, phys, stream=stream)
            if f.pool.numel() > args.sweep_max_gb * 1e9:
                f.close()
                break
            f.set_leaves(leaves)
            f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
            for _ in range(warm):
                f.step(0.0)
            # the step's three phases (refine, evolve, coarsen) between events on the stream
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps + 1)]
            torch.cuda.synchronize()
            ev[0].record(stream)
            for k in range(steps):
                f.refine_all()
                ev[3 * k + 1].record(stream)
                f.rk4_step(0.0)
                ev[3 * k + 2].record(stream)
                n_after, _ = f.coarsen()
                ev[3 * k + 3].record(stream)
            ev[-1].synchronize()
            ms = ev[0].elapsed_time(ev[-1]) / steps
            phase = [sum(ev[3 * k + q].elapsed_time(ev[3 * k + q + 1]) for k in range(steps)) for q in range(3)]
            assert n_after == len(leaves)
            gb = f.pool.numel() / 1e9
            f.close()
        del f
        torch.cuda.empty_cache()
        pts = evolved * Bs ** 3 * 4
        tot = sum(phase)
        rows.append({"n_blocks": len(leaves), "evolved_blocks": evolved, "ms_per_step": ms,
                     "ns_per_point_rhs": ms * 1e6 / pts, "point_updates_per_s": pts / (ms * 1e-3), "pool_gb": gb,
                     "fractions": {"refine": phase[0] / tot, "evolve": phase[1] / tot, "coarsen": phase[2] / tot}})
    clocks = sampler.stop()
    print(json.dumps({"metric": "device time per evolved point and RHS evaluation (random grids, Sec. 5.4)",
                      "unit": "ns", "higher_is_better": False, "n_gpus": 1, "steps": steps, "warmup": warm,
                      "dtype": "f32" if args.precision == 32 else "f64", "data": "synthetic",
                      "config": {"workload": "random 2:1-graded grids of blocks of 17^3, periodic unit cube, "
                                             "Taylor-Green, refine-evolve-coarsen with coarsening forced "
                                             "everywhere (the grid is fixed)"},
                      "sweep": rows, "clocks": clocks}))


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on all host cores at once (one spawned
    process per core, each evaluating the RHS of its own copy of the sample), on a bounded sample
    of the same workload: the sphere case built by the oracle's own initial-grid procedure with
    levels 2..3, refined once (1024 blocks), or -- when K + W evaluations of that would exceed
    about 150 s -- the initial grid itself; one step = one oracle RHS evaluation (ghost sync +
    right-hand side of every block) in every process."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import acm as oacm
    from oracle.adapt import Solver
    from oracle.forest import Forest as OForest
    grid, phys, mask, ic, cfg = sphere_setup(Jmax=3)
    fo = OForest(nroot=grid["nroot"], root_len=grid["root_len"], Bs=grid["Bs"], Jmin=grid["Jmin"],
                 Jmax=grid["Jmax"], max_blocks=1 << 14)
    ph = oacm.Physics(nu=phys["nu"], c0=phys["c0"], C_eta=phys["C_eta"], C_gamma=phys["C_gamma"],
                      C_sp=phys["C_sp"], u_inf=phys["u_inf"], p_inf=phys["p_inf"])
    cx, cy, cz, R, d = mask
    S = Solver(fo, ph, eps=phys["eps"], dealias=True, mask_thr=phys["mask_range_thr"],
               ic=lambda X, Y, Z: oacm.ic_uniform(X, Y, Z),
               mask=lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, (cx, cy, cz), R, d),
               sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, phys["sponge_L"], phys["sponge_width"],
                                                       phys["sponge_delta"]))
    S.initial_grid()
    initial = (list(fo.sorted_leaves()), [S.U[fo.leaves[l]].copy() for l in fo.sorted_leaves()])
    S.refine_all()
    refined = (list(fo.sorted_leaves()), [S.U[fo.leaves[l]].copy() for l in fo.sorted_leaves()])
    # one RHS evaluation of the refined sample on one core decides the sample size
    t0 = time.perf_counter()
    S.rhs(S.U)
    t1 = time.perf_counter() - t0
    leaves, U, kind = (refined + ("refined once",)) if (args.steps + args.warmup) * t1 <= 150.0 else \
        (initial + ("initial grid",))
    cores = args.cpu_cores or os.cpu_count() or 1
    value, slowest = oracle_all_cores(leaves, U, grid, phys, mask, cores, steps=args.steps, warmup=args.warmup)
    n = len(leaves)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * slowest / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(grid), "sample": f"levels 2..3, {kind}: {n} blocks of 17^3; one step = "
                   f"one oracle RHS evaluation (sync + RHS of every block) in each of {cores} processes"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n} blocks x 17^3, {args.steps} RHS evaluations per process, {cores} processes "
                                   f"(nproc = {os.cpu_count()}); one core alone: {n * grid['Bs'] ** 3 / t1:.4g} "
                                   f"point-updates/s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--Jmax", type=int, default=5)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-blocks", type=int, default=40000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-uniform", action="store_true")
    ap.add_argument("--no-cdf44", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint workload")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 run of the sphere workload")
    ap.add_argument("--no-run200", action="store_true", help="skip the 200-step adaptive run of the sphere workload")
    ap.add_argument("--no-fullscale", action="store_true", help="skip the full-scale plate case")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="host cores for the oracle's all-core figure (default: all, os.cpu_count())")
    ap.add_argument("--wavelet", type=int, default=40, choices=[40, 44],
                    help="wavelet of the main line: 40 = CDF 4/0 (default), 44 = CDF 4/4")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint workload (and its at-scale case) and print its JSON")
    ap.add_argument("--fullscale-only", action="store_true",
                    help="run only the full-scale plate case and print its JSON")
    ap.add_argument("--sweep", action="store_true",
                    help="run the random-grid performance study (Sec. 5.4) instead of the benchmark")
    ap.add_argument("--sweep-blocks", default="1000,2000,4000,8000,16000,24000")
    ap.add_argument("--sweep-max-gb", type=float, default=150.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        if not any(a.startswith("--steps") for a in sys.argv[1:]):
            args.steps = 15
        return random_grid_sweep(args)
    if args.fullscale_only:
        import torch
        from paper_1912_05371_gb300 import acm as A
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            out = fullscale_plate(A, stream)
        print(json.dumps({"fullscale": out}))
        return 0
    if args.adjoint_only:
        import torch
        from paper_1912_05371_gb300 import acm as A
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            out = adjoint_measurement(A, stream)
            out["at_scale"] = adjoint_at_scale(A, stream)
        print(json.dumps({"adjoint": out}))
        return 0

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1912_05371_gb300 import acm as A

    grid, phys, mask, ic, cfg = sphere_setup(Jmax=args.Jmax, precision=args.precision,
                                             max_blocks=args.max_blocks)
    grid["wavelet"] = args.wavelet
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        f = A.Forest(grid, phys, stream=stream)
        f.set_mask(A.ACM_MASK_SPHERE, mask)
        f.init_grid(A.ACM_IC_UNIFORM, ic)
        Bs3 = grid["Bs"] ** 3
        for _ in range(args.warmup):
            f.step(0.0)
        # autotune the launch knobs on the evolved (refined) grid, then finish that step
        f.refine_all()
        tuned = f.autotune()
        tuning = f.tuning()
        f.rk4_step(0.0)
        f.coarsen()
        f.enable_timing(True)

        def barrier():
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()

        clocks = ClockSampler(local)
        clocks.start()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = f.launch_count()
        h0 = f.last_step_stats()
        pu = 0
        stage_ms = 0.0
        sync_ms = 0.0
        stage_bytes = 0.0
        nev, nst = [], []
        # events between the step's three phases (refine, evolve, coarsen), as the paper splits
        # its step time (Sec. 5.4)
        pev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
        ev0.record(stream)
        for k in range(args.steps):
            f.refine_all()
            pev[3 * k].record(stream)
            n_ev = f.n_blocks()
            f.rk4_step(0.0)
            pev[3 * k + 1].record(stream)
            n_after, _ = f.coarsen()
            pev[3 * k + 2].record(stream)
            st = f.last_step_stats()
            stage_ms += st["stage_ms"]
            sync_ms += st["sync_ms"]
            stage_bytes += st["stage_bytes"]
            pu += 4 * n_ev * Bs3
            nev.append(n_ev)
            nst.append(n_after)
        ev1.record(stream)
        barrier()
        ph_ms = [0.0, 0.0, 0.0]
        prev = ev0
        for k in range(args.steps):
            for q in range(3):
                ph_ms[q] += prev.elapsed_time(pev[3 * k + q])
                prev = pev[3 * k + q]
        launches = f.launch_count() - l0
        h1 = f.last_step_stats()
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        f.enable_timing(False)
        t_max, pu_all = reduce_over_ranks(ms, pu, dist, "cuda")
        value = pu_all / (t_max * 1e-3)

        # roofline of the dominant kernel (fused RHS + RK4 stage): algorithmic bytes / event time
        peak, peak_kind = measured_peaks()
        achieved = stage_bytes / (stage_ms * 1e-3) / 1e9
        traffic_ppu, capture = profiled_traffic()
        launches_stage = 4 * args.steps
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "kernel": "k_stage<float,17> (fused RHS + RK4 stage)",
                "bytes_per_launch": stage_bytes / launches_stage,
                "avg_launch_ms": stage_ms / launches_stage,
                "traffic": (traffic_ppu * float(np.mean(nev)) * Bs3 if traffic_ppu is not None else None),
                "traffic_capture": capture,
                "stage_share_of_step": round(stage_ms / t_max, 4),
                # the fused RHS + ghost-sync path: the stage kernels' algorithmic bytes over the
                # time of the stage kernels and the per-stage synchronisation (fine wins and the
                # coarse-face slabs) together
                "path": {"achieved": round(stage_bytes / ((stage_ms + sync_ms) * 1e-3) / 1e9, 1),
                         "frac": round(stage_bytes / ((stage_ms + sync_ms) * 1e-3) / 1e9 / peak, 4),
                         "sync_ms_per_stage": sync_ms / launches_stage,
                         "stage_ms_per_stage": stage_ms / launches_stage}}
        roof["kernel"] = {0: "k_stage_pair<17> (fused RHS + RK4 stage, 2 points per thread)",
                          1: "k_stage<float,17> (fused RHS + RK4 stage)",
                          2: "k_stage<float,17,TMA> (fused RHS + RK4 stage, bulk-copy staging)"}[tuning["stage_variant"]]

        # end to end through the C-ABI with host buffers: write state, step, read state
        e2e = None
        if not args.no_e2e:
            nmax = min(grid["max_blocks"], 2 * max(nev))
            esz = 4 if args.precision == 32 else 8
            tdt = torch.float32 if args.precision == 32 else torch.float64
            host = torch.empty(nmax * 4 * Bs3, dtype=tdt).pin_memory()
            n0 = f.n_blocks()
            f.read_fields(host[: n0 * 4 * Bs3])
            barrier()
            t0 = time.perf_counter()
            pu_e, h2d, d2h = 0, 0, 0
            for _ in range(args.steps):
                nb = f.n_blocks()
                f.write_fields(host[: nb * 4 * Bs3])
                h2d += nb * 4 * Bs3 * esz
                f.refine_all()
                pu_e += 4 * f.n_blocks() * Bs3
                f.rk4_step(0.0)
                f.coarsen()
                nb = f.n_blocks()
                f.read_fields(host[: nb * 4 * Bs3])
                d2h += nb * 4 * Bs3 * esz
            barrier()
            te = time.perf_counter() - t0
            e2e = {"value": pu_e / te, "unit": UNIT, "h2d_bytes_per_step": h2d // args.steps,
                   "d2h_bytes_per_step": d2h // args.steps}

        graph = graph_comparison(A, stream, args.precision) if rank == 0 and not args.no_graph else None
        uniform = uniform_roofline(A, stream, args.precision) if rank == 0 and not args.no_uniform else None
        batched = batched_comparison(A, args.precision) if rank == 0 and not args.no_batched else None
        cdf44 = (wavelet_comparison(A, stream, args.precision, args.Jmax, args.max_blocks)
                 if rank == 0 and not args.no_cdf44 and args.wavelet == 40 else None)
        run200 = (adaptive_run(A, stream, args.precision, args.Jmax, args.max_blocks)
                  if rank == 0 and not args.no_run200 else None)
        fullscale = None
        if rank == 0 and not args.no_fullscale and args.precision == 32:
            try:
                fullscale = fullscale_plate(A, stream)
            except Exception as e:  # noqa: BLE001
                fullscale = {"error": f"{type(e).__name__}: {e}"}
        fp64 = None
        if rank == 0 and not args.no_fp64 and args.precision == 32:
            try:
                fp64 = fp64_measurement(A, stream, args.Jmax, args.max_blocks)
            except Exception as e:  # noqa: BLE001
                fp64 = {"error": f"{type(e).__name__}: {e}"}
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            # bounded sample (10-30 s of one core): the same workload with levels 2..4, its grid
            # built and refined by the library, the oracle evaluating one RHS on that state
            g4, p4, m4, ic4, _ = sphere_setup(Jmax=min(args.Jmax, 4), precision=args.precision, max_blocks=8000)
            f4 = A.Forest(g4, p4, stream=stream)
            f4.set_mask(A.ACM_MASK_SPHERE, m4)
            f4.init_grid(A.ACM_IC_UNIFORM, ic4)
            f4.refine_all()
            topo = f4.topology()
            leaves = list(zip(topo["level"].tolist(), topo["gx"].tolist(), topo["gy"].tolist(),
                              topo["gz"].tolist()))
            U = f4.read_fields().astype(np.float64)
            del f4
            v, secs, nb = oracle_rhs_sample(leaves, U, g4, p4, m4)
            cores = args.cpu_cores or os.cpu_count() or 1
            try:
                vall, sall = oracle_all_cores(leaves, U, g4, p4, m4, cores)
            except Exception as e:  # noqa: BLE001
                vall, sall = None, f"{type(e).__name__}: {e}"
            cpu = {"value": vall if vall is not None else v, "unit": UNIT,
                   "cores": cores if vall is not None else 1, "kind": "oracle",
                   "sample": f"one FP64 oracle RHS evaluation (ghost sync + RHS) over the same workload at "
                             f"levels {g4['Jmin']}..{g4['Jmax']} after refinement, {nb} blocks x 17^3, on each of "
                             f"{cores} host processes at once (value: all together; nproc = {os.cpu_count()})",
                   "all_cores_seconds": sall,
                   "single_core": {"value": v, "cores": 1, "seconds": secs}}

        # the last GPU work of the run: a side measurement whose errors are reported, not raised
        adjoint = None
        if rank == 0 and not args.no_adjoint:
            try:
                adjoint = adjoint_measurement(A, stream)
                adjoint["at_scale"] = adjoint_at_scale(A, stream)
            except Exception as e:  # noqa: BLE001
                adjoint = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(grid), "Bs": grid["Bs"], "levels": [grid["Jmin"], grid["Jmax"]],
                       "precision": f"fp{args.precision}", "wavelet": f"CDF 4/{args.wavelet % 10}",
                       "blocks_evolved_mean": float(np.mean(nev)),
                       "points_evolved_mean": float(np.mean(nev)) * Bs3,
                       "l2": f"inputs larger than L2: state {4 * float(np.mean(nev)) * Bs3 * 4 * (args.precision // 8) / 1e9:.2f} GB per RK register x 4 registers",
                       "parallelism": f"replicas x{world}"},
            "n_blocks_over_time": {"evolved": nev[::10], "after_coarsening": nst[::10], "every": 10,
                                   "evolved_min_max": [min(nev), max(nev)]},
            "phase_fractions": {"refine": ph_ms[0] / sum(ph_ms), "evolve": ph_ms[1] / sum(ph_ms),
                                "coarsen": ph_ms[2] / sum(ph_ms)},
            "step_breakdown_ms": {
                "stage_kernels": stage_ms / args.steps,
                "sync_kernels": sync_ms / args.steps,
                "host_topology": (h1["host_topology_ms"] - h0["host_topology_ms"]) / args.steps,
                "host_tree": (h1["host_tree_ms"] - h0["host_tree_ms"]) / args.steps,
                "total": t_max / args.steps},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "rk4_graph": graph,
            "batched": batched,
            "cdf44": cdf44,
            "fp64": fp64,
            "adaptive_200_steps": run200,
            "fullscale": fullscale,
            "adjoint": adjoint,
            "uniform_roofline": uniform,
            "autotune": {"fine_wins_ctas_per_sm": tuned[0], "slab_ctas_per_sm": tuned[1],
                         "stage_kernel": {0: "pair (2 points/thread, packed f32x2)",
                                          1: "point (1 point/thread)",
                                          2: "point, bulk-copy (TMA) staging of U/acc/chi",
                                          3: "point, a block's rows over two CTAs"}[tuning["stage_variant"]],
                         "stage2_ms": {"pair": tuning["stage_ms"][0], "point": tuning["stage_ms"][1],
                                       "point_tma": tuning["stage_ms"][2], "point_rows": tuning["stage_ms"][3]}},
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    try:
        f.close()
    except Exception as e:  # noqa: BLE001
        # reported, not raised: the line above is complete; a failed side measurement (listed
        # under its key) may have left the device in an error state
        print(f"bench: forest close failed after the measurements: {e}", file=sys.stderr)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
