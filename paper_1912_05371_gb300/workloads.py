"""Seeded synthetic inputs: workload parameters and random block layouts.

This module holds recipes only -- parameter values, seeded random draws and random block
layouts -- and none of the solver's arithmetic.  Both the CUDA path (through the C-ABI) and
the FP64 CPU oracle consume what it returns.

Workloads (the paper's own cases need geometries, kinematics and reference data that are not
available, so these synthetic cases stand in for them, with the sizes of its runs):

* ``taylor_green``: periodic unit cube, 4x4x4 blocks of 17^3 points (level 2), Taylor-Green
  velocity of amplitude 1, p = 0, nu = 1e-2, c0 = 10, no mask, CFL 0.5, 20 steps, FP64.
* ``sphere``: periodic box 4x2x2 (2x1x1 roots of side 2), uniform flow u = (1, 0, 0), sphere of
  radius 0.25 at (1, 1, 1) as a tanh-smoothed mask over 1.5 dx_max, C_eta = 1e-3, nu = 1e-3,
  c0 = 20, Bs = 17, levels 2..5, C_eps = 1e-3, dealiasing, sponge of width 0.25 at the box
  faces with C_sp = L_sp / (c0 tau), tau = 20, u_inf = (1, 0, 0), C_gamma = 0.
* ``random_forest``: the paper's performance method (Sec. 5.4) draws random graded grids of a
  prescribed block count; :func:`random_graded_leaves` does this with a seed.
* ``plate_fullscale``: the full-scale case -- a rigid plate (chord 1, span 3, thickness 0.05)
  flapping with stroke +-60 deg and pitch +-45 deg at frequency 1 about its root at the centre
  of the periodic box 8^3 (one root of side 8), fluid at rest, nu = 1/2000, C_eta = 1e-4,
  c0 = 30, C_eps = 1e-3, levels 2..Jmax, the mask's layer 1.5 dx at Jmax.
"""
from __future__ import annotations

import math

import numpy as np


def taylor_green():
    return dict(
        grid=dict(nroot=(1, 1, 1), root_len=1.0, Bs=17, g=4, Jmin=2, Jmax=2),
        phys=dict(nu=1e-2, c0=10.0, C_eta=1e-3, C_gamma=1.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25),
        ic=("taylor_green", dict(k=2.0 * math.pi, amp=1.0)),
        mask=None, sponge=None, J0=2, steps=20, eps=1e-3, dealias=False,
    )


def sphere(Jmax=5, Jmin=2):
    L_sp, tau, c0 = 0.25, 20.0, 20.0
    root_len, Bs = 2.0, 17
    dx_max = root_len / ((1 << Jmax) * (Bs - 1))
    return dict(
        grid=dict(nroot=(2, 1, 1), root_len=root_len, Bs=Bs, g=4, Jmin=Jmin, Jmax=Jmax),
        phys=dict(nu=1e-3, c0=c0, C_eta=1e-3, C_gamma=0.0, C_sp=L_sp / (c0 * tau),
                  u_inf=(1.0, 0.0, 0.0), p_inf=0.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25),
        ic=("uniform", dict(u0=(1.0, 0.0, 0.0), p0=0.0)),
        mask=("sphere", dict(centre=(1.0, 1.0, 1.0), R=0.25, delta=1.5 * dx_max)),
        sponge=dict(L=(4.0, 2.0, 2.0), L_sp=L_sp, delta=1.5 * dx_max),
        steps=200, eps=1e-3, dealias=True, mask_thr=1e-5,
    )


def plate_fullscale(Jmax=7, Jmin=2, Bs=17):
    root_len = 8.0
    dx_max = root_len / ((1 << Jmax) * (Bs - 1))
    return dict(
        grid=dict(nroot=(1, 1, 1), root_len=root_len, Bs=Bs, g=4, Jmin=Jmin, Jmax=Jmax),
        phys=dict(nu=1.0 / 2000.0, c0=30.0, C_eta=1e-4, C_gamma=0.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25),
        ic=("uniform", dict(u0=(0.0, 0.0, 0.0), p0=0.0)),
        # chord, span, thickness, stroke and pitch amplitudes (rad), frequency, root, layer width
        plate=dict(chord=1.0, span=3.0, thickness=0.05, phi_m=math.radians(60.0), alpha_m=math.radians(45.0),
                   freq=1.0, root=(4.0, 4.0, 4.0), delta=1.5 * dx_max),
        eps=1e-3, dealias=True, mask_thr=1e-5,
    )


def _box_key(J, g):
    return (J,) + tuple(int(v) for v in g)


def random_graded_leaves(seed, nroot=(1, 1, 1), J0=1, Jmax=3, n_target=64, p_refine=0.5):
    """Random 2:1-graded (26-neighbour) layout of leaves (J, gx, gy, gz) on a periodic forest.

    Starts from the uniform level-J0 grid and refines randomly chosen leaves (each refinement
    followed by refining every coarser neighbour until the grading holds) until at least
    ``n_target`` leaves exist or nothing below Jmax is left.  Deterministic for a seed."""
    rng = np.random.default_rng(seed)
    nr = np.array(nroot)
    leaves = set()
    nb0 = nr << J0
    for z in range(nb0[2]):
        for y in range(nb0[1]):
            for x in range(nb0[0]):
                leaves.add((J0, x, y, z))

    def wrap(J, g):
        nb = nr << J
        return tuple(int(g[a]) % int(nb[a]) for a in range(3))

    def covering_leaf(J, g):
        """Leaf whose box contains level-J box g, searching coarser levels (or None)."""
        g = wrap(J, g)
        for L in range(J, -1, -1):
            s = J - L
            k = (L, g[0] >> s, g[1] >> s, g[2] >> s)
            if k in leaves:
                return k
        return None

    def refine(leaf):
        J, gx, gy, gz = leaf
        leaves.discard(leaf)
        for c in range(8):
            leaves.add((J + 1, 2 * gx + (c & 1), 2 * gy + ((c >> 1) & 1), 2 * gz + ((c >> 2) & 1)))
        # grading: every box touching a child must be covered by a leaf of level >= J
        stack = [(J + 1, 2 * gx + (c & 1), 2 * gy + ((c >> 1) & 1), 2 * gz + ((c >> 2) & 1))
                 for c in range(8)]
        while stack:
            k = stack.pop()
            if k not in leaves:
                continue
            Jk = k[0]
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if dx == dy == dz == 0:
                            continue
                        cov = covering_leaf(Jk, (k[1] + dx, k[2] + dy, k[3] + dz))
                        if cov is not None and cov[0] < Jk - 1:
                            Jc, cx, cy, cz = cov
                            leaves.discard(cov)
                            kids = [(Jc + 1, 2 * cx + (c & 1), 2 * cy + ((c >> 1) & 1),
                                     2 * cz + ((c >> 2) & 1)) for c in range(8)]
                            leaves.update(kids)
                            stack.extend(kids)
                            stack.append(k)

    while len(leaves) < n_target:
        cand = sorted(l for l in leaves if l[0] < Jmax)
        if not cand:
            break
        pick = cand[int(rng.integers(len(cand)))]
        refine(pick)
    return sorted(leaves)


def random_pulse_ring(seed, n):
    """Per-instance random parameters: Gaussian pressure pulse (width 0.05-0.2, amplitude
    0.01-1, centre in the unit cube) and vortex ring (radius 0.1-0.3, circulation 0.5-2,
    random axis), drawn from one seed."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        out.append(dict(width=float(rng.uniform(0.05, 0.2)), amp=float(rng.uniform(0.01, 1.0)),
                        centre=tuple(float(v) for v in rng.uniform(0, 1, 3)),
                        ring_radius=float(rng.uniform(0.1, 0.3)),
                        circulation=float(rng.uniform(0.5, 2.0)), axis=tuple(float(v) for v in ax)))
    return out


def smooth_periodic_field(seed, L, nmodes=3, kmax=2):
    """Coefficients of a random smooth periodic field: per component, a few Fourier modes
    (integer wave vectors up to kmax per axis, random amplitude and phase) on the box L."""
    rng = np.random.default_rng(seed)
    comps = []
    for _ in range(4):
        modes = []
        for _ in range(nmodes):
            k = tuple(int(v) for v in rng.integers(-kmax, kmax + 1, 3))
            modes.append((k, float(rng.uniform(0.2, 1.0)), float(rng.uniform(0, 2 * math.pi))))
        comps.append(modes)
    return dict(L=tuple(float(v) for v in L), comps=comps)


def cubic_coefficients(seed):
    """Random coefficients c[f][a][b][c] (a, b, c <= 3) of a polynomial of degree <= 3 in each
    coordinate, per component (tensor-product cubic)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(4, 4, 4, 4))


def batched_instances(seed=0, n=64, nb_range=(8, 512), Jmax=5):
    """Independent instances of the batched workload, all drawn from one seed: each a periodic
    unit cube with a random 2:1-graded layout of about N_b ~ U{8..512} blocks (from level 2, or
    level 1 when N_b < 64, up to Jmax), a Gaussian pressure pulse (width U[0.05, 0.2], amplitude
    U[0.01, 1], centre uniform) and a vortex ring (radius U[0.1, 0.3], circulation parameter
    U[0.5, 2], centre uniform, axis uniform on the sphere, core width a quarter of the radius).
    Returns a list of dicts with leaves and the 17 ACM_IC_PULSE_RING parameters."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nb = int(rng.integers(nb_range[0], nb_range[1] + 1))
        J0 = 2 if nb >= 64 else 1
        leaves = random_graded_leaves(int(rng.integers(0, 2 ** 31)), nroot=(1, 1, 1), J0=J0, Jmax=Jmax, n_target=nb)
        pc = rng.uniform(0.0, 1.0, 3)
        width = rng.uniform(0.05, 0.2)
        amp = rng.uniform(0.01, 1.0)
        rc = rng.uniform(0.0, 1.0, 3)
        ax = rng.normal(size=3)
        ax = ax / np.linalg.norm(ax)
        R = rng.uniform(0.1, 0.3)
        gamma = rng.uniform(0.5, 2.0)
        params = [*pc, width, amp, 1.0, 1.0, 1.0, *rc, *ax, R, gamma, 0.25 * R]
        out.append(dict(leaves=leaves, ic=[float(v) for v in params], J0=J0,
                        pulse=(tuple(pc), width, amp), ring=(tuple(rc), tuple(ax), R, gamma, 0.25 * R)))
    return out
