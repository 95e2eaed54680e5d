"""Shared helpers of the GPU parity tests: the same seeded inputs for the CUDA path (through
the C-ABI) and for the FP64 oracle."""
import math

import numpy as np

from oracle import acm as oacm
from oracle.adapt import Solver
from oracle.forest import Forest as OForest


def smooth_field(X, Y, Z, L=(1.0, 1.0, 1.0), seed=0):
    """A smooth periodic 4-component field on the box L (a few low Fourier modes)."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(4):
        v = np.zeros_like(X)
        for _ in range(3):
            k = rng.integers(-2, 3, 3)
            a, ph = rng.uniform(0.2, 1.0), rng.uniform(0, 2 * math.pi)
            v = v + a * np.sin(2 * math.pi * (k[0] * X / L[0] + k[1] * Y / L[1] + k[2] * Z / L[2]) + ph)
        out.append(v)
    return np.stack(out)


def oracle_forest(grid, leaves=None, J=None, max_blocks=1 << 16):
    fo = OForest(nroot=grid["nroot"], root_len=grid["root_len"], Bs=grid["Bs"], Jmin=grid["Jmin"],
                 Jmax=grid["Jmax"], max_blocks=max_blocks)
    if leaves is not None:
        fo.set_leaves(leaves)
    elif J is not None:
        fo.init_uniform(J)
    return fo


def oracle_physics(phys):
    keys = ("nu", "c0", "C_eta", "C_gamma", "C_sp", "u_inf", "p_inf", "cfl", "cfl_eta", "cfl_nu")
    kw = {k: phys[k] for k in keys if k in phys}
    if "fd_scheme" in phys:
        kw["scheme"] = "tam_webb" if phys["fd_scheme"] == 1 else "classic"
    if not phys.get("sponge", 0):
        kw.pop("C_sp", None)
    return oacm.Physics(**kw)


def oracle_solver(fo, phys, ic=None, mask=None, sponge=None, wavelet=40):
    ph = oracle_physics(phys)
    S = Solver(fo, ph, eps=phys.get("eps", 1e-3), dealias=bool(phys.get("dealias", 0)),
               mask_thr=phys.get("mask_range_thr", 1e-5), ic=ic, mask=mask, sponge=sponge,
               wavelet={40: "cdf40", 44: "cdf44"}[wavelet],
               coarsen_everywhere=bool(phys.get("coarsen_everywhere", 0)))
    return S


def block_order_fields(S):
    fo = S.fo
    return np.stack([S.U[fo.leaves[l]] for l in fo.sorted_leaves()])


def fill_from_function(S, fn):
    for leaf, s in S.fo.leaves.items():
        S.U[s] = fn(*oacm.block_coords(S.fo, leaf))


def rel_linf(a, b):
    """Per-component max |a - b| / scale: the velocity components share the scale
    max(|u|, |v|, |w|) of the velocity field; the pressure uses max(max |p|, max |u|^2), i.e.
    at least the dynamic pressure (density 1): an ACM pressure that starts from zero is an
    O(dt) quantity whose error relative to itself is unbounded in any precision.  A zero
    scale means absolute error."""
    out = []
    four = b.shape[1] == 4
    vscale = float(np.abs(b[:, :3]).max()) if four else 0.0
    for f in range(a.shape[1]):
        if four and f < 3:
            den = vscale
        elif four:
            den = max(float(np.abs(b[:, f]).max()), vscale * vscale)
        else:
            den = float(np.abs(b[:, f]).max())
        err = float(np.abs(a[:, f] - b[:, f]).max())
        out.append(err / den if den > 0 else err)
    return out


def sponge_fn(phys):
    L, w, d = phys["sponge_L"], phys["sponge_width"], phys["sponge_delta"]
    return lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, L, w, d)


def sphere_fn(params):
    cx, cy, cz, R, delta = params
    return lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, (cx, cy, cz), R, delta)


def uniform_neighbourhood(get, nb, gx, gy, gz, M, r):
    """The level-J lattice values around block (gx, gy, gz) of a uniform periodic grid of nb
    blocks per axis, r <= M points beyond each face: (4, M + 1 + 2r, ...)^3, indexed (f, z, y,
    x); get(gx, gy, gz) gives a block's (4, M + 1, M + 1, M + 1) values."""
    big = np.empty((4,) + (3 * M + 1,) * 3)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                b = get((gx + dx) % nb[0], (gy + dy) % nb[1], (gz + dz) % nb[2])
                z0, y0, x0 = (dz + 1) * M, (dy + 1) * M, (dx + 1) * M
                big[:, z0:z0 + M + 1, y0:y0 + M + 1, x0:x0 + M + 1] = b
    return big[:, M - r:2 * M + r + 1, M - r:2 * M + r + 1, M - r:2 * M + r + 1]


def rk4_on_neighbourhood(E, M, h, ph, dt):
    """One classical RK4 step (Sec. 2.3) of one block of a uniform periodic grid without mask or
    sponge, from its state E widened by 12 points per side (four stages times the 3-point reach
    of the stencils): the stages' right-hand sides are the oracle's block right-hand side over
    the block widened by 9, 6, 3 and 0 points.  On such a grid every ghost value of the oracle
    solver's step is a neighbour's value, so this is that step on the block."""
    g = 3

    def U(r):
        o = 12 - r
        n = M + 1 + 2 * r
        return E[:, o:o + n, o:o + n, o:o + n]

    def inner(K, r):
        return K[:, r:K.shape[1] - r, r:K.shape[2] - r, r:K.shape[3] - r]

    K1 = oacm.rhs_block(E, g, M + 18, h, ph)
    K2 = oacm.rhs_block(U(9) + 0.5 * dt * K1, g, M + 12, h, ph)
    K3 = oacm.rhs_block(U(6) + 0.5 * dt * K2, g, M + 6, h, ph)
    K4 = oacm.rhs_block(U(3) + dt * K3, g, M, h, ph)
    return U(0) + dt / 6.0 * (inner(K1, 9) + 2.0 * inner(K2, 6) + 2.0 * inner(K3, 3) + K4)
