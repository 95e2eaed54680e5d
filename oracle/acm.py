"""Artificial-compressibility model with volume penalization on the block grid (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 2.1-2.2, eqs. "u_eqn-1" and "p_eqn-1":
    du/dt = -(u.grad)u - grad p + nu lap u - chi/C_eta (u - u_s) - chi_sp/C_sp (u - u_inf)
    dp/dt = -C_0^2 div u - C_gamma p - chi_sp/C_sp (p - p_inf)
Sec. 2.2: force F = C_eta^{-1} int chi (u - u_s) dV by the midpoint rule; the mask chi is a
smoothed indicator with a layer proportional to the grid spacing.
Sec. 2.3: 4th-order centred differences -- the Tam & Webb optimised first derivative and the
classical 4th-order second derivative -- and classical RK4; the time step obeys
dt < min(CFL dx_min/u_eig, CFL_eta C_eta, CFL_nu dx_min^2/nu), u_eig = |u_max| + sqrt(u_max^2 + C_0^2).

Readings (the paper's Appendix A is not available):
* First derivative: (1/h) sum_{j=1..3} a_j (f_{i+j} - f_{i-j}) with the 4th-order family
  a1 = 2/3 + 5 a3, a2 = -1/12 - 4 a3.  Tam & Webb pick a3 by minimising the integrated
  dispersion error over kh in [0, pi/2]; that minimiser is a3 = 0.0265199520614978
  (published to 8 digits as 0.02651995).  a3 = 0 gives the classical (8, -1)/12 stencil.
* Second derivative: (-f_{i-2} + 16 f_{i-1} - 30 f_i + 16 f_{i+1} - f_{i+2}) / (12 h^2).
* The right-hand side is evaluated at all Bs^3 points of every block, faces included.
* u_max is the largest velocity magnitude; the C_eta limit applies only when a mask is set.
* Force and energy sum each physical point once: the half-open points [0, Bs-2]^3 of a block.
"""
from __future__ import annotations

import math

import numpy as np

TAM_WEBB_A3 = 0.0265199520614978


def d1_coeffs(scheme="tam_webb"):
    a3 = TAM_WEBB_A3 if scheme == "tam_webb" else 0.0
    return (2.0 / 3.0 + 5.0 * a3, -1.0 / 12.0 - 4.0 * a3, a3)


def _sh(e, g, axis, k, M):
    """Slice of the extended array e (..., n, n, n) at offset k along axis (0=x,1=y,2=z),
    restricted to the interior in all axes."""
    lo, hi = g, g + M + 1
    sl = [slice(lo, hi)] * 3
    sl[axis] = slice(lo + k, hi + k)
    # array axes are (z, y, x): axis 0 (x) -> last
    return e[(Ellipsis, sl[2], sl[1], sl[0])]


def d1(e, g, M, h, axis, coeffs):
    a = coeffs
    out = a[0] * (_sh(e, g, axis, 1, M) - _sh(e, g, axis, -1, M))
    out = out + a[1] * (_sh(e, g, axis, 2, M) - _sh(e, g, axis, -2, M))
    out = out + a[2] * (_sh(e, g, axis, 3, M) - _sh(e, g, axis, -3, M))
    return out / h


def d2(e, g, M, h, axis):
    return (-_sh(e, g, axis, -2, M) + 16.0 * _sh(e, g, axis, -1, M) - 30.0 * _sh(e, g, axis, 0, M)
            + 16.0 * _sh(e, g, axis, 1, M) - _sh(e, g, axis, 2, M)) / (12.0 * h * h)


class Physics:
    """Parameters of the model equations (names follow the paper)."""

    def __init__(self, nu=1e-2, c0=10.0, C_eta=1e-3, C_gamma=1.0, C_sp=1.0, u_inf=(0.0, 0.0, 0.0),
                 p_inf=0.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25, scheme="tam_webb"):
        self.nu, self.c0, self.C_eta, self.C_gamma, self.C_sp = nu, c0, C_eta, C_gamma, C_sp
        self.u_inf = tuple(u_inf)
        self.p_inf = p_inf
        self.cfl, self.cfl_eta, self.cfl_nu = cfl, cfl_eta, cfl_nu
        self.scheme = scheme


def rhs_block(e, g, M, h, ph, chi=None, us=None, chisp=None):
    """Right-hand side (4, M+1, M+1, M+1) of one block from its extended state e (4, n, n, n)
    (faces of depth >= 3 filled).  chi, chisp: (M+1,)^3 or None; us: (3, M+1,...) or None."""
    a = d1_coeffs(ph.scheme)
    u = [_sh(e[f], g, 0, 0, M) for f in range(4)]
    du = [[d1(e[f], g, M, h, ax, a) for ax in range(3)] for f in range(4)]
    out = np.empty((4, M + 1, M + 1, M + 1))
    for i in range(3):
        conv = u[0] * du[i][0] + u[1] * du[i][1] + u[2] * du[i][2]
        lap = d2(e[i], g, M, h, 0) + d2(e[i], g, M, h, 1) + d2(e[i], g, M, h, 2)
        r = -conv - du[3][i] + ph.nu * lap
        if chi is not None:
            usi = 0.0 if us is None else us[i]
            r = r - chi / ph.C_eta * (u[i] - usi)
        if chisp is not None:
            r = r - chisp / ph.C_sp * (u[i] - ph.u_inf[i])
        out[i] = r
    div = du[0][0] + du[1][1] + du[2][2]
    rp = -ph.c0 ** 2 * div - ph.C_gamma * u[3]
    if chisp is not None:
        rp = rp - chisp / ph.C_sp * (u[3] - ph.p_inf)
    out[3] = rp
    return out


# ---- masks and initial conditions (analytic, evaluated at integer-derived coordinates) ------

def block_coords(forest, leaf):
    """Coordinates X, Y, Z (M+1,)^3 (arrays indexed z, y, x) of a leaf's points: x = i h_J,
    i the global lattice index wrapped into [0, N_J), so that every block holding a point
    (across the periodic seam too) computes bitwise identical coordinates."""
    J, gx, gy, gz = leaf
    M = forest.M
    h = forest.h(J)
    N = forest.npoints(J)
    i = np.arange(M + 1)
    x = np.mod(gx * M + i, N[0]) * h       # the periodic seam x = L is taken as x = 0
    y = np.mod(gy * M + i, N[1]) * h
    z = np.mod(gz * M + i, N[2]) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def smooth_step(d, delta):
    """chi = (1 - tanh(d / delta)) / 2 for signed distance d (negative inside)."""
    return 0.5 * (1.0 - np.tanh(d / delta))


def sphere_mask(X, Y, Z, centre, R, delta):
    d = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2) - R
    return smooth_step(d, delta)


def sponge_mask(X, Y, Z, L, L_sp, delta):
    """Sponge indicator: 1 within L_sp of any face of the periodic box [0, L]^3, smoothed by
    the same tanh profile; the largest of the three axis profiles."""
    out = None
    for c, Lc in zip((X, Y, Z), L):
        dist = np.minimum(c, Lc - c)
        s = smooth_step(dist - L_sp, delta)
        out = s if out is None else np.maximum(out, s)
    return out


def ic_taylor_green(X, Y, Z, k=2.0 * math.pi, amp=1.0):
    u = amp * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z)
    v = -amp * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z)
    w = np.zeros_like(X)
    p = np.zeros_like(X)
    return np.stack([u, v, w, p])


def ic_uniform(X, Y, Z, u0=(1.0, 0.0, 0.0), p0=0.0):
    return np.stack([np.full_like(X, u0[0]), np.full_like(X, u0[1]), np.full_like(X, u0[2]),
                     np.full_like(X, p0)])


def ic_pulse(X, Y, Z, centre, width, amp, L):
    """Gaussian pressure pulse, u = 0; distance taken to the nearest periodic image."""
    r2 = 0.0
    for c, c0, Lc in zip((X, Y, Z), centre, L):
        d = c - c0
        d = d - Lc * np.round(d / Lc)
        r2 = r2 + d * d
    p = amp * np.exp(-r2 / (width * width))
    z = np.zeros_like(X)
    return np.stack([z, z.copy(), z.copy(), p])


def _nearest_image(c, c0, Lc):
    d = c - c0
    return d - Lc * np.round(d / Lc)


def ic_vortex_ring(X, Y, Z, centre, axis, R, gamma, sigma, L):
    """Vortex ring velocity u = curl(psi e_theta), p = 0 (a synthetic divergence-free field).

    In ring coordinates about the centre (nearest periodic image) and the unit axis n: zeta =
    d.n, r_perp = d - zeta n, rho = |r_perp|, e_theta = n x r_perp / rho.  The azimuthal vector
    potential psi = gamma / (2 pi) (rho / R) exp(-((rho - R)^2 + zeta^2) / sigma^2) vanishes on the
    axis; its curl in cylindrical coordinates, u_rho = -d psi/d zeta and
    u_zeta = (1/rho) d(rho psi)/d rho, is with E the exponential and K = gamma E / (2 pi R)
        u = K [ (2 zeta / sigma^2) r_perp + (2 - 2 rho (rho - R) / sigma^2) n ]."""
    n = np.asarray(axis, dtype=np.float64)
    n = n / np.linalg.norm(n)
    d = [_nearest_image(c, c0, Lc) for c, c0, Lc in zip((X, Y, Z), centre, L)]
    zeta = d[0] * n[0] + d[1] * n[1] + d[2] * n[2]
    rp = [d[a] - zeta * n[a] for a in range(3)]
    rho = np.sqrt(rp[0] ** 2 + rp[1] ** 2 + rp[2] ** 2)
    E = np.exp(-((rho - R) ** 2 + zeta ** 2) / (sigma * sigma))
    K = gamma * E / (2.0 * math.pi * R)
    a_r = K * 2.0 * zeta / (sigma * sigma)
    a_n = K * (2.0 - 2.0 * rho * (rho - R) / (sigma * sigma))
    u = [a_r * rp[a] + a_n * n[a] for a in range(3)]
    return np.stack([u[0], u[1], u[2], np.zeros_like(X)])


def vortex_ring_potential(X, Y, Z, centre, axis, R, gamma, sigma, L):
    """The vector potential psi e_theta of ic_vortex_ring (for checks of its curl)."""
    n = np.asarray(axis, dtype=np.float64)
    n = n / np.linalg.norm(n)
    d = [_nearest_image(c, c0, Lc) for c, c0, Lc in zip((X, Y, Z), centre, L)]
    zeta = d[0] * n[0] + d[1] * n[1] + d[2] * n[2]
    rp = [d[a] - zeta * n[a] for a in range(3)]
    rho = np.sqrt(rp[0] ** 2 + rp[1] ** 2 + rp[2] ** 2)
    psi_over_rho = gamma / (2.0 * math.pi * R) * np.exp(-((rho - R) ** 2 + zeta ** 2) / (sigma * sigma))
    # psi e_theta = (psi / rho) (n x r_perp)
    cx = n[1] * rp[2] - n[2] * rp[1]
    cy = n[2] * rp[0] - n[0] * rp[2]
    cz = n[0] * rp[1] - n[1] * rp[0]
    return np.stack([psi_over_rho * cx, psi_over_rho * cy, psi_over_rho * cz])


def ic_pulse_ring(X, Y, Z, pulse, ring, L):
    """Gaussian pressure pulse plus vortex-ring velocity: pulse = (centre, width, amp), ring =
    (centre, axis, R, gamma, sigma)."""
    out = ic_vortex_ring(X, Y, Z, *ring, L)
    out[3] = ic_pulse(X, Y, Z, *pulse, L)[3]
    return out


# ---- time step, RK4 ---------------------------------------------------------------------------

def time_step(ph, u_max, h_min, masked):
    """Sec. 2.3: dt = min(CFL h/u_eig, CFL_eta C_eta, CFL_nu h^2/nu)."""
    u_eig = abs(u_max) + math.sqrt(u_max * u_max + ph.c0 * ph.c0)
    dt = ph.cfl * h_min / u_eig
    if masked:
        dt = min(dt, ph.cfl_eta * ph.C_eta)
    if ph.nu > 0:
        dt = min(dt, ph.cfl_nu * h_min * h_min / ph.nu)
    return dt
