"""Moving rigid plate: time-dependent mask and solid velocity (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Sec. 2.2: the solid enters through the smoothed mask chi (tanh of the signed distance) and the
solid velocity u_s in the penalization term -chi/C_eta (u - u_s), and the force integrates
chi (u - u_s).  Sec. 5.2 flaps a rectangular rigid wing whose kinematics are given in the work
it cites; the plate here is a synthetic stand-in with the dimensions and amplitudes of the
full-scale configuration (chord 1, span 3, thickness 0.05, stroke +-60 deg, pitch +-45 deg,
frequency 1).  Readings:

* Body frame: x_b along the chord, y_b along the span with the root at y_b = 0, z_b across the
  thickness; the plate is the box |x_b| <= c/2, 0 <= y_b <= b, |z_b| <= t/2 (the pitch axis runs
  along the span through mid-chord).
* Body to world: x = x_root + R(t) x_b with R(t) = R_z(phi(t)) R_y(alpha(t)): pitch alpha about
  the span axis, then stroke phi about the vertical z axis (a horizontal stroke plane).
* phi(t) = phi_m sin(2 pi f t), alpha(t) = alpha_m cos(2 pi f t): the pitch is a quarter period
  ahead of the stroke (largest at stroke reversal), so the two half strokes mirror each other.
* u_s = omega x (x - x_root) with omega = phi' e_z + alpha' R_z(phi) e_y (rigid rotation about
  the root); chi and u_s are evaluated at every RK4 stage time.
"""
from __future__ import annotations

import math

import numpy as np

from . import acm
from .adapt import Solver
from .sync import sync


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def box_sdf(P, lo, hi):
    """Signed distance (negative inside) of points P (..., 3) to the axis-aligned box [lo, hi]."""
    c = 0.5 * (np.asarray(lo) + np.asarray(hi))
    h = 0.5 * (np.asarray(hi) - np.asarray(lo))
    q = np.abs(P - c) - h
    outside = np.sqrt((np.maximum(q, 0.0) ** 2).sum(axis=-1))
    inside = np.minimum(q.max(axis=-1), 0.0)
    return outside + inside


class Plate:
    """A rigid plate flapping about a root point (readings in the module docstring)."""

    def __init__(self, chord=1.0, span=3.0, thickness=0.05, phi_m=math.radians(60.0),
                 alpha_m=math.radians(45.0), freq=1.0, root=(4.0, 4.0, 4.0), delta=0.01):
        self.c, self.b, self.t = chord, span, thickness
        self.phi_m, self.alpha_m, self.f = phi_m, alpha_m, freq
        self.root = np.asarray(root, dtype=np.float64)
        self.delta = delta
        self.lo = np.array([-chord / 2, 0.0, -thickness / 2])
        self.hi = np.array([chord / 2, span, thickness / 2])

    def angles(self, t):
        """(phi, alpha, dphi/dt, dalpha/dt) at time t."""
        w = 2.0 * math.pi * self.f
        return (self.phi_m * math.sin(w * t), self.alpha_m * math.cos(w * t),
                self.phi_m * w * math.cos(w * t), -self.alpha_m * w * math.sin(w * t))

    def rotation(self, t):
        phi, alpha, _, _ = self.angles(t)
        return rot_z(phi) @ rot_y(alpha)

    def omega(self, t):
        phi, _, dphi, dalpha = self.angles(t)
        return dphi * np.array([0.0, 0.0, 1.0]) + dalpha * (rot_z(phi) @ np.array([0.0, 1.0, 0.0]))

    def fields(self, X, Y, Z, t):
        """chi (...) and u_s (3, ...) at world points (X, Y, Z) and time t."""
        R = self.rotation(t)
        r = np.stack([X - self.root[0], Y - self.root[1], Z - self.root[2]], axis=-1)
        xb = r @ R                                   # R^T r, row-vector form
        chi = acm.smooth_step(box_sdf(xb, self.lo, self.hi), self.delta)
        us = np.moveaxis(np.cross(self.omega(t), r), -1, 0)
        return chi, us


class MovingSolver(Solver):
    """``adapt.Solver`` with the plate's mask and solid velocity evaluated at every stage time
    of RK4 (the classical nodes t, t + dt/2, t + dt/2, t + dt) and the force of Sec. 2.2 with
    u - u_s."""

    def __init__(self, forest, ph, plate, **kw):
        kw.pop("mask", None)
        super().__init__(forest, ph, **kw)
        self.plate = plate
        self.us = {}

    def eval_moving(self, t):
        for leaf, s in self.fo.leaves.items():
            X, Y, Z = acm.block_coords(self.fo, leaf)
            self.chi[s], self.us[s] = self.plate.fields(X, Y, Z, t)

    def eval_mask(self):
        super().eval_mask()
        self.eval_moving(self.t)

    def rhs_at(self, F, t):
        self.eval_moving(t)
        g = 3
        ext = sync(self.fo, F, g, "faces")
        K = np.zeros_like(F)
        for leaf, s in self.fo.leaves.items():
            K[s] = acm.rhs_block(ext[s], g, self.fo.M, self.fo.h(leaf[0]), self.ph, chi=self.chi[s],
                                 us=self.us[s], chisp=self.chisp.get(s))
        return K

    def rk4(self, dt):
        U, t = self.U, self.t
        K1 = self.rhs_at(U, t)
        K2 = self.rhs_at(U + 0.5 * dt * K1, t + 0.5 * dt)
        K3 = self.rhs_at(U + 0.5 * dt * K2, t + 0.5 * dt)
        K4 = self.rhs_at(U + dt * K3, t + dt)
        self.U = U + dt / 6.0 * (K1 + 2.0 * K2 + 2.0 * K3 + K4)
        self.t = t + dt
        self.eval_moving(self.t)

    def diagnostics(self):
        fo = self.fo
        M = fo.M
        F = np.zeros(3)
        E = 0.0
        for leaf, s in fo.leaves.items():
            h3 = fo.h(leaf[0]) ** 3
            u = self.U[s][:, :M, :M, :M]
            E += 0.5 * float((u[0] ** 2 + u[1] ** 2 + u[2] ** 2).sum()) * h3
            chi = self.chi[s][:M, :M, :M]
            for i in range(3):
                F[i] += float((chi * (u[i] - self.us[s][i][:M, :M, :M])).sum()) * h3 / self.ph.C_eta
        return F, E
