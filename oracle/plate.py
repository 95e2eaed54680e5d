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
from .adjoint import rhs_block_vjp
from .checkpointing import reverse
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


# ---- adjoint of the moving case: the gradient with respect to the pitch amplitude ---------------

def box_sdf_grad(P, lo, hi):
    """Gradient of ``box_sdf`` (..., 3): outside the box the unit vector from the nearest box
    point, inside the outward normal of the nearest face (undefined on the measure-zero set of
    points equidistant from several faces or on the box edges)."""
    c = 0.5 * (np.asarray(lo) + np.asarray(hi))
    h = 0.5 * (np.asarray(hi) - np.asarray(lo))
    sgn = np.where(P - c >= 0.0, 1.0, -1.0)
    q = np.abs(P - c) - h
    qp = np.maximum(q, 0.0)
    n = np.sqrt((qp ** 2).sum(axis=-1, keepdims=True))
    outside = n > 0.0
    onehot = (q == q.max(axis=-1, keepdims=True)).astype(np.float64)
    return np.where(outside, qp / np.where(outside, n, 1.0), onehot) * sgn


def plate_alpha_derivatives(plate, X, Y, Z, t):
    """d chi / d alpha_m (...) and d u_s / d alpha_m (3, ...) of ``Plate.fields`` at world points
    and time t.  alpha = alpha_m cos(w t), so dR/dalpha_m = R_z(phi) R_y'(alpha) cos(w t), and
    d omega / d alpha_m = -w sin(w t) R_z(phi) e_y."""
    phi, alpha, _, _ = plate.angles(t)
    w = 2.0 * math.pi * plate.f
    ca, sa = math.cos(alpha), math.sin(alpha)
    dRy = np.array([[-sa, 0.0, ca], [0.0, 0.0, 0.0], [-ca, 0.0, -sa]])
    dR = rot_z(phi) @ dRy * math.cos(w * t)
    R = plate.rotation(t)
    r = np.stack([X - plate.root[0], Y - plate.root[1], Z - plate.root[2]], axis=-1)
    xb = r @ R
    dxb = r @ dR
    d = box_sdf(xb, plate.lo, plate.hi)
    dchi_dd = -0.5 / plate.delta * (1.0 - np.tanh(d / plate.delta) ** 2)
    dchi = dchi_dd * (box_sdf_grad(xb, plate.lo, plate.hi) * dxb).sum(axis=-1)
    domega = -w * math.sin(w * t) * (rot_z(phi) @ np.array([0.0, 1.0, 0.0]))
    dus = np.moveaxis(np.cross(domega, r), -1, 0)
    return dchi, dus


class MovingPlateAdjoint:
    """Gradient of J = (1/N) sum_{n=1..N} [F_x(U_n, t_n) + w E(U_n)] for N fixed-dt RK4 steps of a
    ``MovingSolver`` on its frozen grid, with respect to the initial state and the pitch
    amplitude alpha_m.  F_x integrates chi (u - u_s) at the step's time.  The forward step is
    the solver's (mask and solid velocity at each stage time); the adjoint step is that of
    ``oracle.adjoint`` with the stage's mask and solid velocity, whose sensitivities are turned
    into d/d alpha_m with ``plate_alpha_derivatives`` at the stage time."""

    def __init__(self, solver, dt, nsteps, checkpoint_every=10, w_energy=0.1):
        from .adjoint import G_RHS, SyncMatrices
        self.S = solver
        self.fo = solver.fo
        self.ph = solver.ph
        self.dt, self.N, self.c, self.we = dt, nsteps, checkpoint_every, w_energy
        self.g = G_RHS
        self.mats = SyncMatrices(self.fo)
        M = self.fo.M
        self.half = np.zeros((M + 1,) * 3)
        self.half[:M, :M, :M] = 1.0
        self.t0 = solver.t

    def _fields(self, t):
        chi, us = {}, {}
        for leaf, s in self.fo.leaves.items():
            X, Y, Z = acm.block_coords(self.fo, leaf)
            chi[s], us[s] = self.S.plate.fields(X, Y, Z, t)
        return chi, us

    def _step(self, U, t):
        """The solver's step from (U, t): (U', [ext_s], [(chi_s, us_s)], [t_s])."""
        dt = self.dt
        V = U.copy()
        Ks, exts, fields, times = [], [], [], []
        for st, ts in enumerate((t, t + 0.5 * dt, t + 0.5 * dt, t + dt)):
            Y = V if st == 0 else V + (dt if st == 3 else 0.5 * dt) * Ks[-1]
            chi, us = self._fields(ts)
            ext = sync(self.fo, Y, self.g, "faces")
            K = np.zeros_like(Y)
            for leaf, s in self.fo.leaves.items():
                K[s] = acm.rhs_block(ext[s], self.g, self.fo.M, self.fo.h(leaf[0]), self.ph, chi=chi[s],
                                     us=us[s], chisp=self.S.chisp.get(s))
            Ks.append(K)
            exts.append(ext)
            fields.append((chi, us))
            times.append(ts)
        return V + dt / 6.0 * (Ks[0] + 2.0 * Ks[1] + 2.0 * Ks[2] + Ks[3]), exts, fields, times

    def _objective_terms(self, U, t):
        chi, us = self._fields(t)
        F = E = 0.0
        for leaf, s in self.fo.leaves.items():
            h3 = self.fo.h(leaf[0]) ** 3
            u = U[s]
            E += 0.5 * float(((u[0] ** 2 + u[1] ** 2 + u[2] ** 2) * self.half).sum()) * h3
            F += float((chi[s] * (u[0] - us[s][0]) * self.half).sum()) * h3 / self.ph.C_eta
        return F, E

    def _alpha_from(self, gchi, gus, t):
        """sum over blocks of <gchi, d chi/d alpha_m> + <gus, d u_s/d alpha_m> at time t."""
        out = 0.0
        for leaf, s in self.fo.leaves.items():
            X, Y, Z = acm.block_coords(self.fo, leaf)
            dchi, dus = plate_alpha_derivatives(self.S.plate, X, Y, Z, t)
            out += float((gchi[s] * dchi).sum()) + float((gus[s] * dus).sum())
        return out

    def _direct(self, U, t, lam):
        """Direct terms of (1/N)(F_x + w E) at (U, t): into lam; returns their d/d alpha_m."""
        chi, us = self._fields(t)
        wN = 1.0 / self.N
        gchi, gus = {}, {}
        for leaf, s in self.fo.leaves.items():
            h3 = self.fo.h(leaf[0]) ** 3
            u = U[s]
            lam[s, 0] += wN * (chi[s] / self.ph.C_eta + self.we * u[0]) * self.half * h3
            lam[s, 1] += wN * self.we * u[1] * self.half * h3
            lam[s, 2] += wN * self.we * u[2] * self.half * h3
            gchi[s] = wN * (u[0] - us[s][0]) * self.half * h3 / self.ph.C_eta
            gus[s] = np.zeros((3,) + u[0].shape)
            gus[s][0] = -wN * chi[s] * self.half * h3 / self.ph.C_eta
        return self._alpha_from(gchi, gus, t)

    def _G_T(self, ext, kappa, chi, us):
        """(J_G^T kappa in the register layout, d/d alpha_m contribution is returned by the caller
        from the mask and solid-velocity sensitivities (gchi, gus))."""
        m = self.mats
        M, g = self.fo.M, self.g
        de = np.zeros((4, m.nb, m.ne, m.ne, m.ne))
        gchi, gus = {}, {}
        for leaf, s in self.fo.leaves.items():
            e = np.nan_to_num(ext[s], nan=0.0)
            d, dc, du = rhs_block_vjp(e, g, M, self.fo.h(leaf[0]), self.ph, kappa[s], chi=chi[s],
                                      chisp=self.S.chisp.get(s), us=us[s], with_us=True)
            de[:, m.pos[s]] = d
            gchi[s], gus[s] = dc, du
        flat = de.reshape(4, -1)
        v = np.stack([m.S.T @ flat[f] for f in range(4)])
        return m.to_reg(v, np.zeros_like(kappa)), gchi, gus

    def _step_adjoint(self, U, t, lam):
        """lam = dJ/dU' -> (dJ/dU, d/d alpha_m through this step)."""
        dt = self.dt
        _, exts, fields, times = self._step(U, t)
        ga = 0.0
        kap = dt / 6.0 * lam
        nus = []
        for st, coef in ((3, None), (2, dt), (1, 0.5 * dt), (0, 0.5 * dt)):
            if st < 3:
                base = (dt / 3.0 if st > 0 else dt / 6.0) * lam
                kap = base + coef * nus[-1]
            nu, gchi, gus = self._G_T(exts[st], kap, *fields[st])
            ga += self._alpha_from(gchi, gus, times[st])
            nus.append(nu)
        m = self.mats
        tot = m.to_vec(lam + nus[0] + nus[1] + nus[2] + nus[3])
        v = np.stack([m.W.T @ tot[f] for f in range(4)])
        return m.to_reg(v, np.zeros_like(lam)), ga

    def gradient(self, U0, snapshots=None):
        """(J, dJ/dU_0 in the register layout, dJ/d alpha_m).  snapshots = S recomputes the
        states by binomial checkpointing with S stored states instead of segments."""
        if snapshots is not None:
            return self._gradient_binomial(U0, snapshots)
        dt, N, c = self.dt, self.N, self.c
        U = U0.copy()
        ckpt = {0: U.copy()}
        J = 0.0
        for n in range(1, N + 1):
            U = self._step(U, self.t0 + (n - 1) * dt)[0]
            F, E = self._objective_terms(U, self.t0 + n * dt)
            J += (F + self.we * E) / N
            if n % c == 0 and n < N:
                ckpt[n] = U.copy()
        lam = np.zeros_like(U0)
        ga = 0.0
        starts = sorted(ckpt)
        for a, b in reversed(list(zip(starts, starts[1:] + [N]))):
            states = [ckpt[a]]
            for k in range(a, b):
                states.append(self._step(states[-1], self.t0 + k * dt)[0])
            if b == N:
                ga += self._direct(states[-1], self.t0 + N * dt, lam)
            for n in range(b - 1, a - 1, -1):
                lam, g_step = self._step_adjoint(states[n - a], self.t0 + n * dt, lam)
                ga += g_step
                if n >= 1:
                    ga += self._direct(states[n - a], self.t0 + n * dt, lam)
        return J, lam, ga

    def vjp(self, U0, lamN, snapshots=None):
        """For L = <lamN, U_N> (lamN in the register layout): (U_N, dL/dU_0, dL/d alpha_m), the
        gradient's sweep without the objective's direct terms, from lam = lamN; the states are
        recomputed with `snapshots` stored states (default: all of them)."""
        dt, N = self.dt, self.N
        st = {"lam": lamN.copy(), "ga": 0.0, "UN": None}

        def advance(U, k):
            return self._step(U, self.t0 + k * dt)[0]

        def turn(U, k):
            if k == N - 1:
                st["UN"] = self._step(U, self.t0 + k * dt)[0]
            st["lam"], g_step = self._step_adjoint(U, self.t0 + k * dt, st["lam"])
            st["ga"] += g_step

        self.last_advances = reverse(N, snapshots or N, U0, advance, turn)
        return st["UN"], st["lam"], st["ga"]

    def _gradient_binomial(self, U0, snapshots):
        """As ``gradient``, the states recomputed by ``oracle.checkpointing.reverse``; the
        objective's terms are summed when a state is first reached."""
        dt, N = self.dt, self.N
        st = {"lam": np.zeros_like(U0), "J": 0.0, "ga": 0.0, "hi": 0}

        def reached(U, k):
            if k > st["hi"]:
                F, E = self._objective_terms(U, self.t0 + k * dt)
                st["J"] += (F + self.we * E) / N
                st["hi"] = k

        def advance(U, k):
            U1 = self._step(U, self.t0 + k * dt)[0]
            reached(U1, k + 1)
            return U1

        def turn(U, k):
            if k == N - 1:
                UN = self._step(U, self.t0 + k * dt)[0]
                reached(UN, N)
                st["ga"] += self._direct(UN, self.t0 + N * dt, st["lam"])
            st["lam"], g_step = self._step_adjoint(U, self.t0 + k * dt, st["lam"])
            st["ga"] += g_step
            if k >= 1:
                st["ga"] += self._direct(U, self.t0 + k * dt, st["lam"])

        self.last_advances = reverse(N, snapshots, U0, advance, turn)
        return st["J"], st["lam"], st["ga"]
