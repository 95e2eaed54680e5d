"""Discrete adjoint of RK4 steps on a frozen block grid (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

The forward map is the oracle's own time step (``adapt.Solver.rk4``, Sec. 2.3) repeated N times
with a fixed step dt on a fixed grid.  One step is

    V = W U,  Y1 = V,  Y2 = V + dt/2 K1,  Y3 = V + dt/2 K2,  Y4 = V + dt K3,  K_s = G(Y_s),
    U' = V + dt/6 (K1 + 2 K2 + 2 K3 + K4),

where W is the fine-wins projection that the synchronisation applies to the state (Sec. 4.2 and
the ghost-value reading of ``oracle.sync``) and G(Y) is the block-local right-hand side of eqs.
(u_eqn-1, p_eqn-1) (Sec. 2.1-2.2) evaluated on the synchronised extended arrays E W Y.  W and E
are linear; the synchronisation is built here as sparse matrices from the same point-value rule
(finest leaf holding a point, else the tensor DD-4 prediction one level up, Sec. 3.1).

The objective is J = (1/N) sum_{n=1..N} [F_x(U_n) + 0.1 E(U_n)] with the force and energy of
Sec. 2.2 (midpoint rule over every block's half-open points).  Its parameters are the initial
state U_0 and the sphere's centre and radius, which enter through the analytic mask chi
(Sec. 2.2): in the penalization term of G and in F_x.

The adjoint of one step, with lam' = dJ/dU' and nu_s = J_G(Y_s)^T kappa_s:

    kappa_4 = dt/6 lam',            kappa_3 = dt/3 lam' + dt nu_4,
    kappa_2 = dt/3 lam' + dt/2 nu_3, kappa_1 = dt/6 lam' + dt/2 nu_2,
    lam = W^T (lam' + nu_1 + nu_2 + nu_3 + nu_4),   J_G(Y)^T = W^T E^T J_loc(E W Y)^T,

and the mask collects sum_s (dG/dchi)(Y_s)^T kappa_s.  The paper has no adjoint; readings:

* The grid is frozen: grid adaptation is not differentiable, so the gradient is that of the RK4
  steps on the grid a forward run uses (recorded and replayed), here one fixed grid.
* dt is fixed (recorded), not differentiated through the CFL rule; the mask is static.
* Checkpointing keeps the state at every c-th step; the backward sweep over a segment recomputes
  the states inside it from its checkpoint (one level of recompute).  Alternatively S snapshots
  and binomial checkpointing (``oracle.checkpointing``) recompute the fewest steps for that
  memory; the arithmetic of every step is the same, so all schedules give the same gradient.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import acm
from .checkpointing import reverse
from .sync import PointValues, local_points, sync

W_DD4 = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0
G_RHS = 3          # ghost layers the right-hand side reads (faces only)


class SyncMatrices:
    """Fine wins W (register -> register) and ghost fill E (register -> extended arrays of
    depth g, 'faces' points) of a fixed forest, over the scalar register of its leaves in slot
    order: vector index ((k (M+1) + z) (M+1) + y) (M+1) + x for the k-th smallest leaf slot."""

    def __init__(self, forest, g=G_RHS, which="faces"):
        self.fo = forest
        self.g = g
        self.M = forest.M
        self.n = forest.M + 1
        self.ne = forest.M + 1 + 2 * g
        self.slots = np.array(sorted(forest.leaves.values()), dtype=np.int64)
        self.pos = {int(s): k for k, s in enumerate(self.slots)}
        self.nb = len(self.slots)
        self.pv = PointValues(forest, None)      # only its leaf tables are used
        self.W = self._fine_wins()
        self.E = self._ghost_fill(which)
        self.S = (self.E @ self.W).tocsr()

    # ---- vector layout -----------------------------------------------------------------
    def _index(self, slot, loc):
        n = self.n
        k = np.array([self.pos[int(s)] for s in np.atleast_1d(slot)], dtype=np.int64)
        return ((k * n + loc[:, 2]) * n + loc[:, 1]) * n + loc[:, 0]

    def to_vec(self, F):
        """Register F[slot, f, z, y, x] -> (4, nb n^3) vectors of the leaves."""
        return F[self.slots].transpose(1, 0, 2, 3, 4).reshape(F.shape[1], -1)

    def to_reg(self, v, F):
        """Write vectors (4, nb n^3) into a register F of the oracle's shape."""
        n = self.n
        F[self.slots] = v.reshape(v.shape[0], self.nb, n, n, n).transpose(1, 0, 2, 3, 4)
        return F

    def ext_of(self, x):
        """Extended arrays (4, nb, ne, ne, ne) from a vector of extended values (4, nb ne^3)."""
        ne = self.ne
        return x.reshape(x.shape[0], self.nb, ne, ne, ne)

    # ---- point values as sparse rows ------------------------------------------------------------
    def _finest(self, J, P, min_level):
        """Vector index of the finest leaf of level >= min_level holding each level-J point
        (-1 where none): the lookup of ``PointValues.finest``."""
        out = -np.ones(P.shape[0], dtype=np.int64)
        todo = np.ones(P.shape[0], dtype=bool)
        for L in sorted((l for l in self.pv.levels if l >= min_level), reverse=True):
            if not todo.any():
                break
            idx = np.nonzero(todo)[0]
            slot, loc = self.pv._leaf_at_level(L, P[idx] * (1 << (L - J)))
            hit = slot >= 0
            if hit.any():
                out[idx[hit]] = self._index(slot[hit], loc[hit])
                todo[idx[hit]] = False
        return out

    def _rows(self, J, P):
        """V_J at the level-J points P (n, 3) as sparse rows: (row, col, weight) arrays."""
        N = np.array(self.fo.npoints(J), dtype=np.int64)
        P = np.mod(np.asarray(P, dtype=np.int64), N)
        col = self._finest(J, P, J)
        hit = col >= 0
        rows = [np.nonzero(hit)[0]]
        cols = [col[hit]]
        wts = [np.ones(int(hit.sum()))]
        miss = np.nonzero(~hit)[0]
        if miss.size:
            Pm = P[miss]
            # tensor DD-4 weights per axis: 4 coarse samples at (p + {-3,-1,1,3}) / 2 if p is odd,
            # the coarse sample p / 2 itself if p is even
            co = np.zeros((miss.size, 3, 4), dtype=np.int64)
            w = np.zeros((miss.size, 3, 4))
            for a in range(3):
                p = Pm[:, a]
                odd = (p % 2) == 1
                for j, dj in enumerate((-3, -1, 1, 3)):
                    co[:, a, j] = np.where(odd, (p + dj) // 2, p // 2)
                    w[:, a, j] = np.where(odd, W_DD4[j], 1.0 if j == 0 else 0.0)
            Q, wq, parent = [], [], []
            for kz in range(4):
                for ky in range(4):
                    for kx in range(4):
                        wk = w[:, 0, kx] * w[:, 1, ky] * w[:, 2, kz]
                        nz = wk != 0.0
                        Q.append(np.stack([co[nz, 0, kx], co[nz, 1, ky], co[nz, 2, kz]], axis=1))
                        wq.append(wk[nz])
                        parent.append(miss[nz])
            Q = np.concatenate(Q)
            wq = np.concatenate(wq)
            parent = np.concatenate(parent)
            r2, c2, w2 = self._rows(J - 1, Q)
            rows.append(parent[r2])
            cols.append(c2)
            wts.append(wq[r2] * w2)
        return np.concatenate(rows), np.concatenate(cols), np.concatenate(wts)

    def _fine_wins(self):
        """W: identity, except that a leaf's boundary point that a strictly finer leaf holds takes
        that leaf's value (``oracle.sync.fine_wins``)."""
        M, n = self.M, self.n
        N = self.nb * n ** 3
        Pl = local_points(M, 0, "cube")
        bnd = Pl[((Pl == 0) | (Pl == M)).any(axis=1)]
        keep = np.ones(N, dtype=bool)
        rows, cols = [], []
        top = self.pv.levels[-1]
        for (J, gx, gy, gz), s in self.fo.leaves.items():
            if J >= top:
                continue
            col = self._finest(J, bnd + np.array([gx, gy, gz]) * M, J + 1)
            hit = col >= 0
            if hit.any():
                r = self._index(np.full(int(hit.sum()), s), bnd[hit])
                keep[r] = False
                rows.append(r)
                cols.append(col[hit])
        ident = np.nonzero(keep)[0]
        rows = np.concatenate([ident] + rows)
        cols = np.concatenate([ident] + cols)
        return sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(N, N))

    def _ghost_fill(self, which):
        """E: the extended array of every leaf (interior + g layers, points of ``which``), every
        point V_J from the (fine-won) register, as ``oracle.sync.sync`` fills it.  A point on a
        block face is looked up like a ghost point; a same-level copy may answer, which is the
        same value whenever redundant points agree (always, for states of the method), but not
        for an arbitrary perturbation: the matrix follows the lookup, so that it is the exact
        linear map of the oracle's synchronisation on every input."""
        M, g, ne, n = self.M, self.g, self.ne, self.n
        Pl = local_points(M, g, which)
        rows, cols, wts = [], [], []
        for (J, gx, gy, gz), s in self.fo.leaves.items():
            k = self.pos[s]
            erow = ((k * ne + Pl[:, 2] + g) * ne + Pl[:, 1] + g) * ne + Pl[:, 0] + g
            r, c, w = self._rows(J, Pl + np.array([gx, gy, gz]) * M)
            rows.append(erow[r])
            cols.append(c)
            wts.append(w)
        rows, cols, wts = np.concatenate(rows), np.concatenate(cols), np.concatenate(wts)
        return sp.csr_matrix((wts, (rows, cols)), shape=(self.nb * ne ** 3, self.nb * n ** 3))


# ---- the block right-hand side and its transposed Jacobian --------------------------------------

def _sh_add(out, g, axis, k, M, val):
    """Transpose of ``acm._sh``: add val (interior-shaped) into out at offset k along axis."""
    lo, hi = g, g + M + 1
    sl = [slice(lo, hi)] * 3
    sl[axis] = slice(lo + k, hi + k)
    out[(Ellipsis, sl[2], sl[1], sl[0])] += val


def d1_T(w, out, g, M, h, axis, coeffs):
    """out += D1^T w for the first derivative along axis (``acm.d1``)."""
    for j, a in enumerate(coeffs, start=1):
        _sh_add(out, g, axis, j, M, a * w / h)
        _sh_add(out, g, axis, -j, M, -a * w / h)


def d2_T(w, out, g, M, h, axis):
    """out += D2^T w for the second derivative along axis (``acm.d2``)."""
    c = 1.0 / (12.0 * h * h)
    for k, a in ((-2, -1.0), (-1, 16.0), (0, -30.0), (1, 16.0), (2, -1.0)):
        _sh_add(out, g, axis, k, M, a * c * w)


def rhs_block_vjp(e, g, M, h, ph, kappa, chi=None, chisp=None, us=None, with_us=False):
    """Transposed Jacobian of ``acm.rhs_block`` at the extended state e (4, ne, ne, ne) applied
    to kappa (4, M+1, M+1, M+1): (d e (4, ne, ne, ne), d chi (M+1,)^3 or None), and with
    ``with_us`` also d u_s (3, M+1, M+1, M+1) (the solid velocity us, default 0)."""
    a = acm.d1_coeffs(ph.scheme)
    u = [acm._sh(e[f], g, 0, 0, M) for f in range(4)]
    du = [[acm.d1(e[f], g, M, h, ax, a) for ax in range(3)] for f in range(4)]
    de = np.zeros_like(e)
    dint = np.zeros((4, M + 1, M + 1, M + 1))
    dchi = None if chi is None else np.zeros((M + 1, M + 1, M + 1))
    for i in range(3):
        k = kappa[i]
        # -(u . grad) u_i = -sum_j u_j D1_j u_i
        for j in range(3):
            dint[j] -= k * du[i][j]
            d1_T(-u[j] * k, de[i], g, M, h, j, a)
        # -D1_i p
        d1_T(-k, de[3], g, M, h, i, a)
        # nu sum_ax D2_ax u_i
        for ax in range(3):
            d2_T(ph.nu * k, de[i], g, M, h, ax)
        if chi is not None:
            usi = 0.0 if us is None else us[i]
            dint[i] -= chi / ph.C_eta * k
            dchi -= (u[i] - usi) / ph.C_eta * k
        if chisp is not None:
            dint[i] -= chisp / ph.C_sp * k
    k = kappa[3]
    for j in range(3):
        d1_T(-ph.c0 ** 2 * k, de[j], g, M, h, j, a)
    dint[3] -= ph.C_gamma * k
    if chisp is not None:
        dint[3] -= chisp / ph.C_sp * k
    for f in range(4):
        _sh_add(de[f], g, 0, 0, M, dint[f])
    if with_us:
        dus = np.zeros((3, M + 1, M + 1, M + 1))
        if chi is not None:
            for i in range(3):
                dus[i] = chi / ph.C_eta * kappa[i]
        return de, dchi, dus
    return de, dchi


# ---- the mask and its parameter derivatives -------------------------------------------------------

def sphere_mask_grad(X, Y, Z, centre, R, delta):
    """d chi / d (cx, cy, cz, R) of ``acm.sphere_mask``: chi = (1 - tanh(d/delta))/2 with
    d = |x - c| - R, so d chi/d d = -sech^2(d/delta) / (2 delta)."""
    rx, ry, rz = X - centre[0], Y - centre[1], Z - centre[2]
    r = np.sqrt(rx * rx + ry * ry + rz * rz)
    d = r - R
    s = 0.5 / delta * (1.0 - np.tanh(d / delta) ** 2)      # = -d chi / d d
    rs = np.where(r > 0, r, 1.0)
    return np.stack([s * rx / rs, s * ry / rs, s * rz / rs, s])


# ---- objective, forward and backward sweeps ---------------------------------------------------------

class FrozenGridAdjoint:
    """Gradient of J = (1/N) sum_{n=1..N} [F_x(U_n) + 0.1 E(U_n)] for N fixed-dt RK4 steps of a
    ``adapt.Solver`` whose grid stays fixed, with respect to U_0 and the sphere's centre and
    radius.  The solver's mask must be the sphere (centre, R, delta) given here."""

    def __init__(self, solver, centre, R, delta, dt, nsteps, checkpoint_every=10, w_energy=0.1):
        self.S = solver
        self.fo = solver.fo
        self.ph = solver.ph
        self.centre = None if centre is None else tuple(centre)
        self.R, self.delta = R, delta
        self.dt, self.N, self.c, self.we = dt, nsteps, checkpoint_every, w_energy
        self.mats = SyncMatrices(self.fo)
        M = self.fo.M
        self.half = np.zeros((M + 1,) * 3)
        self.half[:M, :M, :M] = 1.0                     # the half-open points [0, M-1]^3

    # objective terms of one state (U in the solver's register layout)
    def objective_terms(self, U):
        F = 0.0
        E = 0.0
        for leaf, s in self.fo.leaves.items():
            h3 = self.fo.h(leaf[0]) ** 3
            u = U[s]
            E += 0.5 * float(((u[0] ** 2 + u[1] ** 2 + u[2] ** 2) * self.half).sum()) * h3
            F += float((self.S.chi[s] * u[0] * self.half).sum()) * h3 / self.ph.C_eta
        return F, E

    def _dJ_dU(self, U, lam, gchi):
        """Add the direct terms of one state's contribution (1/N)(F_x + w E) to lam (register
        layout) and to the mask gradient gchi (slot -> array)."""
        wN = 1.0 / self.N
        for leaf, s in self.fo.leaves.items():
            h3 = self.fo.h(leaf[0]) ** 3
            u = U[s]
            lam[s, 0] += wN * (self.S.chi[s] / self.ph.C_eta + self.we * u[0]) * self.half * h3
            lam[s, 1] += wN * self.we * u[1] * self.half * h3
            lam[s, 2] += wN * self.we * u[2] * self.half * h3
            gchi[s] += wN * u[0] * self.half * h3 / self.ph.C_eta

    def _step(self, U):
        """The oracle's RK4 step on a copy: returns (U', [Y_s after fine wins], [ext_s])."""
        S = self.S
        dt = self.dt
        ys, exts, Ks = [], [], []
        V = U.copy()
        for st in range(4):
            if st == 0:
                Y = V
            else:
                Y = V + (dt if st == 3 else 0.5 * dt) * Ks[-1]
            ext = sync(self.fo, Y, G_RHS, "faces")            # fine wins applied to Y in place
            K = np.zeros_like(Y)
            for leaf, s in self.fo.leaves.items():
                K[s] = acm.rhs_block(ext[s], G_RHS, self.fo.M, self.fo.h(leaf[0]), self.ph,
                                     chi=S.chi.get(s), chisp=S.chisp.get(s))
            ys.append(Y)
            exts.append(ext)
            Ks.append(K)
        Un = V + dt / 6.0 * (Ks[0] + 2.0 * Ks[1] + 2.0 * Ks[2] + Ks[3])
        return Un, ys, exts

    def _G_T(self, ext, kappa, gchi):
        """J_G(Y)^T kappa (register layout) from Y's synchronised extended arrays; the mask part
        is added to gchi."""
        m = self.mats
        M, g = self.fo.M, G_RHS
        de = np.zeros((4, m.nb, m.ne, m.ne, m.ne))
        for leaf, s in self.fo.leaves.items():
            e = np.nan_to_num(ext[s], nan=0.0)     # points the right-hand side does not read
            d, dc = rhs_block_vjp(e, g, M, self.fo.h(leaf[0]), self.ph, kappa[s],
                                  chi=self.S.chi.get(s), chisp=self.S.chisp.get(s))
            de[:, m.pos[s]] = d
            if dc is not None:
                gchi[s] += dc
        flat = de.reshape(4, -1)
        v = np.stack([m.S.T @ flat[f] for f in range(4)])
        return m.to_reg(v, np.zeros_like(kappa))

    def _step_adjoint(self, U, lam, gchi):
        """lam (dJ/dU') -> dJ/dU through one step from U; mask contributions into gchi."""
        dt = self.dt
        _, ys, exts = self._step(U)
        nu4 = self._G_T(exts[3], dt / 6.0 * lam, gchi)
        nu3 = self._G_T(exts[2], dt / 3.0 * lam + dt * nu4, gchi)
        nu2 = self._G_T(exts[1], dt / 3.0 * lam + 0.5 * dt * nu3, gchi)
        nu1 = self._G_T(exts[0], dt / 6.0 * lam + 0.5 * dt * nu2, gchi)
        m = self.mats
        tot = m.to_vec(lam + nu1 + nu2 + nu3 + nu4)
        v = np.stack([m.W.T @ tot[f] for f in range(4)])
        return m.to_reg(v, np.zeros_like(lam))

    def forward(self, U0):
        """J and the checkpoints {n: U_n} for n = 0, c, 2c, ... (< N)."""
        U = U0.copy()
        ckpt = {0: U.copy()}
        J = 0.0
        for n in range(1, self.N + 1):
            U, _, _ = self._step(U)
            F, E = self.objective_terms(U)
            J += (F + self.we * E) / self.N
            if n % self.c == 0 and n < self.N:
                ckpt[n] = U.copy()
        return J, ckpt

    def gradient(self, U0, store_all=False, snapshots=None):
        """(J, dJ/dU_0 in the register layout, dJ/d(cx, cy, cz, R)).  store_all keeps every
        state instead of recomputing segments (the same arithmetic, for comparison); snapshots
        = S reverses with S stored states by binomial checkpointing (``oracle.checkpointing``;
        the count of recomputed steps is left in ``last_advances``)."""
        if snapshots is not None:
            return self._gradient_binomial(U0, snapshots)
        c = 1 if store_all else self.c
        saved_c, self.c = self.c, c
        J, ckpt = self.forward(U0)
        self.c = saved_c
        gchi = {s: np.zeros_like(self.S.chi[s]) for s in self.fo.leaves.values()}
        lam = np.zeros_like(U0)
        starts = sorted(ckpt)
        ends = starts[1:] + [self.N]
        for a, b in reversed(list(zip(starts, ends))):
            # recompute U_a .. U_b within the segment from its checkpoint
            states = [ckpt[a]]
            for _ in range(a, b):
                states.append(self._step(states[-1])[0])
            if b == self.N:
                self._dJ_dU(states[-1], lam, gchi)
            for n in range(b - 1, a - 1, -1):
                lam = self._step_adjoint(states[n - a], lam, gchi)
                if n >= 1:
                    self._dJ_dU(states[n - a], lam, gchi)
        return J, lam, self._theta(gchi)

    def vjp(self, U0, lamN, snapshots=None):
        """The vector-Jacobian product of the N-step map U_0 -> U_N: for L = <lamN, U_N> (lamN in
        the register layout) returns (U_N, dL/dU_0, dL/d(cx, cy, cz, R)).  The backward sweep is
        the gradient's without the objective's direct terms, from lam = lamN; the states are
        recomputed with `snapshots` stored states (default: all of them)."""
        N = self.N
        gchi = {s: np.zeros_like(U0[s][0]) for s in self.fo.leaves.values()}
        st = {"lam": lamN.copy(), "UN": None}

        def advance(U, k):
            return self._step(U)[0]

        def turn(U, k):
            if k == N - 1:
                st["UN"] = self._step(U)[0]
            st["lam"] = self._step_adjoint(U, st["lam"], gchi)

        self.last_advances = reverse(N, snapshots or N, U0, advance, turn)
        return st["UN"], st["lam"], self._theta(gchi)

    def _theta(self, gchi):
        """dJ/d(cx, cy, cz, R) from the mask gradient (zero without a sphere: centre None)."""
        gtheta = np.zeros(4)
        if self.centre is None:
            return gtheta
        for leaf, s in self.fo.leaves.items():
            X, Y, Z = acm.block_coords(self.fo, leaf)
            dchi = sphere_mask_grad(X, Y, Z, self.centre, self.R, self.delta)
            gtheta += (dchi * gchi[s]).reshape(4, -1).sum(axis=1)
        return gtheta

    def _gradient_binomial(self, U0, snapshots):
        """The gradient with the states recomputed by binomial checkpointing: the objective's
        terms are summed when a state is first reached (U_1 .. U_N in order), the adjoint steps
        run N-1 .. 0 as in the segment sweep."""
        N = self.N
        gchi = {s: np.zeros_like(self.S.chi[s]) for s in self.fo.leaves.values()}
        st = {"lam": np.zeros_like(U0), "J": 0.0, "hi": 0}

        def reached(U, k):
            if k > st["hi"]:
                F, E = self.objective_terms(U)
                st["J"] += (F + self.we * E) / N
                st["hi"] = k

        def advance(U, k):
            U1 = self._step(U)[0]
            reached(U1, k + 1)
            return U1

        def turn(U, k):
            if k == N - 1:
                UN = self._step(U)[0]
                reached(UN, N)
                self._dJ_dU(UN, st["lam"], gchi)
            st["lam"] = self._step_adjoint(U, st["lam"], gchi)
            if k >= 1:
                self._dJ_dU(U, st["lam"], gchi)

        self.last_advances = reverse(N, snapshots, U0, advance, turn)
        return st["J"], st["lam"], self._theta(gchi)
