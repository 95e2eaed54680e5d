"""Time stepping and grid adaptation of the oracle: the refine / evolve / coarsen cycle (FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 3.5: one time step (1) refines every block by one level (up to J_max), filling the
children by prediction, (2) advances eqs. (u_eqn-1, p_eqn-1) with RK4 on that grid, (3) computes
the details of every block, tags blocks whose largest normalised detail is below C_eps, drops
tags that would break the grading, merges tagged sister groups, and repeats (3) until nothing
changes.  With the dealiasing option, blocks at J_max are always tagged; blocks whose mask
varies (max chi - min chi > thr) keep their level unless dealiasing forces the tag.  The
initial grid starts at J_min and repeats {refine all, evaluate the initial condition and the
mask, coarsen} until the grid no longer changes.  Sec. 3.3: a block is coarsened only if all
its details are below C_eps, with each component normalised by its global L-infinity norm
(Sec. 3.4).  Sec. 2.3: classical RK4.

Readings: the norms are taken once per coarsening phase, before its first pass; a component
with zero norm is skipped; the mask-range threshold is 1e-5.  Merging is decimation with the
CDF 4/0 wavelet.  With CDF 4/4 (Sec. 3.2.1; the paper's choice for its later runs) the parent
takes the lifted analysis low-pass h~ of the level-(J+1) point values V_{J+1} (the values the
ghost synchronisation defines, so the 4 fine points outside the sister group come from its
neighbours) at its interior points; its boundary points keep the decimated value.  The
boundary reading keeps redundant points shared with a same-level leaf that is not merged in
the same pass bitwise equal in both blocks (that leaf holds the decimated value after fine
wins), and the 13-tap filter then needs 4 fine ghost layers, not 6.
"""
from __future__ import annotations

import numpy as np

from . import acm
from .forest import DIRECTIONS, Forest
from .mra import block_details, cdf44_lowpass, lowpass_decimate_axis, predict_3d
from .sync import PointValues, local_points, sync


class Solver:
    """State of one simulation: forest, register U (slot-indexed) and the analytic mask."""

    def __init__(self, forest: Forest, ph: acm.Physics, eps=1e-3, dealias=True,
                 mask_thr=1e-5, ic=None, mask=None, sponge=None, wavelet="cdf40", coarsen_everywhere=False):
        assert wavelet in ("cdf40", "cdf44")
        self.wavelet = wavelet
        # the performance cycle of Sec. 5.4 ("coarsen everywhere" on random data): instead of
        # thresholding, every block made by the last refine_all is tagged, so coarsening
        # restores the grid the step started from (reading: a block goes back at most one level)
        self.coarsen_everywhere = coarsen_everywhere
        self.last_refined = set()
        self.fo = forest
        self.ph = ph
        self.eps, self.dealias, self.mask_thr = eps, dealias, mask_thr
        n = forest.Bs
        self.U = np.zeros((forest.max_blocks, 4, n, n, n))
        self.ic = ic            # callable (X, Y, Z) -> (4, ...)
        self.mask = mask        # callable (X, Y, Z) -> chi, or None
        self.sponge = sponge    # callable (X, Y, Z) -> chi_sp, or None
        self.chi = {}
        self.chisp = {}
        self.t = 0.0

    # ---- analytic fields -------------------------------------------------------------------
    def eval_ic(self, leaves=None):
        for leaf in (self.fo.leaves if leaves is None else leaves):
            X, Y, Z = acm.block_coords(self.fo, leaf)
            self.U[self.fo.leaves[leaf]] = self.ic(X, Y, Z)

    def eval_mask(self):
        self.chi, self.chisp = {}, {}
        for leaf, s in self.fo.leaves.items():
            X, Y, Z = acm.block_coords(self.fo, leaf)
            if self.mask is not None:
                self.chi[s] = self.mask(X, Y, Z)
            if self.sponge is not None:
                self.chisp[s] = self.sponge(X, Y, Z)

    # ---- right-hand side and RK4 --------------------------------------------------------------
    def rhs(self, F):
        """K = RHS(F) for every leaf; F is synchronised in place first (fine wins)."""
        g = 3
        ext = sync(self.fo, F, g, "faces")
        K = np.zeros_like(F)
        for leaf, s in self.fo.leaves.items():
            h = self.fo.h(leaf[0])
            K[s] = acm.rhs_block(ext[s], g, self.fo.M, h, self.ph,
                                 chi=self.chi.get(s), chisp=self.chisp.get(s))
        return K

    def rk4(self, dt):
        U = self.U
        K1 = self.rhs(U)
        K2 = self.rhs(U + 0.5 * dt * K1)
        K3 = self.rhs(U + 0.5 * dt * K2)
        K4 = self.rhs(U + dt * K3)
        self.U = U + dt / 6.0 * (K1 + 2.0 * K2 + 2.0 * K3 + K4)
        self.t += dt

    # ---- reductions ---------------------------------------------------------------------------
    def slots(self):
        return np.array(sorted(self.fo.leaves.values()), dtype=np.int64)

    def u_max(self):
        s = self.slots()
        u = self.U[s]
        return float(np.sqrt(u[:, 0] ** 2 + u[:, 1] ** 2 + u[:, 2] ** 2).max())

    def norms(self):
        s = self.slots()
        return np.abs(self.U[s]).max(axis=(0, 2, 3, 4))

    def h_min(self):
        return self.fo.h(max(l[0] for l in self.fo.leaves))

    def dt_cfl(self):
        return acm.time_step(self.ph, self.u_max(), self.h_min(), self.mask is not None)

    # ---- details and flags -----------------------------------------------------------------
    def indicators(self, norms):
        """Per leaf: (largest normalised detail, range of chi), from the synchronised U."""
        g = 2
        ext = sync(self.fo, self.U, g, "cube")
        out = {}
        for leaf, s in self.fo.leaves.items():
            d = block_details(ext[s], g, self.fo.M)
            ind = 0.0
            for f in range(4):
                if norms[f] > 0.0:
                    ind = max(ind, float(np.abs(d[f]).max()) / norms[f])
            chi = self.chi.get(s)
            rng = 0.0 if chi is None else float(chi.max() - chi.min())
            out[leaf] = (ind, rng)
        return out, ext

    def tags(self, ind):
        tags = {}
        for leaf, (d, rng) in ind.items():
            J = leaf[0]
            t = False
            if J > self.fo.Jmin:
                if self.dealias and J == self.fo.Jmax:
                    t = True
                else:
                    t = (d < self.eps) and not (rng > self.mask_thr)
            tags[leaf] = t
        return tags

    def coarsenable_groups(self, tags):
        fo = self.fo
        out = []
        for parent in fo.sister_groups():
            kids = fo.children_of(parent)
            if not all(tags[k] for k in kids):
                continue
            ok = True
            for k in kids:
                J, g = k[0], k[1:]
                for d in DIRECTIONS:
                    st = fo.box_status(J, (g[0] + d[0], g[1] + d[1], g[2] + d[2]))
                    if st[0] == "refined":
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                out.append(parent)
        return out

    def lowpass_parent(self, parent, src):
        """CDF 4/4 values of ``parent`` at its interior points 1..M-1 (per axis), (4, M-1, M-1,
        M-1): V_{J+1} of the current forest on the fine points -4..2M+4 around the parent's
        box (parent point i sits at fine point 2i), low-passed along x, then y, then z."""
        fo = self.fo
        M = fo.M
        g = 4
        J, px, py, pz = parent
        Pl = local_points(2 * M, g, "cube")                 # x fastest, then y, then z
        P = Pl + 2 * M * np.array([px, py, pz])
        vals = PointValues(fo, src).value(J + 1, P)         # (n, 4)
        n = 2 * M + 1 + 2 * g
        e = np.moveaxis(vals.reshape(n, n, n, -1), -1, 0)   # (4, z, y, x)
        ht = cdf44_lowpass()
        a = lowpass_decimate_axis(e, -1, ht, g, M)
        a = lowpass_decimate_axis(a, -2, ht, g, M)
        return lowpass_decimate_axis(a, -3, ht, g, M)

    def merge(self, groups, src):
        """Replace each sister group by its parent; parent points are decimated children points
        taken from ``src`` (slot-indexed synchronised interiors); with CDF 4/4 the interior
        points then take the low-passed values (``lowpass_parent``, on the forest before the
        merge)."""
        fo = self.fo
        M = fo.M
        half = M // 2
        lp = {p: self.lowpass_parent(p, src) for p in groups} if self.wavelet == "cdf44" else {}
        old = {p: [fo.leaves[k] for k in fo.children_of(p)] for p in groups}
        removed = [k for p in groups for k in fo.children_of(p)]
        new = fo.apply_pass(removed, list(groups))
        i = np.arange(M + 1)
        c = (i > half).astype(int)          # child half holding parent point i
        li = 2 * (i - half * c)            # its index in that child
        CZ, CY, CX = np.meshgrid(c, c, c, indexing="ij")
        LZ, LY, LX = np.meshgrid(li, li, li, indexing="ij")
        cn = CX + 2 * CY + 4 * CZ          # child number per parent point
        for p in groups:
            kid_slots = np.array(old[p])
            P = src[kid_slots[cn], :, LZ, LY, LX]          # (z, y, x, 4)
            self.U[new[p]] = np.moveaxis(P, -1, 0)
            if p in lp:
                self.U[new[p]][:, 1:M, 1:M, 1:M] = lp[p]
        return new

    def coarsen(self, max_passes=64):
        norms = self.norms()
        npass = 0
        for _ in range(max_passes):
            if self.coarsen_everywhere:
                tags = {l: l[0] > 0 and (l[0] - 1, l[1] >> 1, l[2] >> 1, l[3] >> 1) in self.last_refined
                        for l in self.fo.leaves}
            else:
                ind, ext = self.indicators(norms)
                tags = self.tags(ind)
            groups = self.coarsenable_groups(tags)
            if not groups:
                break
            src = self.U.copy()
            self.merge(groups, src)
            self.eval_mask()
            npass += 1
        return npass

    def refine_all(self, analytic=False):
        """Split every leaf below J_max into 8 children; children are predicted from the
        synchronised parent (or evaluated analytically when ``analytic``)."""
        fo = self.fo
        M = fo.M
        half = M // 2
        parents = [l for l in fo.sorted_leaves() if l[0] < fo.Jmax]
        self.last_refined = set(parents)
        if not parents:
            return
        g = 2
        ext = None if analytic else sync(fo, self.U, g, "cube")
        old = {p: fo.leaves[p] for p in parents}
        created = [k for p in parents for k in fo.children_of(p)]
        new = fo.apply_pass(parents, created)
        if analytic:
            self.eval_ic(created)
        else:
            for p in parents:
                e = ext[old[p]]
                for c, k in enumerate(fo.children_of(p)):
                    o = [(c & 1) * half, ((c >> 1) & 1) * half, ((c >> 2) & 1) * half]
                    # parent samples o-1 .. o+half+1 along each axis (ext index +g)
                    sub = e[:, o[2] - 1 + g:o[2] + half + 2 + g, o[1] - 1 + g:o[1] + half + 2 + g,
                            o[0] - 1 + g:o[0] + half + 2 + g]
                    fine = predict_3d(sub)
                    self.U[new[k]] = fine[:, 2:2 + M + 1, 2:2 + M + 1, 2:2 + M + 1]
        self.eval_mask()

    # ---- the time step of Sec. 3.5 -------------------------------------------------------------
    def step(self, dt=None):
        self.refine_all()
        dt = self.dt_cfl() if dt is None else dt
        self.rk4(dt)
        self.coarsen()
        return dt

    def initial_grid(self, max_iter=32):
        fo = self.fo
        fo.init_uniform(fo.Jmin)
        self.eval_ic()
        self.eval_mask()
        for _ in range(max_iter):
            before = set(fo.leaves)
            self.refine_all(analytic=True)
            self.coarsen()
            if set(fo.leaves) == before:
                return
        raise RuntimeError("initial grid did not converge")

    # ---- diagnostics ------------------------------------------------------------------------------
    def diagnostics(self):
        """Force C_eta^{-1} sum chi (u - u_s) h^3 and energy 1/2 sum |u|^2 h^3 over the
        half-open points [0, Bs-2]^3 of every leaf (each physical point once)."""
        fo = self.fo
        M = fo.M
        F = np.zeros(3)
        E = 0.0
        for leaf, s in fo.leaves.items():
            h3 = fo.h(leaf[0]) ** 3
            u = self.U[s][:, :M, :M, :M]
            E += 0.5 * float((u[0] ** 2 + u[1] ** 2 + u[2] ** 2).sum()) * h3
            if s in self.chi:
                chi = self.chi[s][:M, :M, :M]
                for i in range(3):
                    F[i] += float((chi * u[i]).sum()) * h3 / self.ph.C_eta
        return F, E
