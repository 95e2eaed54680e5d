"""Ghost-node values on the redundant block grid (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 4.2: each block carries n_g ghost layers that overlap its neighbours; during
synchronisation the data are restricted (decimated) or predicted as needed and copied into
the ghost layers.  Sec. 3.1 fixes the two operators: decimation u_i^J = u_{2i}^{J+1} and the
DD-4 prediction.  The precise interface rules are in the paper's unavailable Appendix B; this
module writes out the reading used throughout:

* Point value of the level-J lattice.  V_J(p) is the value that the finest leaf containing the
  point p (as one of its grid points) holds there, searching leaves of level >= J.  A level-J
  lattice point is a grid point of every leaf of level >= J whose closed box contains it, so
  this is a copy (same level) or a decimation (finer leaf).  Redundant points shared by leaves
  of the same level hold bitwise equal values, so any of them may be taken.
* If no leaf of level >= J contains p, V_J(p) is the tensor-product DD-4 prediction of V_{J-1}
  on the coarse lattice (even coordinates): along x, then y, then z.
* Synchronisation of a register: (1) every leaf's own boundary points that a finer leaf also
  holds take the finer value ("fine wins"); (2) every block's extended array (interior plus
  g ghost layers) is filled with V_J at its points.

The lookup is done on whole arrays of points at once with dense per-level leaf tables; it is
slow but each step is the definition above.
"""
from __future__ import annotations

import numpy as np

from .mra import DD4


class PointValues:
    """V_J(p) for arrays of level-J lattice points, for one register ``F[slot, f, z, y, x]``."""

    def __init__(self, forest, F):
        self.fo = forest
        self.F = F
        self.tabs = forest.leaf_lookup_tables()
        self.levels = sorted(self.tabs)

    def _leaf_at_level(self, L, PL):
        """For points PL (n,3) on the level-L lattice: slot and local index of a level-L leaf
        holding the point (slot -1 where none)."""
        fo = self.fo
        M = fo.M
        nb = np.array(fo.nblocks(L))
        NL = np.array(fo.npoints(L))
        PL = np.mod(PL, NL)
        base = PL // M
        on = (PL % M) == 0
        slot = -np.ones(PL.shape[0], dtype=np.int64)
        loc = np.zeros_like(PL)
        tab = self.tabs[L]
        for c in range(8):
            off = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
            valid = np.all(on | (off == 0), axis=1)
            b = np.mod(base - off, nb)
            lc = PL - (base - off) * M            # in [0, M]
            s = tab[b[:, 2], b[:, 1], b[:, 0]]
            take = (slot < 0) & valid & (s >= 0)
            slot[take] = s[take]
            loc[take] = lc[take]
        return slot, loc

    def finest(self, J, P, min_level=None):
        """Values of the finest leaf of level >= min_level (default J) holding each level-J
        point; NaN rows where there is none.  Returns (values (n,4), level (n,))."""
        min_level = J if min_level is None else min_level
        n = P.shape[0]
        vals = np.full((n, self.F.shape[1]), np.nan)
        lev = -np.ones(n, dtype=np.int64)
        todo = np.ones(n, dtype=bool)
        for L in sorted((l for l in self.levels if l >= min_level), reverse=True):
            if not todo.any():
                break
            idx = np.nonzero(todo)[0]
            PL = P[idx] * (1 << (L - J)) if L >= J else None
            if PL is None:
                continue
            slot, loc = self._leaf_at_level(L, PL)
            hit = slot >= 0
            if hit.any():
                ii = idx[hit]
                s, lc = slot[hit], loc[hit]
                vals[ii] = self.F[s, :, lc[:, 2], lc[:, 1], lc[:, 0]]
                lev[ii] = L
                todo[ii] = False
        return vals, lev

    def value(self, J, P):
        """V_J(P) for points P (n,3) (x, y, z order) of the level-J lattice."""
        P = np.mod(np.asarray(P, dtype=np.int64), np.array(self.fo.npoints(J)))
        # each distinct lattice point is looked up once
        N = np.array(self.fo.npoints(J), dtype=np.int64)
        key = P[:, 0] + N[0] * (P[:, 1] + N[1] * P[:, 2])
        ukey, inv = np.unique(key, return_inverse=True)
        Pu = np.stack([ukey % N[0], (ukey // N[0]) % N[1], ukey // (N[0] * N[1])], axis=1)
        vals, _ = self.finest(J, Pu)
        miss = np.isnan(vals[:, 0])
        if miss.any():
            vals[miss] = self.predicted(J, Pu[miss])
        return vals[inv.ravel()]

    def predicted(self, J, P):
        """Tensor DD-4 prediction of V_{J-1} at level-J points P: x, then y, then z."""
        n = P.shape[0]
        nf = self.F.shape[1]
        # per axis 4 coarse coordinates and weights; an even coordinate is a copy
        co = np.zeros((n, 3, 4), dtype=np.int64)
        w = np.zeros((n, 3, 4))
        for a in range(3):
            p = P[:, a]
            odd = (p % 2) == 1
            for j, dj in enumerate((-3, -1, 1, 3)):
                co[:, a, j] = np.where(odd, (p + dj) // 2, p // 2)
                w[:, a, j] = np.where(odd, DD4[j], 1.0 if j == 0 else 0.0)
        Q = np.empty((n, 4, 4, 4, 3), dtype=np.int64)   # [n, kz, ky, kx, axis]
        for kz in range(4):
            for ky in range(4):
                for kx in range(4):
                    Q[:, kz, ky, kx, 0] = co[:, 0, kx]
                    Q[:, kz, ky, kx, 1] = co[:, 1, ky]
                    Q[:, kz, ky, kx, 2] = co[:, 2, kz]
        cv = self.value(J - 1, Q.reshape(-1, 3)).reshape(n, 4, 4, 4, nf)
        # along x
        vx = np.zeros((n, 4, 4, nf))
        for kx in range(4):
            vx = vx + w[:, 0, kx][:, None, None, None] * cv[:, :, :, kx, :]
        vy = np.zeros((n, 4, nf))
        for ky in range(4):
            vy = vy + w[:, 1, ky][:, None, None] * vx[:, :, ky, :]
        vz = np.zeros((n, nf))
        for kz in range(4):
            vz = vz + w[:, 2, kz][:, None] * vy[:, kz, :]
        return vz


def local_points(M, g, which="cube"):
    """Local indices (n,3) x,y,z of an extended block: 'cube' = all of [-g, M+g]^3,
    'faces' = interior plus the six face slabs of depth g (no edges or corners)."""
    r = np.arange(-g, M + g + 1)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    P = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    if which == "faces":
        out = ((P < 0) | (P > M)).sum(axis=1)
        P = P[out <= 1]
    return P


def fine_wins(forest, F):
    """Step (1) of the synchronisation: each leaf's boundary points take the value of the
    finest strictly finer leaf holding them.  Modifies F in place; returns F."""
    M = forest.M
    pv = PointValues(forest, F.copy())
    Pl = local_points(M, 0, "cube")
    bnd = Pl[((Pl == 0) | (Pl == M)).any(axis=1)]
    for (J, gx, gy, gz), s in forest.leaves.items():
        if J >= pv.levels[-1]:
            continue
        P = bnd + np.array([gx, gy, gz]) * M
        vals, _ = pv.finest(J, P, min_level=J + 1)
        hit = ~np.isnan(vals[:, 0])
        if hit.any():
            b = bnd[hit]
            F[s, :, b[:, 2], b[:, 1], b[:, 0]] = vals[hit]
    return F


def sync(forest, F, g, which="cube"):
    """Synchronise register F: fine-wins update of F (in place), then the extended arrays.

    Returns ``ext`` of shape (max_slot+1, nf, M+1+2g, M+1+2g, M+1+2g); points outside
    ``which`` are NaN.  Interior points of ext equal F after step (1)."""
    M = forest.M
    fine_wins(forest, F)
    pv = PointValues(forest, F)
    Pl = local_points(M, g, which)
    n = M + 1 + 2 * g
    leaves = list(forest.leaves.items())
    nslot = max(s for _, s in leaves) + 1 if leaves else 0
    ext = np.full((nslot, F.shape[1], n, n, n), np.nan)
    # batch all blocks of one level together
    for J in sorted({l[0][0] for l in leaves}):
        blk = [(l, s) for l, s in leaves if l[0] == J]
        P = np.concatenate([Pl + np.array(l[1:]) * M for l, _ in blk], axis=0)
        vals = pv.value(J, P)
        k = Pl.shape[0]
        for i, (_, s) in enumerate(blk):
            v = vals[i * k:(i + 1) * k]
            ext[s, :, Pl[:, 2] + g, Pl[:, 1] + g, Pl[:, 0] + g] = v   # (n, nf): advanced indices first
    return ext


def redundant_points_consistent(forest, F):
    """True iff every lattice point held by several leaves of the same level has bitwise equal
    values in all of them (the invariant the synchronisation relies on)."""
    M = forest.M
    seen = {}
    Pl = local_points(M, 0, "cube")
    bnd = Pl[((Pl == 0) | (Pl == M)).any(axis=1)]
    for (J, gx, gy, gz), s in forest.leaves.items():
        NL = np.array(forest.npoints(J))
        P = np.mod(bnd + np.array([gx, gy, gz]) * M, NL)
        v = F[s, :, bnd[:, 2], bnd[:, 1], bnd[:, 0]]     # (n, nf)
        for i in range(P.shape[0]):
            key = (J,) + tuple(P[i])
            if key in seen:
                if not np.array_equal(seen[key], v[i]):
                    return False
            else:
                seen[key] = v[i]
    return True
