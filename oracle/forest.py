"""Block forest of the oracle: treecodes, leaves, slot map and neighbour tables.

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 4.1: all blocks hold Bs^D points, live in one preallocated contiguous array, and
their position in the tree is an octal (Gargantini) number from which level, position and
neighbour ids are computed.  Sec. 3.1: the nested grids x_i^J = i/2^J have an odd number of
points and x_{2i}^{J+1} = x_i^J, so neighbouring blocks share their face points (redundant grid).

Readings of what the paper leaves open (its Appendix B is not available):

* A block at level J with global block coordinates (gx, gy, gz) covers the closed box
  [g*M*h_J, (g+1)*M*h_J] per axis, M = Bs-1, h_J = L_root / (2^J M).  Its point i sits at
  global lattice index g*M + i of level J.  All domains are periodic.
* Treecode: digit c = bx + 2 by + 4 bz per level (x fastest), packed most significant level
  first, 3 bits per level for 18 levels, root number in bits 56..63; the level is kept apart.
* Ordering key of a block: (treecode, level); listing order of the API is ascending key.
* Slots: in one adaptation pass the slots of removed blocks are returned first, then the new
  blocks, in ascending key order, each take the lowest free slot.
* Neighbour table: 26 directions in the order produced by iterating dz, dy, dx over -1, 0, 1
  (x fastest), split into faces, edges, corners in that order.  Per block 56 slot entries:
  face k -> [4k, 4k+4), edge k -> 24 + [2k, 2k+2), corner k -> 48 + k; plus 26 relative levels
  (0 same, -1 coarser, +1 finer).  A same-level or coarser neighbour fills the first entry of
  its group; finer neighbours fill the group with the touching children in ascending child
  number c = cx + 2 cy + 4 cz.  Unused entries are -1.
* Grading: 26-neighbour 2:1 balance.
"""
from __future__ import annotations

import itertools

import numpy as np

ROOT_SHIFT = 56
LEVEL_BITS = 18


def _directions():
    faces, edges, corners = [], [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                n = abs(dx) + abs(dy) + abs(dz)
                if n == 1:
                    faces.append((dx, dy, dz))
                elif n == 2:
                    edges.append((dx, dy, dz))
                elif n == 3:
                    corners.append((dx, dy, dz))
    return faces + edges + corners


DIRECTIONS = _directions()          # 26 tuples (dx, dy, dz)


def group_start(k):
    """First entry of direction k in the 56-entry neighbour table and the group size."""
    if k < 6:
        return 4 * k, 4
    if k < 18:
        return 24 + 2 * (k - 6), 2
    return 48 + (k - 18), 1


def touching_children(d):
    """Child numbers c = cx + 2cy + 4cz of the box at offset d that touch the block, ascending."""
    out = []
    for c in range(8):
        cc = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        ok = True
        for a in range(3):
            if d[a] == 1 and cc[a] != 0:
                ok = False
            if d[a] == -1 and cc[a] != 1:
                ok = False
        if ok:
            out.append(c)
    return out


class Forest:
    """Leaves of the block tree, their slots, and the grid geometry."""

    def __init__(self, nroot=(1, 1, 1), root_len=1.0, Bs=17, Jmin=0, Jmax=18, max_blocks=1 << 20):
        assert Bs % 2 == 1 and Bs >= 5
        self.nroot = tuple(int(n) for n in nroot)
        self.root_len = float(root_len)
        self.Bs = int(Bs)
        self.M = self.Bs - 1
        self.Jmin, self.Jmax = int(Jmin), int(Jmax)
        self.max_blocks = int(max_blocks)
        self.leaves: dict[tuple, int] = {}     # (J, gx, gy, gz) -> slot
        self.free = list(range(self.max_blocks))  # kept sorted ascending

    # ---- geometry -------------------------------------------------------------------------
    def nblocks(self, J):
        return tuple(n << J for n in self.nroot)

    def h(self, J):
        return self.root_len / ((1 << J) * self.M)

    def npoints(self, J):
        """Points per axis of the periodic level-J lattice."""
        return tuple(n * self.M for n in self.nblocks(J))

    def wrap(self, J, g):
        nb = self.nblocks(J)
        return tuple(int(g[a]) % nb[a] for a in range(3))

    # ---- treecode -------------------------------------------------------------------------
    def treecode(self, J, g):
        rx, ry, rz = (g[0] >> J, g[1] >> J, g[2] >> J)
        root = rx + self.nroot[0] * (ry + self.nroot[1] * rz)
        code = root << ROOT_SHIFT
        for l in range(1, J + 1):
            sh = J - l
            c = ((g[0] >> sh) & 1) | (((g[1] >> sh) & 1) << 1) | (((g[2] >> sh) & 1) << 2)
            code |= c << (3 * (LEVEL_BITS - l))
        return code

    def decode(self, code, J):
        root = code >> ROOT_SHIFT
        rx = root % self.nroot[0]
        ry = (root // self.nroot[0]) % self.nroot[1]
        rz = root // (self.nroot[0] * self.nroot[1])
        b = [0, 0, 0]
        for l in range(1, J + 1):
            c = (code >> (3 * (LEVEL_BITS - l))) & 7
            for a in range(3):
                b[a] = (b[a] << 1) | ((c >> a) & 1)
        return (rx * (1 << J) + b[0], ry * (1 << J) + b[1], rz * (1 << J) + b[2])

    def key(self, leaf):
        J, gx, gy, gz = leaf
        return (self.treecode(J, (gx, gy, gz)), J)

    def sorted_leaves(self):
        return sorted(self.leaves, key=self.key)

    # ---- slots ----------------------------------------------------------------------------
    def _alloc(self):
        if not self.free:
            raise MemoryError("slot pool exhausted")
        return self.free.pop(0)

    def _release(self, slot):
        self.free.append(slot)
        self.free.sort()

    def apply_pass(self, removed, created):
        """One adaptation pass: free the slots of ``removed`` leaves, then give the ``created``
        leaves the lowest free slots in ascending key order.  Returns {leaf: slot} of created."""
        if len(created) - len(removed) > len(self.free):
            raise MemoryError("slot pool exhausted")
        for leaf in removed:
            self._release(self.leaves.pop(leaf))
        out = {}
        for leaf in sorted(created, key=self.key):
            s = self._alloc()
            self.leaves[leaf] = s
            out[leaf] = s
        return out

    def set_leaves(self, leaves):
        """Start from an empty pool and create ``leaves`` (J, gx, gy, gz) in one pass."""
        self.leaves.clear()
        self.free = list(range(self.max_blocks))
        self.apply_pass([], [tuple(int(v) for v in l) for l in leaves])

    def init_uniform(self, J):
        self.leaves.clear()
        self.free = list(range(self.max_blocks))
        nb = self.nblocks(J)
        created = [(J, x, y, z) for z in range(nb[2]) for y in range(nb[1]) for x in range(nb[0])]
        self.apply_pass([], created)

    # ---- topology queries -----------------------------------------------------------------
    def is_leaf(self, J, g):
        return (J,) + self.wrap(J, g) in self.leaves

    def box_status(self, J, g):
        """Status of the level-J box g: ('leaf', slot) | ('coarser', slot, octant) |
        ('refined', {child: slot}) -- children listed only where they are leaves."""
        g = self.wrap(J, g)
        if (J,) + g in self.leaves:
            return ("leaf", self.leaves[(J,) + g])
        if J > 0:
            p = (g[0] >> 1, g[1] >> 1, g[2] >> 1)
            if (J - 1,) + p in self.leaves:
                octant = (g[0] & 1, g[1] & 1, g[2] & 1)
                return ("coarser", self.leaves[(J - 1,) + p], octant)
        kids = {}
        for c in range(8):
            cg = (2 * g[0] + (c & 1), 2 * g[1] + ((c >> 1) & 1), 2 * g[2] + ((c >> 2) & 1))
            if (J + 1,) + cg in self.leaves:
                kids[c] = self.leaves[(J + 1,) + cg]
        if kids:
            return ("refined", kids)
        return ("none",)

    def neighbour_table(self, order=None):
        """(nbr[N,56] int32, rel[N,26] int8) in ``order`` (default: ascending key)."""
        order = self.sorted_leaves() if order is None else order
        nbr = -np.ones((len(order), 56), dtype=np.int32)
        rel = np.zeros((len(order), 26), dtype=np.int8)
        for i, leaf in enumerate(order):
            J, g = leaf[0], leaf[1:]
            for k, d in enumerate(DIRECTIONS):
                st = self.box_status(J, (g[0] + d[0], g[1] + d[1], g[2] + d[2]))
                s0, n = group_start(k)
                if st[0] == "leaf":
                    nbr[i, s0] = st[1]
                    rel[i, k] = 0
                elif st[0] == "coarser":
                    nbr[i, s0] = st[1]
                    rel[i, k] = -1
                elif st[0] == "refined":
                    tc = touching_children(d)
                    assert len(tc) == n
                    for j, c in enumerate(tc):
                        if c not in st[1]:
                            raise ValueError("grid is not 2:1 graded")
                        nbr[i, s0 + j] = st[1][c]
                    rel[i, k] = 1
                else:
                    raise ValueError("grid is not 2:1 graded")
        return nbr, rel

    def topology(self):
        """Arrays listed in ascending key order: treecode u64, level u8, slot i32, nbr, rel."""
        order = self.sorted_leaves()
        tc = np.array([self.treecode(l[0], l[1:]) for l in order], dtype=np.uint64)
        lv = np.array([l[0] for l in order], dtype=np.uint8)
        sl = np.array([self.leaves[l] for l in order], dtype=np.int32)
        nbr, rel = self.neighbour_table(order)
        return tc, lv, sl, nbr, rel

    # ---- structural checks (used by tests) ------------------------------------------------
    def box_int(self, leaf, Jref):
        """Integer box [lo, hi) of a leaf on the level-Jref block grid (Jref >= leaf level)."""
        J = leaf[0]
        s = 1 << (Jref - J)
        return tuple((leaf[1 + a] * s, (leaf[1 + a] + 1) * s) for a in range(3))

    def is_graded(self):
        for leaf in self.leaves:
            J, g = leaf[0], leaf[1:]
            for d in DIRECTIONS:
                st = self.box_status(J, (g[0] + d[0], g[1] + d[1], g[2] + d[2]))
                if st[0] == "none":
                    return False
                if st[0] == "refined" and len(st[1]) != 8:
                    # a finer neighbour box must consist of leaves only where it touches
                    if any(c not in st[1] for c in touching_children(d)):
                        return False
        return True

    def covers_domain_exactly(self):
        Jref = max(l[0] for l in self.leaves)
        nb = self.nblocks(Jref)
        total = 0
        for leaf in self.leaves:
            total += (1 << (Jref - leaf[0])) ** 3
        if total != nb[0] * nb[1] * nb[2]:
            return False
        occ = np.zeros(nb[::-1], dtype=np.int32)
        for leaf in self.leaves:
            (x0, x1), (y0, y1), (z0, z1) = self.box_int(leaf, Jref)
            occ[z0:z1, y0:y1, x0:x1] += 1
        return bool((occ == 1).all())

    def sister_groups(self):
        """Parents (J-1, p) whose 8 children are all leaves."""
        cnt = {}
        for (J, gx, gy, gz) in self.leaves:
            if J > 0:
                p = (J - 1, gx >> 1, gy >> 1, gz >> 1)
                cnt[p] = cnt.get(p, 0) + 1
        return sorted([p for p, n in cnt.items() if n == 8], key=self.key)

    @staticmethod
    def children_of(parent):
        J, gx, gy, gz = parent
        return [(J + 1, 2 * gx + (c & 1), 2 * gy + ((c >> 1) & 1), 2 * gz + ((c >> 2) & 1))
                for c in range(8)]

    def leaf_lookup_tables(self):
        """Dense per-level arrays [nz, ny, nx] of leaf slots (-1 where no leaf)."""
        levels = sorted({l[0] for l in self.leaves})
        tabs = {}
        for J in range(min(levels), max(levels) + 1):
            nb = self.nblocks(J)
            tabs[J] = -np.ones(nb[::-1], dtype=np.int64)
        for (J, gx, gy, gz), s in self.leaves.items():
            tabs[J][gz, gy, gx] = s
        return tabs


def brute_force_adjacency(forest):
    """Touching leaf pairs by box geometry alone (O(N^2)), periodic: {leaf: set(leaves)}."""
    leaves = list(forest.leaves)
    Jref = max(l[0] for l in leaves)
    nb = forest.nblocks(Jref)
    boxes = {l: forest.box_int(l, Jref) for l in leaves}
    out = {l: set() for l in leaves}
    for a, b in itertools.combinations(leaves, 2):
        touch = True
        for ax in range(3):
            (a0, a1), (b0, b1) = boxes[a][ax], boxes[b][ax]
            n = nb[ax]
            ok = False
            for sh in (-n, 0, n):
                if b0 + sh <= a1 and a0 <= b1 + sh:
                    ok = True
            if not ok:
                touch = False
                break
        if touch:
            out[a].add(b)
            out[b].add(a)
    return out
