"""Binomial checkpointing of a reverse sweep over time steps (oracle).

Test infrastructure only (see ``oracle/__init__``).

The adjoint of N steps U_{k+1} = Phi_k(U_k) visits the states in the order U_{N-1}, ..., U_0.
With room for S stored states (snapshots; one of them holds U_0 for the whole sweep) the states
are recomputed from stored ones.  The recursion below is binomial checkpointing (Griewank,
"Achieving logarithmic growth of temporal and spatial complexity in reverse automatic
differentiation", 1992; Griewank and Walther, revolve, ACM TOMS 26, 2000): to reverse the steps
a..b-1 from U_a (stored) with F further free snapshots,

* one step (b = a + 1): take the step and its adjoint from U_a (a "turn");
* no free snapshot: for k = b-1 down to a, advance U_a to U_k and turn;
* otherwise advance to U_m for some a < m < b, store it, reverse m..b-1 with F - 1 free
  snapshots, restore U_a and reverse a..m-1 with the F free snapshots again.

The number of plain forward steps ("advances", turns not counted) is minimal when m minimises
m - a + C(b - m, F - 1) + C(m - a, F), with C(1, .) = 0 and C(n, 0) = n (n - 1) / 2.  Here the
minimum is found by brute force over every m (``min_advances``); the split is the smallest
minimiser.  The paper has no adjoint; this is the memory-bounded variant of the checkpointing
its adjoint extension uses.
"""
from __future__ import annotations

from functools import lru_cache


@lru_cache(maxsize=None)
def _cost(n, free):
    """Fewest advances to reverse n steps from a stored first state with `free` more snapshots,
    and the smallest split achieving it (0 where no split is made)."""
    if n <= 1:
        return 0, 0
    if free == 0:
        return n * (n - 1) // 2, 0
    best, arg = None, 0
    for m in range(1, n):
        c = m + _cost(n - m, free - 1)[0] + _cost(m, free)[0]
        if best is None or c < best:
            best, arg = c, m
    return best, arg


def min_advances(n, snapshots):
    """Fewest forward steps (turns excluded) that reverse n steps with `snapshots` stored states,
    U_0's included, by the brute-force recursion."""
    if n < 1 or snapshots < 1:
        raise ValueError("need n >= 1 and at least one snapshot")
    return _cost(n, snapshots - 1)[0]


def schedule(n, snapshots):
    """The reversal as a list of actions: ("store", j) keeps the current state in snapshot j,
    ("restore", j) makes snapshot j current, ("advance", k) takes the plain step k -> k + 1,
    ("turn", k) takes step k with its adjoint (the current state is used up)."""
    if n < 1 or snapshots < 1:
        raise ValueError("need n >= 1 and at least one snapshot")
    out = [("store", 0)]

    def rev(a, b, home, free):
        # the current state is U_a, also held in snapshot `home`
        if b - a == 1:
            out.append(("turn", a))
            return
        if not free:
            for k in range(b - 1, a - 1, -1):
                if k < b - 1:
                    out.append(("restore", home))
                out.extend(("advance", i) for i in range(a, k))
                out.append(("turn", k))
            return
        m = a + _cost(b - a, len(free))[1]
        out.extend(("advance", i) for i in range(a, m))
        out.append(("store", free[0]))
        rev(m, b, free[0], free[1:])
        out.append(("restore", home))
        rev(a, m, home, free)

    rev(0, n, 0, list(range(1, snapshots)))
    return out


def reverse(n, snapshots, U0, advance, turn):
    """Run the reversal on states: advance(U, k) -> U_{k+1}; turn(U, k) takes step k's adjoint
    from U_k.  Returns the number of advances taken."""
    snaps = {}
    cur = U0.copy()
    count = 0
    for op, k in schedule(n, snapshots):
        if op == "store":
            snaps[k] = cur.copy()
        elif op == "restore":
            cur = snaps[k].copy()
        elif op == "advance":
            cur = advance(cur, k)
            count += 1
        else:
            turn(cur, k)
            cur = None
    return count
