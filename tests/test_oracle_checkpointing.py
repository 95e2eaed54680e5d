"""Pins of the oracle's binomial checkpointing (the adjoint's reverse sweep; an extension).

The brute-force recursion's minimum is pinned by the closed form of Griewank's theorem: with S
snapshots and r the least integer with C(S + r, S) >= n, reversing n steps takes r n -
C(S + r, r - 1) forward steps besides the n taped ones.  The schedule is pinned by simulating it
on step indices: every step's adjoint is taken once, from its own state, in the order n-1 .. 0,
with at most S snapshots, U_0 never overwritten, and exactly the minimal number of advances.
"""
from math import comb

import numpy as np
import pytest

from oracle.checkpointing import min_advances, reverse, schedule


def _closed_form(n, S):
    r = 0
    while comb(S + r, S) < n:
        r += 1
    return r * n - (comb(S + r, r - 1) if r >= 1 else 0)


def simulate(actions, n, S):
    """Replays a schedule on step indices; returns the number of advances."""
    snaps, cur, expect, adv = {}, 0, n - 1, 0
    for i, (op, k) in enumerate(actions):
        if op == "store":
            assert 0 <= k < S and cur is not None
            assert k != 0 or (i == 0 and cur == 0)       # U_0's snapshot is written once, first
            snaps[k] = cur
        elif op == "restore":
            assert k in snaps
            cur = snaps[k]
        elif op == "advance":
            assert cur == k and k < n - 1
            cur, adv = k + 1, adv + 1
        else:
            assert op == "turn" and cur == k == expect
            cur, expect = None, expect - 1
    assert expect == -1
    return adv


@pytest.mark.parametrize("S", range(1, 9))
def test_minimum_is_the_binomial_closed_form(S):
    for n in range(1, 41):
        assert min_advances(n, S) == _closed_form(n, S), (n, S)
    assert min_advances(7, 1) == 21                        # U_0 only: 0 + 1 + ... + 6
    assert min_advances(9, 9) == 8                         # room for every state


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 21, 34])
def test_schedule_reverses_every_step_with_the_fewest_advances(n):
    for S in range(1, 7):
        assert simulate(schedule(n, S), n, S) == min_advances(n, S)


def test_reverse_runs_the_schedule_on_states():
    seen = []
    U0 = np.zeros(1)
    count = reverse(6, 2, U0, lambda U, k: U + 1.0, lambda U, k: seen.append((k, float(U[0]))))
    assert seen == [(k, float(k)) for k in range(5, -1, -1)]
    assert count == min_advances(6, 2) == _closed_form(6, 2)
