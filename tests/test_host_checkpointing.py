"""The library's checkpoint schedules (csrc/checkpoint.hpp, through acm_checkpoint_schedule; host
only, no GPU) replayed on step indices: every step's adjoint is taken once, from its own state,
in the order n-1 .. 0; snapshot indices stay within the reported count and the workspace's; U_0's
snapshot is written once, first; every state is first reached in the order U_1 .. U_n (where the
objective's terms are summed).  The binomial schedule takes exactly the oracle's brute-force
minimum of recomputed steps; the equidistant one recomputes every segment but the last once."""
import numpy as np
import pytest

from oracle.checkpointing import min_advances

OPS = ("store", "restore", "advance", "turn")


@pytest.fixture(scope="module")
def A():
    from paper_1912_05371_gb300 import acm, build
    build.build()
    acm.lib()
    return acm


def replay(sched, n, slots):
    """Checks a schedule on step indices; returns the number of advances."""
    snaps, cur, expect, adv, hi, first = {}, 0, n - 1, 0, 0, []
    for i, (op, k) in enumerate(sched["actions"]):
        if op == "store":
            assert 0 <= k < slots and cur is not None
            assert k != 0 or (i == 0 and cur == 0)
            snaps[k] = cur
        elif op == "restore":
            assert k in snaps
            cur = snaps[k]
        elif op == "advance":
            assert cur == k and 0 <= k < n - 1
            cur, adv = k + 1, adv + 1
        else:
            assert op == "turn" and cur == k == expect
            cur, expect = None, expect - 1
        if op in ("advance", "turn") and k + 1 > hi:      # both steps reach U_{k+1}
            hi = k + 1
            first.append(hi)
    assert expect == -1
    assert first == list(range(1, n + 1))
    assert sched["actions"][0] == ("store", 0)
    assert adv == sched["advances"]
    assert max(a for o, a in sched["actions"] if o in ("store", "restore")) + 1 == sched["snapshots"]
    return adv


def test_binomial_schedule_is_valid_and_minimal(A):
    for n in range(1, 61):
        for S in range(1, 9):
            sch = A.checkpoint_schedule(n, snapshots=S)
            assert sch["snapshots"] <= min(S, n)
            assert replay(sch, n, min(S, n)) == min_advances(n, S), (n, S)


@pytest.mark.parametrize("n,S", [(100, 18), (100, 5), (1000, 3), (4096, 12), (30000, 2)])
def test_binomial_schedule_at_larger_sizes(A, n, S):
    from math import comb
    r = 0
    while comb(S + r, S) < n:
        r += 1
    sch = A.checkpoint_schedule(n, snapshots=S)
    assert sch["advances"] == r * n - (comb(S + r, r - 1) if r else 0)
    if n <= 4096:
        replay(sch, n, S)


def test_equidistant_schedule(A):
    for n in range(1, 61):
        for c in range(1, 13):
            cc = min(c, n)
            nck = (n - 1) // cc + 1
            slots = nck + max(cc - 2, 0)
            sch = A.checkpoint_schedule(n, ckpt_every=c)
            assert sch["snapshots"] <= slots
            assert replay(sch, n, slots) == (n - 1) + (nck - 1) * (cc - 1), (n, c)
    # the adjoint benchmark's setting: 100 steps, every 10th state kept
    assert A.checkpoint_schedule(100, ckpt_every=10)["advances"] == 99 + 9 * 9


def test_invalid_requests(A):
    import ctypes as C
    L = A.lib()
    na = C.c_int64(-1)
    assert L.acm_checkpoint_schedule(0, 2, None, None, None, None, 0, C.byref(na)) == 1
    assert L.acm_checkpoint_schedule(10, 0, None, None, None, None, 0, C.byref(na)) == 1
    assert L.acm_checkpoint_schedule((1 << 20) + 1, -4, None, None, None, None, 0, C.byref(na)) == 1
    ops = np.zeros(4, np.int8)
    args = np.zeros(4, np.int32)
    assert L.acm_checkpoint_schedule(10, -2, None, None, ops.ctypes.data_as(C.c_void_p),
                                     args.ctypes.data_as(C.c_void_p), 4, C.byref(na)) == 1
    assert na.value > 4
    with pytest.raises(ValueError):
        A.checkpoint_schedule(10, snapshots=0)
    # too many recomputed steps for the memory given: refused at once, not built
    assert L.acm_checkpoint_schedule(1 << 20, -2, None, None, None, None, 0, C.byref(na)) == 1
    assert A.checkpoint_schedule(1 << 20, snapshots=64)["advances"] < (1 << 26)
