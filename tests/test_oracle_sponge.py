"""Pins of the oracle's sponge profile (Sec. 2.2, the sponge terms of eqs. u_eqn-1 and p_eqn-1).

The paper's Appendix D, which would give the sponge's shape, is not available.  The reading the
oracle follows: on the periodic box [0, L0] x [0, L1] x [0, L2], chi_sp is the mask's tanh profile
of (distance to the nearest face of one axis - L_sp), and the largest of the three axis profiles.
What that reading fixes, checked here without re-evaluating the oracle's expression:
  * chi_sp = 1/2 exactly at distance L_sp from a face, far from the other faces;
  * chi_sp -> 1 on a face and -> 0 in the interior;
  * one delta further in, the logistic form 1 / (1 + e^2) of (1 - tanh 1) / 2;
  * each axis measures to its own two faces (both ends, its own box length);
  * at an edge or corner the profile is the largest of the per-axis profiles.
Planted slips (min for max over axes, a one-sided face distance, a dropped L_sp, a swapped box
length, a halved layer width) each fail one of these checks.
"""
import math

import numpy as np

from oracle import acm

L = (4.0, 2.0, 2.0)          # the sphere workload's box
L_SP = 0.25
DELTA = 0.01


def _eval(fn, pts):
    p = np.asarray(pts, dtype=np.float64)
    return fn(p[:, 0], p[:, 1], p[:, 2], L, L_SP, DELTA)


def _failures(fn):
    """Names of the reading's properties that fn(X, Y, Z, L, L_sp, delta) violates."""
    bad = []
    mid = [Lc / 2 for Lc in L]
    # 1/2 at distance L_sp from each of the six faces, the other coordinates at the box centre
    half = []
    for a in range(3):
        for at in (L_SP, L[a] - L_SP):
            q = list(mid)
            q[a] = at
            half.append(q)
    if np.max(np.abs(_eval(fn, half) - 0.5)) > 1e-15:
        bad.append("half at L_sp")
    # on a face -> 1 (tanh(-L_sp/delta) = -1 to rounding), at the centre -> 0
    face = []
    for a in range(3):
        for at in (0.0, L[a]):
            q = list(mid)
            q[a] = at
            face.append(q)
    if np.min(_eval(fn, face)) < 1.0 - 1e-12:
        bad.append("one on the faces")
    if _eval(fn, [mid])[0] > 1e-12:
        bad.append("zero inside")
    # one layer width inside the half-value surface: (1 - tanh 1)/2 = 1/(1 + e^2); one outside:
    # 1 - that
    logistic = 1.0 / (1.0 + math.exp(2.0))
    inner, outer = [], []
    for a in range(3):
        q = list(mid)
        q[a] = L_SP + DELTA
        inner.append(q)
        q = list(mid)
        q[a] = L[a] - (L_SP - DELTA)
        outer.append(q)
    if np.max(np.abs(_eval(fn, inner) - logistic)) > 1e-14:
        bad.append("layer width")
    if np.max(np.abs(_eval(fn, outer) - (1.0 - logistic))) > 1e-14:
        bad.append("layer width (far face)")
    # mirror symmetry of each axis about its own centre
    rng = np.random.default_rng(7)
    pts = rng.uniform(0.0, 1.0, (200, 3)) * np.array(L)
    mir = pts.copy()
    a = rng.integers(0, 3, 200)
    mir[np.arange(200), a] = np.array(L)[a] - pts[np.arange(200), a]
    if np.max(np.abs(_eval(fn, pts) - _eval(fn, mir))) > 1e-14:
        bad.append("mirror symmetry")
    # edges and corners: the largest of the single-axis profiles, each taken with the other
    # coordinates at the centre
    corner = rng.uniform(0.0, 3 * L_SP, (200, 3))
    single = []
    for a in range(3):
        q = np.tile(np.array(mid), (200, 1))
        q[:, a] = corner[:, a]
        single.append(_eval(fn, q))
    if np.max(np.abs(_eval(fn, corner) - np.maximum.reduce(single))) > 1e-15:
        bad.append("largest over axes")
    return bad


def test_sponge_profile_follows_the_reading():
    assert _failures(acm.sponge_mask) == []


def _planted(kind):
    def fn(X, Y, Z, Lb, L_sp, delta):
        out = None
        lens = (Lb[1], Lb[0], Lb[2]) if kind == "swapped length" else Lb
        for c, Lc in zip((X, Y, Z), lens):
            dist = c if kind == "one-sided" else np.minimum(c, Lc - c)
            arg = dist if kind == "no L_sp" else dist - L_sp
            s = acm.smooth_step(arg, delta / 2 if kind == "half width" else delta)
            if out is None:
                out = s
            else:
                out = np.minimum(out, s) if kind == "min" else np.maximum(out, s)
        return out
    return fn


def test_planted_sponge_slips_fail_the_pin():
    for kind in ("min", "one-sided", "no L_sp", "swapped length", "half width"):
        assert _failures(_planted(kind)), kind
    # the planted form without a slip passes, so the failures come from the slips alone
    assert _failures(_planted("none")) == []
