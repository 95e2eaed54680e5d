"""Pins of the oracle's CDF 4/4 coarsening (Sec. 3.2.1 lifting, Sec. 3.5 merge).

The lifted low-pass h~ is pinned by what the lifting must give (normalisation, the moments
that make it reproduce cubics, the alternating moments that are the lifted wavelet's vanishing
moments), by the two-step lifting form (details, then the update of the even samples), and by
its exact action on a sinusoid.  The 3D merge is pinned on grids: sinusoids on a uniform grid
(exact tensor transfer function), cubics next to coarser neighbours (whose ghost values come
from the DD-4 prediction, exact for cubics), the alternating modes (annihilated), and the
boundary reading (decimated face points, redundant points consistent).
"""
import math

import numpy as np
import pytest

from oracle import acm, mra
from oracle.adapt import Solver
from oracle.forest import Forest
from oracle.sync import fine_wins, redundant_points_consistent
from paper_1912_05371_gb300.workloads import cubic_coefficients, random_graded_leaves


def _poly(C, X, Y, Z):
    return np.stack([sum(C[f, a, b, c] * X ** a * Y ** b * Z ** c
                         for a in range(4) for b in range(4) for c in range(4)) for f in range(4)])


def _solver(fo, fn, wavelet="cdf44", **kw):
    S = Solver(fo, acm.Physics(), ic=fn, wavelet=wavelet, **kw)
    S.eval_ic()
    S.eval_mask()
    return S


def _transfer(ht, w):
    """sum_n h~_n cos(n w): the filter's response to a sinusoid (h~ is symmetric)."""
    return sum(v * math.cos(n * w) for n, v in ht.items())


# ---- the 1D filter ----------------------------------------------------------------------------

def test_lowpass_moments():
    ht = mra.cdf44_lowpass()
    assert set(ht) == {-6, -4, -3, -2, -1, 0, 1, 2, 3, 4, 6}
    for n in ht:
        assert abs(ht[n] - ht[-n]) < 1e-15
    m = mra.moments(ht, 5)
    assert abs(m[0] - 1.0) < 1e-14
    assert np.allclose(m[1:4], 0.0, atol=1e-12)          # reproduces cubics
    assert abs(m[4]) > 1.0                                # but not quartics
    alt = {n: (-1.0) ** (n % 2) * v for n, v in ht.items()}
    assert np.allclose(mra.moments(alt, 4), 0.0, atol=1e-12)   # kills (-1)^n x cubic
    # dyadic rationals with denominator 512 (the update weights are multiples of 1/32, the
    # prediction weights of 1/16)
    for v in ht.values():
        assert abs(v * 512 - round(v * 512)) < 1e-10


def test_lowpass_equals_the_two_lifting_steps():
    """Filter form against the lifting form on a periodic signal: details at the odd points
    (u - P R u), then each even sample updated by the four details around it."""
    h, ht0, g, gt = mra.dd4_filters()
    s = mra.lifting_coefficients(h, g, 4, [-1, 0, 1, 2])
    ht = mra.cdf44_lowpass()
    rng = np.random.default_rng(5)
    f = rng.normal(size=64)
    n = f.size
    d = mra.details_1d_periodic(f)[1::2]                  # d_j at fine point 2j+1
    nc = n // 2
    lifted = np.array([f[2 * i] + sum(s[k] * d[(i - k) % nc] for k in s) for i in range(nc)])
    filt = np.array([sum(v * f[(2 * i + m) % n] for m, v in ht.items()) for i in range(nc)])
    assert np.abs(lifted - filt).max() < 1e-13


def test_lowpass_of_a_sinusoid_is_the_transfer_function():
    ht = mra.cdf44_lowpass()
    M, g = 16, 4
    x = np.arange(-g, 2 * M + g + 1)
    for k, ph in ((0.3, 0.2), (1.1, -0.7), (2.9, 1.3)):
        f = np.sin(k * x + ph)[None, :]
        c = mra.lowpass_decimate_axis(f, -1, ht, g, M)[0]
        i = np.arange(1, M)
        assert np.abs(c - _transfer(ht, k) * np.sin(2 * k * i + ph)).max() < 1e-14
    # fourth order: 1 - H(w) = O(w^4)
    r = [(1.0 - _transfer(ht, w)) for w in (0.2, 0.1)]
    assert 15.0 < r[0] / r[1] < 17.0


# ---- the 3D merge ----------------------------------------------------------------------------

def test_uniform_grid_merge_is_the_tensor_transfer_function():
    fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 10)
    fo.init_uniform(3)
    a, b, c = 1, 2, 3
    p = (0.3, -0.4, 1.1)

    def fn(X, Y, Z):
        v = np.sin(2 * math.pi * a * X + p[0]) * np.sin(2 * math.pi * b * Y + p[1]) * np.sin(
            2 * math.pi * c * Z + p[2])
        return np.stack([v, 2 * v, -v, 0.5 * v])

    S = _solver(fo, fn)
    ht = mra.cdf44_lowpass()
    h = fo.h(3)
    gain = (_transfer(ht, 2 * math.pi * a * h) * _transfer(ht, 2 * math.pi * b * h)
            * _transfer(ht, 2 * math.pi * c * h))
    M = fo.M
    for parent in [(2, 1, 1, 1), (2, 0, 3, 2), (2, 3, 0, 0)]:   # the last two touch the seam
        lp = S.lowpass_parent(parent, S.U)
        X, Y, Z = acm.block_coords(fo, parent)
        want = gain * fn(X, Y, Z)[:, 1:M, 1:M, 1:M]
        assert np.abs(lp - want).max() < 1e-13


def test_merge_reproduces_cubics_next_to_coarser_and_same_level_neighbours():
    C = cubic_coefficients(21)
    nroot = (1, 1, 1)
    fo = Forest(nroot=nroot, root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 10)
    # level-2 grid with two neighbouring blocks refined: the group of parent (2,1,1,1) has
    # level-3 neighbours on +x and level-2 neighbours elsewhere
    leaves = [(2, x, y, z) for z in range(4) for y in range(4) for x in range(4)
              if (x, y, z) not in ((1, 1, 1), (2, 1, 1))]
    leaves += list(Forest.children_of((2, 1, 1, 1))) + list(Forest.children_of((2, 2, 1, 1)))
    fo.set_leaves(leaves)
    assert fo.is_graded()
    S = _solver(fo, lambda X, Y, Z: _poly(C, X, Y, Z))
    M = fo.M
    for parent in [(2, 1, 1, 1), (2, 2, 1, 1)]:
        lp = S.lowpass_parent(parent, S.U)
        X, Y, Z = acm.block_coords(fo, parent)
        want = _poly(C, X, Y, Z)[:, 1:M, 1:M, 1:M]
        assert np.abs(lp - want).max() < 1e-12 * np.abs(want).max()


def test_merge_annihilates_the_alternating_modes():
    fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 10)
    fo.init_uniform(3)
    C = cubic_coefficients(22)
    h = fo.h(3)

    def fn(X, Y, Z):
        sgn = sum((-1.0) ** np.rint(V / h).astype(np.int64) for V in (X, Y, Z))
        return sgn * _poly(C, X, Y, Z)

    S = _solver(fo, fn)
    lp = S.lowpass_parent((2, 1, 1, 1), S.U)
    assert np.abs(lp).max() < 1e-12 * np.abs(S.U).max()
    # each axis pass matters: the x-alternating mode alone is not removed by y and z
    S2 = _solver(fo, lambda X, Y, Z: (-1.0) ** np.rint(X / h).astype(np.int64) * _poly(C, X, Y, Z),
                 wavelet="cdf44")
    assert np.abs(S2.lowpass_parent((2, 1, 1, 1), S2.U)).max() < 1e-12 * np.abs(S2.U).max()


@pytest.mark.parametrize("seed", [31, 32])
def test_merge_keeps_decimated_faces_and_redundancy(seed):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=90)
    L = (2.0, 1.0, 1.0)

    def fn(X, Y, Z):
        return np.stack([np.sin(2 * math.pi * (k * X / L[0] + Y + 2 * Z) + k) for k in range(1, 5)])

    out = {}
    for wl in ("cdf40", "cdf44"):
        fo = Forest(nroot=(2, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 12)
        fo.set_leaves(leaves)
        S = _solver(fo, fn, wavelet=wl)
        fine_wins(fo, S.U)
        groups = S.coarsenable_groups({l: True for l in fo.leaves})
        assert groups
        new = S.merge(groups, S.U.copy())
        out[wl] = (fo, S, new)
    fo, S44, new = out["cdf44"]
    _, S40, new40 = out["cdf40"]
    assert new == new40
    M = fo.M
    inner = (slice(None), slice(1, M), slice(1, M), slice(1, M))
    for p, s in new.items():
        a, b = S44.U[s].copy(), S40.U[s].copy()
        assert not np.array_equal(a[inner], b[inner])
        a[inner] = 0.0
        b[inner] = 0.0
        assert np.array_equal(a, b)                       # faces, edges, corners: decimated
    assert redundant_points_consistent(fo, S44.U)


def test_refine_then_cdf44_coarsen_restores_any_field():
    """Biorthogonality, sum_n h_n h~_{n+2k} = delta_k: the lifted analysis undoes the interpolating
    prediction, so refining every block and merging all groups back with CDF 4/4 returns the
    original blocks for an arbitrary (here random) field on a uniform periodic grid."""
    rng = np.random.default_rng(9)
    N = 2 * 8
    lat = rng.normal(size=(4, N, N, N))
    fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=2, max_blocks=256)
    fo.init_uniform(1)
    h = fo.h(1)

    def field(X, Y, Z):
        ix, iy, iz = (np.rint(V / h).astype(int) % N for V in (X, Y, Z))
        return lat[:, iz, iy, ix]

    S = _solver(fo, field, eps=1e30, dealias=False)
    before = {l: S.U[s].copy() for l, s in fo.leaves.items()}
    S.refine_all()
    assert all(l[0] == 2 for l in fo.leaves)
    S.coarsen()
    assert set(fo.leaves) == set(before)
    err = max(np.abs(S.U[s] - before[l]).max() for l, s in fo.leaves.items())
    assert err < 1e-13 * np.abs(lat).max()
