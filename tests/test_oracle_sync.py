"""Pins of the oracle's ghost-node synchronisation (Sec. 4.2 with the Sec. 3.1 operators)."""
import numpy as np
import pytest

from oracle.acm import block_coords
from oracle.forest import DIRECTIONS, Forest
from oracle.sync import fine_wins, redundant_points_consistent, sync
from paper_1912_05371_gb300.workloads import cubic_coefficients, random_graded_leaves


def _poly(C, X, Y, Z):
    return np.stack([sum(C[f, a, b, c] * X ** a * Y ** b * Z ** c
                         for a in range(4) for b in range(4) for c in range(4)) for f in range(4)])


def _fill(fo, fn):
    n = fo.Bs
    F = np.zeros((fo.max_blocks, 4, n, n, n))
    for leaf, s in fo.leaves.items():
        F[s] = fn(*block_coords(fo, leaf))
    return F


def test_uniform_grid_ghosts_are_the_periodic_neighbours():
    fo = Forest(nroot=(2, 1, 1), root_len=1.0, Bs=9, max_blocks=64)
    fo.init_uniform(1)
    rng = np.random.default_rng(0)
    N = fo.npoints(1)
    glob = rng.normal(size=(4, N[2], N[1], N[0]))
    M = fo.M
    F = np.zeros((64, 4, 9, 9, 9))
    for (J, gx, gy, gz), s in fo.leaves.items():
        iz = np.mod(gz * M + np.arange(9), N[2])
        iy = np.mod(gy * M + np.arange(9), N[1])
        ix = np.mod(gx * M + np.arange(9), N[0])
        F[s] = glob[:, iz][:, :, iy][:, :, :, ix]
    g = 4
    ext = sync(fo, F, g)
    for (J, gx, gy, gz), s in fo.leaves.items():
        r = np.arange(-g, M + g + 1)
        iz, iy, ix = (np.mod(gz * M + r, N[2]), np.mod(gy * M + r, N[1]), np.mod(gx * M + r, N[0]))
        ref = glob[:, iz][:, :, iy][:, :, :, ix]
        assert np.array_equal(ext[s], ref)


@pytest.mark.parametrize("seed", [3, 5])
def test_adaptive_ghosts_reproduce_cubics(seed):
    """DD-4 prediction and decimation are exact for cubic polynomials, so every ghost value of
    a tensor-cubic field equals the polynomial -- wherever the periodic seam is not involved."""
    leaves = random_graded_leaves(seed, nroot=(2, 2, 2), J0=1, Jmax=3, n_target=120)
    fo = Forest(nroot=(2, 2, 2), root_len=1.0, Bs=9, max_blocks=4096)
    fo.set_leaves(leaves)
    assert len({l[0] for l in leaves}) == 3
    C = cubic_coefficients(seed)
    F = _fill(fo, lambda X, Y, Z: _poly(C, X, Y, Z))
    g = 4
    ext = sync(fo, F, g)
    M = fo.M
    checked = 0
    for leaf, s in fo.leaves.items():
        J = leaf[0]
        h = fo.h(J)
        N = fo.npoints(J)
        r = np.arange(-g, M + g + 1)
        gi = [leaf[1 + a] * M + r for a in range(3)]
        inside = [(v >= 10) & (v <= N[a] - 10) for a, v in enumerate(gi)]
        mz, my, mx = np.meshgrid(inside[2], inside[1], inside[0], indexing="ij")
        m = mz & my & mx
        if not m.any():
            continue
        Z, Y, X = np.meshgrid(gi[2] * h, gi[1] * h, gi[0] * h, indexing="ij")
        ref = _poly(C, X, Y, Z)
        assert np.abs(ext[s] - ref)[:, m].max() < 1e-12
        checked += 1
    assert checked > 20
    assert not np.isnan(ext[sorted(fo.leaves.values())]).any()


def test_ghosts_reproduce_cubics_with_33_cubed_blocks():
    """The same exactness for blocks of 33^3 (the full-scale case's block size): two roots, the
    second refined once, so that a level-0 block meets level-1 blocks across the root faces."""
    leaves = [(0, 0, 0, 0)] + [(1, 2 + (c & 1), (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
    fo = Forest(nroot=(2, 1, 1), root_len=1.0, Bs=33, max_blocks=16)
    fo.set_leaves(leaves)
    C = cubic_coefficients(33)
    F = _fill(fo, lambda X, Y, Z: _poly(C, X, Y, Z))
    g = 4
    ext = sync(fo, F, g)
    M = fo.M
    checked = 0
    for leaf, s in fo.leaves.items():
        J = leaf[0]
        h = fo.h(J)
        N = fo.npoints(J)
        r = np.arange(-g, M + g + 1)
        gi = [leaf[1 + a] * M + r for a in range(3)]
        inside = [(v >= 10) & (v <= N[a] - 10) for a, v in enumerate(gi)]
        mz, my, mx = np.meshgrid(inside[2], inside[1], inside[0], indexing="ij")
        m = mz & my & mx
        if not m.any():
            continue
        Z, Y, X = np.meshgrid(gi[2] * h, gi[1] * h, gi[0] * h, indexing="ij")
        assert np.abs(ext[s] - _poly(C, X, Y, Z))[:, m].max() < 1e-12
        checked += 1
    assert checked == 9
    assert not np.isnan(ext[sorted(fo.leaves.values())]).any()


def test_fine_wins_and_redundancy():
    leaves = random_graded_leaves(7, nroot=(1, 1, 1), J0=1, Jmax=3, n_target=60)
    fo = Forest(nroot=(1, 1, 1), Bs=9, max_blocks=4096)
    fo.set_leaves(leaves)
    rng = np.random.default_rng(7)
    F = _fill(fo, lambda X, Y, Z: np.stack([np.sin(6 * X + f) * np.cos(5 * Y) + Z for f in range(4)]))
    # perturb so that coarse and fine copies of shared points disagree before the sync
    for s in fo.leaves.values():
        F[s] += 1e-3 * rng.normal(size=F[s].shape)
    # after synchronisation same-level copies are not yet equal (random noise), but every
    # point a finer leaf holds must carry that finer leaf's value in the coarser leaf
    G = F.copy()
    fine_wins(fo, G)
    M = fo.M
    n_checked = 0
    for leaf, s in fo.leaves.items():
        J, g = leaf[0], leaf[1:]
        for k, d in enumerate(DIRECTIONS[:6]):
            st = fo.box_status(J, (g[0] + d[0], g[1] + d[1], g[2] + d[2]))
            if st[0] != "refined":
                continue
            a = [i for i in range(3) if d[i] != 0][0]
            face = 0 if d[a] < 0 else M
            for c, cs in st[1].items():
                cc = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
                if cc[a] != (1 if d[a] < 0 else 0):
                    continue
                # child face points at even indices coincide with the coarse face; those off the
                # child's own face boundary are held by this child alone (noise makes the
                # copies of the others differ)
                for j in range(2, M - 1, 2):
                    for i in range(2, M - 1, 2):
                        loc = [0, 0, 0]
                        loc[a] = M if d[a] < 0 else 0
                        others = [b for b in range(3) if b != a]
                        loc[others[0]] = i
                        loc[others[1]] = j
                        cl = list(loc)
                        pl = [0, 0, 0]
                        pl[a] = face
                        pl[others[0]] = cc[others[0]] * M // 2 + i // 2
                        pl[others[1]] = cc[others[1]] * M // 2 + j // 2
                        assert np.array_equal(G[s, :, pl[2], pl[1], pl[0]], F[cs, :, cl[2], cl[1], cl[0]])
                        n_checked += 1
    assert n_checked > 0
    # a field that starts consistent stays consistent through the sync
    H = _fill(fo, lambda X, Y, Z: np.stack([np.sin(6 * X + f) * np.cos(5 * Y) + Z for f in range(4)]))
    sync(fo, H, 2)
    assert redundant_points_consistent(fo, H)
