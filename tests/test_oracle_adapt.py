"""Pins of the oracle's refine / coarsen cycle and initial grid (Sec. 3.3, 3.5)."""
import math

import numpy as np
import pytest

from oracle import acm
from oracle.adapt import Solver
from oracle.forest import Forest
from paper_1912_05371_gb300.workloads import cubic_coefficients, random_graded_leaves


def _poly(C, X, Y, Z):
    return np.stack([sum(C[f, a, b, c] * X ** a * Y ** b * Z ** c
                         for a in range(4) for b in range(4) for c in range(4)) for f in range(4)])


def _solver(leaves, nroot=(2, 2, 2), Jmin=1, Jmax=3, ic=None, **kw):
    fo = Forest(nroot=nroot, root_len=1.0, Bs=9, Jmin=Jmin, Jmax=Jmax, max_blocks=1 << 12)
    fo.set_leaves(leaves)
    S = Solver(fo, acm.Physics(), ic=ic, **kw)
    S.eval_ic()
    S.eval_mask()
    return S


def _interior_field(S):
    return {leaf: S.U[s].copy() for leaf, s in S.fo.leaves.items()}


def test_refine_predicts_cubics_exactly_with_33_cubed_blocks():
    """Refinement of 33^3 blocks (the full-scale case's block size) is exact on cubics too: eight
    roots, one of them refined once, all refined again."""
    C = cubic_coefficients(12)
    leaves = [(0, x, y, z) for z in range(2) for y in range(2) for x in range(2) if (x, y, z) != (1, 1, 1)]
    leaves += [(1, 2 + (c & 1), 2 + ((c >> 1) & 1), 2 + ((c >> 2) & 1)) for c in range(8)]
    fo = Forest(nroot=(2, 2, 2), root_len=1.0, Bs=33, Jmin=0, Jmax=2, max_blocks=160)
    fo.set_leaves(leaves)
    S = Solver(fo, acm.Physics(), ic=lambda X, Y, Z: _poly(C, X, Y, Z), eps=1e3, dealias=False)
    S.eval_ic()
    S.eval_mask()
    S.refine_all()
    assert len(fo.leaves) == 7 * 8 + 8 * 8 and fo.is_graded()
    nchk = 0
    for leaf, s in fo.leaves.items():
        X, Y, Z = acm.block_coords(fo, leaf)
        if min(X.min(), Y.min(), Z.min()) < 0.3 or max(X.max(), Y.max(), Z.max()) > 1.7:
            continue                    # the parent's stencils would cross the periodic seam
        assert np.abs(S.U[s] - _poly(C, X, Y, Z)).max() < 1e-11
        nchk += 1
    assert nchk > 10


def test_refine_predicts_cubics_exactly_and_coarsen_restores():
    C = cubic_coefficients(11)
    leaves = random_graded_leaves(4, nroot=(2, 2, 2), J0=1, Jmax=2, n_target=80)
    S = _solver(leaves, ic=lambda X, Y, Z: _poly(C, X, Y, Z), Jmax=3, eps=1e3, dealias=False)
    before = _interior_field(S)
    S.refine_all()
    assert S.fo.is_graded() and S.fo.covers_domain_exactly()
    M = S.fo.M
    nchk = 0
    for leaf, s in S.fo.leaves.items():
        X, Y, Z = acm.block_coords(S.fo, leaf)
        lo = min(X.min(), Y.min(), Z.min())
        hi = max(X.max(), Y.max(), Z.max())
        if lo < 0.3 or hi > 1.7:
            continue                    # the parent's stencils would cross the periodic seam
        assert np.abs(S.U[s] - _poly(C, X, Y, Z)).max() < 1e-11
        nchk += 1
    assert nchk > 10
    # uniform level-2 grid, J_min = 2: with every detail below a huge threshold, coarsening
    # undoes the refinement exactly (R o P = Id)
    fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=2, Jmax=3, max_blocks=1 << 10)
    fo.init_uniform(2)
    S = Solver(fo, acm.Physics(), ic=lambda X, Y, Z: _poly(C, X, Y, Z), eps=1e3, dealias=False)
    S.eval_ic()
    before = _interior_field(S)
    S.refine_all()
    assert {l[0] for l in fo.leaves} == {3}
    S.coarsen()
    assert set(S.fo.leaves) == set(before)
    for leaf, s in S.fo.leaves.items():
        assert np.array_equal(S.U[s], before[leaf])


def test_coarsen_refine_error_below_threshold_and_grid_invariants():
    eps = 2e-3
    leaves = random_graded_leaves(5, nroot=(1, 1, 1), J0=1, Jmax=3, n_target=120)
    ic = lambda X, Y, Z: np.stack([np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y),
                                   np.cos(2 * math.pi * Z), np.sin(4 * math.pi * (X + Y)) * 0.3,
                                   np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / 0.01)])
    S = _solver(leaves, nroot=(1, 1, 1), ic=ic, eps=eps, dealias=False)
    ref = _interior_field(S)
    norms = S.norms()
    S.coarsen(max_passes=1)          # one pass: merged blocks are one level coarser
    fo = S.fo
    assert fo.is_graded() and fo.covers_domain_exactly()
    merged = set(ref) - set(fo.leaves)
    assert merged, "some groups must coarsen"
    # refine the merged parents back: the error is the dropped details, below eps * ||f||
    S.refine_all()
    for leaf in merged:
        if leaf in fo.leaves:
            err = np.abs(S.U[fo.leaves[leaf]] - ref[leaf]).max(axis=(1, 2, 3))
            assert np.all(err < eps * norms + 1e-14)
    # after a full coarsening no sister group is left that could still coarsen
    S2 = _solver(leaves, nroot=(1, 1, 1), ic=ic, eps=eps, dealias=False)
    S2.coarsen()
    ind, _ = S2.indicators(S2.norms())
    assert not S2.coarsenable_groups(S2.tags(ind))
    assert S2.fo.is_graded() and S2.fo.covers_domain_exactly()


def test_initial_grid_tracks_the_mask_interface():
    delta = 1.5 / (8 * 8)
    for dealias, top in ((True, 2), (False, 3)):
        fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 10)
        S = Solver(fo, acm.Physics(), eps=1e-3, dealias=dealias,
                   ic=lambda X, Y, Z: acm.ic_uniform(X, Y, Z),
                   mask=lambda X, Y, Z: acm.sphere_mask(X, Y, Z, (0.5, 0.5, 0.5), 0.2, delta))
        S.initial_grid()
        assert fo.is_graded() and fo.covers_domain_exactly()
        levels = {l[0] for l in fo.leaves}
        assert max(levels) == top
        for leaf, s in fo.leaves.items():
            rng = float(S.chi[s].max() - S.chi[s].min())
            if rng > S.mask_thr:
                assert leaf[0] == top      # the interface sits on the finest level kept


def test_adaptive_run_stays_within_the_threshold_error_of_the_uniform_run():
    """Sec. 3.4: an adaptive run (refine, RK4, coarsen per step) differs from the same steps on the
    uniform finest grid by at most about N_t C_eps ||u||: each step's coarsening drops details
    below C_eps ||u|| and the (stable) scheme carries the dropped parts along."""
    eps, steps = 1e-3, 3
    ph = acm.Physics(nu=1e-2, c0=3.0, C_gamma=0.5)
    ic = lambda X, Y, Z: np.stack([np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y),
                                   0.5 * np.cos(2 * math.pi * X) * np.sin(2 * math.pi * Z),
                                   0.2 * np.sin(2 * math.pi * (Y + Z)), np.zeros_like(X)])
    fa = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=3, max_blocks=1 << 10)
    A = Solver(fa, ph, eps=eps, dealias=False, ic=ic)
    A.initial_grid()
    fu = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=3, Jmax=3, max_blocks=1 << 10)
    fu.init_uniform(3)
    Uni = Solver(fu, ph, ic=ic)
    Uni.eval_ic()
    assert len(fa.leaves) < len(fu.leaves)        # the adaptive grid is coarser somewhere
    scale = float(np.abs(np.stack([Uni.U[s] for s in fu.leaves.values()])[:, :3]).max())
    for _ in range(steps):
        A.refine_all()
        dt = A.dt_cfl()
        A.rk4(dt)
        A.coarsen()
        Uni.rk4(dt)
    # compare on the adaptive grid's points (each is a point of the uniform level-3 lattice)
    M = fa.M
    err = 0.0
    for (J, gx, gy, gz), s in fa.leaves.items():
        k = 1 << (3 - J)
        for c in range(8 ** (3 - J)):
            cx, cy, cz = c % k, (c // k) % k, c // (k * k)
            leaf3 = (3, gx * k + cx, gy * k + cy, gz * k + cz)
            u3 = Uni.U[fu.leaves[leaf3]]
            # points of the level-3 block that lie on the level-J lattice
            sub = u3[:3, ::k, ::k, ::k]
            n = M // k
            ua = A.U[s][:3, cz * n:cz * n + n + 1, cy * n:cy * n + n + 1, cx * n:cx * n + n + 1]
            err = max(err, float(np.abs(ua - sub).max()))
    assert err <= steps * eps * scale, (err, steps * eps * scale)
    assert err > 0.0


@pytest.mark.parametrize("seed", [51])
def test_coarsen_everywhere_restores_the_step_grid(seed):
    """The performance cycle of Sec. 5.4 with coarsening forced everywhere (reading: every block
    made by the step's refinement is tagged, thresholds ignored): refine-all then coarsening
    restores the starting layout, and with CDF 4/0 the state bitwise (prediction copies the
    coincident points to the children, decimation copies them back); over full steps
    (refine, RK4, coarsen) the layout stays the same."""
    from oracle.sync import fine_wins
    from tests.gpu_util import fill_from_function, oracle_forest, smooth_field
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=60)
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=4)
    fo = oracle_forest(grid, leaves=leaves, max_blocks=4096)
    S = Solver(fo, acm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5), coarsen_everywhere=True)
    fill_from_function(S, lambda X, Y, Z: smooth_field(X, Y, Z, (2.0, 1.0, 1.0), seed))
    S.eval_mask()
    fine_wins(fo, S.U)
    before = {l: S.U[s].copy() for l, s in fo.leaves.items()}
    S.refine_all()
    assert len(fo.leaves) > len(before)
    assert S.coarsen() >= 2                                    # finest groups first (grading)
    assert set(fo.leaves) == set(before)
    assert all(np.array_equal(S.U[s], before[l]) for l, s in fo.leaves.items())
    S.refine_all()
    S.rk4(1e-3)
    S.coarsen()
    assert set(fo.leaves) == set(before)
