"""Blocks of 33^3 points (the full-scale configuration's block size, FP32 fields): the CUDA path
through the C-ABI against the FP64 oracle, element by element.

A 33^3 block has 1089 (x, y) columns, more than a CTA's 1024 threads: the stage kernel splits a
block by rows over three CTAs that read each other's rows like a halo, the column kernels take two
columns per thread, the block indicator keeps one component's coarse samples in shared memory at
a time and refinement predicts one child per CTA.  The layout is two roots of 33^3 along x, the
second refined: one level-0 block and eight level-1 blocks, so that every face type occurs (same
level, finer, coarser; in y and z the roots are their own periodic neighbours).  Tolerances as in
the other FP32 parity tests: 2e-5 relative per field (gpu_util.rel_linf), topology bit-exact.
"""
import numpy as np
import pytest

from oracle import acm as oacm
from tests.gpu_util import (block_order_fields, fill_from_function, oracle_forest, oracle_solver, rel_linf,
                            smooth_field, sphere_fn, sponge_fn)

pytestmark = pytest.mark.gpu

LEAVES = [(0, 0, 0, 0)] + [(1, 2 + (c & 1), (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]
MASK = (1.2, 0.5, 0.5, 0.2, 0.04)


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _grid(Jmax=1, wavelet=40, precision=32):
    return dict(nroot=(2, 1, 1), root_len=1.0, Bs=33, g=4, Jmin=0, Jmax=Jmax, precision=precision,
                max_blocks=96, fd_scheme=1, wavelet=wavelet)


def _phys(**kw):
    p = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5, eps=1e-3, dealias=0, mask_range_thr=1e-5,
             sponge=1, C_sp=0.05, u_inf=(0.4, -0.1, 0.2), p_inf=0.1, sponge_L=(2.0, 1.0, 1.0),
             sponge_width=0.2, sponge_delta=0.05)
    p.update(kw)
    return p


def _pair(A, grid, phys, leaves=LEAVES, seed=3, mask=MASK):
    f = A.Forest(grid, phys)
    f.set_leaves(leaves)
    fo = oracle_forest(grid, leaves=leaves, max_blocks=grid["max_blocks"])
    S = oracle_solver(fo, phys, mask=sphere_fn(mask) if mask else None,
                      sponge=sponge_fn(phys) if phys.get("sponge") else None, wavelet=grid["wavelet"])
    fill_from_function(S, lambda X, Y, Z: smooth_field(X, Y, Z, (2.0, 1.0, 1.0), seed))
    S.eval_mask()
    if mask:
        f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.write_fields(block_order_fields(S))
    return f, S


def _same_topology(f, fo):
    t = f.topology()
    tc, lv, sl, nbr, rel = fo.topology()
    assert np.array_equal(t["treecode"], tc) and np.array_equal(t["level"], lv)
    assert np.array_equal(t["slot"], sl) and np.array_equal(t["nbr"], nbr) and np.array_equal(t["rel"], rel)


def test_bs33_forest_is_fp32_and_cdf40_only(A):
    for bad in (_grid(precision=64), _grid(wavelet=44)):
        with pytest.raises(A.AcmError):
            A.Forest(bad, _phys())
    f = A.Forest(_grid(), _phys())
    f.set_leaves(LEAVES)
    _same_topology(f, oracle_forest(_grid(), leaves=LEAVES, max_blocks=96))


def test_bs33_sync_ghosts_matches_oracle(A):
    """Every block's extended array (interior and 4 ghost layers, edges and corners included:
    copies, decimations and DD-4 predictions) against the oracle's synchronisation."""
    from oracle.sync import sync as osync
    f, S = _pair(A, _grid(), _phys())
    gpu = f.sync_ghosts()
    ext = osync(S.fo, S.U, 4, "cube")
    ref = np.stack([ext[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    assert not np.isnan(ref).any()
    err = rel_linf(gpu.astype(np.float64), ref)
    assert max(err) < 1e-6, err


def test_bs33_mask_matches_oracle(A):
    f, S = _pair(A, _grid(), _phys())
    chi = f.read_mask().astype(np.float64)
    ref = np.stack([S.chi[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    assert np.abs(chi - ref).max() <= 1e-5


def test_bs33_fused_rhs_matches_oracle(A):
    """One right-hand side (mask, sponge) on the row-split stage kernel."""
    f, S = _pair(A, _grid(), _phys())
    gpu = f.rhs().astype(np.float64)
    K = S.rhs(S.U.copy())
    ref = np.stack([K[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    U32 = S.U.astype(np.float32).astype(np.float64)
    K32 = S.rhs(U32)
    ref32 = np.stack([K32[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    err, err32 = rel_linf(gpu, ref), rel_linf(gpu, ref32)
    print("bs33 fp32 rhs err vs fp64 state", err, "vs rounded state", err32)
    assert max(err32) < 2e-5, err32
    assert max(err) < 2e-5, err


def test_bs33_rk4_steps_match_oracle(A):
    f, S = _pair(A, _grid(), _phys(sponge=0))
    f.rk4_step(1e-3)
    S.rk4(1e-3)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < 2e-5, err


def test_bs33_row_tiles_are_bitwise_equal(A):
    """The stage kernel's two tiles for 33^3 blocks (three CTAs of 11 rows, four of 9) compute
    bitwise the same RK4 steps (mask and sponge on, FP32)."""
    out = []
    for variant in (A.ACM_STAGE_POINT, A.ACM_STAGE_POINT_ROWS):
        f = A.Forest(_grid(), _phys())
        f.set_leaves(LEAVES)
        f.set_mask(A.ACM_MASK_SPHERE, MASK)
        f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2.0 * np.pi, 1.0])
        f.set_stage_variant(variant)
        for _ in range(2):
            f.rk4_step(1e-3)
        out.append(f.read_fields())
    assert np.array_equal(out[0], out[1])


def test_bs33_indicators_match_oracle(A):
    f, S = _pair(A, _grid(), _phys(sponge=0))
    ind, rng = f.block_indicators()
    oind, _ = S.indicators(S.norms())
    order = S.fo.sorted_leaves()
    ref = np.array([oind[l][0] for l in order])
    rref = np.array([oind[l][1] for l in order])
    assert np.abs(ind - ref).max() <= 1e-4 * ref.max()
    assert np.abs(rng - rref).max() <= 1e-6


def test_bs33_refine_matches_oracle(A):
    """Every leaf below J = 2 split into 8 children: the level-1 blocks next to the level-0 block
    have a coarser neighbour, so their children's parent samples beyond the face are predicted."""
    grid = _grid(Jmax=2)
    f, S = _pair(A, grid, _phys(sponge=0))
    f.refine_all()
    S.refine_all()
    _same_topology(f, S.fo)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < 2e-5, err


def test_bs33_coarsen_matches_oracle(A):
    """Every block tagged (no mask, which would keep the blocks it crosses): the eight level-1
    blocks merge into their root (decimation)."""
    f, S = _pair(A, _grid(), _phys(sponge=0, eps=1e30), mask=None)
    nb, npass = f.coarsen()
    opass = S.coarsen()
    assert nb == len(S.fo.leaves) == 2 and npass == opass
    _same_topology(f, S.fo)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < 2e-5, err


def test_bs33_adaptive_step_matches_oracle(A):
    """One refine-evolve-coarsen step of the sphere case from its initial grid (Jmin 0, Jmax 1)."""
    grid = _grid(Jmax=1)
    dxm = 1.0 / (2 * 32)
    phys = dict(nu=1e-3, c0=5.0, C_eta=1e-2, C_gamma=0.0, C_sp=0.25 / (5.0 * 20.0), u_inf=(1.0, 0.0, 0.0),
                p_inf=0.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25, eps=1e-3, dealias=1, mask_range_thr=1e-5,
                sponge=1, sponge_L=(2.0, 1.0, 1.0), sponge_width=0.25, sponge_delta=1.5 * dxm)
    mask = (0.6, 0.5, 0.5, 0.15, 1.5 * dxm)
    f = A.Forest(grid, phys)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    nb = f.init_grid(A.ACM_IC_UNIFORM, [1.0, 0.0, 0.0, 0.0])
    fo = oracle_forest(grid, max_blocks=96)
    S = oracle_solver(fo, phys, ic=lambda X, Y, Z: oacm.ic_uniform(X, Y, Z), mask=sphere_fn(mask),
                      sponge=sponge_fn(phys))
    S.initial_grid()
    assert nb == len(fo.leaves)
    _same_topology(f, fo)
    dt, n = f.step(0.0)
    S.refine_all()
    dto = S.dt_cfl()
    assert abs(dt - dto) <= 1e-6 * dto
    S.rk4(dto)
    S.coarsen()
    _same_topology(f, fo)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < 2e-5, err


def test_bs33_vjp_matches_the_oracle(A):
    """The discrete adjoint on 33^3 blocks (the adjoint stage kernel split by rows, as the
    forward one): dL/dU_0 and dL/d(centre, radius) of L = <lam, U_1> (one RK4 step, sphere and
    sponge, lam random on every copy of every point) against the oracle's vector-Jacobian
    product, which is pinned by central differences; FP32 within 1e-4 as at Bs 17."""
    from oracle.adapt import Solver
    from oracle.adjoint import FrozenGridAdjoint
    from oracle.forest import Forest as OForest
    from tests.test_gpu_adjoint import _per_point
    from tests.test_oracle_adjoint import L, _field
    fo = OForest(nroot=(2, 1, 1), root_len=1.0, Bs=33, Jmin=0, Jmax=1, max_blocks=96)
    fo.set_leaves(LEAVES)
    delta = 1.5 * fo.h(1)
    centre, R, dt = (1.3, 0.5, 0.5), 0.2, 1e-3
    ph = oacm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0))
    S = Solver(fo, ph, ic=lambda X, Y, Z: _field(X, Y, Z, 41),
               mask=lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, centre, R, delta),
               sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, L, 0.2, delta))
    S.eval_ic()
    S.eval_mask()
    order = fo.sorted_leaves()
    rng = np.random.default_rng(23)
    lamB = rng.normal(size=(len(order), 4, 33, 33, 33))
    lam = np.zeros_like(S.U)
    for r, l in enumerate(order):
        lam[fo.leaves[l]] = lamB[r]
    _, go, gtho = FrozenGridAdjoint(S, centre, R, delta, dt=dt, nsteps=1).vjp(S.U.copy(), lam)
    phys = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0), p_inf=0.0,
                sponge=1, sponge_L=L, sponge_width=0.2, sponge_delta=delta)
    f = A.Forest(_grid(), phys)
    f.set_leaves(LEAVES)
    f.set_mask(A.ACM_MASK_SPHERE, (*centre, R, delta))
    f.write_fields(block_order_fields(S))
    gU, gth = f.adjoint_vjp(1, dt, lamB, ckpt_every=1)
    gob = np.stack([go[fo.leaves[l]] for l in order])
    a, b = _per_point(fo, gU, 1), _per_point(fo, gob, 1)
    assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max()
    assert np.abs(gth - gtho).max() <= 1e-4 * np.abs(gtho).max(), (gth, gtho)
