"""CUDA path (through the C-ABI) against the FP64 oracle, element by element.

Tolerances: topology (treecode, level, slot, coordinates, neighbour tables) bit-exact; fields
relative L-infinity per component <= 1e-12 in FP64 and <= 2e-5 in FP32 (FP32 against the
FP64 oracle on the same FP64-evaluated inputs), velocity components relative to the velocity
scale max(|u|,|v|,|w|), pressure relative to max(max |p|, max |u|^2) (see gpu_util.rel_linf).
"""
import math

import numpy as np
import pytest

from oracle import acm as oacm
from oracle.sync import sync as osync
from paper_1912_05371_gb300.workloads import random_graded_leaves
from tests.gpu_util import (block_order_fields, fill_from_function, oracle_forest, oracle_solver,
                            rel_linf, smooth_field, sphere_fn, sponge_fn)

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 2e-5}


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _grid(Bs=9, nroot=(2, 1, 1), root_len=1.0, Jmin=1, Jmax=3, precision=64, max_blocks=4096, g=4, wavelet=40):
    return dict(nroot=nroot, root_len=root_len, Bs=Bs, g=g, Jmin=Jmin, Jmax=Jmax, precision=precision,
                max_blocks=max_blocks, fd_scheme=1, wavelet=wavelet)


def _phys(**kw):
    p = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5, eps=1e-3, dealias=0, mask_range_thr=1e-5)
    p.update(kw)
    return p


def _pair(A, grid, phys, leaves, fn_seed=1, mask=None):
    f = A.Forest(grid, phys)
    f.set_leaves(leaves)
    # the oracle's pool is the forest's: slots follow the same rule and fit the same capacity
    fo = oracle_forest(grid, leaves=leaves, max_blocks=grid["max_blocks"])
    S = oracle_solver(fo, phys, mask=sphere_fn(mask) if mask else None,
                      sponge=sponge_fn(phys) if phys.get("sponge") else None, wavelet=grid.get("wavelet", 40))
    L = tuple(n * grid["root_len"] for n in grid["nroot"])
    fill_from_function(S, lambda X, Y, Z: smooth_field(X, Y, Z, L, fn_seed))
    S.eval_mask()
    if mask:
        f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.write_fields(block_order_fields(S))
    return f, S


@pytest.mark.parametrize("seed,Bs", [(1, 9), (2, 17), (3, 9)])
def test_topology_is_bit_exact(A, seed, Bs):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=80)
    grid = _grid(Bs=Bs)
    f = A.Forest(grid, _phys())
    f.set_leaves(leaves)
    t = f.topology()
    fo = oracle_forest(grid, leaves=leaves)
    tc, lv, sl, nbr, rel = fo.topology()
    order = fo.sorted_leaves()
    assert np.array_equal(t["treecode"], tc)
    assert np.array_equal(t["level"], lv)
    assert np.array_equal(t["slot"], sl)
    assert np.array_equal(t["gx"], [l[1] for l in order])
    assert np.array_equal(t["nbr"], nbr)
    assert np.array_equal(t["rel"], rel)


def test_ungraded_layout_is_rejected(A):
    f = A.Forest(_grid(), _phys())
    bad = [(1, x, y, z) for z in range(2) for y in range(2) for x in range(4) if (x, y, z) != (0, 0, 0)]
    bad += [(3, x, y, z) for z in range(4) for y in range(4) for x in range(4)]  # two levels finer
    with pytest.raises(A.AcmError):
        f.set_leaves(bad)


@pytest.mark.parametrize("prec,Bs,seed", [(64, 9, 4), (64, 17, 5), (32, 9, 6)])
def test_sync_ghosts_matches_oracle(A, prec, Bs, seed):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=Bs, precision=prec)
    f, S = _pair(A, grid, _phys(), leaves, fn_seed=seed)
    gpu = f.sync_ghosts()
    ext = osync(S.fo, S.U, grid["g"], "cube")
    ref = np.stack([ext[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    assert not np.isnan(ref).any()
    err = rel_linf(gpu.astype(np.float64), ref)
    assert max(err) < (1e-13 if prec == 64 else 1e-6), err


# the stage kernel's forms (FP32: two points per thread; one; one with bulk-copy staging; one
# with a block's rows over two CTAs)
PAIR, POINT, TMA, ROWS = 0, 1, 2, 3


@pytest.mark.parametrize("prec,Bs,seed,masked,sponge,variant", [
    (64, 9, 7, True, True, POINT), (64, 17, 8, False, False, POINT), (32, 9, 9, True, True, PAIR),
    (32, 9, 9, True, True, POINT), (32, 17, 14, True, True, PAIR), (32, 17, 14, True, True, POINT),
    (32, 17, 14, True, True, TMA), (32, 9, 9, True, True, TMA), (32, 17, 16, False, False, TMA),
    (32, 17, 14, True, True, ROWS), (64, 9, 10, False, True, POINT)])
def test_fused_rhs_matches_oracle(A, prec, Bs, seed, masked, sponge, variant):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=Bs, precision=prec)
    phys = _phys(sponge=int(sponge), C_sp=0.05, u_inf=(0.4, -0.1, 0.2), p_inf=0.1,
                 sponge_L=(2.0, 1.0, 1.0), sponge_width=0.2, sponge_delta=0.05)
    mask = (0.8, 0.5, 0.5, 0.2, 0.04) if masked else None
    f, S = _pair(A, grid, phys, leaves, fn_seed=seed, mask=mask)
    f.set_stage_variant(variant)
    gpu = f.rhs().astype(np.float64)
    K = S.rhs(S.U.copy())
    ref = np.stack([K[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    err = rel_linf(gpu, ref)
    if prec == 64:
        assert max(err) < 1e-12, err
        return
    # FP32 against the oracle on the same state rounded to FP32: the rounding of the kernel's own
    # arithmetic, within the FP32 field tolerance
    U32 = S.U.astype(np.float32).astype(np.float64)
    K32 = S.rhs(U32)
    ref32 = np.stack([K32[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    err32 = rel_linf(gpu, ref32)
    print("fp32 rhs err vs fp64 state", err, "vs rounded state", err32)
    assert max(err32) < 2e-5, err32
    # against the unrounded FP64 state too (the stencils amplify the input's own rounding by
    # about 1/(k h); measured about 1e-6 here)
    assert max(err) < 2e-5, err


@pytest.mark.parametrize("prec,Bs,seed,variant", [(64, 9, 11, POINT), (64, 17, 12, POINT), (32, 17, 13, PAIR),
                                                  (32, 17, 13, POINT), (32, 9, 15, PAIR), (32, 17, 13, TMA),
                                                  (32, 17, 13, ROWS)])
def test_rk4_steps_match_oracle(A, prec, Bs, seed, variant):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=Bs, precision=prec)
    phys = _phys()
    mask = (1.2, 0.5, 0.5, 0.15, 0.05)
    f, S = _pair(A, grid, phys, leaves, fn_seed=seed, mask=mask)
    f.set_stage_variant(variant)
    dt = 2e-3 if Bs == 9 else 1e-3
    for _ in range(2):
        f.rk4_step(dt)
        S.rk4(dt)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err


@pytest.mark.parametrize("masked,other", [(True, TMA), (False, TMA), (True, ROWS), (False, ROWS)])
def test_bulk_copy_staging_is_bitwise_the_point_kernel(A, masked, other):
    """The one-point stage kernel with U, the accumulator and chi staged by bulk copies, and the
    one with a block's rows over two CTAs, compute bitwise what the one-point kernel with
    per-thread loads over whole blocks computes (FP32, graded layout, RK4 steps)."""
    leaves = random_graded_leaves(17, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=17, precision=32)
    mask = (1.2, 0.5, 0.5, 0.15, 0.05) if masked else None
    out = []
    for variant in (POINT, other):
        f, S = _pair(A, grid, _phys(), leaves, fn_seed=17, mask=mask)
        f.set_stage_variant(variant)
        for _ in range(2):
            f.rk4_step(1e-3)
        out.append(f.read_fields())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec,Bs", [(64, 9), (32, 17), (32, 9)])
def test_mask_matches_oracle(A, prec, Bs):
    """chi of every block (smoothed sphere, Sec. 2.2) against the oracle's FP64 values."""
    leaves = random_graded_leaves(16, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=Bs, precision=prec)
    mask = (0.9, 0.5, 0.5, 0.2, 0.02)
    f, S = _pair(A, grid, _phys(), leaves, fn_seed=16, mask=mask)
    chi = f.read_mask().astype(np.float64)
    ref = np.stack([S.chi[S.fo.leaves[l]] for l in S.fo.sorted_leaves()])
    assert chi.shape == ref.shape
    # FP32: the distance to the surface rounds at about 1e-7 of the box size, 5e-6 of delta in
    # the argument of tanh, so chi (in [0, 1]) is good to about half of that
    assert np.abs(chi - ref).max() <= (1e-14 if prec == 64 else 1e-5)
    assert np.all((chi >= 0.0) & (chi <= 1.0))


@pytest.mark.parametrize("prec,Bs", [(64, 9), (32, 17)])
def test_rk4_steps_device_dt_and_graph_match_host_steps(A, prec, Bs):
    """acm_rk4_steps (time step on the device, CUDA graph replay) gives bitwise the result of the
    same number of acm_rk4_step calls with the CFL rule, and the same simulated time."""
    leaves = random_graded_leaves(17, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=Bs, precision=prec)
    phys = _phys(sponge=1, C_sp=0.05, u_inf=(0.4, -0.1, 0.2), p_inf=0.1, sponge_L=(2.0, 1.0, 1.0),
                 sponge_width=0.2, sponge_delta=0.05)
    mask = (0.8, 0.5, 0.5, 0.2, 0.04)
    import torch
    st = torch.cuda.Stream()
    runs = []
    with torch.cuda.stream(st):
        for mode in ("host", "device", "graph"):
            f, _ = _pair(A, grid, phys, leaves, fn_seed=17, mask=mask)
            used = False
            if mode == "host":
                t = 0.0
                for _ in range(5):
                    t += f.rk4_step(0.0)
            else:
                t, used = f.rk4_steps(5, 0.0, graph=(mode == "graph"))
            runs.append((mode, t, used, f.read_fields()))
    (_, t0, _, u0), (_, t1, g1, u1), (_, t2, g2, u2) = runs
    assert not g1
    assert t1 == t0 and t2 == t0
    assert np.array_equal(u1, u0) and np.array_equal(u2, u0)


def test_autotune_keeps_the_state_and_the_results(A):
    """The autotuner only changes launch knobs: the state is what a synchronisation leaves, and a
    step after it is bitwise the step without it."""
    leaves = random_graded_leaves(18, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=17, precision=32)
    mask = (0.8, 0.5, 0.5, 0.2, 0.04)
    f, _ = _pair(A, grid, _phys(), leaves, fn_seed=18, mask=mask)
    g, _ = _pair(A, grid, _phys(), leaves, fn_seed=18, mask=mask)
    fw, sc = f.autotune()
    assert fw in (2, 4, 8, 16) and 1 <= sc <= 3
    g.sync_ghosts()                      # the same fine-wins update the autotuner made
    assert np.array_equal(f.read_fields(), g.read_fields())
    f.rk4_step(1e-3)
    g.rk4_step(1e-3)
    assert np.array_equal(f.read_fields(), g.read_fields())


@pytest.mark.parametrize("prec", [64, 32])
def test_indicators_match_oracle(A, prec):
    leaves = random_graded_leaves(14, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=70)
    grid = _grid(Bs=9, precision=prec)
    mask = (1.0, 0.5, 0.5, 0.2, 0.03)
    f, S = _pair(A, grid, _phys(), leaves, fn_seed=14, mask=mask)
    ind, rng = f.block_indicators()
    oind, _ = S.indicators(S.norms())
    order = S.fo.sorted_leaves()
    ref = np.array([oind[l][0] for l in order])
    rref = np.array([oind[l][1] for l in order])
    tol = 1e-12 if prec == 64 else 1e-4
    assert np.abs(ind - ref).max() <= tol * ref.max()
    assert np.abs(rng - rref).max() <= (1e-14 if prec == 64 else 1e-6)


@pytest.mark.parametrize("prec", [64, 32])
def test_refine_and_coarsen_match_oracle(A, prec):
    leaves = random_graded_leaves(15, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=40)
    grid = _grid(Bs=9, precision=prec, Jmax=3)
    phys = _phys(eps=3e-3)
    f, S = _pair(A, grid, phys, leaves, fn_seed=15)
    f.refine_all()
    S.refine_all()
    t = f.topology()
    tc, lv, sl, nbr, rel = S.fo.topology()
    assert np.array_equal(t["treecode"], tc) and np.array_equal(t["slot"], sl) and np.array_equal(t["nbr"], nbr)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err
    if prec == 64:
        nb, npass = f.coarsen()
        S.coarsen()
        t = f.topology()
        tc, lv, sl, nbr, rel = S.fo.topology()
        assert nb == len(S.fo.leaves)
        assert np.array_equal(t["treecode"], tc) and np.array_equal(t["slot"], sl)
        assert np.array_equal(t["nbr"], nbr) and np.array_equal(t["rel"], rel)
        err = rel_linf(f.read_fields(), block_order_fields(S))
        assert max(err) < TOL[prec], err


def test_adapt_is_the_coarsening(A):
    """acm_adapt (the adaptation call after a step) leaves the grid and state acm_coarsen leaves."""
    leaves = random_graded_leaves(15, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=40)
    grid = _grid(Bs=9, precision=64, Jmax=3)
    out = []
    for call in ("coarsen", "adapt"):
        f, _ = _pair(A, grid, _phys(eps=3e-3), leaves, fn_seed=15)
        f.refine_all()
        n = f.coarsen()[0] if call == "coarsen" else f.adapt()
        out.append((n, f.topology()["treecode"], f.read_fields()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec,Bs", [(64, 9), (32, 9), (64, 17), (32, 17)])
def test_cdf44_coarsen_to_jmin_matches_oracle(A, prec, Bs):
    """Every block tagged (huge threshold): the merges are decided by the grading alone, so the
    topology does not depend on the precision; several passes of the lifted low-pass."""
    leaves = random_graded_leaves(16 + Bs, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=60 if Bs == 9 else 30)
    grid = _grid(Bs=Bs, precision=prec, Jmax=3, wavelet=44)
    f, S = _pair(A, grid, _phys(eps=1e30), leaves, fn_seed=16)
    nb, npass = f.coarsen()
    opass = S.coarsen()
    assert npass == opass and nb == len(S.fo.leaves) == 16
    t = f.topology()
    tc, lv, sl, nbr, rel = S.fo.topology()
    assert np.array_equal(t["treecode"], tc) and np.array_equal(t["slot"], sl)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err


def test_cdf44_refine_and_coarsen_match_oracle(A):
    leaves = random_graded_leaves(17, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=40)
    grid = _grid(Bs=9, precision=64, Jmax=3, wavelet=44)
    f, S = _pair(A, grid, _phys(eps=3e-3), leaves, fn_seed=17)
    f.refine_all()
    S.refine_all()
    nb, npass = f.coarsen()
    opass = S.coarsen()
    t = f.topology()
    tc, lv, sl, nbr, rel = S.fo.topology()
    assert npass == opass >= 1 and nb == len(S.fo.leaves)
    assert np.array_equal(t["treecode"], tc) and np.array_equal(t["slot"], sl)
    assert np.array_equal(t["nbr"], nbr) and np.array_equal(t["rel"], rel)
    err = rel_linf(f.read_fields(), block_order_fields(S))
    assert max(err) < TOL[64], err
    # the two wavelets give different parents from the same refined state
    g40 = _grid(Bs=9, precision=64, Jmax=3, wavelet=40)
    f40, _ = _pair(A, g40, _phys(eps=3e-3), leaves, fn_seed=17)
    f40.refine_all()
    f40.coarsen()
    if np.array_equal(f40.topology()["treecode"], t["treecode"]):
        assert not np.array_equal(f40.read_fields(), f.read_fields())


def _small_sphere(prec, Jmax=3, wavelet=40):
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=Jmax, precision=prec,
                max_blocks=1 << 14, fd_scheme=1, wavelet=wavelet)
    dxm = 1.0 / ((1 << Jmax) * 8)
    phys = dict(nu=1e-3, c0=5.0, C_eta=1e-2, C_gamma=0.0, C_sp=0.25 / (5.0 * 20.0), u_inf=(1.0, 0.0, 0.0),
                p_inf=0.0, cfl=0.5, cfl_eta=1.0, cfl_nu=0.25, eps=1e-3, dealias=1, mask_range_thr=1e-5,
                sponge=1, sponge_L=(2.0, 1.0, 1.0), sponge_width=0.25, sponge_delta=1.5 * dxm)
    mask = (0.6, 0.5, 0.5, 0.15, 1.5 * dxm)
    return grid, phys, mask


@pytest.mark.parametrize("wavelet", [40, 44])
def test_adaptive_sphere_steps_match_oracle(A, wavelet):
    grid, phys, mask = _small_sphere(64, wavelet=wavelet)
    f = A.Forest(grid, phys)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    nb = f.init_grid(A.ACM_IC_UNIFORM, [1.0, 0.0, 0.0, 0.0])
    fo = oracle_forest(grid)
    S = oracle_solver(fo, phys, ic=lambda X, Y, Z: oacm.ic_uniform(X, Y, Z), mask=sphere_fn(mask),
                      sponge=sponge_fn(phys), wavelet=wavelet)
    S.initial_grid()
    assert nb == len(fo.leaves)
    assert np.array_equal(f.topology()["treecode"], fo.topology()[0])
    for _ in range(2):
        dt, n = f.step(0.0)
        S.refine_all()
        dto = S.dt_cfl()
        assert abs(dt - dto) <= 1e-14 * dto
        S.rk4(dto)
        S.coarsen()
        t = f.topology()
        tc, lv, sl, nbr, rel = fo.topology()
        assert np.array_equal(t["treecode"], tc) and np.array_equal(t["level"], lv)
        assert np.array_equal(t["slot"], sl) and np.array_equal(t["nbr"], nbr)
        err = rel_linf(f.read_fields(), block_order_fields(S))
        assert max(err) < 1e-12, err
    d = f.diagnostics()
    F, E = S.diagnostics()
    assert np.allclose(d["force"], F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
    assert abs(d["energy"] - E) <= 1e-12 * E


@pytest.mark.slow
@pytest.mark.parametrize("prec,steps", [(64, 20), (32, 3)])
def test_taylor_green_config(A, prec, steps):
    """Periodic unit cube, 4x4x4 blocks of 17^3, Taylor-Green, nu = 1e-2, c0 = 10, CFL 0.5."""
    grid = _grid(Bs=17, nroot=(1, 1, 1), Jmin=2, Jmax=2, precision=prec, max_blocks=64)
    phys = dict(nu=1e-2, c0=10.0, C_gamma=1.0, cfl=0.5)
    f = A.Forest(grid, phys)
    f.init_uniform(2)
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    fo = oracle_forest(grid, J=2)
    S = oracle_solver(fo, phys, ic=lambda X, Y, Z: oacm.ic_taylor_green(X, Y, Z))
    S.eval_ic()
    for _ in range(steps):
        dt = f.rk4_step(0.0)
        dto = S.dt_cfl()
        assert abs(dt - dto) <= (1e-15 if prec == 64 else 1e-6) * dto
        S.rk4(dt)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err
    d = f.diagnostics()
    _, E = S.diagnostics()
    assert abs(d["energy"] - E) <= (1e-12 if prec == 64 else 1e-5) * E


@pytest.mark.parametrize("prec,Bs", [(64, 9), (64, 17), (32, 17)])
def test_refine_then_cdf44_coarsen_restores_any_field(A, prec, Bs):
    """Biorthogonality of the lifted wavelet: refining every block (DD-4 prediction) and merging
    every group back with CDF 4/4 returns an arbitrary field on a uniform periodic grid."""
    M = Bs - 1
    N = 2 * M
    rng = np.random.default_rng(61)
    lat = rng.normal(size=(4, N, N, N))
    i = np.arange(Bs)
    blocks = []
    fo = oracle_forest(dict(nroot=(1, 1, 1), root_len=1.0, Bs=Bs, Jmin=1, Jmax=2), J=1, max_blocks=64)
    for (J, gx, gy, gz) in fo.sorted_leaves():
        zz, yy, xx = np.meshgrid((gz * M + i) % N, (gy * M + i) % N, (gx * M + i) % N, indexing="ij")
        blocks.append(lat[:, zz, yy, xx])
    field = np.stack(blocks)
    grid = _grid(Bs=Bs, nroot=(1, 1, 1), Jmin=1, Jmax=2, precision=prec, max_blocks=128, wavelet=44)
    f = A.Forest(grid, _phys(eps=1e30))
    f.init_uniform(1)
    f.write_fields(field)
    before = f.read_fields().astype(np.float64)
    f.refine_all()
    assert f.n_blocks() == 64
    nb, npass = f.coarsen()
    assert nb == 8 and npass == 1
    err = np.abs(f.read_fields().astype(np.float64) - before).max() / np.abs(before).max()
    # FP32: rounding amplified by the summed weights of the prediction and the low-pass (~8 in 3D)
    assert err < (1e-13 if prec == 64 else 5e-6), err


@pytest.mark.parametrize("prec,Bs", [(64, 9), (64, 17), (32, 9)])
def test_single_block_is_its_own_neighbour(A, prec, Bs):
    """The degenerate grid of one root at level 0: every one of the only block's 26 periodic
    neighbours is the block itself.  Neighbour table, two RK4 steps with a sphere mask, refinement
    to 8 blocks and coarsening back to the single block (dealiasing tags every finest block),
    against the oracle."""
    grid = _grid(Bs=Bs, nroot=(1, 1, 1), Jmin=0, Jmax=1, precision=prec, max_blocks=16)
    phys = _phys(eps=1e30, dealias=1)
    mask = (0.45, 0.5, 0.55, 0.2, 0.1)
    f = A.Forest(grid, phys)
    f.set_leaves([(0, 0, 0, 0)])
    fo = oracle_forest(grid, leaves=[(0, 0, 0, 0)], max_blocks=16)
    S = oracle_solver(fo, phys, mask=sphere_fn(mask))
    fill_from_function(S, lambda X, Y, Z: smooth_field(X, Y, Z, (1.0, 1.0, 1.0), 21))
    S.eval_mask()
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.write_fields(block_order_fields(S))
    t = f.topology()
    tc, lv, sl, nbr, rel = fo.topology()
    assert np.array_equal(t["nbr"], nbr) and np.array_equal(t["rel"], rel)
    dt = 2e-3 if Bs == 9 else 1e-3
    for _ in range(2):
        f.rk4_step(dt)
        S.rk4(dt)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err
    f.refine_all()
    S.refine_all()
    assert f.n_blocks() == len(S.fo.leaves) == 8
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err
    nb, npass = f.coarsen()
    S.coarsen()
    assert nb == len(S.fo.leaves) == 1 and npass == 1
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < TOL[prec], err


@pytest.mark.parametrize("prec,Bs", [(64, 9), (32, 17)])
def test_coarsen_everywhere_restores_the_step_grid(A, prec, Bs):
    """The performance cycle's coarsening (coarsen_everywhere = 1): after refine-all, every block
    the refinement made merges back, in as many passes as the grading needs, to the starting
    layout with bit-exact topology against the oracle's and, with CDF 4/0, the state bitwise."""
    from oracle.sync import fine_wins
    leaves = random_graded_leaves(51, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=60)
    grid = _grid(Bs=Bs, precision=prec, Jmax=4)
    phys = _phys(coarsen_everywhere=1)
    f = A.Forest(grid, phys)
    f.set_leaves(leaves)
    S = oracle_solver(oracle_forest(grid, leaves=leaves, max_blocks=grid["max_blocks"]), phys)
    fill_from_function(S, lambda X, Y, Z: smooth_field(X, Y, Z, (2.0, 1.0, 1.0), 51))
    S.eval_mask()
    f.write_fields(block_order_fields(S))
    f.sync_ghosts()                                       # fine wins on U, as refinement does
    fine_wins(S.fo, S.U)
    before = f.read_fields().copy()
    t0 = f.topology()
    f.refine_all()
    S.refine_all()
    nb, npass = f.coarsen()
    opass = S.coarsen()
    assert nb == len(leaves) == len(S.fo.leaves) and npass == opass >= 2
    t = f.topology()
    tc, lv, sl, nbr, rel = S.fo.topology()
    assert np.array_equal(t["treecode"], tc) and np.array_equal(t["slot"], sl) and np.array_equal(t["nbr"], nbr)
    assert np.array_equal(t["treecode"], t0["treecode"]) and np.array_equal(t["level"], t0["level"])
    assert np.array_equal(f.read_fields(), before)
