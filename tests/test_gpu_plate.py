"""The moving plate (time-dependent mask and solid velocity) through the C-ABI against the oracle's
MovingSolver: the state after RK4 steps with the mask evaluated at every stage time, the mask at
the final time, and the force with u - u_s."""
import math

import numpy as np
import pytest

from oracle import acm as oacm
from oracle.plate import MovingSolver, Plate
from tests.gpu_util import block_order_fields, oracle_forest, rel_linf

pytestmark = pytest.mark.gpu

PLATE = dict(chord=0.25, span=0.3, thickness=0.06, phi_m=math.radians(60.0), alpha_m=math.radians(45.0),
             freq=1.0, root=(0.5, 0.5, 0.5), delta=0.03)


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


GRID = dict(nroot=(1, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=2, Jmax=2, max_blocks=128, fd_scheme=1)
DT, NSTEPS = 2e-3, 3


@pytest.fixture(scope="module")
def oracle_run():
    fo = oracle_forest(GRID, J=2, max_blocks=256)
    S = MovingSolver(fo, oacm.Physics(nu=1e-2, c0=5.0, C_eta=1e-2, C_gamma=0.5), Plate(**PLATE),
                     ic=lambda X, Y, Z: oacm.ic_taylor_green(X, Y, Z))
    S.eval_ic()
    S.eval_mask()
    for _ in range(NSTEPS):
        S.rk4(DT)
    return S


@pytest.mark.parametrize("prec", [64, 32])
def test_moving_plate_steps_match_oracle(A, oracle_run, prec):
    grid = dict(GRID, precision=prec)
    phys = dict(nu=1e-2, c0=5.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5)
    f = A.Forest(grid, phys)
    f.init_uniform(2)
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    P = PLATE
    f.set_mask(A.ACM_MASK_PLATE, [P["chord"], P["span"], P["thickness"], P["phi_m"], P["alpha_m"], P["freq"],
                                  *P["root"], P["delta"]])
    for _ in range(NSTEPS):
        f.rk4_step(DT)
    S = oracle_run
    fo = S.fo
    tol = 1e-12 if prec == 64 else 2e-5
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < tol, err
    chi = np.stack([S.chi[fo.leaves[l]] for l in fo.sorted_leaves()])
    # FP32: the signed distance carries ~1e-7 absolute rounding, i.e. ~3e-6 of d/delta at delta = 0.03
    assert np.abs(f.read_mask().astype(np.float64) - chi).max() < (1e-14 if prec == 64 else 1e-5)
    d = f.diagnostics()
    F, E = S.diagnostics()
    ftol = 1e-11 if prec == 64 else 1e-4
    assert np.abs(np.asarray(d["force"]) - F).max() <= ftol * np.abs(F).max(), (d["force"], F)
    assert abs(d["energy"] - E) <= ftol * E


@pytest.mark.parametrize("ckpt,prec", [(dict(ckpt_every=1), 64), (dict(snapshots=1), 64), (dict(ckpt_every=2), 32)])
def test_moving_plate_adjoint_matches_oracle(A, ckpt, prec):
    """The gradient of the moving case with respect to the pitch amplitude (8 blocks of 9^3, 2
    steps) against the oracle's adjoint, which is pinned by central differences: FP64 with
    equidistant checkpoints or binomial checkpointing with U_0 as the only snapshot, to rounding;
    FP32 (states, adjoint variables and the box's per-point sensitivity in FP32, the sums onto the
    parameter in FP64) within the FP32 rounding of the mask's signed distance."""
    from oracle.forest import Forest as OForest
    from oracle.plate import MovingPlateAdjoint
    from tests.test_gpu_adjoint import _per_point
    P = dict(chord=0.3, span=0.35, thickness=0.1, phi_m=math.radians(60.0), alpha_m=math.radians(45.0), freq=1.0,
             root=(0.5, 0.5, 0.5), delta=0.06)
    ic = lambda X, Y, Z: np.stack([np.sin(2 * math.pi * Y), 0.3 * np.cos(2 * math.pi * Z),
                                   0.2 * np.sin(2 * math.pi * X), 0.0 * X])
    fo = OForest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=1, max_blocks=16)
    fo.init_uniform(1)
    S = MovingSolver(fo, oacm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5), Plate(**P), ic=ic)
    S.eval_ic()
    S.eval_mask()
    dt, n = 2e-3, 2
    Jo, gUo, gao = MovingPlateAdjoint(S, dt, n, checkpoint_every=1).gradient(S.U.copy())
    grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=1, precision=prec, max_blocks=16,
                fd_scheme=1)
    f = A.Forest(grid, dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5))
    f.init_uniform(1)
    f.write_fields(block_order_fields(S))
    f.set_mask(A.ACM_MASK_PLATE, [P["chord"], P["span"], P["thickness"], P["phi_m"], P["alpha_m"], P["freq"],
                                  *P["root"], P["delta"]])
    before = f.read_fields().copy()
    J, ga, gU = f.adjoint_plate_pitch(n, dt, w_energy=0.1, **ckpt)
    assert np.array_equal(f.read_fields(), before) and f.diagnostics()["time"] == 0.0
    go = np.stack([gUo[fo.leaves[l]] for l in fo.sorted_leaves()])
    a, b = _per_point(fo, gU, 1), _per_point(fo, go, 1)
    tol_J, tol_g = (1e-12, 1e-10) if prec == 64 else (1e-5, 1e-4)
    print(f"plate adjoint FP{prec}: J {J} vs {Jo}, dJ/dalpha_m {ga} vs {gao}")
    assert abs(J - Jo) <= tol_J * abs(Jo), (J, Jo)
    assert abs(ga - gao) <= tol_g * abs(gao), (ga, gao)
    assert np.abs(a - b).max() <= tol_g * np.abs(b).max()


def test_moving_plate_vjp_matches_oracle(A):
    """The vector-Jacobian product of 2 steps of the moving case (FP64, 8 blocks of 9^3, random
    lam on every copy of every point, binomial checkpointing with one snapshot): dL/dU_0 per
    physical point and dL/d alpha_m against the oracle's product, which is pinned by central
    differences."""
    from oracle.forest import Forest as OForest
    from oracle.plate import MovingPlateAdjoint
    from tests.test_gpu_adjoint import _per_point
    P = dict(chord=0.3, span=0.35, thickness=0.1, phi_m=math.radians(60.0), alpha_m=math.radians(45.0), freq=1.0,
             root=(0.5, 0.5, 0.5), delta=0.06)
    ic = lambda X, Y, Z: np.stack([np.sin(2 * math.pi * Y), 0.3 * np.cos(2 * math.pi * Z),
                                   0.2 * np.sin(2 * math.pi * X), 0.0 * X])
    fo = OForest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=1, max_blocks=16)
    fo.init_uniform(1)
    S = MovingSolver(fo, oacm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5), Plate(**P), ic=ic)
    S.eval_ic()
    S.eval_mask()
    order = fo.sorted_leaves()
    lamB = np.random.default_rng(31).normal(size=(len(order), 4, 9, 9, 9))
    lam = np.zeros_like(S.U)
    for r, l in enumerate(order):
        lam[fo.leaves[l]] = lamB[r]
    dt, n = 2e-3, 2
    _, go, gao = MovingPlateAdjoint(S, dt, n).vjp(S.U.copy(), lam)
    grid = dict(nroot=(1, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=1, precision=64, max_blocks=16, fd_scheme=1)
    f = A.Forest(grid, dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5))
    f.init_uniform(1)
    f.write_fields(block_order_fields(S))
    f.set_mask(A.ACM_MASK_PLATE, [P["chord"], P["span"], P["thickness"], P["phi_m"], P["alpha_m"], P["freq"],
                                  *P["root"], P["delta"]])
    gU, gth = f.adjoint_vjp(n, dt, lamB, snapshots=1)
    assert f.diagnostics()["time"] == 0.0
    gob = np.stack([go[fo.leaves[l]] for l in order])
    a, b = _per_point(fo, gU, 1), _per_point(fo, gob, 1)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    assert abs(gth[0] - gao) <= 1e-10 * abs(gao), (gth[0], gao)


@pytest.mark.slow
@pytest.mark.parametrize("Bs,Jmax,precs", [(17, 5, (64, 32)), (33, 4, (32,))])
def test_fullscale_twin_force_series(A, Bs, Jmax, precs):
    """The full-scale plate case on its coarsened twin (box 8^3, fluid at rest, nu = 1/2000,
    C_eta = 1e-4, c0 = 30): blocks of 17^3 at levels 2..5 (FP64 and FP32 fields) and the
    configuration's blocks of 33^3 at levels 2..4 (FP32; the same finest spacing): the initial
    grid of the paper's procedure (built by the first precision's path), then 4 RK4 steps of fixed
    dt on that grid against the oracle's MovingSolver: the force F = C_eta^-1 int chi (u - u_s)
    after every step.  Run with -s to print the series."""
    from oracle.forest import Forest as OForest
    from paper_1912_05371_gb300 import workloads as W
    cfg = W.plate_fullscale(Jmax=Jmax, Bs=Bs)
    pl = cfg["plate"]
    params = [pl["chord"], pl["span"], pl["thickness"], pl["phi_m"], pl["alpha_m"], pl["freq"], *pl["root"],
              pl["delta"]]
    phys = dict(cfg["phys"], eps=cfg["eps"], dealias=1, mask_range_thr=cfg["mask_thr"])
    forests = {}
    leaves = None
    for prec in precs:
        f = A.Forest(dict(cfg["grid"], precision=prec, max_blocks=4096, fd_scheme=1), phys)
        f.set_mask(A.ACM_MASK_PLATE, params)
        if leaves is None:
            f.init_grid(A.ACM_IC_UNIFORM, [0.0, 0.0, 0.0, 0.0])
            t = f.topology()
            leaves = list(zip(t["level"].tolist(), t["gx"].tolist(), t["gy"].tolist(), t["gz"].tolist()))
        else:
            f.set_leaves(leaves)
            f.set_mask(A.ACM_MASK_PLATE, params)
        forests[prec] = f
    g = cfg["grid"]
    # the oracle's pool holds these leaves only (its registers are dense over the pool's slots)
    fo = OForest(nroot=g["nroot"], root_len=g["root_len"], Bs=g["Bs"], Jmin=g["Jmin"], Jmax=g["Jmax"],
                 max_blocks=len(leaves) + 8)
    fo.set_leaves(leaves)
    ph = oacm.Physics(nu=phys["nu"], c0=phys["c0"], C_eta=phys["C_eta"], C_gamma=phys["C_gamma"])
    plate = Plate(chord=pl["chord"], span=pl["span"], thickness=pl["thickness"], phi_m=pl["phi_m"],
                  alpha_m=pl["alpha_m"], freq=pl["freq"], root=pl["root"], delta=pl["delta"])
    S = MovingSolver(fo, ph, plate, ic=lambda X, Y, Z: oacm.ic_uniform(X, Y, Z, (0.0, 0.0, 0.0), 0.0))
    S.eval_ic()
    S.eval_mask()
    dt = 1e-4
    print(f"\n{len(leaves)} blocks of {Bs}^3; step  F_x oracle  rel. error " + "  ".join(f"FP{p}" for p in precs))
    for step in range(1, 5):
        S.rk4(dt)
        F, _ = S.diagnostics()
        errs = {}
        for prec, f in forests.items():
            f.rk4_step(dt)
            d = f.diagnostics()
            errs[prec] = float(np.abs(np.asarray(d["force"]) - F).max() / np.abs(F).max())
        print(f"{step:4d}  {F[0]: .6e}  " + "  ".join(f"{errs[p]:.2e}" for p in precs))
        assert errs.get(64, 0.0) <= 1e-11 and errs[32] <= 1e-4, (step, errs)
