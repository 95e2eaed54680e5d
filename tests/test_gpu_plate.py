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
    assert np.abs(f.read_mask().astype(np.float64) - chi).max() < (1e-14 if prec == 64 else 1e-6)
    d = f.diagnostics()
    F, E = S.diagnostics()
    ftol = 1e-11 if prec == 64 else 1e-4
    assert np.abs(np.asarray(d["force"]) - F).max() <= ftol * np.abs(F).max(), (d["force"], F)
    assert abs(d["energy"] - E) <= ftol * E
