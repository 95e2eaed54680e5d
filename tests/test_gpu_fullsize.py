"""Parity at the benchmark's full size: the sphere workload (box 4x2x2, levels 2..5, Bs = 17)
after the initial grid and one refinement -- 4608 blocks, 22.6 M points, the grid every RK4 stage
of the benchmark runs on -- with the fused right-hand side evaluated through the C-ABI in the
benchmark's launch configuration and by the FP64 oracle on the same state, element by element."""
import numpy as np
import pytest

from oracle import acm as oacm
from paper_1912_05371_gb300 import workloads as W
from tests.gpu_util import oracle_forest, oracle_solver, rel_linf

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


@pytest.mark.parametrize("prec", [32, 64])
def test_full_size_sphere_rhs_matches_oracle(A, prec):
    cfg = W.sphere(Jmax=5)
    grid = dict(cfg["grid"], precision=prec, max_blocks=6000, fd_scheme=1)
    sp = cfg["sponge"]
    phys = dict(cfg["phys"], eps=cfg["eps"], dealias=int(cfg["dealias"]), mask_range_thr=cfg["mask_thr"],
                sponge=1, sponge_L=sp["L"], sponge_width=sp["L_sp"], sponge_delta=sp["delta"])
    m = cfg["mask"][1]
    mask = (*m["centre"], m["R"], m["delta"])
    f = A.Forest(grid, phys)
    f.set_mask(A.ACM_MASK_SPHERE, mask)
    f.init_grid(A.ACM_IC_UNIFORM, [*cfg["ic"][1]["u0"], cfg["ic"][1]["p0"]])
    f.step(0.0)                       # a developed (non-uniform) state on the benchmark's grids
    f.refine_all()
    t = f.topology()
    assert len(t["level"]) == 4608
    leaves = list(zip(t["level"].tolist(), t["gx"].tolist(), t["gy"].tolist(), t["gz"].tolist()))
    U = f.read_fields().astype(np.float64)
    K = f.rhs().astype(np.float64)
    fo = oracle_forest(grid, leaves=leaves, max_blocks=6000)
    cx, cy, cz, R, d = mask
    S = oracle_solver(fo, phys, mask=lambda X, Y, Z: oacm.sphere_mask(X, Y, Z, (cx, cy, cz), R, d),
                      sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, phys["sponge_L"], phys["sponge_width"],
                                                              phys["sponge_delta"]))
    order = fo.sorted_leaves()
    assert np.array_equal(t["slot"], np.array([fo.leaves[l] for l in order]))
    for i, l in enumerate(order):
        S.U[fo.leaves[l]] = U[i]
    S.eval_mask()
    Ko = S.rhs(S.U.copy())
    ref = np.stack([Ko[fo.leaves[l]] for l in order])
    err = rel_linf(K, ref)
    # FP32: one derivative evaluation of FP32 data (see test_fused_rhs_matches_oracle)
    assert max(err) < (1e-12 if prec == 64 else 1e-4), err
