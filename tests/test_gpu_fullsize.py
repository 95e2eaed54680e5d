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
    print(f"full-size rhs FP{prec} rel. Linf per field", err)
    # the oracle evaluates the right-hand side of the forest's own (FP32-rounded) state, so the
    # difference is the FP32 arithmetic of one evaluation
    assert max(err) < (1e-12 if prec == 64 else 2e-5), err


def check_cdf44_parents(grid, pre_leaves, pre_U, post_leaves, post_U, nsample=4, tol=2e-5):
    """Parents made by the first CDF 4/4 merging pass against the oracle's low-pass of the state
    before coarsening (after fine wins, as the coarsening applies them): boundary points bitwise
    (decimated), interior points within tol of the velocity scale.  With tags that do not change
    between passes (huge threshold: only the mask range keeps blocks), a surviving parent whose
    children were leaves and whose 56 surrounding child-sized boxes held no finer leaf was merged
    in the first pass.  Returns the number of parents checked."""
    from oracle.adapt import Solver
    from oracle.forest import Forest as OForest
    from oracle.sync import fine_wins
    fo = oracle_forest(grid, leaves=pre_leaves, max_blocks=grid["max_blocks"])
    order = fo.sorted_leaves()
    src = np.zeros((grid["max_blocks"], 4) + (grid["Bs"],) * 3)
    for i, l in enumerate(order):
        src[fo.leaves[l]] = pre_U[i]
    fine_wins(fo, src)
    S = Solver(fo, oacm.Physics(), wavelet="cdf44")
    pre = set(pre_leaves)
    post_idx = {l: i for i, l in enumerate(post_leaves)}

    def no_finer_around(p):
        J, px, py, pz = p
        for bz in range(-1, 3):
            for by in range(-1, 3):
                for bx in range(-1, 3):
                    if not (0 <= bx <= 1 and 0 <= by <= 1 and 0 <= bz <= 1):
                        if fo.box_status(J + 1, (2 * px + bx, 2 * py + by, 2 * pz + bz))[0] == "refined":
                            return False
        return True

    firsts = [p for p in post_leaves if all(k in pre for k in OForest.children_of(p)) and no_finer_around(p)]
    assert firsts, "no parent of the first merging pass"
    pick = [firsts[int(i)] for i in np.linspace(0, len(firsts) - 1, min(nsample, len(firsts)))]
    M = fo.M
    half = M // 2
    scale = float(np.abs(pre_U[:, :3]).max())
    for p in pick:
        got = post_U[post_idx[p]]
        lp = S.lowpass_parent(p, src)
        assert np.abs(got[:, 1:M, 1:M, 1:M] - lp).max() <= tol * scale
        kids = [fo.leaves[k] for k in OForest.children_of(p)]
        for z in range(M + 1):
            for y in range(M + 1):
                for x in range(M + 1):
                    if 0 < x < M and 0 < y < M and 0 < z < M:
                        continue
                    c = (x > half) | ((y > half) << 1) | ((z > half) << 2)
                    v = src[kids[c], :, 2 * z - (z > half) * M, 2 * y - (y > half) * M, 2 * x - (x > half) * M]
                    assert np.array_equal(got[:, z, y, x], v)
    return len(pick)


def test_full_size_sphere_cdf44_parents_match_oracle(A):
    """The benchmark's sphere workload and procedure (initial grid, a step, refinement, RK4) with the
    CDF 4/4 wavelet in FP32, with a threshold so large that only the mask range keeps blocks from
    merging: the parents of the first merging pass of the coarsening against the oracle."""
    cfg = W.sphere(Jmax=5)
    grid = dict(cfg["grid"], precision=32, max_blocks=6000, fd_scheme=1, wavelet=44)
    sp = cfg["sponge"]
    phys = dict(cfg["phys"], eps=1e30, dealias=int(cfg["dealias"]), mask_range_thr=cfg["mask_thr"],
                sponge=1, sponge_L=sp["L"], sponge_width=sp["L_sp"], sponge_delta=sp["delta"])
    m = cfg["mask"][1]
    f = A.Forest(grid, phys)
    f.set_mask(A.ACM_MASK_SPHERE, (*m["centre"], m["R"], m["delta"]))
    f.init_grid(A.ACM_IC_UNIFORM, [*cfg["ic"][1]["u0"], cfg["ic"][1]["p0"]])
    f.step(0.0)
    f.refine_all()
    f.rk4_step(0.0)
    t = f.topology()
    pre_leaves = list(zip(t["level"].tolist(), t["gx"].tolist(), t["gy"].tolist(), t["gz"].tolist()))
    pre_U = f.read_fields().astype(np.float64)
    f.coarsen()
    t = f.topology()
    post_leaves = list(zip(t["level"].tolist(), t["gx"].tolist(), t["gy"].tolist(), t["gz"].tolist()))
    post_U = f.read_fields().astype(np.float64)
    assert len(post_leaves) < len(pre_leaves)
    assert check_cdf44_parents(grid, pre_leaves, pre_U, post_leaves, post_U) >= 1
