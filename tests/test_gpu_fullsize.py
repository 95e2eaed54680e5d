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


def test_full_size_33_cubed_offsets_past_2_31_rk4_step_matches_oracle(A):
    """Blocks of 33^3 in slots whose element offsets pass 2^31, as in the full-scale plate case
    (up to 29,000 blocks of 33^3, 4.2e9 elements per register): a uniform periodic grid of 16,384
    blocks (box 4x1x1, level 4, 589 M points, a 56 GB pool) with a smooth state that differs
    between the four roots, one RK4 step through the stage kernels; sampled blocks -- the two
    highest slots, the slots around the first one whose block starts past 2^31 elements, and
    the first slot, whose -x neighbour across the periodic seam is in the last root -- against
    the oracle's step on their neighbourhood."""
    import math

    import torch

    from tests.gpu_util import oracle_physics, rk4_on_neighbourhood, uniform_neighbourhood
    Bs, J, nroot = 33, 4, (4, 1, 1)
    M = Bs - 1
    grid = dict(nroot=nroot, root_len=1.0, Bs=Bs, g=4, Jmin=J, Jmax=J, precision=32, max_blocks=16400,
                fd_scheme=1)
    phys = dict(nu=1e-2, c0=10.0, C_gamma=1.0, cfl=0.5)
    f = A.Forest(grid, phys)
    f.init_uniform(J)
    t = f.topology()
    n = len(t["slot"])
    assert n == 16384
    nb = tuple(r << J for r in nroot)
    h = 1.0 / ((1 << J) * M)
    dev = torch.device("cuda", torch.cuda.current_device())
    # a few Fourier modes of the box 4x1x1 (seeded), plus one of period 4 in x, at x = i h with i
    # the wrapped global lattice index, built on the device
    rng = np.random.default_rng(71)
    modes = [[(rng.integers(-2, 3, 3), rng.uniform(0.2, 1.0), rng.uniform(0, 2 * math.pi)) for _ in range(3)]
             for _ in range(4)]
    Lb = [float(r) for r in nroot]
    i = torch.arange(Bs, device=dev, dtype=torch.float64)
    gxyz = [torch.as_tensor(t[k].astype(np.int64), device=dev) for k in ("gx", "gy", "gz")]
    U0 = torch.empty((n, 4, Bs, Bs, Bs), dtype=torch.float32, device=dev)
    for c0 in range(0, n, 1024):
        sl = slice(c0, min(n, c0 + 1024))
        X, Y, Z = (((g[sl, None] * M + i) % (nb[a] * M)) * h for a, g in enumerate(gxyz))
        X, Y, Z = X[:, None, None, :], Y[:, None, :, None], Z[:, :, None, None]
        for fc in range(4):
            v = 0.3 * torch.sin(2 * math.pi * X / Lb[0])
            for k, a, ph in modes[fc]:
                v = v + a * torch.sin(2 * math.pi * (int(k[0]) * X / Lb[0] + int(k[1]) * Y / Lb[1]
                                                     + int(k[2]) * Z / Lb[2]) + ph)
            U0[sl, fc] = v.to(torch.float32)
    f.write_fields(U0)
    dt = 5e-5
    f.rk4_step(dt)
    U1 = torch.empty_like(U0)
    f.read_fields(out=U1)
    torch.cuda.synchronize()

    slot = t["slot"].astype(np.int64)
    past = -(-(1 << 31) // (4 * Bs ** 3))   # a register's block stride is at least 4 Bs^3 elements
    assert slot.max() >= past + 1
    by_slot = {int(s): b for b, s in enumerate(slot)}
    by_xyz = {(int(t["gx"][b]), int(t["gy"][b]), int(t["gz"][b])): b for b in range(n)}
    cache = {}

    def get(x, y, z):
        b = by_xyz[(x, y, z)]
        if b not in cache:
            cache[b] = U0[b].double().cpu().numpy()
        return cache[b]

    ph = oracle_physics(phys)
    got, ref, moved = [], [], 0.0
    for s in (n - 1, n - 2, past - 1, past, past + 1, 0):
        b = by_slot[s]
        xyz = (int(t["gx"][b]), int(t["gy"][b]), int(t["gz"][b]))
        E = uniform_neighbourhood(get, nb, *xyz, M, 12)
        ref.append(rk4_on_neighbourhood(E, M, h, ph, dt))
        got.append(U1[b].double().cpu().numpy())
        moved = max(moved, float(np.abs(ref[-1] - get(*xyz)).max()))
    err = rel_linf(np.stack(got), np.stack(ref))
    print("33^3 blocks past 2^31 elements: RK4 step rel. Linf per field", err, "largest change", moved)
    assert max(err) < 2e-5, err
    assert moved > 1e-3                     # the step changed the state well above the tolerance
