"""The CUDA discrete adjoint (frozen grid, fixed dt, FP64) against the oracle's.

The objective and its gradient with respect to the sphere's centre and radius are compared
directly; the gradient with respect to U_0 is compared per physical point, summed over the
blocks that hold the point (the two forward maps read a shared point from different copies, so
only the sum over the copies is the same linear functional)."""
import numpy as np
import pytest

from oracle.adjoint import FrozenGridAdjoint
from tests.gpu_util import block_order_fields
from tests.test_oracle_adjoint import CENTRE, RADIUS, L, _setup
from paper_1912_05371_gb300.workloads import random_graded_leaves

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _gpu_forest(A, S, delta, seed=41, n_target=18, precision=64):
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=2, precision=precision, max_blocks=256,
                fd_scheme=1)
    phys = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0), p_inf=0.0,
                sponge=1, sponge_L=L, sponge_width=0.2, sponge_delta=delta)
    f = A.Forest(grid, phys)
    f.set_leaves(random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=n_target))
    f.set_mask(A.ACM_MASK_SPHERE, (*CENTRE, RADIUS, delta))
    f.write_fields(block_order_fields(S))
    return f


def _per_point(fo, blocks, Jmax):
    """Sum block-order arrays (n, 4, Bs, Bs, Bs) over the copies of each physical point."""
    M = fo.M
    Nf = np.array(fo.npoints(Jmax))
    keys, vals = [], []
    i = np.arange(M + 1)
    for r, (J, gx, gy, gz) in enumerate(fo.sorted_leaves()):
        sc = 1 << (Jmax - J)
        Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
        gxi = np.mod((gx * M + X) * sc, Nf[0])
        gyi = np.mod((gy * M + Y) * sc, Nf[1])
        gzi = np.mod((gz * M + Z) * sc, Nf[2])
        keys.append(((gzi * Nf[1] + gyi) * Nf[0] + gxi).ravel())
        vals.append(blocks[r].reshape(4, -1))
    keys = np.concatenate(keys)
    vals = np.concatenate(vals, axis=1)
    uk, inv = np.unique(keys, return_inverse=True)
    out = np.zeros((4, uk.size))
    for c in range(4):
        np.add.at(out[c], inv.ravel(), vals[c])
    return out


DT, N, C = 2e-3, 4, 2


@pytest.fixture(scope="module")
def oracle_gradient():
    S, delta = _setup()
    adj = FrozenGridAdjoint(S, CENTRE, RADIUS, delta, dt=DT, nsteps=N, checkpoint_every=C)
    Jo, gUo, gtho = adj.gradient(S.U.copy())
    return S, delta, Jo, gUo, gtho


@pytest.mark.parametrize("prec,tol_J,tol_g", [(64, 1e-12, 1e-10), (32, 1e-5, 1e-4)])
def test_adjoint_matches_the_oracle(A, oracle_gradient, prec, tol_J, tol_g):
    """FP64: the same arithmetic up to rounding.  FP32 forward states (the adjoint variables
    and sums stay FP64): within the FP32 rounding of the states the coefficients come from."""
    S, delta, Jo, gUo, gtho = oracle_gradient
    f = _gpu_forest(A, S, delta, precision=prec)
    before = f.read_fields().copy()
    J, gth, gU = f.adjoint_sphere(N, DT, ckpt_every=C, w_energy=0.1)
    assert np.array_equal(f.read_fields(), before)
    fo = S.fo
    go = np.stack([gUo[fo.leaves[l]] for l in fo.sorted_leaves()])
    a, b = _per_point(fo, gU, 2), _per_point(fo, go, 2)
    info = (J, Jo, gth, gtho, [float(np.abs(a[k] - b[k]).max() / np.abs(b).max()) for k in range(4)])
    assert abs(J - Jo) <= tol_J * abs(Jo), info
    assert np.abs(gth - gtho).max() <= tol_g * np.abs(gtho).max(), info
    assert np.abs(a - b).max() <= tol_g * np.abs(b).max(), info


@pytest.mark.parametrize("ckpt", [dict(snapshots=1), dict(snapshots=2), dict(snapshots=3), dict(ckpt_every=1),
                                  dict(ckpt_every=3), dict(ckpt_every=8)])
def test_every_checkpoint_schedule_gives_the_oracles_gradient(A, oracle_gradient, ckpt):
    """Binomial checkpointing with 1-3 snapshots and equidistant checkpoints at other spacings
    take the same steps in the same arithmetic (FP64): the oracle's gradient, which is itself
    the same for every schedule, and the forest's state and time unchanged."""
    S, delta, Jo, gUo, gtho = oracle_gradient
    f = _gpu_forest(A, S, delta, precision=64)
    before = f.read_fields().copy()
    J, gth, gU = f.adjoint_sphere(N, DT, w_energy=0.1, **ckpt)
    assert np.array_equal(f.read_fields(), before) and f.diagnostics()["time"] == 0.0
    fo = S.fo
    go = np.stack([gUo[fo.leaves[l]] for l in fo.sorted_leaves()])
    a, b = _per_point(fo, gU, 2), _per_point(fo, go, 2)
    assert abs(J - Jo) <= 1e-12 * abs(Jo), (J, Jo)
    assert np.abs(gth - gtho).max() <= 1e-10 * np.abs(gtho).max(), (gth, gtho)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()


def test_adjoint_through_autograd(A):
    import torch
    S, delta = _setup()
    f = _gpu_forest(A, S, delta)
    Fn = A.sphere_objective_function()
    U0 = torch.tensor(block_order_fields(S), dtype=torch.float64, requires_grad=True)
    th = torch.tensor([*CENTRE, RADIUS, delta], dtype=torch.float64, requires_grad=True)
    J = Fn.apply(f, U0, th, 3, 2e-3, 2, 0.1)
    J.backward()
    J2, gth, gU = f.adjoint_sphere(3, 2e-3, ckpt_every=2, w_energy=0.1)
    # the scatter and the parameter sums add with FP64 atomics: equal up to their order
    assert float(J.detach()) == J2
    assert np.allclose(th.grad.numpy()[:4], gth, rtol=0, atol=1e-12 * np.abs(gth).max())
    assert th.grad.numpy()[4] == 0.0
    assert np.allclose(U0.grad.numpy(), gU, rtol=0, atol=1e-12 * np.abs(gU).max())


NV = 3


@pytest.fixture(scope="module")
def oracle_vjp():
    S, delta = _setup()
    fo = S.fo
    order = fo.sorted_leaves()
    rng = np.random.default_rng(23)
    lamB = rng.normal(size=(len(order), 4, fo.M + 1, fo.M + 1, fo.M + 1))
    lam = np.zeros_like(S.U)
    for r, l in enumerate(order):
        lam[fo.leaves[l]] = lamB[r]
    adj = FrozenGridAdjoint(S, CENTRE, RADIUS, delta, dt=DT, nsteps=NV)
    UN, g, gth = adj.vjp(S.U.copy(), lam)
    return S, delta, lamB, UN, g, gth


@pytest.mark.parametrize("prec,tol,ckpt", [(64, 1e-10, dict(ckpt_every=2)), (64, 1e-10, dict(snapshots=1)),
                                           (32, 1e-4, dict(snapshots=2))])
def test_vjp_matches_the_oracle(A, oracle_vjp, prec, tol, ckpt):
    """dL/dU_0 and dL/d(centre, radius) of L = <lam, U_N> (3 steps, lam random on every copy of
    every point) against the oracle's vector-Jacobian product, which is pinned by central
    differences: FP64 to rounding; an FP32 forward (FP64 adjoint) within the FP32 rounding of the
    states its coefficients come from.  The forest's state is unchanged."""
    S, delta, lamB, UNo, go, gtho = oracle_vjp
    f = _gpu_forest(A, S, delta, precision=prec)
    before = f.read_fields().copy()
    gU, gth = f.adjoint_vjp(NV, DT, lamB, **ckpt)
    assert np.array_equal(f.read_fields(), before) and f.diagnostics()["time"] == 0.0
    fo = S.fo
    gob = np.stack([go[fo.leaves[l]] for l in fo.sorted_leaves()])
    a, b = _per_point(fo, gU, 2), _per_point(fo, gob, 2)
    assert np.abs(a - b).max() <= tol * np.abs(b).max()
    assert np.abs(gth - gtho).max() <= tol * np.abs(gtho).max(), (gth, gtho)


def test_step_map_through_autograd(A, oracle_vjp):
    """U_N of the autograd step map equals the forest's own steps and the oracle's; the gradient
    of a loss of U_N equals the direct vector-Jacobian product (up to the order of FP64 atomic
    sums); the forest is left at U_0 and time 0."""
    import torch
    S, delta, lamB, UNo, go, gtho = oracle_vjp
    f = _gpu_forest(A, S, delta, precision=64)
    Fn = A.step_map_function()
    U0 = torch.tensor(block_order_fields(S), dtype=torch.float64, requires_grad=True)
    th = torch.tensor([*CENTRE, RADIUS, delta], dtype=torch.float64, requires_grad=True)
    W = torch.tensor(lamB)
    UN = Fn.apply(f, U0, th, NV, DT, 2)
    fo = S.fo
    UNob = np.stack([UNo[fo.leaves[l]] for l in fo.sorted_leaves()])
    assert np.abs(UN.detach().numpy() - UNob).max() <= 1e-12 * np.abs(UNob).max()
    assert np.array_equal(f.read_fields(), block_order_fields(S)) and f.diagnostics()["time"] == 0.0
    (UN * W).sum().backward()
    gU, gth = f.adjoint_vjp(NV, DT, lamB, ckpt_every=2)
    assert np.allclose(U0.grad.numpy(), gU, rtol=0, atol=1e-12 * np.abs(gU).max())
    assert np.allclose(th.grad.numpy()[:4], gth, rtol=0, atol=1e-12 * np.abs(gth).max())
    assert th.grad.numpy()[4] == 0.0


def test_vjp_without_a_mask_matches_the_oracle(A):
    """The vector-Jacobian product of a flow without a body (sponge only; 2 steps, FP64) against
    the oracle's, which is pinned by central differences."""
    from oracle import acm as oacm
    from oracle.adapt import Solver
    from oracle.forest import Forest as OForest
    from tests.test_oracle_adjoint import _field
    leaves = random_graded_leaves(41, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=18)
    fo = OForest(nroot=(2, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=2, max_blocks=256)
    fo.set_leaves(leaves)
    delta = 1.5 * fo.h(2)
    S = Solver(fo, oacm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0)),
               ic=lambda X, Y, Z: _field(X, Y, Z, 41),
               sponge=lambda X, Y, Z: oacm.sponge_mask(X, Y, Z, L, 0.2, delta))
    S.eval_ic()
    S.eval_mask()
    order = fo.sorted_leaves()
    lamB = np.random.default_rng(29).normal(size=(len(order), 4, 9, 9, 9))
    lam = np.zeros_like(S.U)
    for r, l in enumerate(order):
        lam[fo.leaves[l]] = lamB[r]
    _, go, _ = FrozenGridAdjoint(S, None, None, None, dt=DT, nsteps=2).vjp(S.U.copy(), lam)
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=2, precision=64, max_blocks=256, fd_scheme=1)
    phys = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0), p_inf=0.0,
                sponge=1, sponge_L=L, sponge_width=0.2, sponge_delta=delta)
    f = A.Forest(grid, phys)
    f.set_leaves(leaves)
    f.write_fields(block_order_fields(S))
    gU, gth = f.adjoint_vjp(2, DT, lamB, snapshots=1)
    assert not gth.any()
    gob = np.stack([go[fo.leaves[l]] for l in order])
    a, b = _per_point(fo, gU, 2), _per_point(fo, gob, 2)
    assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
