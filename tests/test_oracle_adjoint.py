"""Pins of the oracle's discrete adjoint (frozen grid, fixed dt).

The synchronisation matrices are checked against the oracle's synchronisation itself; the
block right-hand side's transposed Jacobian against central differences of the right-hand side
(exact for its quadratic and linear terms); one RK4 step's adjoint by the dot-product identity
against central differences of the oracle's own step; the whole gradient against central finite
differences with h = 1e-4 in FP64 of the objective computed by the oracle's solver and
diagnostics; checkpointed and stored-state sweeps against each other.
"""
import math

import numpy as np
import pytest

from oracle import acm
from oracle.adapt import Solver
from oracle.adjoint import FrozenGridAdjoint, SyncMatrices, rhs_block_vjp, sphere_mask_grad
from oracle.forest import Forest
from oracle.sync import fine_wins, local_points, sync
from paper_1912_05371_gb300.workloads import random_graded_leaves

L = (2.0, 1.0, 1.0)
CENTRE, RADIUS = (1.0, 0.5, 0.5), 0.2


def _field(X, Y, Z, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for f in range(4):
        v = np.full_like(X, 1.0 if f == 0 else 0.0)
        for _ in range(3):
            k = rng.integers(-2, 3, 3)
            a, ph = rng.uniform(0.05, 0.3), rng.uniform(0, 2 * math.pi)
            v = v + a * np.sin(2 * math.pi * (k[0] * X / L[0] + k[1] * Y / L[1] + k[2] * Z / L[2]) + ph)
        out.append(v)
    return np.stack(out)


def _setup(seed=41, n_target=18, centre=CENTRE, R=RADIUS, sponge=True):
    leaves = random_graded_leaves(seed, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=n_target)
    fo = Forest(nroot=(2, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=2, max_blocks=256)
    fo.set_leaves(leaves)
    delta = 1.5 * fo.h(2)
    ph = acm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0))
    S = Solver(fo, ph, ic=lambda X, Y, Z: _field(X, Y, Z, seed),
               mask=lambda X, Y, Z: acm.sphere_mask(X, Y, Z, centre, R, delta),
               sponge=(lambda X, Y, Z: acm.sponge_mask(X, Y, Z, L, 0.2, delta)) if sponge else None)
    S.eval_ic()
    S.eval_mask()
    return S, delta


def _objective(S, dt, nsteps, w=0.1):
    """J through the oracle's own solver and diagnostics."""
    J = 0.0
    for _ in range(nsteps):
        S.rk4(dt)
        F, E = S.diagnostics()
        J += (F[0] + w * E) / nsteps
    return J


def test_sync_matrices_equal_the_synchronisation():
    S, _ = _setup(seed=42, n_target=30)
    fo = S.fo
    m = SyncMatrices(fo)
    rng = np.random.default_rng(1)
    F = np.zeros_like(S.U)
    F[m.slots] = rng.normal(size=F[m.slots].shape)
    Fw = fine_wins(fo, F.copy())
    v = m.to_vec(F)
    assert np.array_equal(m.to_reg(np.stack([m.W @ v[f] for f in range(4)]), np.zeros_like(F))[m.slots],
                          Fw[m.slots])
    W = m.W.tocoo()
    assert (W.row != W.col).sum() > 0                 # some points are taken from finer leaves
    ext = sync(fo, F.copy(), 3, "faces")
    got = m.ext_of(np.stack([m.S @ v[f] for f in range(4)]))
    Pl = local_points(fo.M, 3, "faces") + 3
    for k, s in enumerate(m.slots):
        a = got[:, k][:, Pl[:, 2], Pl[:, 1], Pl[:, 0]]
        b = ext[s][:, Pl[:, 2], Pl[:, 1], Pl[:, 0]]
        assert np.abs(a - b).max() <= 1e-14 * np.abs(F).max()


def test_rhs_transpose_against_central_differences():
    S, _ = _setup()
    fo = S.fo
    leaf, s = next((l, s) for l, s in fo.leaves.items() if S.chi[s].max() > 1e-3)
    g, M, h = 3, fo.M, fo.h(leaf[0])
    rng = np.random.default_rng(2)
    ne = M + 1 + 2 * g
    e = 1.0 + 0.3 * rng.normal(size=(4, ne, ne, ne))
    v = rng.normal(size=e.shape)
    kap = rng.normal(size=(4, M + 1, M + 1, M + 1))
    chi, chisp = S.chi[s], S.chisp[s]
    de, dchi = rhs_block_vjp(e, g, M, h, S.ph, kap, chi=chi, chisp=chisp)
    eps = 1e-3        # the right-hand side is quadratic in e: central differences are exact
    rp = acm.rhs_block(e + eps * v, g, M, h, S.ph, chi=chi, chisp=chisp)
    rm = acm.rhs_block(e - eps * v, g, M, h, S.ph, chi=chi, chisp=chisp)
    lhs = float(((rp - rm) / (2 * eps) * kap).sum())
    assert abs(lhs - float((v * de).sum())) <= 1e-10 * abs(lhs)
    c = rng.normal(size=chi.shape)
    rp = acm.rhs_block(e, g, M, h, S.ph, chi=chi + eps * c, chisp=chisp)
    rm = acm.rhs_block(e, g, M, h, S.ph, chi=chi - eps * c, chisp=chisp)
    lhs = float(((rp - rm) / (2 * eps) * kap).sum())
    assert abs(lhs - float((c * dchi).sum())) <= 1e-10 * abs(lhs)


def test_mask_derivative_against_central_differences():
    X, Y, Z = np.meshgrid(*(np.linspace(0.3, 0.7, 9),) * 3, indexing="ij")
    c, R, d = (0.51, 0.48, 0.5), 0.12, 0.03
    g = sphere_mask_grad(X, Y, Z, c, R, d)
    h = 1e-6
    for a in range(4):
        th = list(c) + [R]
        tp, tm = list(th), list(th)
        tp[a] += h
        tm[a] -= h
        fd = (acm.sphere_mask(X, Y, Z, tp[:3], tp[3], d) - acm.sphere_mask(X, Y, Z, tm[:3], tm[3], d)) / (2 * h)
        assert np.abs(fd - g[a]).max() <= 1e-6 * np.abs(g[a]).max()


def test_one_step_adjoint_dot_product():
    S, delta = _setup()
    adj = FrozenGridAdjoint(S, CENTRE, RADIUS, delta, dt=2e-3, nsteps=1)
    rng = np.random.default_rng(3)
    U = S.U.copy()
    v = np.zeros_like(U)
    w = np.zeros_like(U)
    sl = adj.mats.slots
    v[sl] = rng.normal(size=v[sl].shape)
    w[sl] = rng.normal(size=w[sl].shape)
    eps = 1e-5
    up = adj._step(U + eps * v)[0]
    um = adj._step(U - eps * v)[0]
    lhs = float(((up - um) / (2 * eps) * w).sum())
    gchi = {s: np.zeros_like(S.chi[s]) for s in S.fo.leaves.values()}
    rhs = float((v * adj._step_adjoint(U, w, gchi)).sum())
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)
    # the step is the oracle solver's own step
    S2 = Solver(S.fo, S.ph)
    S2.U, S2.chi, S2.chisp = U.copy(), S.chi, S.chisp
    S2.rk4(2e-3)
    assert np.array_equal(S2.U[sl], adj._step(U)[0][sl])


@pytest.fixture(scope="module")
def grad_case():
    S, delta = _setup()
    dt, N = 2e-3, 4
    adj = FrozenGridAdjoint(S, CENTRE, RADIUS, delta, dt=dt, nsteps=N, checkpoint_every=2)
    U0 = S.U.copy()
    J, gU, gth = adj.gradient(U0)
    return S, delta, dt, N, adj, U0, J, gU, gth


def test_gradient_against_central_finite_differences(grad_case):
    S0, delta, dt, N, adj, U0, J, gU, gth = grad_case
    S, _ = _setup()
    assert abs(_objective(S, dt, N) - J) <= 1e-13 * abs(J)
    h = 1e-4
    theta = list(CENTRE) + [RADIUS]
    for a in range(4):
        tp, tm = list(theta), list(theta)
        tp[a] += h
        tm[a] -= h
        Sp, _ = _setup(centre=tp[:3], R=tp[3])
        Sm, _ = _setup(centre=tm[:3], R=tm[3])
        fd = (_objective(Sp, dt, N) - _objective(Sm, dt, N)) / (2 * h)
        assert abs(fd - gth[a]) <= 2e-4 * np.abs(gth).max(), (a, fd, gth[a])
    # initial state: a random direction over all entries, and single entries
    rng = np.random.default_rng(4)
    sl = adj.mats.slots
    d = np.zeros_like(U0)
    d[sl] = rng.normal(size=d[sl].shape)
    vals = []
    for sgn in (1, -1):
        S, _ = _setup()
        S.U = U0 + sgn * h * d
        vals.append(_objective(S, dt, N))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - float((gU * d).sum())) <= 1e-7 * abs(fd)
    idx = np.argwhere(np.abs(gU) > 0.1 * np.abs(gU).max())[:3]
    for s, f, z, y, x in idx:
        vals = []
        for sgn in (1, -1):
            S, _ = _setup()
            S.U = U0.copy()
            S.U[s, f, z, y, x] += sgn * h
            vals.append(_objective(S, dt, N))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gU[s, f, z, y, x]) <= 1e-6 * abs(gU).max()


def test_checkpointing_reproduces_the_stored_state_sweep(grad_case):
    S, delta, dt, N, adj, U0, J, gU, gth = grad_case
    J2, gU2, gth2 = adj.gradient(U0, store_all=True)
    assert J2 == J and np.array_equal(gU2, gU) and np.array_equal(gth2, gth)
    # binomial checkpointing with 2 snapshots: 4 recomputed steps (the closed form 2*4 - C(4,1))
    J3, gU3, gth3 = adj.gradient(U0, snapshots=2)
    assert adj.last_advances == 4
    assert J3 == J and np.array_equal(gU3, gU) and np.array_equal(gth3, gth)


def test_vector_jacobian_product_against_central_differences():
    """L = <lam, U_N> over 3 steps for a random lam: the oracle's vector-Jacobian product against
    central differences of L through the oracle solver's own steps, in a random direction of U_0
    and in the sphere's centre and radius; binomial checkpointing gives it bitwise."""
    S, delta = _setup()
    dt, N = 2e-3, 3
    adj = FrozenGridAdjoint(S, CENTRE, RADIUS, delta, dt=dt, nsteps=N)
    U0 = S.U.copy()
    sl = adj.mats.slots
    rng = np.random.default_rng(12)
    lam = np.zeros_like(U0)
    lam[sl] = rng.normal(size=lam[sl].shape)
    UN, g, gth = adj.vjp(U0, lam)

    def L(T):
        for _ in range(N):
            T.rk4(dt)
        return float((lam[sl] * T.U[sl]).sum())

    assert L(_setup()[0]) == float((lam[sl] * UN[sl]).sum())
    h = 1e-4
    v = np.zeros_like(U0)
    v[sl] = rng.normal(size=v[sl].shape)
    vals = []
    for sgn in (1, -1):
        T, _ = _setup()
        T.U = U0 + sgn * h * v
        vals.append(L(T))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - float((g * v).sum())) <= 1e-7 * abs(fd)
    theta = list(CENTRE) + [RADIUS]
    for a in range(4):
        tp, tm = list(theta), list(theta)
        tp[a] += h
        tm[a] -= h
        fd = (L(_setup(centre=tp[:3], R=tp[3])[0]) - L(_setup(centre=tm[:3], R=tm[3])[0])) / (2 * h)
        assert abs(fd - gth[a]) <= 2e-4 * np.abs(gth).max(), (a, fd, gth[a])
    UN2, g2, gth2 = adj.vjp(U0, lam, snapshots=1)
    assert adj.last_advances == 3
    assert np.array_equal(UN2, UN) and np.array_equal(g2, g) and np.array_equal(gth2, gth)


def test_vector_jacobian_product_without_a_mask():
    """The same product for a flow without a body (sponge only): central differences of
    L = <lam, U_N> in a random direction of U_0."""
    leaves = random_graded_leaves(41, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=18)
    fo = Forest(nroot=(2, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=2, max_blocks=256)
    fo.set_leaves(leaves)
    delta = 1.5 * fo.h(2)
    ph = acm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, C_sp=0.05, u_inf=(1.0, 0.0, 0.0))

    def make():
        S = Solver(fo, ph, ic=lambda X, Y, Z: _field(X, Y, Z, 41),
                   sponge=lambda X, Y, Z: acm.sponge_mask(X, Y, Z, L, 0.2, delta))
        S.eval_ic()
        S.eval_mask()
        return S

    S = make()
    dt, N = 2e-3, 2
    adj = FrozenGridAdjoint(S, None, None, None, dt=dt, nsteps=N)
    U0 = S.U.copy()
    sl = adj.mats.slots
    rng = np.random.default_rng(13)
    lam = np.zeros_like(U0)
    lam[sl] = rng.normal(size=lam[sl].shape)
    _, g, gth = adj.vjp(U0, lam)
    assert not gth.any()
    h = 1e-4
    v = np.zeros_like(U0)
    v[sl] = rng.normal(size=v[sl].shape)
    vals = []
    for sgn in (1, -1):
        T = make()
        T.U = U0 + sgn * h * v
        for _ in range(N):
            T.rk4(dt)
        vals.append(float((lam[sl] * T.U[sl]).sum()))
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - float((g * v).sum())) <= 1e-7 * abs(fd)
