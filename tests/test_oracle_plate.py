"""Pins of the oracle's moving plate (Sec. 2.2 mask and solid velocity, time-dependent)."""
import math

import numpy as np

from oracle import acm
from oracle.adapt import Solver
from oracle.forest import Forest
from oracle.plate import MovingSolver, Plate, box_sdf, rot_y, rot_z


def test_rotations_and_angular_velocity():
    P = Plate()
    for t in (0.0, 0.13, 0.37, 0.8):
        R = P.rotation(t)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-15) and abs(np.linalg.det(R) - 1.0) < 1e-14
        h = 1e-5
        dR = (P.rotation(t + h) - P.rotation(t - h)) / (2 * h)
        Wm = dR @ R.T                                   # [omega]_x
        assert np.allclose(Wm, -Wm.T, atol=1e-7)
        w = np.array([Wm[2, 1], Wm[0, 2], Wm[1, 0]])
        assert np.allclose(w, P.omega(t), atol=1e-7)
    # t = 0: no stroke, full pitch; t = 1/4: full stroke, no pitch
    assert np.allclose(P.rotation(0.0), rot_y(math.radians(45.0)), atol=1e-15)
    assert np.allclose(P.rotation(0.25), rot_z(math.radians(60.0)), atol=1e-15)


def test_solid_velocity_is_the_material_derivative():
    P = Plate()
    rng = np.random.default_rng(0)
    xb = rng.uniform([-0.5, 0.0, -0.025], [0.5, 3.0, 0.025], size=(5, 3))
    for t in (0.05, 0.4, 0.77):
        h = 1e-5
        pos = lambda s: P.root + xb @ P.rotation(s).T      # x = root + R x_b
        v_fd = (pos(t + h) - pos(t - h)) / (2 * h)
        x = pos(t)
        _, us = P.fields(x[:, 0], x[:, 1], x[:, 2], t)
        assert np.abs(us.T - v_fd).max() < 1e-7 * np.abs(v_fd).max()


def test_box_signed_distance_against_a_sampled_surface():
    lo, hi = np.array([-0.5, 0.0, -0.1]), np.array([0.5, 2.0, 0.1])
    d = 0.01
    faces = []
    for a in range(3):
        b, c = [k for k in range(3) if k != a]
        u = np.arange(lo[b], hi[b] + d / 2, d)
        v = np.arange(lo[c], hi[c] + d / 2, d)
        U, V = np.meshgrid(u, v, indexing="ij")
        for side in (lo[a], hi[a]):
            F = np.zeros(U.shape + (3,))
            F[..., a], F[..., b], F[..., c] = side, U, V
            faces.append(F.reshape(-1, 3))
    S = np.concatenate(faces)
    rng = np.random.default_rng(1)
    P = rng.uniform(lo - 0.4, hi + 0.4, size=(300, 3))
    dist = np.sqrt(((P[:, None, :] - S[None, :, :]) ** 2).sum(-1)).min(axis=1)
    inside = np.all((P >= lo) & (P <= hi), axis=1)
    sd = box_sdf(P, lo, hi)
    assert np.all((sd < 0) == inside)
    assert np.abs(np.abs(sd) - dist).max() <= d * math.sqrt(2) / 2 + 1e-12
    # exact values on the axes through the centre
    c = (lo + hi) / 2
    assert box_sdf(c, lo, hi) == -0.1 and abs(box_sdf(c + [0.0, 0.0, 0.3], lo, hi) - 0.2) < 1e-15


def test_mask_is_one_half_on_the_plate_surface():
    P = Plate(delta=0.02)
    t = 0.3
    R = P.rotation(t)
    pts_b = np.array([[0.5, 1.0, 0.0], [0.0, 3.0, 0.0], [0.1, 2.0, 0.025], [-0.5, 0.5, -0.01]])
    x = P.root + pts_b @ R.T
    chi, _ = P.fields(x[:, 0], x[:, 1], x[:, 2], t)
    assert np.allclose(chi, 0.5, atol=1e-12)
    far = P.root + np.array([[0.0, -1.0, 0.0]]) @ R.T      # behind the root
    chi, _ = P.fields(far[:, 0], far[:, 1], far[:, 2], t)
    assert chi[0] < 1e-12


def _forest():
    fo = Forest(nroot=(1, 1, 1), root_len=8.0, Bs=9, Jmin=2, Jmax=2, max_blocks=128)
    fo.init_uniform(2)
    return fo


def test_moving_solver_uses_the_stage_times():
    fo = _forest()
    ph = acm.Physics(nu=1e-3, c0=5.0, C_eta=1e-2, C_gamma=0.0)
    S = MovingSolver(fo, ph, Plate(delta=0.3), ic=lambda X, Y, Z: np.zeros((4,) + X.shape))
    S.eval_ic()
    S.eval_mask()
    # from rest the right-hand side is the penalization alone: chi(t) u_s(t) / C_eta, p' = 0
    for t in (0.0, 0.21):
        K = S.rhs_at(S.U.copy(), t)
        for leaf, s in fo.leaves.items():
            X, Y, Z = acm.block_coords(fo, leaf)
            chi, us = S.plate.fields(X, Y, Z, t)
            assert np.allclose(K[s, :3], chi * us / ph.C_eta, rtol=0, atol=1e-12 * max(1.0, np.abs(us).max()) / ph.C_eta)
            assert np.all(K[s, 3] == 0.0)
    times = []
    orig = S.rhs_at
    S.rhs_at = lambda F, t: (times.append(t), orig(F, t))[1]
    S.t = 0.1
    S.rk4(0.02)
    assert np.allclose(times, [0.1, 0.11, 0.11, 0.12], rtol=0, atol=1e-15) and times[1] == times[2]
    assert abs(S.t - 0.12) < 1e-15


def test_static_plate_equals_the_static_solver():
    fo = _forest()
    ph = acm.Physics(nu=1e-3, c0=5.0, C_eta=1e-2, C_gamma=0.0)
    plate = Plate(phi_m=0.0, alpha_m=0.0, delta=0.3)
    ic = lambda X, Y, Z: np.stack([np.sin(X), np.cos(Y), 0.1 * np.sin(Z), 0.0 * X])
    A = MovingSolver(fo, ph, plate, ic=ic)
    A.eval_ic()
    A.eval_mask()
    B = Solver(fo, ph, ic=ic, mask=lambda X, Y, Z: plate.fields(X, Y, Z, 0.0)[0])
    B.eval_ic()
    B.eval_mask()
    for _ in range(2):
        A.rk4(0.01)
        B.rk4(0.01)
    sl = sorted(fo.leaves.values())
    assert np.array_equal(A.U[sl], B.U[sl])
    Fa, Ea = A.diagnostics()
    Fb, Eb = B.diagnostics()
    assert np.array_equal(Fa, Fb) and Ea == Eb


def test_fluid_moving_with_the_plate_feels_no_force():
    fo = _forest()
    ph = acm.Physics(nu=1e-3, c0=5.0, C_eta=1e-2, C_gamma=0.0)
    S = MovingSolver(fo, ph, Plate(delta=0.3), ic=lambda X, Y, Z: np.zeros((4,) + X.shape))
    S.eval_ic()
    S.t = 0.17
    S.eval_mask()
    for leaf, s in fo.leaves.items():
        S.U[s, :3] = S.us[s]                 # u = u_s everywhere: no relative motion
    F, E = S.diagnostics()
    assert np.all(F == 0.0) and E > 0
    for leaf, s in fo.leaves.items():
        S.U[s, :3] = 0.0
    F0, _ = S.diagnostics()
    assert np.abs(F0).max() > 0             # while a fluid at rest is pushed


# ---- the moving case's adjoint (gradient with respect to the pitch amplitude) --------------------

def test_alpha_derivatives_against_central_differences():
    from oracle.plate import plate_alpha_derivatives
    P = Plate(chord=0.3, span=0.35, thickness=0.1, root=(0.5, 0.5, 0.5), delta=0.06)
    rng = np.random.default_rng(7)
    X, Y, Z = (rng.uniform(0.2, 0.8, size=400) for _ in range(3))
    h = 1e-6
    for t in (0.1, 0.33, 0.7):
        dchi, dus = plate_alpha_derivatives(P, X, Y, Z, t)
        Pp = Plate(chord=0.3, span=0.35, thickness=0.1, root=(0.5, 0.5, 0.5), delta=0.06, alpha_m=P.alpha_m + h)
        Pm = Plate(chord=0.3, span=0.35, thickness=0.1, root=(0.5, 0.5, 0.5), delta=0.06, alpha_m=P.alpha_m - h)
        cp, up = Pp.fields(X, Y, Z, t)
        cm, um = Pm.fields(X, Y, Z, t)
        assert np.abs((cp - cm) / (2 * h) - dchi).max() <= 1e-6 * np.abs(dchi).max()
        assert np.abs((up - um) / (2 * h) - dus).max() <= 1e-8 * max(np.abs(dus).max(), 1e-30)


def _moving_case(alpha_m=math.radians(45.0)):
    fo = Forest(nroot=(1, 1, 1), root_len=1.0, Bs=9, Jmin=1, Jmax=1, max_blocks=16)
    fo.init_uniform(1)
    ph = acm.Physics(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5)
    plate = Plate(chord=0.3, span=0.35, thickness=0.1, root=(0.5, 0.5, 0.5), delta=0.06, alpha_m=alpha_m)
    S = MovingSolver(fo, ph, plate,
                     ic=lambda X, Y, Z: np.stack([np.sin(2 * math.pi * Y), 0.3 * np.cos(2 * math.pi * Z),
                                                  0.2 * np.sin(2 * math.pi * X), 0.0 * X]))
    S.t = 0.1
    S.eval_ic()
    S.eval_mask()
    return S


def _moving_objective(S, dt, n, w=0.1):
    J = 0.0
    for _ in range(n):
        S.rk4(dt)
        F, E = S.diagnostics()
        J += (F[0] + w * E) / n
    return J


def test_moving_adjoint_against_central_differences():
    from oracle.plate import MovingPlateAdjoint
    dt, n = 2e-3, 2
    S = _moving_case()
    adj = MovingPlateAdjoint(S, dt, n, checkpoint_every=1)
    U0 = S.U.copy()
    J, gU, ga = adj.gradient(U0)
    assert abs(_moving_objective(_moving_case(), dt, n) - J) <= 1e-13 * abs(J)
    h = 1e-4
    a0 = math.radians(45.0)
    fd = (_moving_objective(_moving_case(a0 + h), dt, n) - _moving_objective(_moving_case(a0 - h), dt, n)) / (2 * h)
    assert abs(fd - ga) <= 1e-4 * abs(fd), (fd, ga)
    rng = np.random.default_rng(8)
    sl = sorted(S.fo.leaves.values())
    d = np.zeros_like(U0)
    d[sl] = rng.normal(size=d[sl].shape)
    vals = []
    for sgn in (1, -1):
        T = _moving_case()
        T.U = U0 + sgn * h * d
        vals.append(_moving_objective(T, dt, n))
    fdu = (vals[0] - vals[1]) / (2 * h)
    assert abs(fdu - float((gU * d).sum())) <= 1e-7 * abs(fdu)
    # checkpointing every 2 steps recomputes the same arithmetic
    J2, gU2, ga2 = MovingPlateAdjoint(_moving_case(), dt, n, checkpoint_every=2).gradient(U0)
    assert J2 == J and np.array_equal(gU2, gU) and ga2 == ga
    # and so does binomial checkpointing with U_0 as the only snapshot (1 recomputed step)
    adj1 = MovingPlateAdjoint(_moving_case(), dt, n)
    J3, gU3, ga3 = adj1.gradient(U0, snapshots=1)
    assert adj1.last_advances == 1
    assert J3 == J and np.array_equal(gU3, gU) and ga3 == ga


def test_moving_vector_jacobian_product_against_central_differences():
    """L = <lam, U_N> over 2 steps of the moving case, random lam: the oracle's product against
    central differences of L through the moving solver's own steps, in the pitch amplitude and
    in a random direction of U_0; binomial checkpointing gives it bitwise."""
    from oracle.plate import MovingPlateAdjoint
    dt, n = 2e-3, 2
    S = _moving_case()
    adj = MovingPlateAdjoint(S, dt, n)
    U0 = S.U.copy()
    sl = sorted(S.fo.leaves.values())
    rng = np.random.default_rng(17)
    lam = np.zeros_like(U0)
    lam[sl] = rng.normal(size=lam[sl].shape)
    UN, g, ga = adj.vjp(U0, lam)

    def L(T):
        for _ in range(n):
            T.rk4(dt)
        return float((lam[sl] * T.U[sl]).sum())

    assert L(_moving_case()) == float((lam[sl] * UN[sl]).sum())
    h = 1e-4
    a0 = math.radians(45.0)
    fd = (L(_moving_case(a0 + h)) - L(_moving_case(a0 - h))) / (2 * h)
    assert abs(fd - ga) <= 1e-6 * abs(fd), (fd, ga)             # agreement 1.7e-8
    d = np.zeros_like(U0)
    d[sl] = rng.normal(size=d[sl].shape)
    vals = []
    for sgn in (1, -1):
        T = _moving_case()
        T.U = U0 + sgn * h * d
        vals.append(L(T))
    fdu = (vals[0] - vals[1]) / (2 * h)
    assert abs(fdu - float((g * d).sum())) <= 1e-7 * abs(fdu)
    UN2, g2, ga2 = MovingPlateAdjoint(_moving_case(), dt, n).vjp(U0, lam, snapshots=1)
    assert np.array_equal(UN2, UN) and np.array_equal(g2, g) and ga2 == ga
