"""The caller's mask field (ACM_MASK_FIELD): written as the sphere mask's own chi it gives the
sphere-masked forest's steps and diagnostics bitwise, its vector-Jacobian product (up to the order
of FP64 atomic sums, with no parameter gradient) and a bitwise restart; calls that would change the
grid it belongs to are refused and change nothing."""
import numpy as np
import pytest

from tests.test_gpu_adjoint import DT, _gpu_forest
from tests.test_oracle_adjoint import _setup
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


def _twins(A, prec):
    S, delta = _setup()
    f = _gpu_forest(A, S, delta, precision=prec)          # the sphere mask, evaluated analytically
    g = _gpu_forest(A, S, delta, precision=prec)
    chi = f.read_mask()
    g.set_mask(A.ACM_MASK_FIELD)
    assert not g.read_mask().any()                        # zero until written
    g.write_mask(chi)
    assert np.array_equal(g.read_mask(), chi)
    return f, g


@pytest.mark.parametrize("prec", [64, 32])
def test_field_mask_steps_like_the_sphere(A, prec):
    f, g = _twins(A, prec)
    for _ in range(2):
        f.rk4_step(DT)
        g.rk4_step(DT)
    assert np.array_equal(f.read_fields(), g.read_fields())
    assert f.diagnostics() == g.diagnostics()
    assert f.rk4_step(0.0) == g.rk4_step(0.0)             # the C_eta limit of dt applies to both


def test_field_mask_refuses_grid_changes(A):
    f, g = _twins(A, 64)
    before, n = g.read_fields().copy(), g.n_blocks()
    for call in (g.refine_all, g.coarsen, lambda: g.init_uniform(1),
                 lambda: g.set_leaves(random_graded_leaves(41, nroot=(2, 1, 1), J0=1, Jmax=2, n_target=18))):
        with pytest.raises(A.AcmError, match="status 1"):
            call()
    assert g.n_blocks() == n and np.array_equal(g.read_fields(), before)
    g.set_mask(A.ACM_MASK_NONE)
    g.refine_all()                                        # allowed again without the field
    assert g.n_blocks() > n


def test_field_mask_vjp_and_restart(A, tmp_path):
    f, g = _twins(A, 64)
    lam = np.random.default_rng(37).normal(size=f.read_fields().shape)
    gf, thf = f.adjoint_vjp(2, DT, lam, snapshots=1)
    gg, thg = g.adjoint_vjp(2, DT, lam, snapshots=1)
    assert np.allclose(gg, gf, rtol=0, atol=1e-12 * np.abs(gf).max())
    assert thf.any() and not thg.any()
    path = str(tmp_path / "field.acm")
    g.rk4_step(DT)
    g.save(path)
    h = A.Forest.from_file(path)
    assert np.array_equal(h.read_mask(), g.read_mask()) and np.array_equal(h.read_fields(), g.read_fields())
    g.rk4_step(DT)
    h.rk4_step(DT)
    assert np.array_equal(h.read_fields(), g.read_fields()) and h.diagnostics() == g.diagnostics()


@pytest.mark.parametrize("prec", [64, 32])
def test_field_mask_on_a_grid_whose_slots_are_out_of_block_order(A, prec):
    """After refinement and a partial coarsening the slots are no longer in block order and
    reach far past max_blocks / 4 (the merged parents take the lowest free slots, the kept
    children keep theirs): the field mask written there reads back unchanged and steps like the
    sphere mask it copies, bitwise."""
    delta = 1.5 / (4 * 8)
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=2, precision=prec, max_blocks=128,
                fd_scheme=1)
    phys = dict(nu=1e-2, c0=3.0, C_eta=1e-2, C_gamma=0.5, eps=1e-3, dealias=0)

    def forest():
        f = A.Forest(grid, phys)
        f.init_uniform(1)
        f.set_mask(A.ACM_MASK_SPHERE, (1.0, 0.5, 0.5, 0.2, delta))
        f.set_ic(A.ACM_IC_UNIFORM, (1.0, 0.0, 0.0, 0.0))
        f.refine_all()
        f.coarsen()
        return f

    f, g = forest(), forest()
    slots = f.topology()["slot"]
    n = f.n_blocks()
    assert n > grid["max_blocks"] // 4 and slots.max() >= grid["max_blocks"] // 4
    assert np.any(np.diff(slots) < 0)                     # not in block order
    assert np.array_equal(g.topology()["slot"], slots)
    chi = f.read_mask()
    assert 0.0 < chi.max() and chi.min() < chi.max()
    g.set_mask(A.ACM_MASK_FIELD)
    g.write_mask(chi)
    assert np.array_equal(g.read_mask(), chi)
    # a field that differs from block to block makes a misplaced block visible; an analytic one
    # keeps every copy of a redundant point equal (the synchronisation relies on that)
    for h in (f, g):
        h.set_ic(A.ACM_IC_TAYLOR_GREEN, (2 * np.pi, 1.0))
    U = f.read_fields()
    assert np.array_equal(g.read_fields(), U) and np.abs(np.diff(U[:, 0, 4, 4, 4])).max() > 0
    for _ in range(2):
        f.rk4_step(1e-3)
        g.rk4_step(1e-3)
    assert np.array_equal(f.read_fields(), g.read_fields())
    assert f.diagnostics() == g.diagnostics()
