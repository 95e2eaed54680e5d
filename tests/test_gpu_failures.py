"""Failure detection with the faults made on the host (no kernel is made to fail): a non-finite
value written into the state is reported by the next step that takes its time step from the max
norms (ACM_ENUMERIC, before any stage runs) and the forest stays usable; a refinement that the
block pool cannot hold is refused (ACM_ECAPACITY) with the grid and the state unchanged."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRID = dict(nroot=(1, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=1, Jmax=3, max_blocks=64, fd_scheme=1)
PHYS = dict(nu=1e-2, c0=3.0, C_gamma=0.5, cfl=0.5)


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _forest(A, prec):
    f = A.Forest(dict(GRID, precision=prec), PHYS)
    f.init_uniform(1)
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    return f


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("bad", [math.nan, math.inf, -math.inf])
def test_non_finite_state_is_reported(A, prec, bad):
    f = _forest(A, prec)
    good = f.read_fields().copy()
    planted = good.copy()
    planted[3, 1, 4, 2, 5] = bad                           # one interior point of block 3, v
    f.write_fields(planted)
    with pytest.raises(A.AcmError, match="status 6"):
        f.rk4_step(0.0)
    with pytest.raises(A.AcmError, match="status 6"):
        f.diagnostics()                                    # it reduces the same norms
    f.write_fields(good)
    assert f.diagnostics()["time"] == 0.0                  # the failed step did not advance
    assert f.rk4_step(0.0) > 0.0
    assert np.isfinite(f.read_fields()).all()
    f.close()


@pytest.mark.parametrize("graph", [False, True])
def test_non_finite_state_is_reported_by_device_dt_steps(A, graph):
    """Steps with the time step on the device (plain launches or a CUDA graph) report a NaN
    planted in the state after their steps."""
    f = _forest(A, 32)
    planted = f.read_fields().copy()
    planted[5, 0, 3, 3, 3] = math.nan
    f.write_fields(planted)
    with pytest.raises(A.AcmError, match="status 6"):
        f.rk4_steps(3, 0.0, graph=graph)
    f.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_refinement_beyond_the_pool_is_refused_and_changes_nothing(A, prec):
    f = _forest(A, prec)
    f.refine_all()                                         # 8 -> 64 blocks: the pool is full
    assert f.n_blocks() == 64
    topo, fields = f.topology(), f.read_fields().copy()
    with pytest.raises(A.AcmError, match="status 3"):
        f.refine_all()                                     # 512 blocks do not fit
    after = f.topology()
    assert all(np.array_equal(topo[k], after[k]) for k in topo)
    assert np.array_equal(f.read_fields(), fields)
    assert f.rk4_step(0.0) > 0.0                           # and the forest still steps
    f.close()
