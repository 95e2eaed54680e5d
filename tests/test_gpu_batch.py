"""Batched independent instances (the batched workload's synthetic inputs) through the C-ABI:
the pulse + vortex-ring initial condition against the FP64 oracle, RK4 steps of one instance
against the oracle, and the batched call (one CUDA graph per step for all instances) against the
same steps taken instance by instance, bit for bit."""
import numpy as np
import pytest

from oracle import acm as oacm
from paper_1912_05371_gb300 import workloads as W
from tests.gpu_util import block_order_fields, oracle_forest, oracle_solver, rel_linf

pytestmark = pytest.mark.gpu

PHYS = dict(nu=1e-3, c0=10.0, C_gamma=0.0, cfl=0.5, eps=1e-3)


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _grid(prec, Bs, Jmax, max_blocks=4096):
    return dict(nroot=(1, 1, 1), root_len=1.0, Bs=Bs, g=4, Jmin=1, Jmax=Jmax, precision=prec,
                max_blocks=max_blocks, fd_scheme=1)


def _forest(A, inst, prec, Bs, Jmax, stream=None):
    f = A.Forest(_grid(prec, Bs, Jmax), PHYS, stream=stream)
    f.set_leaves(inst["leaves"])
    f.set_ic(A.ACM_IC_PULSE_RING, inst["ic"])
    return f


def _oracle(inst, Bs, Jmax):
    g = _grid(64, Bs, Jmax)
    fo = oracle_forest(g, leaves=inst["leaves"])
    L = (1.0, 1.0, 1.0)
    S = oracle_solver(fo, PHYS, ic=lambda X, Y, Z: oacm.ic_pulse_ring(X, Y, Z, inst["pulse"], inst["ring"], L))
    S.eval_ic()
    return S


@pytest.mark.parametrize("prec", [64, 32])
def test_pulse_ring_initial_condition_matches_oracle(A, prec):
    inst = W.batched_instances(seed=3, n=1, nb_range=(20, 60), Jmax=3)[0]
    f = _forest(A, inst, prec, 9, 3)
    S = _oracle(inst, 9, 3)
    err = rel_linf(f.read_fields().astype(np.float64), block_order_fields(S))
    assert max(err) < (1e-14 if prec == 64 else 1e-6), err


def test_instance_rk4_steps_match_oracle(A):
    inst = W.batched_instances(seed=4, n=1, nb_range=(20, 60), Jmax=3)[0]
    f = _forest(A, inst, 64, 9, 3)
    S = _oracle(inst, 9, 3)
    total = 0.0
    for _ in range(2):
        dto = S.dt_cfl()
        S.rk4(dto)
        total += dto
    t, _ = f.rk4_steps(2, 0.0, graph=True)
    assert abs(t - total) <= 1e-14 * total
    err = rel_linf(f.read_fields(), block_order_fields(S))
    assert max(err) < 1e-12, err


@pytest.mark.parametrize("prec,Bs,mode", [(64, 9, 1), (32, 17, 1), (32, 17, 2), (64, 9, 2), (32, 9, 2)])
def test_batched_graph_equals_instance_by_instance(A, prec, Bs, mode):
    """The batched steps -- one graph of per-instance launch sequences (mode 1), or the persistent
    form with one stage launch walking the blocks of every instance (mode 2) -- give every instance
    bitwise the steps it takes alone."""
    import torch
    insts = W.batched_instances(seed=5, n=3, nb_range=(8, 80), Jmax=3)
    streams = [torch.cuda.Stream() for _ in insts]
    batch = [_forest(A, i, prec, Bs, 3, stream=s) for i, s in zip(insts, streams)]
    times, used = A.rk4_steps_batch(batch, 4, 0.0, graph=mode)
    assert used == mode
    for inst, s, tb, fb in zip(insts, streams, times, batch):
        f = _forest(A, inst, prec, Bs, 3, stream=s)
        t, _ = f.rk4_steps(4, 0.0, graph=False)
        assert t == tb
        assert np.array_equal(f.read_fields(), fb.read_fields())
