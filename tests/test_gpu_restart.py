"""Restart files through the C-ABI: a forest resumed from a file (acm_save_state, then
acm_read_state_header + acm_load_state) holds the same grid, state, mask, parameters and time,
and continues bitwise like the forest that saved it (adaptive sphere steps in FP32 and FP64, the
moving plate at a time t > 0).  Loads of another grid, into too small a pool, or of a truncated
file are refused and leave the forest unchanged."""
import math

import numpy as np
import pytest

from paper_1912_05371_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm
    acm.lib()
    return acm


def _sphere_forest(A, precision, Jmax=3):
    cfg = W.sphere(Jmax=Jmax)
    grid = dict(cfg["grid"], precision=precision, max_blocks=3000, fd_scheme=1)
    sp = cfg["sponge"]
    phys = dict(cfg["phys"], eps=cfg["eps"], dealias=int(cfg["dealias"]), mask_range_thr=cfg["mask_thr"], sponge=1,
                sponge_L=sp["L"], sponge_width=sp["L_sp"], sponge_delta=sp["delta"])
    m = cfg["mask"][1]
    f = A.Forest(grid, phys)
    f.set_mask(A.ACM_MASK_SPHERE, (*m["centre"], m["R"], m["delta"]))
    f.init_grid(A.ACM_IC_UNIFORM, [*cfg["ic"][1]["u0"], cfg["ic"][1]["p0"]])
    return f


PLATE_GRID = dict(nroot=(1, 1, 1), root_len=1.0, Bs=9, g=4, Jmin=2, Jmax=2, precision=64, max_blocks=128,
                  fd_scheme=1)
PLATE_PHYS = dict(nu=1e-2, c0=5.0, C_eta=1e-2, C_gamma=0.5, cfl=0.5)
PLATE = [0.25, 0.3, 0.06, math.radians(60.0), math.radians(45.0), 1.0, 0.5, 0.5, 0.5, 0.03]


def _plate_forest(A, grid=PLATE_GRID):
    f = A.Forest(grid, PLATE_PHYS)
    f.init_uniform(2)
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    f.set_mask(A.ACM_MASK_PLATE, PLATE)
    return f


def _same(f, g):
    ta, tb = f.topology(), g.topology()
    for k in ("treecode", "level", "gx", "gy", "gz", "rel"):        # slots may differ
        assert np.array_equal(ta[k], tb[k]), k
    assert np.array_equal(f.read_fields(), g.read_fields())
    assert np.array_equal(f.read_mask(), g.read_mask())
    assert f.diagnostics() == g.diagnostics()


@pytest.mark.parametrize("prec", [32, 64])
def test_resumed_sphere_run_continues_bitwise(A, tmp_path, prec):
    f = _sphere_forest(A, prec)
    for _ in range(2):
        f.step()
    path = str(tmp_path / "sphere.acm")
    f.save(path)
    grid, phys, n, t = A.read_state_header(path)
    assert n == f.n_blocks() and t == f.diagnostics()["time"] > 0.0 and grid["precision"] == prec
    g = A.Forest.from_file(path)
    _same(f, g)
    for _ in range(2):
        assert f.step() == g.step()
    _same(f, g)


def test_resumed_plate_run_continues_bitwise(A, tmp_path):
    f = _plate_forest(A)
    for _ in range(3):
        f.rk4_step(2e-3)
    path = str(tmp_path / "plate.acm")
    f.save(path)
    g = A.Forest.from_file(path)
    _same(f, g)
    for _ in range(2):
        f.rk4_step(2e-3)
        g.rk4_step(2e-3)
    _same(f, g)


def test_refused_loads_leave_the_forest_unchanged(A, tmp_path):
    f = _plate_forest(A)
    f.rk4_step(2e-3)
    path = str(tmp_path / "p.acm")
    f.save(path)
    with pytest.raises(A.AcmError, match="status 1"):
        _plate_forest(A, dict(PLATE_GRID, Jmax=3)).load(path)            # another grid
    with pytest.raises(A.AcmError, match="status 3"):
        A.Forest(dict(PLATE_GRID, max_blocks=32), PLATE_PHYS).load(path)  # 64 blocks do not fit
    blob = open(path, "rb").read()
    cut = str(tmp_path / "cut.acm")
    with open(cut, "wb") as fh:
        fh.write(blob[: len(blob) // 2])
    g = _plate_forest(A)
    before, d0 = g.read_fields().copy(), g.diagnostics()
    with pytest.raises(A.AcmError, match="status 1"):
        g.load(cut)
    assert np.array_equal(g.read_fields(), before) and g.diagnostics() == d0
