"""The restart-file header as the library reads it (acm_read_state_header; host only, no GPU):
a file laid out as include/acm.h documents is read back field by field, and foreign, truncated,
other-version or inconsistent files are refused."""
import ctypes as C
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def A():
    from paper_1912_05371_gb300 import acm, build
    build.build()
    acm.lib()
    return acm


def _file(A, path, n=3, version=1, magic=b"ACMSTATE", precision=32, mask_kind=1, max_blocks=100, cut=None):
    g = A.GridParams()
    g.nroot = (C.c_int * 3)(2, 1, 1)
    g.root_len, g.Bs, g.g, g.Jmin, g.Jmax, g.precision, g.max_blocks, g.fd_scheme, g.wavelet = (
        2.0, 9, 4, 1, 4, precision, max_blocks, 1, 44)
    p = A.PhysParams()
    p.nu, p.c0, p.C_eta, p.eps, p.sponge = 1e-3, 20.0, 1e-3, 1e-3, 1
    p.sponge_L = (C.c_double * 3)(4.0, 2.0, 2.0)
    head = magic + struct.pack("<6i", version, precision, C.sizeof(g), C.sizeof(p), mask_kind, 0)
    head += struct.pack("<10d", 1.0, 1.0, 1.0, 0.25, 0.01, 0, 0, 0, 0, 0) + struct.pack("<dq", 0.375, n)
    leaves = np.zeros(4 * n, np.int32)
    fields = np.zeros(n * 4 * 9 ** 3, np.float32 if precision == 32 else np.float64)
    blob = head + bytes(g) + bytes(p) + leaves.tobytes() + fields.tobytes()
    with open(path, "wb") as fh:
        fh.write(blob if cut is None else blob[:cut])
    return g, p


def test_header_fields_read_back(A, tmp_path):
    path = tmp_path / "a.acm"
    g, p = _file(A, path)
    grid, phys, n, t = A.read_state_header(str(path))
    assert n == 3 and t == 0.375
    assert grid["nroot"] == (2, 1, 1) and grid["Bs"] == 9 and grid["wavelet"] == 44 and grid["precision"] == 32
    assert grid["max_blocks"] == 100 and grid["Jmax"] == 4
    assert phys["c0"] == 20.0 and phys["sponge"] == 1 and phys["sponge_L"] == (4.0, 2.0, 2.0)


@pytest.mark.parametrize("bad", [dict(magic=b"ACMSTATX"), dict(version=2), dict(n=0), dict(n=101),
                                 dict(mask_kind=5), dict(precision=16), dict(cut=40), dict(cut=100)])
def test_foreign_or_inconsistent_files_are_refused(A, tmp_path, bad):
    path = tmp_path / "b.acm"
    _file(A, path, **bad)
    with pytest.raises(A.AcmError):
        A.read_state_header(str(path))


def test_missing_file_and_no_forest(A, tmp_path):
    with pytest.raises(A.AcmError):
        A.read_state_header(str(tmp_path / "missing.acm"))
    L = A.lib()
    assert L.acm_load_state(None, b"x") == 1 and L.acm_save_state(None, b"x") == 1
