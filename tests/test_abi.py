"""The C-ABI library loads and exports every entry point include/acm.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "acm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(acm_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1912_05371_gb300 import build
    return build.build()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for n in ("acm_create_forest", "acm_set_mask", "acm_rk4_step", "acm_coarsen", "acm_refine_all",
              "acm_sync_ghosts", "acm_diagnostics", "acm_get_topology"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header_and_pool_size_is_host_only(libpath):
    from paper_1912_05371_gb300 import acm
    assert set(declared_functions()) <= set(acm.EXPORTS)
    L = acm.lib()
    g = acm.GridParams()
    g.nroot = (ctypes.c_int * 3)(2, 1, 1)
    g.root_len, g.Bs, g.g, g.Jmin, g.Jmax, g.precision, g.max_blocks, g.fd_scheme = 2.0, 17, 4, 2, 5, 32, 1000, 1
    n = L.acm_pool_bytes(ctypes.byref(g))
    assert n > 1000 * 4 * 17 ** 3 * 4 * 4          # at least the four RK registers
    g.Bs = 12
    assert L.acm_pool_bytes(ctypes.byref(g)) == 0  # invalid block size is rejected
    assert L.acm_status_string(3) == b"block pool exhausted"


def test_host_only_argument_checks(libpath):
    """Calls that are refused before any device work: an unknown wavelet, and the adjoint entry
    points without a forest."""
    from paper_1912_05371_gb300 import acm
    L = acm.lib()
    g = acm.GridParams()
    g.nroot = (ctypes.c_int * 3)(2, 1, 1)
    g.root_len, g.Bs, g.g, g.Jmin, g.Jmax, g.precision, g.max_blocks, g.fd_scheme = 2.0, 17, 4, 2, 5, 32, 1000, 1
    sizes = {}
    for w in (0, 40, 44, 43):
        g.wavelet = w
        sizes[w] = L.acm_pool_bytes(ctypes.byref(g))
    assert sizes[0] == sizes[40] == sizes[44] > 0 and sizes[43] == 0
    assert L.acm_adjoint_bytes(None, 10, 2) == 0
    J = ctypes.c_double()
    einval = 1
    assert L.acm_adjoint_sphere(None, 4, 1e-3, 2, 0.1, None, 0, ctypes.byref(J), None, None, 0, 0) == einval
    assert L.acm_adjoint_plate_pitch(None, 4, 1e-3, 2, 0.1, None, 0, ctypes.byref(J), None, None, 0, 0) == einval
    assert L.acm_adjoint_vjp(None, 4, 1e-3, 2, None, 0, None, None, 0, 0, None) == einval
    assert L.acm_set_time(None, 0.0) == einval
    assert L.acm_write_mask(None, None, 0, 0) == einval
    assert L.acm_load_state(None, b"missing.acm") == einval and L.acm_save_state(None, b"x.acm") == einval


def test_pool_limits_of_the_33_cubed_blocks(libpath):
    """Blocks of 33^3 take FP32 fields and the CDF 4/0 merge only, and every block size keeps the
    element offsets of a register and of the coarse-face slab buffer within 32 bits: the largest
    accepted max_blocks holds fewer than 2^32 elements in one register of four components, and
    not far fewer (the full-scale plate's 29,000 blocks of 33^3 fit)."""
    from paper_1912_05371_gb300 import acm
    L = acm.lib()
    g = acm.GridParams()
    g.nroot = (ctypes.c_int * 3)(1, 1, 1)
    g.root_len, g.Bs, g.g, g.Jmin, g.Jmax, g.precision, g.max_blocks, g.fd_scheme = 8.0, 33, 4, 2, 7, 32, 29000, 1

    def size(**kw):
        for k, v in kw.items():
            setattr(g, k, v)
        return L.acm_pool_bytes(ctypes.byref(g))

    assert size(precision=32, wavelet=40) > 29000 * 4 * 4 * 33 ** 3 * 4     # four RK registers
    assert size(wavelet=0) == size(wavelet=40)
    assert size(wavelet=44) == 0 and size(wavelet=40, precision=64) == 0
    for Bs, prec in ((9, 32), (17, 32), (17, 64), (33, 32)):
        lo, hi = 1, 1 << 30
        g.precision, g.Bs, g.wavelet = prec, Bs, 40
        assert size(max_blocks=lo) > 0
        while hi - lo > 1:                  # the largest accepted max_blocks
            mid = (lo + hi) // 2
            if size(max_blocks=mid) > 0:
                lo = mid
            else:
                hi = mid
        assert lo * 4 * Bs ** 3 < 1 << 32, (Bs, prec, lo)
        assert lo > 0.9 * (1 << 32) / (4 * (Bs + 2) ** 3), (Bs, prec, lo)  # not far below the cap
