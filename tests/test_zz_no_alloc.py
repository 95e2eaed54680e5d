"""The allocation-free max-norm entry point (acm_max_norms_noalloc) against the forest's own
norms (acm_diagnostics), called through the C-ABI twice in a row on changing data.

It is for callers that cannot allocate device memory when they call it (their memory is owned
by another allocator, or they must avoid the synchronisation an allocation can imply, or they
hold a field array but no forest); its scratch is an array compiled into the library.  This file
is collected last so that a run stopping at its first failure has already run every other test.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [32, 64])
def test_no_alloc_norms_match_the_forest_norms(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_05371_gb300 import acm as A
    from paper_1912_05371_gb300.workloads import random_graded_leaves

    Bs = 17
    grid = dict(nroot=(2, 1, 1), root_len=1.0, Bs=Bs, g=4, Jmin=1, Jmax=3, precision=precision,
                max_blocks=2048, fd_scheme=1)
    phys = dict(nu=1e-2, c0=3.0, C_gamma=0.5, cfl=0.5)
    stream = torch.cuda.current_stream()
    f = A.Forest(grid, phys, stream=stream)
    f.set_leaves(random_graded_leaves(21, nroot=(2, 1, 1), J0=1, Jmax=3, n_target=60))
    f.set_ic(A.ACM_IC_TAYLOR_GREEN, [2 * math.pi, 1.0])
    dtype = torch.float32 if precision == 32 else torch.float64
    tol = 1e-12
    for call in range(2):
        f.rk4_step(1e-3)                      # the data change between the two calls
        n = f.n_blocks()
        dense = torch.empty(n * 4 * Bs ** 3, dtype=dtype, device="cuda")
        f.read_fields(dense)
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        st = A.max_norms_noalloc(dense, n, Bs, precision, out, stream)
        assert st == 0, A.lib().acm_status_string(st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        d = f.diagnostics()
        ref = np.array(list(d["norms"]) + [d["u_max"]])
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= tol * np.abs(ref).max()), (call, got, ref)

    # a NaN and an infinity in the state reach the norms as they reach the forest's own: here
    # an infinity in v and a NaN in p (at other points), so |v| and the speed are infinite
    # and |p| is NaN, while |u| and |w| stay finite
    host = dense.view(n, 4, Bs, Bs, Bs)
    host[n // 2, 1, 3, 4, 5] = float("inf")
    host[n - 1, 3, 6, 2, 1] = float("nan")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    assert A.max_norms_noalloc(dense, n, Bs, precision, out, stream) == 0
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isfinite(got[0]) and np.isfinite(got[2]), got
    assert got[1] == np.inf and got[4] == np.inf and np.isnan(got[3]), got

    # sizes beyond the scratch capacity are refused before anything is launched
    big = A.NOALLOC_MAX_BLOCKS + 1
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    assert A.max_norms_noalloc(dense, big, Bs, precision, out, stream) == 3   # ACM_ECAPACITY
    assert A.max_norms_noalloc(dense, n, 12, precision, out, stream) == 1     # ACM_EINVAL
    f.close()
