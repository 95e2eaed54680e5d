"""Pins of the oracle's multiresolution operators (Sec. 3.1-3.4)."""
import numpy as np

from oracle import mra
from tests.golden_util import load_golden

G = load_golden("paper_constants.txt")


def test_dd4_weights_are_the_papers():
    assert np.array_equal(mra.DD4, np.array(G["dd4_weights"]))


def test_prediction_reproduces_cubics_and_R_P_is_identity():
    rng = np.random.default_rng(0)
    a = rng.uniform(-1, 1, 4)
    x = np.linspace(-1.0, 1.0, 21)          # fine grid, coarse = even points
    f = a[0] + a[1] * x + a[2] * x ** 2 + a[3] * x ** 3
    c = mra.restrict_1d(f)
    p = mra.predict_1d(c)
    ok = ~np.isnan(p)
    assert ok[3:-3].all()
    assert np.max(np.abs(p[ok] - f[ok])) < 1e-14
    assert np.array_equal(mra.restrict_1d(mra.predict_1d(c)), c)   # R o P = Id, bitwise
    cp = rng.normal(size=16)
    assert np.array_equal(mra.restrict_1d(mra.predict_1d_periodic(cp)), cp)


def test_quartic_detail_is_the_interpolation_error():
    # u = x^4, fine spacing h: cubic interpolation at a midpoint of nodes -3h, -h, h, 3h
    # misses f''''/4! * (3h)(h)(h)(3h) = 9 h^4
    h = 0.01
    x = np.arange(-20, 21) * h
    f = x ** 4
    d = f - mra.predict_1d(mra.restrict_1d(f))
    odd = d[5:-5:2] if (5 % 2 == 1) else d[6:-5:2]
    assert np.allclose(odd, 9 * h ** 4, rtol=1e-9, atol=0)
    assert np.all(d[4:-4:2] == 0.0)


def test_block_details_3d():
    M, g = 8, 2
    h = 0.05
    i = np.arange(-g, M + g + 1) * h + 0.3
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    rng = np.random.default_rng(1)
    C = rng.uniform(-1, 1, (4, 4, 4))
    cub = sum(C[a, b, c] * X ** a * Y ** b * Z ** c for a in range(4) for b in range(4) for c in range(4))
    d = mra.block_details(cub[None], g, M)[0]
    assert np.abs(d).max() < 1e-13 * np.abs(cub).max()
    q = X ** 4
    d = mra.block_details(q[None], g, M)[0]
    idx = np.arange(M + 1)
    oddx = (idx % 2 == 1)[None, None, :]
    assert np.allclose(d[np.broadcast_to(oddx, d.shape)], 9 * h ** 4, rtol=1e-8)
    assert np.abs(d[np.broadcast_to(~oddx, d.shape)]).max() < 1e-14


def test_filter_relations_and_wavelet_transform_equal_details():
    h, ht, g, gt = mra.linear_filters()
    assert [h[n] for n in (-1, 0, 1)] == G["linear_h"]
    assert [gt[n] for n in (0, 1, 2)] == G["linear_gt"]
    assert g == {1: 1.0}
    # cubic case: analysing with g~ at odd points gives u - P R u
    h4, ht4, g4, gt4 = mra.dd4_filters()
    rng = np.random.default_rng(2)
    u = rng.normal(size=32)
    d_ref = mra.details_1d_periodic(u)
    n = u.size
    d_fwt = np.array([sum(v * u[(2 * i + k) % n] for k, v in gt4.items()) for i in range(n // 2)])
    assert np.allclose(d_fwt, d_ref[1::2], atol=1e-14)
    # g~ has 4 vanishing moments (it annihilates cubics) -- about its centre n = 1
    mom = [sum(((k - 1) ** p) * v for k, v in gt4.items()) for p in range(5)]
    assert np.allclose(mom[:4], 0.0, atol=1e-14) and abs(mom[4]) > 1


def test_lifting_cdf22():
    h, ht, g, gt = mra.linear_filters()
    s = mra.lifting_coefficients(h, g, 2, [0, 1])
    assert np.allclose([abs(s[0]), abs(s[1])], G["cdf22_s_abs"], atol=1e-15)
    gn, htn = mra.lift_primal(h, ht, g, gt, s)
    # lifted wavelet filter as printed (paper index n = -3..1 is ours shifted by +2)
    assert np.allclose([gn[n] for n in range(-1, 4)], G["cdf22_g"], atol=1e-15)
    assert np.allclose(mra.moments(gn, 2), 0.0, atol=1e-15)
    assert np.allclose([abs(htn[n]) for n in range(-2, 3)], G["cdf22_ht_abs"], atol=1e-15)
    assert abs(sum(htn.values()) - 1.0) < 1e-15
    # biorthogonality survives lifting: sum_n h_n h~_{n+2k} = delta_k
    for k in range(-3, 4):
        v = sum(hv * htn.get(n + 2 * k, 0.0) for n, hv in h.items())
        assert abs(v - (1.0 if k == 0 else 0.0)) < 1e-15


def test_lifting_cdf44_update_weights():
    h, ht, g, gt = mra.dd4_filters()
    s = mra.lifting_coefficients(h, g, 4, [-1, 0, 1, 2])
    assert np.allclose([s[k] for k in (-1, 0, 1, 2)], np.array([-1, 9, 9, -1]) / 32, atol=1e-14)
    gn, htn = mra.lift_primal(h, ht, g, gt, s)
    assert np.allclose(mra.moments(gn, 4), 0.0, atol=1e-13)
    for k in range(-5, 6):
        v = sum(hv * htn.get(n + 2 * k, 0.0) for n, hv in h.items())
        assert abs(v - (1.0 if k == 0 else 0.0)) < 1e-14


def test_thresholding_error_one_level():
    # Sec. 3.3: dropping details below C_eps ||u|| changes u by less than C_eps ||u||
    rng = np.random.default_rng(3)
    x = np.linspace(0, 1, 128, endpoint=False)
    u = np.sin(2 * np.pi * x) + 0.01 * np.sin(2 * np.pi * 23 * x) + 1e-4 * rng.normal(size=128)
    d = mra.details_1d_periodic(u)
    eps = 5e-3
    norm = np.abs(u).max()
    keep = np.abs(d) / norm >= eps
    u_thr = mra.predict_1d_periodic(mra.restrict_1d(u)) + np.where(keep, d, 0.0)
    assert np.abs(u_thr - u).max() < eps * norm
