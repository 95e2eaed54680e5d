"""Point-value multiresolution of the oracle (Harten / Deslauriers-Dubuc), FP64.

Test infrastructure only (see ``oracle/__init__``).

Paper, Sec. 3.1: prediction P_{J->J+1} keeps the even points and fills the odd ones with the
4th-order interpolating subdivision weights (-1, 9, 9, -1)/16; restriction R_{J+1->J} is
decimation u_i^J = u_{2i}^{J+1}; R o P = Id; the details are u - P R u, zero at even points
(eq. "details").  Sec. 3.2: the same operators written as filters, with
g~_n = (-1)^{1-n} h_{1-n} and g_n = (-1)^{1-n} h~_{1-n}.  Sec. 3.2.1: primal lifting of the
linear case with s_0 = s_1 = -1/4 (CDF 2/0 -> CDF 2/2), and of the cubic case
(CDF 4/0 -> CDF 4/4), whose analysis low-pass h~ the CDF 4/4 coarsening applies before
decimation.  Sec. 3.4: tensor products in 3D, each component of a vector field separately,
normalised by its global L-infinity norm.
"""
from __future__ import annotations

import numpy as np

DD4 = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0


def predict_1d(c):
    """P: coarse samples c_0..c_{n-1} -> fine samples f_0..f_{2n-2} (odd points interior only
    where the 4-point stencil fits; the two odd points next to the ends are left NaN)."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    f = np.full(2 * n - 1, np.nan)
    f[0::2] = c
    for i in range(1, n - 2):
        f[2 * i + 1] = DD4[0] * c[i - 1] + DD4[1] * c[i] + DD4[2] * c[i + 1] + DD4[3] * c[i + 2]
    return f


def predict_1d_periodic(c):
    """P on a periodic sequence of n coarse samples -> 2n fine samples."""
    c = np.asarray(c, dtype=np.float64)
    n = c.shape[0]
    f = np.empty(2 * n)
    f[0::2] = c
    for i in range(n):
        f[2 * i + 1] = (DD4[0] * c[(i - 1) % n] + DD4[1] * c[i] + DD4[2] * c[(i + 1) % n]
                        + DD4[3] * c[(i + 2) % n])
    return f


def restrict_1d(f):
    """R: decimation by two."""
    return np.asarray(f)[0::2].copy()


def details_1d_periodic(f):
    """u - P R u on a periodic fine sequence (zero at even points)."""
    return np.asarray(f, dtype=np.float64) - predict_1d_periodic(restrict_1d(f))


def predict_axis(a, axis):
    """Apply P along one axis of an array whose extent along ``axis`` is m (coarse samples),
    returning extent 2m-1 (odd points without a full stencil are NaN)."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, -1)
    n = a.shape[-1]
    out = np.full(a.shape[:-1] + (2 * n - 1,), np.nan)
    out[..., 0::2] = a
    out[..., 3:2 * n - 4:2] = (DD4[0] * a[..., 0:n - 3] + DD4[1] * a[..., 1:n - 2]
                               + DD4[2] * a[..., 2:n - 1] + DD4[3] * a[..., 3:n])
    return np.moveaxis(out, -1, axis)


def predict_3d(c):
    """Tensor-product prediction of a coarse cube (..., nz, ny, nx): along x, then y, then z."""
    out = predict_axis(c, -1)
    out = predict_axis(out, -2)
    out = predict_axis(out, -3)
    return out


def block_details(ext, g, M):
    """Details of one block from its synchronised extended array.

    ``ext``: (..., M+1+2g, M+1+2g, M+1+2g) point values at local indices -g .. M+g (g even,
    g >= 2).  The coarse samples are the even local indices -g .. M+g; they are predicted back
    to the fine lattice and subtracted (Sec. 3.1, eq. "details").  Returns the details on the
    interior (..., M+1, M+1, M+1).
    """
    assert g % 2 == 0 and g >= 2
    c = ext[..., 0::2, 0::2, 0::2]
    p = predict_3d(c)                    # fine indices -g .. M+g
    sl = slice(g, g + M + 1)
    u = ext[..., sl, sl, sl]
    return u - p[..., sl, sl, sl]


# ---- biorthogonal filter view (Sec. 3.2) ---------------------------------------------------

def dd4_filters():
    """Filters of the point-value MRA with cubic interpolation (CDF 4/0), as dicts n -> value.

    h: refinement filter of phi (the prediction written as a filter), h~ = delta_0,
    g_n = (-1)^{1-n} h~_{1-n}  (so g = delta_1), g~_n = (-1)^{1-n} h_{1-n}.
    """
    h = {-3: -1 / 16, -1: 9 / 16, 0: 1.0, 1: 9 / 16, 3: -1 / 16}
    ht = {0: 1.0}
    g = {n: (-1.0) ** (1 - n) * ht[1 - n] for n in range(-10, 11) if (1 - n) in ht}
    gt = {n: (-1.0) ** (1 - n) * h[1 - n] for n in range(-10, 11) if (1 - n) in h}
    return h, ht, g, gt


def linear_filters():
    """Linear interpolation (CDF 2/0): h = {1/2, 1, 1/2}_{-1..1}, h~ = delta_0 (Sec. 3.2)."""
    h = {-1: 0.5, 0: 1.0, 1: 0.5}
    ht = {0: 1.0}
    gt = {n: (-1.0) ** (1 - n) * h[1 - n] for n in range(-10, 11) if (1 - n) in h}
    g = {n: (-1.0) ** (1 - n) * ht[1 - n] for n in range(-10, 11) if (1 - n) in ht}
    return h, ht, g, gt


def lift_primal(h, ht, g, gt, s):
    """Primal lifting (Sec. 3.2.1) on the filters.

    The wavelet is updated with coarse scaling functions, psi = psi_old - sum_k s_k phi(x-k),
    i.e. g_new[m] = g[m] - sum_k s_k h[m-2k].  Biorthogonality then fixes the dual update
    phi~ = phi~_old + sum_k s_k psi~_old(x+k), i.e. h~_new[m] = h~[m] + sum_k s_k g~[m+2k];
    phi and psi~ are unchanged.  ``s``: dict k -> s_k.  Returns (g_new, ht_new)."""
    g_new = dict(g)
    for k, sk in s.items():
        for m, hm in h.items():
            g_new[m + 2 * k] = g_new.get(m + 2 * k, 0.0) - sk * hm
    ht_new = dict(ht)
    for k, sk in s.items():
        for m, gm in gt.items():
            ht_new[m - 2 * k] = ht_new.get(m - 2 * k, 0.0) + sk * gm
    g_new = {m: v for m, v in g_new.items() if v != 0.0}
    ht_new = {m: v for m, v in ht_new.items() if v != 0.0}
    return g_new, ht_new


def lifting_coefficients(h, g, nvanish, ks):
    """Solve for s_k (k in ``ks``) so that g_new = g - sum_k s_k h(.-2k) has ``nvanish``
    vanishing moments (Sec. 3.2.1: 'requiring that the new psi has M vanishing moments')."""
    A = np.zeros((nvanish, len(ks)))
    b = np.zeros(nvanish)
    for p in range(nvanish):
        b[p] = sum((float(m) ** p) * v for m, v in g.items())
        for j, k in enumerate(ks):
            A[p, j] = sum((float(m + 2 * k) ** p) * v for m, v in h.items())
    sol = np.linalg.lstsq(A, b, rcond=None)[0]
    return {k: float(sol[j]) for j, k in enumerate(ks)}


def moments(filt, pmax):
    """sum_n n^p f_n for p = 0..pmax-1."""
    return [sum((float(n) ** p) * v for n, v in filt.items()) for p in range(pmax)]


# ---- CDF 4/4: the lifted analysis low-pass (Sec. 3.2.1) ------------------------------------------

def cdf44_lowpass():
    """Analysis low-pass h~ of CDF 4/4 as a dict n -> h~_n (n = -6..6).

    Sec. 3.2.1: the cubic interpolating MRA (CDF 4/0: h~ = delta_0) is lifted with update
    weights s_k chosen so that the new primal wavelet has 4 vanishing moments; the dual scaling
    filter then changes to h~_new[m] = h~[m] + sum_k s_k g~[m + 2k] (``lift_primal``).  The
    weights are solved for, not typed in: four unknowns s_{-1..2} (the four details around an
    even point), four moment equations."""
    h, ht, g, gt = dd4_filters()
    s = lifting_coefficients(h, g, 4, [-1, 0, 1, 2])
    _, ht_new = lift_primal(h, ht, g, gt, s)
    return ht_new


def lowpass_decimate_axis(a, axis, ht, g, M):
    """Coarse values at coarse indices 1..M-1 along ``axis``: c_i = sum_n h~_n f_{2i+n}.

    ``a`` holds fine samples at local fine indices -g..2M+g along ``axis`` (array index
    fine index + g); the filter's reach max|n| must be <= g + 2, so that c_1 and c_{M-1} find
    all their samples."""
    reach = max(abs(n) for n in ht)
    assert reach <= g + 2
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis, -1)
    assert a.shape[-1] == 2 * M + 1 + 2 * g
    out = np.zeros(a.shape[:-1] + (M - 1,))
    for i in range(1, M):
        acc = np.zeros(a.shape[:-1])
        for n in sorted(ht):
            acc = acc + ht[n] * a[..., g + 2 * i + n]
        out[..., i - 1] = acc
    return np.moveaxis(out, -1, axis)
