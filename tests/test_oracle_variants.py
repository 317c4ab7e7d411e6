"""Pins for the oracle's variants of the method (beyond Eq. 1-3 as printed):

* normalised interpolation xhat_n = sum_p w_pn y_p / sum_p w_pn (map ->
  samples): with the circular kernel it equals Eq. 1-3 with the roles of
  targets and samples exchanged (computed by the brute-force gridder, a
  different routine); a constant map interpolates to the constant; a single
  target's value reaches exactly the samples within r, NaN elsewhere;
* one weight per sample and channel: a 0 / 1 weight equals gridding the
  subset of samples with weight 1 (removed from the input arrays instead);
  scaling one channel's weights leaves its map unchanged and scales its
  weight map; the weights of one channel do not affect another.
"""
import math

import numpy as np
import pytest

import oracle


def _field(seed, n, P, side=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    lon_s = 50.0 + rng.uniform(-side, side, n)
    lat_s = 10.0 + rng.uniform(-side, side, n)
    g = np.linspace(-0.8 * side, 0.8 * side, P)
    lat_t, lon_t = np.meshgrid(10.0 + g, 50.0 + g, indexing="ij")
    return rng, lon_s, lat_s, lon_t.ravel(), lat_t.ravel()


def test_interp_equals_swapped_gridding():
    rng, lon_s, lat_s, lon_t, lat_t = _field(41, 400, 12)
    k = oracle.gauss1d(0.1, 0.3)
    y = rng.normal(size=(lon_t.size, 3))
    xh, v = oracle.interp_bruteforce(lon_t, lat_t, lon_s, lat_s, y, k)
    sw = oracle.grid_bruteforce(lon_s, lat_s, lon_t, lat_t, y, k)
    on = sw.wsum > 0
    assert np.array_equal(on, v > 0)
    assert np.allclose(v[on], sw.wsum[on], rtol=1e-13, atol=0)
    assert np.allclose(xh[on], sw.out[on], rtol=1e-12, atol=1e-13)
    assert np.all(np.isnan(xh[~on]))


def test_interp_constant_and_single_target():
    rng, lon_s, lat_s, lon_t, lat_t = _field(43, 300, 8)
    k = oracle.gauss2d(0.12, 0.07, 35.0, 0.3)
    xh, v = oracle.interp_bruteforce(lon_t, lat_t, lon_s, lat_s, np.full((lon_t.size, 2), 3.25), k)
    on = v > 0
    assert on.any() and np.allclose(xh[on], 3.25, rtol=1e-14)
    # one target: the samples within r see its value, the others NaN
    x1, v1 = oracle.interp_bruteforce(lon_t[:1], lat_t[:1], lon_s, lat_s, [[7.5]], k)
    d = np.array([oracle.haversine(lon_t[0], lat_t[0], a, b) for a, b in zip(lon_s, lat_s)])
    inside = d <= math.radians(0.3)
    assert np.array_equal(v1 > 0, inside)
    assert np.allclose(x1[inside, 0], 7.5, rtol=1e-14)
    assert np.all(np.isnan(x1[~inside, 0]))


def test_pcw_mask_equals_subset():
    rng, lon_s, lat_s, lon_t, lat_t = _field(47, 500, 10)
    k = oracle.gauss1d(0.1, 0.3)
    C = 3
    data = rng.normal(size=(lon_s.size, C))
    om = (rng.random((lon_s.size, C)) < 0.6).astype(float)
    R, W, _ = oracle.grid_bruteforce_pcw(lon_t, lat_t, lon_s, lat_s, data, k, om)
    for c in range(C):
        keep = om[:, c] > 0
        sub = oracle.grid_bruteforce(lon_t, lat_t, lon_s[keep], lat_s[keep], data[keep, c:c + 1], k)
        on = sub.wsum > 0
        assert np.array_equal(on, W[:, c] > 0)
        assert np.allclose(W[on, c], sub.wsum[on], rtol=1e-13, atol=0)
        assert np.allclose(R[on, c], sub.out[on, 0], rtol=1e-12, atol=1e-13)


def test_pcw_scaling_and_independence():
    rng, lon_s, lat_s, lon_t, lat_t = _field(53, 400, 9)
    k = oracle.gauss1d(0.1, 0.3)
    data = rng.normal(size=(lon_s.size, 2))
    om = rng.uniform(0.2, 3.0, (lon_s.size, 2))
    R, W, _ = oracle.grid_bruteforce_pcw(lon_t, lat_t, lon_s, lat_s, data, k, om)
    om2 = om.copy()
    om2[:, 1] *= 4.0
    R2, W2, _ = oracle.grid_bruteforce_pcw(lon_t, lat_t, lon_s, lat_s, data, k, om2)
    on = W[:, 1] > 0
    assert np.allclose(R2[on, 1], R[on, 1], rtol=1e-12, atol=1e-13)
    assert np.allclose(W2[on, 1], 4.0 * W[on, 1], rtol=1e-13, atol=0)
    assert np.array_equal(R2[:, 0], R[:, 0], equal_nan=True)


def test_tapered_sinc_closed_forms():
    """sin(x)/x at x = pi d / a, taper exp(-d^2 / b^2): zeros at d = a, 2a;
    1 at d = 0; 2/pi at d = a / 2 and -2/(3 pi) at d = 3a/2 (times the
    taper); evaluated for a target at (0, 0) and samples on the equator."""
    a, b = 0.2, 0.35
    k = oracle.tapered_sinc(a, b, 1.0)
    L = oracle.lib()
    val = lambda d: L.or_kernel_value(k, 0.0, 0.0, d, 0.0)
    assert val(0.0) == 1.0
    assert abs(val(a)) < 1e-15 and abs(val(2 * a)) < 1e-15
    assert math.isclose(val(a / 2), (2 / math.pi) * math.exp(-(a / 2 / b) ** 2), rel_tol=1e-12)
    assert math.isclose(val(1.5 * a), (-2 / (3 * math.pi)) * math.exp(-(1.5 * a / b) ** 2),
                        rel_tol=1e-12)
    assert val(1.01) == 0.0                      # beyond the support


def test_tapered_sinc_single_sample():
    """One sample: R = D wherever its (signed) weight is positive; where the
    weight map is negative (the sinc's negative lobe) R is NaN (W > 0 rule)."""
    a, b = 0.2, 0.5
    k = oracle.tapered_sinc(a, b, 0.6)
    lon_t = np.linspace(-0.55, 0.55, 45)
    lat_t = np.zeros_like(lon_t)
    res = oracle.grid_bruteforce(lon_t, lat_t, [0.0], [0.0], [[2.5]], k)
    d = np.abs(lon_t)
    pos = np.sin(np.pi * d / a) / np.where(d > 0, np.pi * d / a, 1.0)
    pos = np.where(d > 0, pos, 1.0) > 1e-9
    assert np.allclose(res.out[pos, 0], 2.5, rtol=1e-13)
    neg = (res.wsum < 0)
    assert neg.any() and np.all(np.isnan(res.out[neg, 0]))
