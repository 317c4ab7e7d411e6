"""Pins for the oracle's gridding arithmetic (paper Eq. 1-3, Sect. 2.1-2.2,
Sect. 3.5 Eq. 6, App. A flux conservation).

The paper prints no gridded value, so every pin is a closed form, an invariant
or an independent computation of the same quantity:

* distances: textbook values and an independent formula (Vincenty / atan2);
* a single sample reproduces the sampled kernel (closed form);
* constant data gives a constant map where W > 0, NaN elsewhere (Eq. 3);
* integer sample weights equal repeated samples (weights in Eq. 1-2);
* brute force == HEALPix lookup (Sect. 2.2), for several nside, with the
  per-sample disc and the ring-shifted disc of Eq. 4-5;
* sum_p W_p Omega_p == N x (spherical integral of the kernel) (Eq. 2);
* a densely sampled Gaussian source keeps its flux and its width grows as
  sqrt(sigma_k^2 + sigma_s^2) (Eq. 6, flux conservation);
* linearity, the adjoint identity <G x, y> = <x, G^T y>, and d/dsigma against
  central finite differences;
* sort / CSR / ring offsets against numpy's stable argsort and unique.

``check_*`` functions hold the pins so that the mutation tests at the end can
re-run them against copies of the oracle with a planted mistake.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
from scipy import integrate

import oracle
import workloads

DEG = math.pi / 180.0
ARCMIN = 1.0 / 60.0


def vincenty(l1, b1, l2, b2):
    """Great-circle distance (rad) by the atan2 (Vincenty) form, numpy."""
    p1, p2 = np.radians(b1), np.radians(b2)
    dl = np.radians(np.asarray(l2) - np.asarray(l1))
    y = np.hypot(np.cos(p2) * np.sin(dl),
                 np.cos(p1) * np.sin(p2) - np.sin(p1) * np.cos(p2) * np.cos(dl))
    x = np.sin(p1) * np.sin(p2) + np.cos(p1) * np.cos(p2) * np.cos(dl)
    return np.arctan2(y, x)


# ----------------------------------------------------------------------------
# pins
# ----------------------------------------------------------------------------

def check_distances():
    h = oracle.haversine
    assert abs(h(0, 0, 90, 0) - math.pi / 2) < 1e-15
    assert abs(h(0, 0, 0, 90) - math.pi / 2) < 1e-15
    assert abs(h(0, 89, 180, 89) - 2 * DEG) < 1e-14
    assert abs(h(10, -30, 190, 30) - math.pi) < 1e-12
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(300):
        l1, l2 = rng.uniform(0, 360, 2)
        b1, b2 = np.degrees(np.arcsin(rng.uniform(-1, 1, 2)))
        if rng.random() < 0.5:          # small separations, the gridding regime
            l2, b2 = l1 + rng.normal(0, 0.2), np.clip(b1 + rng.normal(0, 0.2), -90, 90)
        assert abs(h(l1, b1, l2, b2) - vincenty(l1, b1, l2, b2)) < 2e-13
    # bearings from the equator: north 0, east +90 deg, west -90 deg
    assert abs(oracle.bearing(0, 0, 0, 1)) < 1e-15
    assert abs(oracle.bearing(0, 0, 1, 0) - math.pi / 2) < 1e-15
    assert abs(oracle.bearing(0, 0, -1, 0) + math.pi / 2) < 1e-15


def check_single_sample():
    sig, r = 0.05, 0.15
    k = oracle.gauss1d(sig, r)
    lon_t, lat_t = workloads.car_grid(40.0, 60.0, 15, 15, 0.02)
    ls, bs = np.array([40.013]), np.array([60.007])
    res = oracle.grid_bruteforce(lon_t, lat_t, ls, bs, np.array([[2.5, -1.0]]), k)
    d = vincenty(lon_t, lat_t, ls[0], bs[0])
    w = np.where(d <= r * DEG, np.exp(-(d / (sig * DEG)) ** 2 / 2), 0.0)
    assert np.all(np.abs(res.wsum - w) <= 1e-12 * w)
    on = w > 0
    assert np.all(np.abs(res.out[on] - np.array([2.5, -1.0])) < 1e-14)
    assert np.all(np.isnan(res.out[~on]))
    assert res.npairs == int(on.sum())


def check_constant_data():
    wl = workloads.random_field(41, 400, 12, 3, 10.0, 45.0, 1.0, 2.0 * ARCMIN, weights=True)
    k = oracle.gauss1d(2.0 * ARCMIN, 6.0 * ARCMIN)
    data = np.tile(np.array([1.25, -7.0, 0.0]), (wl.n_samples, 1))
    res = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, data, k, wl.omega)
    on = res.wsum > 0
    assert on.sum() > 10 and (~on).sum() >= 0
    assert np.all(np.abs(res.out[on] - np.array([1.25, -7.0, 0.0])) <= 1e-14 * 7)
    assert np.all(np.isnan(res.out[~on]))


def check_weights_equal_repeats():
    wl = workloads.random_field(42, 150, 8, 2, 300.0, -20.0, 0.6, 2.0 * ARCMIN)
    k = oracle.gauss1d(2.0 * ARCMIN, 6.0 * ARCMIN)
    rng = np.random.Generator(np.random.PCG64(5))
    rep = rng.integers(1, 4, wl.n_samples)
    a = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, k,
                               rep.astype(np.float64))
    b = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, np.repeat(wl.lon_s, rep),
                               np.repeat(wl.lat_s, rep), np.repeat(wl.data, rep, axis=0), k)
    assert np.allclose(a.wsum, b.wsum, rtol=1e-13, atol=0)
    on = a.wsum > 0
    assert np.allclose(a.out[on], b.out[on], rtol=1e-12, atol=1e-13)


def _cases_for_lookup():
    yield workloads.random_field(51, 300, 10, 2, 0.2, 1.0, 1.2, 3.0 * ARCMIN, weights=True)
    yield workloads.random_field(52, 300, 10, 1, 200.0, 88.9, 2.2, 4.0 * ARCMIN)
    yield workloads.random_field(53, 300, 10, 3, 359.8, -41.8, 1.0, 3.0 * ARCMIN)
    # all-sky plate-carree with the elliptical kernel
    rng = np.random.Generator(np.random.PCG64(54))
    n = 3000
    z = rng.uniform(-1, 1, n)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    lon_t, lat_t = workloads.allsky_car(36, 18)
    wl = workloads.Workload("allsky-tiny", lon, lat, rng.normal(0, 1, (n, 2)), None, lon_t,
                            lat_t, {"type": "gauss2d", "smaj": 6.0, "smin": 3.0, "pa": 30.0},
                            18.0, 1.5)
    yield wl


def _kernel_of(wl):
    kk = wl.kernel
    if kk["type"] == "gauss1d":
        return oracle.gauss1d(kk["sigma"], wl.support)
    return oracle.gauss2d(kk["smaj"], kk["smin"], kk["pa"], wl.support)


def check_lookup_equals_bruteforce():
    for wl in _cases_for_lookup():
        k = _kernel_of(wl)
        a = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, k, wl.omega)
        base = oracle.nside_for_resolution(wl.hpx_maxres)
        for ns, shifted in ((base, False), (base, True), (max(1, base // 8), False),
                            (base * 2, False)):
            b = oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, k,
                                   wl.omega, shifted=shifted)
            assert a.npairs == b.npairs, (wl.name, ns, shifted, a.npairs, b.npairs)
            assert a.npairs > 0
            assert np.allclose(a.wsum, b.wsum, rtol=1e-12, atol=1e-300)
            on = a.wsum > 0
            assert np.array_equal(on, b.wsum > 0)
            assert np.allclose(a.out[on], b.out[on], rtol=1e-12, atol=1e-12)


def check_weight_sum_normalisation():
    """sum_p W_p Omega_p = N * 2 pi int_0^r exp(-t^2/2s^2) sin t dt for samples
    whose support lies inside a finely pixelised target field."""
    sig = 0.1
    r = 5 * sig
    h = sig / 4
    lon_t, lat_t = workloads.car_grid(80.0, 20.0, 81, 81, h)
    rng = np.random.Generator(np.random.PCG64(61))
    n = 40
    ls = 80.0 + rng.uniform(-1.0, 1.0, n) * (40 * h - r - 2 * h) / math.cos(math.radians(23))
    bs = 20.0 + rng.uniform(-1.0, 1.0, n) * (40 * h - r - 2 * h)
    res = oracle.grid_bruteforce(lon_t, lat_t, ls, bs, np.ones((n, 1)), oracle.gauss1d(sig, r))
    omega = (h * DEG) * (np.sin(np.radians(lat_t + h / 2)) - np.sin(np.radians(lat_t - h / 2)))
    total = float((res.wsum * omega).sum())
    s, R = sig * DEG, r * DEG
    one = 2 * math.pi * integrate.quad(lambda t: math.exp(-t * t / (2 * s * s)) * math.sin(t),
                                       0.0, R, epsabs=0, epsrel=1e-13)[0]
    assert abs(total / (n * one) - 1.0) < 2e-4, total / (n * one)


def check_eq6_flux_and_width():
    """Densely sampled Gaussian source (sigma_s) gridded with sigma_k: the map
    keeps the source flux and has sigma_out^2 = sigma_s^2 + sigma_k^2 (Eq. 6)."""
    sig_s, sig_k = 0.05, 0.025
    step = sig_k / 5
    half = 0.45
    g = np.arange(-half, half + 1e-9, step)
    lat_s, lon_s = np.meshgrid(g, g, indexing="ij")
    lon_s, lat_s = lon_s.ravel(), lat_s.ravel()
    val = np.exp(-(lon_s ** 2 + lat_s ** 2) / (2 * sig_s ** 2))
    h = sig_k / 2
    lon_t, lat_t = workloads.car_grid(0.0, 0.0, 61, 61, h)
    res = oracle.grid_bruteforce(lon_t, lat_t, lon_s, lat_s, val, oracle.gauss1d(sig_k, 5 * sig_k))
    R = res.out[:, 0]
    on = np.isfinite(R)
    flux = float((R[on]).sum() * h * h)
    assert abs(flux / (2 * math.pi * sig_s ** 2) - 1) < 2e-3, flux
    m2 = float((R[on] * lon_t[on] ** 2).sum() / R[on].sum())
    want = sig_s ** 2 + sig_k ** 2
    assert abs(m2 / want - 1) < 1e-2, (m2, want)


def check_elliptical_closed_forms():
    smaj, smin, r = 0.2, 0.1, 1.0
    for pa in (0.0, 30.0, 90.0, 135.0):
        k = oracle.gauss2d(smaj, smin, pa, r)
        for d, beta in ((0.15, 0.0), (0.12, 90.0), (0.2, 45.0), (0.3, -60.0)):
            # target on the equator; the sample at distance d along bearing beta
            b = math.radians(beta)
            dr = math.radians(d)
            lat = math.degrees(math.asin(math.sin(dr) * math.cos(b)))
            lon = math.degrees(math.atan2(math.sin(b) * math.sin(dr), math.cos(dr)))
            a_ = d * math.cos(b - math.radians(pa))
            b_ = d * math.sin(b - math.radians(pa))
            want = math.exp(-a_ ** 2 / (2 * smaj ** 2) - b_ ** 2 / (2 * smin ** 2))
            got = oracle.kernel_value(k, 0.0, 0.0, lon, lat)
            assert abs(got - want) < 1e-12 * max(1.0, want) + 1e-300, (pa, d, beta, got, want)
        # PA and PA+180 describe the same ellipse
        k2 = oracle.gauss2d(smaj, smin, pa + 180.0, r)
        assert abs(oracle.kernel_value(k, 5, 40, 5.1, 40.05)
                   - oracle.kernel_value(k2, 5, 40, 5.1, 40.05)) < 1e-14
    # circular limit
    kc = oracle.gauss2d(0.1, 0.1, 77.0, 0.5)
    k1 = oracle.gauss1d(0.1, 0.5)
    for (lt, bt, ls, bs) in ((10, 10, 10.2, 10.1), (0, 89.9, 180, 89.95)):
        assert abs(oracle.kernel_value(kc, lt, bt, ls, bs)
                   - oracle.kernel_value(k1, lt, bt, ls, bs)) < 1e-14


def _tiny_linear_case():
    wl = workloads.random_field(71, 120, 9, 3, 150.0, 35.0, 0.5, 1.5 * ARCMIN, weights=True)
    return wl, oracle.gauss1d(1.5 * ARCMIN, 4.5 * ARCMIN)


def check_linearity_and_adjoint():
    wl, k = _tiny_linear_case()
    rng = np.random.Generator(np.random.PCG64(72))
    x = rng.normal(0, 1, (wl.n_samples, 3))
    y = rng.normal(0, 1, (wl.n_samples, 3))
    gx = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, x, k, wl.omega).out
    gy = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, y, k, wl.omega).out
    gz = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, 2.0 * x - 3.0 * y, k,
                                wl.omega).out
    on = np.isfinite(gx[:, 0])
    assert np.allclose(gz[on], 2.0 * gx[on] - 3.0 * gy[on], rtol=1e-12, atol=1e-12)
    ymap = rng.normal(0, 1, (wl.n_targets, 3))
    xhat = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, ymap, k, wl.omega)
    lhs = float(np.sum(np.where(on[:, None], gx, 0.0) * ymap))
    rhs = float(np.sum(x * xhat))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)), (lhs, rhs)


def check_dsigma_fd():
    wl, k = _tiny_linear_case()
    sig = k.sigma_deg
    an = oracle.dsigma_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, k, wl.omega)
    h = 1e-5 * sig
    kp = oracle.gauss1d(sig + h, k.support_deg)
    km = oracle.gauss1d(sig - h, k.support_deg)
    rp = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, kp, wl.omega).out
    rm = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, km, wl.omega).out
    fd = (rp - rm) / (2 * h)
    on = np.isfinite(an[:, 0])
    scale = np.abs(an[on]).max()
    assert scale > 0
    assert np.max(np.abs(fd[on] - an[on])) < 1e-6 * scale


def check_sort_csr():
    rng = np.random.Generator(np.random.PCG64(81))
    keys = rng.integers(0, 50, 2000)
    perm = oracle.sort_stable(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    sk = keys[perm]
    uniq, off = oracle.csr(sk)
    u2, first = np.unique(sk, return_index=True)
    assert np.array_equal(uniq, u2)
    assert np.array_equal(off[:-1], first) and off[-1] == sk.size
    ns = 4
    pix = rng.integers(0, 12 * ns * ns, 500)
    spix = np.sort(pix)
    ro = oracle.ring_offsets(ns, spix)
    rings = np.array([oracle.pix2ring(ns, int(p)) for p in spix])
    assert np.array_equal(ro, np.searchsorted(rings, np.arange(4 * ns + 1), side="left"))


# ----------------------------------------------------------------------------
# tests
# ----------------------------------------------------------------------------

def test_distances():
    check_distances()


def test_single_sample_closed_form():
    check_single_sample()


def test_constant_data():
    check_constant_data()


def test_weights_equal_repeats():
    check_weights_equal_repeats()


def test_lookup_equals_bruteforce():
    check_lookup_equals_bruteforce()


def test_weight_sum_normalisation():
    check_weight_sum_normalisation()


def test_eq6_flux_and_width():
    check_eq6_flux_and_width()


def test_elliptical_closed_forms():
    check_elliptical_closed_forms()


def test_linearity_and_adjoint():
    check_linearity_and_adjoint()


def test_dsigma_fd():
    check_dsigma_fd()


def test_sort_csr():
    check_sort_csr()


def check_nonfinite_ieee():
    """Eq. 1 with a non-finite channel value, summed as IEEE arithmetic
    defines it: a target reached by a +Inf sample gets +Inf, one reached by
    +Inf and -Inf samples NaN, one reached by a NaN sample NaN; every other
    target equals the sum over the finite samples alone (the same map with
    those samples removed, where they do not reach)."""
    rng = np.random.Generator(np.random.PCG64(4242))
    n = 300
    lon = 10.0 + rng.uniform(-0.5, 0.5, n)
    lat = 5.0 + rng.uniform(-0.5, 0.5, n)
    lon[:3] = [9.8, 10.2, 10.21]
    lat[:3] = [5.0, 5.0, 5.0]
    data = rng.normal(0, 1, (n, 2)) + 2.0
    data[0, 0] = np.nan
    data[1, 1] = np.inf
    data[2, 1] = -np.inf
    lon_t, lat_t = workloads.car_grid(10.0, 5.0, 24, 24, 1.0 / 24.0)
    k = oracle.gauss1d(2.0 * ARCMIN, 6.0 * ARCMIN)
    ref = oracle.grid_bruteforce(lon_t, lat_t, lon, lat, data, k)
    d = np.array([[oracle.haversine(a, b, c, e) for c, e in zip(lon[:3], lat[:3])]
                  for a, b in zip(lon_t, lat_t)])
    reach = d <= math.radians(6.0 * ARCMIN)
    on = ref.wsum > 0
    r0, r1, r2 = reach[:, 0] & on, reach[:, 1] & on, reach[:, 2] & on
    assert r0.any() and (r1 & ~r2).any() and (r1 & r2).any()
    assert np.all(np.isnan(ref.out[r0, 0]))
    assert np.all(ref.out[r1 & ~r2, 1] == np.inf)
    assert np.all(ref.out[r2 & ~r1, 1] == -np.inf)
    assert np.all(np.isnan(ref.out[r1 & r2, 1]))
    clean = oracle.grid_bruteforce(lon_t, lat_t, lon[3:], lat[3:], data[3:], k)
    # (the clean map lacks all three samples, so compare where none reaches)
    keep0 = keep1 = on & ~(r0 | r1 | r2) & (clean.wsum > 0)
    # away from the bad samples' supports both maps sum the same terms
    assert np.all(np.isfinite(ref.num[keep0, 0])) and np.all(np.isfinite(ref.num[keep1, 1]))
    assert np.allclose(ref.num[keep0, 0], clean.num[keep0, 0], rtol=1e-13, atol=1e-13)
    assert np.allclose(ref.num[keep1, 1], clean.num[keep1, 1], rtol=1e-13, atol=1e-13)


def test_nonfinite_ieee():
    check_nonfinite_ieee()


# ----------------------------------------------------------------------------
# planted mistakes: each copy of the oracle with one plausible error must fail
# at least one pin
# ----------------------------------------------------------------------------

MUTATIONS = {
    "haversine_wrong_cos": ("cos(p1) * cos(p2) * sdl * sdl", "cos(p1) * cos(p1) * sdl * sdl",
                            [check_distances, check_single_sample]),
    "kernel_sigma_not_squared": ("exp(-(d * d) / (2.0 * s * s))", "exp(-(d * d) / (2.0 * s))",
                                 [check_single_sample, check_weight_sum_normalisation]),
    "weight_dropped_from_numerator": ("acc_add(&anum[p * C + c], ww * data[n * C + c]);",
                                      "acc_add(&anum[p * C + c], w * data[n * C + c]);",
                                      [check_weights_equal_repeats]),
    "bearing_sign": ("const double y = sin(dl) * cos(p2);",
                     "const double y = -sin(dl) * cos(p2);",
                     [check_distances, check_elliptical_closed_forms]),
    "ellipse_axes_swapped": ("(a * a) / (2.0 * s1 * s1) - (b * b) / (2.0 * s2 * s2)",
                             "(a * a) / (2.0 * s2 * s2) - (b * b) / (2.0 * s1 * s1)",
                             [check_elliptical_closed_forms]),
    "ring_phase_flipped": ("*phase = ((i - ns) % 2 == 0) ? 0.5 : 0.0;",
                           "*phase = ((i - ns) % 2 == 0) ? 0.0 : 0.5;",
                           [check_lookup_equals_bruteforce]),
    "disc_without_pixel_margin": ("const double W = hw + 0.5 * dphi + 1e-12;",
                                  "const double W = hw + 1e-12;",
                                  [check_lookup_equals_bruteforce]),
    "dsigma_missing_R_term": ("(acc_get(&anp[p * C + c]) - R * Wp) / W",
                              "(acc_get(&anp[p * C + c])) / W", [check_dsigma_fd]),
    "degrid_not_normalised": ("const double g = w * (omega ? omega[n] : 1.0) / W;",
                              "const double g = w * (omega ? omega[n] : 1.0);",
                              [check_linearity_and_adjoint]),
    "compensation_on_nonfinite": ("  if (isfinite(t)) {\n", "  if (1) {\n", [check_nonfinite_ieee]),
    "cut_not_applied": ("if (!(d <= r)) { *inside = 0; return 0.0; }",
                        "if (0) { *inside = 0; return 0.0; }", [check_single_sample]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    old, new, checks = MUTATIONS[name]
    src = open(oracle._build.SRC).read()
    assert src.count(old) >= 1, name
    tmp = tempfile.mkdtemp(prefix="cgmut_")
    try:
        cpath = os.path.join(tmp, "m.c")
        with open(cpath, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "libm.so")
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", so, cpath, "-lm"])
        good = oracle.lib()
        monkeypatch.setattr(oracle, "_lib", None)
        monkeypatch.setattr(oracle._build, "build", lambda force=False: so)
        caught = False
        for chk in checks:
            try:
                chk()
            except AssertionError:
                caught = True
                break
        monkeypatch.setattr(oracle, "_lib", good)
        assert caught, f"planted mistake {name} was not caught"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
