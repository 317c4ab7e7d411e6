"""Pins for the oracle's HEALPix RING geometry (paper Sect. 2.2, 3.2-3.3;
tessellation of Gorski et al. 2005).

The paper prints no HEALPix values, so the oracle is pinned by facts the
tessellation fixes independently of the index formulas: the base-pixel
layout, ring sizes and centres, the round trip pixel -> centre -> pixel, the
equal-area property, the pixel extent used by the disc query, and a brute-force
superset check of query-disc.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def _lonlat_of(z, phi):
    return np.degrees(phi), np.degrees(np.arcsin(np.clip(z, -1, 1)))


def test_base_pixels_nside1():
    g = _load("healpix_base_nside1.txt")
    for pix, z, phi_deg in g:
        zz, pp = oracle.pix2ang(1, int(pix))
        assert abs(zz[0] - z) < 1e-15
        assert abs(math.degrees(pp[0]) - phi_deg) < 1e-12
        # the centre maps back to its own base pixel
        assert oracle.ang2pix(1, [phi_deg], [math.degrees(math.asin(z))])[0] == int(pix)


def test_ring_layout_nside2():
    g = _load("healpix_rings_nside2.txt")
    for ring, z, count, first in g:
        c, f, zz, _ = oracle.ring_info(2, int(ring))
        assert (c, f) == (int(count), int(first))
        assert abs(zz - z) < 1e-15


# the RING scheme is defined for any nside >= 1, not only powers of two
@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 8, 12, 16, 64])
def test_ring_counts_sum(ns):
    total = 0
    prev_first = 0
    for i in range(1, 4 * ns):
        c, f, z, ph = oracle.ring_info(ns, i)
        assert f == prev_first
        prev_first = f + c
        total += c
        # ring centres move monotonically south
        if i > 1:
            assert z < oracle.ring_info(ns, i - 1)[2]
    assert total == 12 * ns * ns


@pytest.mark.parametrize("ns", [1, 2, 3, 4, 5, 8, 12, 64, 100])
def test_roundtrip_all_pixels(ns):
    npix = 12 * ns * ns
    pix = np.arange(npix)
    z, phi = oracle.pix2ang(ns, pix)
    lon, lat = _lonlat_of(z, phi)
    back = oracle.ang2pix(ns, lon, lat)
    assert np.array_equal(back, pix)
    # ring of every pixel matches the ring that holds its centre
    for p in pix[:: max(1, npix // 200)]:
        r = oracle.pix2ring(ns, int(p))
        c, f, zr, _ = oracle.ring_info(ns, r)
        assert f <= p < f + c
        assert abs(zr - z[p]) < 1e-15


@pytest.mark.parametrize("ns", [8, 5])
def test_equal_area_counts(ns):
    """Uniform points on the sphere fill every pixel equally (chi^2)."""
    npix = 12 * ns * ns
    rng = np.random.Generator(np.random.PCG64(7))
    n = 1_200_000
    z = rng.uniform(-1, 1, n)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    cnt = np.bincount(oracle.ang2pix(ns, lon, lat), minlength=npix)
    assert cnt.size == npix
    exp = n / npix
    chi2 = float(((cnt - exp) ** 2 / exp).sum())
    dof = npix - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof), chi2


@pytest.mark.parametrize("ns", [1, 2, 3, 4, 16, 1000, 4096, 12345])
def test_pixel_box_contains_point(ns):
    """Every point lies between the centres of the rings adjacent to its own
    ring and within half a pixel spacing of its pixel centre in phi: the box
    the disc query relies on."""
    rng = np.random.Generator(np.random.PCG64(11 + ns))
    n = 4000
    z = rng.uniform(-1, 1, n)
    # concentrate some points near the poles and the cap/belt transition
    z[:500] = 1 - rng.uniform(0, 1e-3, 500)
    z[500:1000] = -(1 - rng.uniform(0, 1e-3, 500))
    z[1000:1500] = 2 / 3 + rng.uniform(-1e-3, 1e-3, 500)
    lon = rng.uniform(0, 360, n)
    lat = np.degrees(np.arcsin(z))
    zz = np.sin(np.radians(lat))
    pix = oracle.ang2pix(ns, lon, lat)
    assert pix.min() >= 0 and pix.max() < 12 * ns * ns
    for k in range(n):
        r = oracle.pix2ring(ns, int(pix[k]))
        c, f, zc, ph = oracle.ring_info(ns, r)
        zn = 1.0 if r == 1 else oracle.ring_info(ns, r - 1)[2]
        zs = -1.0 if r == 4 * ns - 1 else oracle.ring_info(ns, r + 1)[2]
        assert zs - 1e-12 <= zz[k] <= zn + 1e-12
        phic = (pix[k] - f + ph) * 2 * math.pi / c
        dphi = (math.radians(lon[k]) - phic + math.pi) % (2 * math.pi) - math.pi
        assert abs(dphi) <= math.pi / c + 1e-12


@pytest.mark.parametrize("ns", [1, 4, 64, 256])
def test_boundary_ring_corners(ns):
    """Points on the cap/belt boundary |z| = 2/3 at pixel-corner longitudes
    (and one ulp either side) get a pixel whose box holds them (a corner
    belongs to the pixels that meet there, on the boundary ring or the next
    belt ring): the belt formula alone can round such a point to ring 0 or
    2 ns + 2, outside the belt, i.e. a pixel of the neighbouring cap ring
    several spacings away."""
    zb = 2.0 / 3.0
    for sign in (1.0, -1.0):
        lat0 = math.degrees(math.asin(sign * zb))
        lats = np.array([lat0, np.nextafter(lat0, 90.0), np.nextafter(lat0, -90.0)])
        lon0 = np.arange(0, 4 * ns + 1) * (90.0 / ns)
        lons = np.concatenate([lon0, np.nextafter(lon0, 400.0), np.nextafter(lon0, -400.0)])
        lon, lat = np.meshgrid(lons, lats)
        lon, lat = lon.ravel(), lat.ravel()
        pix = oracle.ang2pix(ns, lon, lat)
        zz = np.sin(np.radians(lat))
        for k in range(pix.size):
            r = oracle.pix2ring(ns, int(pix[k]))
            c, f, zc, ph = oracle.ring_info(ns, r)
            zn = 1.0 if r == 1 else oracle.ring_info(ns, r - 1)[2]
            zs = -1.0 if r == 4 * ns - 1 else oracle.ring_info(ns, r + 1)[2]
            assert zs - 1e-12 <= zz[k] <= zn + 1e-12
            phic = (pix[k] - f + ph) * 2 * math.pi / c
            dphi = (math.radians(lon[k]) - phic + math.pi) % (2 * math.pi) - math.pi
            assert abs(dphi) <= math.pi / c + 1e-12


def test_lookup_equals_bruteforce_on_sightlines():
    """The lookup oracle finds every pair the brute force finds when the
    targets are the pixel centres of a coarser HEALPix grid -- they sit on
    ring latitudes and pixel corners of the lookup's finer grid (the cap /
    belt boundary ring included)."""
    import workloads
    lon_t, lat_t = workloads.healpix_centres(8)
    rng = np.random.Generator(np.random.PCG64(29))
    n = 30000
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    lon = rng.uniform(0, 360, n)
    data = rng.normal(size=(n, 1))
    k = oracle.gauss1d(2.0, 6.0)
    a = oracle.grid_lookup(64, lon_t, lat_t, lon, lat, data, k)
    b = oracle.grid_bruteforce(lon_t, lat_t, lon, lat, data, k)
    assert a.npairs == b.npairs
    assert np.allclose(a.wsum, b.wsum, rtol=1e-12, atol=0)


def test_lon_fold_and_poles():
    ns = 16
    lat = np.array([10.0, 10.0, 10.0, 10.0, 90.0, -90.0, 0.0])
    lon = np.array([-30.0, 330.0, 690.0, -390.0, 0.0, 0.0, 360.0])
    p = oracle.ang2pix(ns, lon, lat)
    assert p[0] == p[1] == p[2] == p[3]
    assert p[4] == 0                      # north pole -> first pixel of ring 1
    assert p[5] == 12 * ns * ns - 4       # south pole -> first pixel of last ring
    assert p[6] == oracle.ang2pix(ns, [0.0], [0.0])[0]
    assert oracle.lib().or_lon_fold_deg(-1e-20) == 0.0


@pytest.mark.parametrize("shifted", [False, True])
@pytest.mark.parametrize("ns", [8, 16])
def test_query_disc_superset_bruteforce(ns, shifted):
    """Every pixel that holds a point within R of the centre is returned."""
    rng = np.random.Generator(np.random.PCG64(23 + ns + (100 if shifted else 0)))
    pts_z = rng.uniform(-1, 1, 300_000)
    pts_lon = rng.uniform(0, 360, 300_000)
    pts_lat = np.degrees(np.arcsin(pts_z))
    pts_pix = oracle.ang2pix(ns, pts_lon, pts_lat)
    cz, sz = np.cos(np.radians(pts_lat)), np.sin(np.radians(pts_lat))
    centres = [(0.5, 0.0), (359.9, 45.0), (123.0, 89.0), (200.0, -88.5), (17.0, 90.0),
               (45.0, 41.8), (300.0, -41.8), (10.0, 3.0)]
    for (lc, bc) in centres:
        for R_deg in (0.7, 3.0, 11.0):
            R = math.radians(R_deg)
            # angular distance via the unit-vector dot product (independent of
            # the oracle's haversine)
            cb, sb = math.cos(math.radians(bc)), math.sin(math.radians(bc))
            dot = cz * cb * np.cos(np.radians(pts_lon - lc)) + sz * sb
            inside = np.arccos(np.clip(dot, -1, 1)) <= R
            need = set(np.unique(pts_pix[inside]).tolist())
            got = set(oracle.query_disc(ns, lc, bc, R, shifted=shifted).tolist())
            assert need <= got, (lc, bc, R_deg, sorted(need - got)[:5])
            # and not absurdly large: at most the pixels of a disc of radius
            # R + 2 pixel sizes (+ a few whole rings near a pole)
            pixsz = math.sqrt(math.pi / 3) / ns
            area = 2 * math.pi * (1 - math.cos(min(math.pi, R + 3 * pixsz)))
            assert len(got) <= 3 * area / (4 * math.pi / (12 * ns * ns)) + 8 * 4 * ns


def test_nside_rule_golden():
    for res_arcmin, ns in _load("nside_rule.txt"):
        assert oracle.nside_for_resolution(res_arcmin / 60.0) == int(ns)
