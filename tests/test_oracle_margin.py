"""Pins for the oracle's ang2pix decision margin (paper Sect. 2.2 step 3a; the
RING tessellation of Gorski et al. 2005).

``oracle.ang2pix_margin`` returns how far, in the units of the quantities that
ang2pix truncates, a direction lies from the nearest pixel boundary.  The GPU
key tests excuse a key mismatch only where that margin is below 1e-9, so a
margin that is too small somewhere would hide a real GPU error.  It is pinned
by facts the tessellation fixes, not by its own formulas:

* at every pixel centre the margin is exactly one half (the centre is half a
  unit from each of the lines that bound its pixel), except on the two rings
  that lie on the cap/belt switch |z| = 2/3, where it is zero;
* on a pixel boundary -- found by bisecting a short segment whose end points
  ang2pix puts in different pixels, so the boundary is where ang2pix changes,
  whatever formula produced it -- the margin is zero;
* random directions have a margin above 1e-9 (the chance of one falling that
  close to a boundary is ~1e-8 per point).

Planted mistakes (a dropped line family, an offset in the cap's in-ring index,
the zone switch left out) each fail at least one of these.
"""
import math

import numpy as np
import pytest

import oracle
from _mutate import with_mutated_oracle


def _lonlat(z, phi):
    return np.degrees(phi), np.degrees(np.arcsin(np.clip(z, -1.0, 1.0)))


def check_centres(nsides=(2, 4, 8, 16)):
    for ns in nsides:
        npix = 12 * ns * ns
        pix = np.arange(npix)
        z, phi = oracle.pix2ang(ns, pix)
        lon, lat = _lonlat(z, phi)
        m = oracle.ang2pix_margin(ns, lon, lat)
        ring = np.array([oracle.pix2ring(ns, int(p)) for p in pix])
        on_switch = (ring == ns) | (ring == 3 * ns)
        assert np.all(m[on_switch] < 1e-9), (ns, m[on_switch].max())
        off = ~on_switch
        assert np.max(np.abs(m[off] - 0.5)) < 1e-7, (ns, np.abs(m[off] - 0.5).max())


def _boundary_points(ns, n, seed):
    """Points on pixel boundaries: random short segments in (phi, z) whose end
    points ang2pix assigns to different pixels, bisected to 1e-14."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pix_rad = math.sqrt(math.pi / 3.0) / ns
    pts = []
    tries = 0
    while len(pts) < n and tries < 50 * n:
        tries += 1
        z0 = rng.uniform(-0.999, 0.999)
        if rng.uniform() < 0.3:                       # extra points near the switch
            z0 = math.copysign(2.0 / 3.0, rng.uniform(-1, 1)) + rng.uniform(-2, 2) * pix_rad
        p0 = rng.uniform(0.0, 2.0 * math.pi)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        step = 0.6 * pix_rad
        z1 = float(np.clip(z0 + step * math.sin(ang), -0.999, 0.999))
        p1 = p0 + step * math.cos(ang) / math.sqrt(max(1e-6, 1.0 - z0 * z0))
        ends = np.array([[z0, p0], [z1, p1]])
        lon, lat = _lonlat(ends[:, 0], ends[:, 1])
        k = oracle.ang2pix(ns, lon, lat)
        if k[0] == k[1]:
            continue
        a, b, ka = ends[0].copy(), ends[1].copy(), k[0]
        for _ in range(200):
            if np.max(np.abs(b - a)) < 1e-14:
                break
            mid = 0.5 * (a + b)
            lo, la = _lonlat(np.array([mid[0]]), np.array([mid[1]]))
            if oracle.ang2pix(ns, lo, la)[0] == ka:
                a = mid
            else:
                b = mid
        pts.append(0.5 * (a + b))
    assert len(pts) == n
    return np.array(pts)


def check_boundaries(nsides=(1, 4, 64, 4096), n=150):
    for ns in nsides:
        pts = _boundary_points(ns, n, seed=900 + ns)
        lon, lat = _lonlat(pts[:, 0], pts[:, 1])
        m = oracle.ang2pix_margin(ns, lon, lat)
        # a boundary point is within ~1e-14 rad of the line: ns * 1e-13 units
        assert np.all(m < 1e-9 + ns * 1e-12), (ns, m.max(), pts[np.argmax(m)])


def check_random_points(nsides=(1, 8, 512, 8192), n=20000):
    for ns in nsides:
        rng = np.random.Generator(np.random.PCG64(77 + ns))
        z = rng.uniform(-1.0, 1.0, n)
        lon = rng.uniform(-360.0, 720.0, n)
        lat = np.degrees(np.arcsin(z))
        m = oracle.ang2pix_margin(ns, lon, lat)
        assert np.all(m > 1e-9), (ns, m.min())
        assert np.all(m <= 0.5 + 1e-12), (ns, m.max())


def test_margin_at_pixel_centres():
    check_centres()


def test_margin_zero_on_boundaries():
    check_boundaries()


def test_margin_random_points():
    check_random_points()


MUTATIONS = {
    "descending_lines_dropped": ("    q[nq++] = u + v;\n", "\n", [check_boundaries]),
    "cap_in_ring_index_offset": ("q[nq++] = tt * (double)k;", "q[nq++] = tt * (double)(k + 1);",
                                 [check_centres]),
    "zone_switch_dropped": ("double m = fabs(za - 2.0 / 3.0) * dns;", "double m = 1.0;",
                            [check_centres]),
    "cap_line_scaled": ("q[nq++] = (1.0 - t) * x;", "q[nq++] = (1.0 - t) * x * 0.5;",
                        [check_centres, check_boundaries]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_margin_mistake_is_caught(name, monkeypatch):
    old, new, checks = MUTATIONS[name]
    assert with_mutated_oracle(monkeypatch, old, new, checks), \
        "planted mistake %s was not caught" % name
