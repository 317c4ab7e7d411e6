"""GPU HEALPix index, sort and ring offsets against the FP64 oracle: bit-exact
(paper Sect. 2.2 step 3a; the sorted replacement for the hash tables of
Sect. 3.4).  Samples closer than 1e-9 (in the units of the floored quantities)
to a pixel boundary may legitimately land in either neighbour; the oracle
flags them and only they may differ (none are expected)."""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def adversarial(ns, rng):
    lon, lat = [], []
    # poles, equator, lon wrap, cap/belt transition
    for b in (90.0, -90.0, 0.0, -0.0, math.degrees(math.asin(2 / 3)),
              -math.degrees(math.asin(2 / 3)), 89.999999, -89.999999):
        for l in (0.0, -0.0, 360.0, 720.0, -360.0, 359.9999999999, -1e-300, 1e-300, 45.0, 90.0,
                  180.0, 270.0, -45.0):
            lon.append(l)
            lat.append(b)
    # either side of the pole thresholds of the fast paths (1 - |z| = 1e-5,
    # 1e-6), where the error of z is magnified most
    for dz in (3e-5, 1.2e-5, 1e-5, 0.8e-5, 3e-6, 1e-6, 3e-7):
        b = math.degrees(math.asin(1.0 - dz))
        for l in rng.uniform(0.0, 360.0, 24):
            lon += [l, l]
            lat += [b, -b]
    # ring centres and pixel-centre / pixel-edge longitudes of a few rings
    for i in sorted(set([1, 2, ns - 1, ns, ns + 1, 2 * ns, 3 * ns, 3 * ns + 1, 4 * ns - 1])):
        if i < 1 or i > 4 * ns - 1:
            continue
        c, f, z, ph = oracle.ring_info(ns, i)
        b = math.degrees(math.asin(z))
        for j in list(range(min(c, 6))) + [c - 1]:
            for off in (0.0, 0.5, 0.25):
                lon.append((j + ph + off) * 360.0 / c)
                lat.append(b)
    n = len(lon)
    return np.array(lon), np.array(lat)


@pytest.mark.parametrize("ns", [1, 2, 3, 16, 1000, 1024, 2048, 4096, 8192, 12345])
def test_ang2pix_bit_exact(ns):
    from paper_1604_06667_gb300 import ang2pix_ring
    rng = np.random.Generator(np.random.PCG64(100 + ns))
    n = 400_000
    lon = rng.uniform(-720, 720, n)
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, n)))
    al, ab = adversarial(ns, rng)
    lon = np.concatenate([lon, al])
    lat = np.concatenate([lat, ab])
    got = ang2pix_ring(ns, lon, lat).cpu().numpy()
    ref = oracle.ang2pix(ns, lon, lat)
    bad = np.nonzero(got != ref)[0]
    if bad.size:
        margins = oracle.ang2pix_margin(ns, lon[bad], lat[bad])
        assert np.all(margins < 1e-9), (bad[:5], got[bad[:5]], ref[bad[:5]], margins[:5])
    assert bad.size <= 2


@pytest.mark.parametrize("ns", [16, 1024, 4096, 8192])
def test_sample_keys_bit_exact(ns):
    """The gridder's own per-sample keys (the double-float path for ordinary
    angles, FP64 near boundaries and pixel-edge or quadrant-edge values, near
    the poles and for |lon| >= 2048)
    sorted and exported: equal to the oracle's sort of its keys."""
    import torch
    from paper_1604_06667_gb300 import Gridder
    rng = np.random.Generator(np.random.PCG64(200 + ns))
    n = 300_000
    lon = np.concatenate([rng.uniform(-720, 720, n), rng.uniform(-5000, 5000, 2000)])
    lat = np.degrees(np.arcsin(rng.uniform(-1, 1, lon.size)))
    al, ab = adversarial(ns, rng)
    lon = np.concatenate([lon, al])
    lat = np.concatenate([lat, ab])
    g = Gridder(np.array([0.0]), np.array([0.0]), n_channels=1)
    sigma = math.degrees(math.sqrt(math.pi / 3) / ns)
    g.set_kernel("gauss1d", (sigma,), 3 * sigma, nside=ns)
    g.grid(lon, lat, torch.zeros((lon.size, 1)))
    pix, perm, _ = g.export_index(lon.size)
    g.sync()
    pix, perm = pix.cpu().numpy(), perm.cpu().numpy()
    g.close()
    got = np.empty_like(pix)
    got[perm] = pix
    ref = oracle.ang2pix(ns, lon, lat)
    bad = np.nonzero(got != ref)[0]
    if bad.size:
        margins = oracle.ang2pix_margin(ns, lon[bad], lat[bad])
        assert np.all(margins < 1e-9), (bad[:5], got[bad[:5]], ref[bad[:5]], margins[:5])
    assert bad.size <= 2


def test_ang2pix_invalid_inputs():
    from paper_1604_06667_gb300 import ang2pix_ring
    lon = np.array([0.0, np.nan, 10.0, np.inf, 10.0, 5.0])
    lat = np.array([0.0, 0.0, 90.0000001, 0.0, np.nan, -91.0])
    got = ang2pix_ring(64, lon, lat).cpu().numpy()
    assert got[0] == oracle.ang2pix(64, [0.0], [0.0])[0]
    assert np.all(got[1:] == -1)


@pytest.mark.parametrize("case", ["cube", "allsky", "dup", "dup_many_tiles", "allsky_many_waves"])
def test_sort_and_ring_offsets_bit_exact(case):
    import torch
    from paper_1604_06667_gb300 import Gridder
    if case == "cube":
        wl = workloads.cube(scale=0.02, n_channels=4)
    elif case == "allsky":
        wl = workloads.allsky(scale=0.01, n_channels=2)
    elif case == "allsky_many_waves":
        # 2e6 samples = 489 sort tiles: more than one wave of resident tiles,
        # so the passes rank block-wide (fewer tiles rank per warp)
        wl = workloads.allsky(scale=0.2, n_channels=1)
    else:
        # many exact duplicates: ties must keep ascending sample order (the
        # larger case spans 40 sort tiles of 4096 keys with a ragged last one)
        base = workloads.plain2d(scale=0.05 if case == "dup" else 1.0)
        rep = 7 if case == "dup" else 8
        wl = workloads.Workload("dup", np.repeat(base.lon_s, rep), np.repeat(base.lat_s, rep),
                                np.repeat(base.data, rep, axis=0), None, base.lon_t, base.lat_t,
                                base.kernel, base.support, base.hpx_maxres)
        rng = np.random.Generator(np.random.PCG64(5))
        p = rng.permutation(wl.n_samples)
        wl.lon_s, wl.lat_s, wl.data = wl.lon_s[p], wl.lat_s[p], wl.data[p]
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    kt, kp = ("gauss1d", (wl.kernel["sigma"],)) if wl.kernel["type"] == "gauss1d" else \
        ("gauss2d", (wl.kernel["smaj"], wl.kernel["smin"], wl.kernel["pa"]))
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    ns = g.info()["nside"]
    assert ns == oracle.nside_for_resolution(wl.hpx_maxres)
    g.grid(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data))
    pix, perm, ring = g.export_index(wl.n_samples)
    g.sync()
    pix, perm, ring = pix.cpu().numpy(), perm.cpu().numpy(), ring.cpu().numpy()
    ref_pix = oracle.ang2pix(ns, wl.lon_s, wl.lat_s)
    ref_perm = oracle.sort_stable(ref_pix)
    assert np.array_equal(perm, ref_perm)
    assert np.array_equal(pix, ref_pix[ref_perm])
    assert np.array_equal(ring, oracle.ring_offsets(ns, ref_pix[ref_perm]))
    uniq, off = oracle.csr(pix)
    assert off[-1] == wl.n_samples and uniq.size <= wl.n_samples
    g.close()


def test_unit_vectors_double_float():
    """Sample unit vectors (double-float sine/cosine on the FP32 pipes) against
    the FP64 definition: |error| <= 1e-13 per component, including quadrant
    and table-interval boundaries, large longitudes and the poles."""
    from paper_1604_06667_gb300 import unit_vectors
    rng = np.random.Generator(np.random.PCG64(4242))
    n = 200_000
    lon = np.concatenate([rng.uniform(-1080, 1080, n),
                          np.array([0.0, -0.0, 45.0, -45.0, 90.0, 135.0, 180.0, 225.0, 270.0,
                                    315.0, 360.0, 1e-12, -1e-12, 44.999999999, 45.000000001,
                                    0.5 * 180 / math.pi / 64, 1.5 * 180 / math.pi / 64,
                                    720.0, -720.0, 1e6 + 0.123]),
                          # table-interval edges j/64 +- 1/128 rad in degrees
                          np.degrees((np.arange(-52, 53) + 0.5) / 64.0)])
    lat = np.concatenate([np.degrees(np.arcsin(rng.uniform(-1, 1, n))),
                          np.array([0.0, 90.0, -90.0, 89.9999999, -89.9999999, 45.0, -45.0,
                                    1e-300, 30.0, 60.0, 0.0, 0.0, 0.0, 10.0, -10.0, 20.0,
                                    20.0, 0.0, 0.0, 5.0]),
                          np.clip(np.degrees((np.arange(-52, 53) + 0.5) / 64.0), -90, 90)])
    got = unit_vectors(lon, lat).cpu().numpy()
    # reduce the longitude in degrees first (exact), as radians(1e6 deg) alone
    # would carry an FP64 rounding error of ~1e-12 rad
    b, l = np.radians(lat), np.radians(np.fmod(lon, 360.0))
    ref = np.stack([np.cos(b) * np.cos(l), np.cos(b) * np.sin(l), np.sin(b)], axis=1)
    err = np.abs(got - ref).max()
    assert err <= 1e-13, err
    assert np.abs(np.linalg.norm(got, axis=1) - 1.0).max() <= 2e-13
