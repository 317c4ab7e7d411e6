"""Seeded synthetic inputs for the gridding workloads.

This module only synthesises inputs (sample coordinates, channel data, target
coordinates and kernel parameters).  It contains none of the gridding
arithmetic, so both the CUDA path and the FP64 oracle can consume it.

All randomness comes from ``numpy.random.Generator(PCG64(seed))`` with
``seed = 1604_06667 + config id`` unless overridden.

Workloads (sizes at ``scale = 1``):

* ``plain2d``  -- 20,000 samples uniform in a 5 x 5 deg field at (30, 0); value =
  5 Gaussian sources (FWHM 6', amplitude U[1,10]) + N(0, 0.1) noise; unit
  weights; 100 x 100 plate-carree targets at 3'; gauss1d sigma = 2.5',
  support 3 sigma, hpx_maxres = sigma / 2.  (The shape of the paper's
  Example 1, Sect. 4: uniform random positions and a noise-like signal.)
* ``cube``     -- 1e6 samples on a basket-weave raster (1' rows, 0.5' along scan,
  pointing jitter N(0, 0.2')) over lon 115-125, lat 25-35; 256 channels
  (3 Gaussian lines of width 5 channels with spatially smooth amplitude,
  + N(0,1) noise); 512 x 512 targets; gauss1d sigma = 3', support 9'.
* ``allsky``   -- 1e7 samples uniform on the sphere (poles included); 32
  channels of smooth random fields (16 blobs of FWHM 5 deg shared by all
  channels with per-channel amplitudes) + N(0, 0.1); 4096 x 2048 full-sky
  plate-carree targets (pixel centres off the poles, longitude wrap);
  elliptical Gaussian sigma_maj = 10', sigma_min = 6', PA = 30 deg, support
  3 sigma_maj, hpx_maxres = sigma_min / 2.
* ``diff``     -- 2e5 samples uniform in 512' x 512' at (200, -20); 16 channels;
  256 x 256 targets at 2'; sigma = 4', support 12'.

``scale < 1`` shrinks a workload for fast parity tests while keeping its
sample density, pixel size and kernel (field side scales as sqrt(scale)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1604_06667
ARCMIN = 1.0 / 60.0


@dataclass
class Workload:
    name: str
    lon_s: np.ndarray            # float64 [N] degrees
    lat_s: np.ndarray            # float64 [N] degrees
    data: np.ndarray             # float32 [N][C]
    omega: np.ndarray | None     # float32 [N] or None (unit weights)
    lon_t: np.ndarray            # float64 [P] degrees
    lat_t: np.ndarray            # float64 [P] degrees
    kernel: dict                 # {"type": "gauss1d", "sigma": deg, ...}
    support: float               # degrees
    hpx_maxres: float            # degrees
    grid_shape: tuple = ()       # (ny, nx) of the plate-carree target grid
    meta: dict = field(default_factory=dict)

    @property
    def n_samples(self) -> int:
        return int(self.lon_s.size)

    @property
    def n_targets(self) -> int:
        return int(self.lon_t.size)

    @property
    def n_channels(self) -> int:
        return int(self.data.shape[1])


def rng_for(cid: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + cid if seed is None else seed))


def car_grid(lon0: float, lat0: float, nx: int, ny: int, dpix: float):
    """Plate-carree target centres around (lon0, lat0), row-major (lat outer)."""
    xs = lon0 + (np.arange(nx) - 0.5 * (nx - 1)) * dpix
    ys = lat0 + (np.arange(ny) - 0.5 * (ny - 1)) * dpix
    lat, lon = np.meshgrid(ys, xs, indexing="ij")
    return lon.ravel().astype(np.float64), lat.ravel().astype(np.float64)


def allsky_car(nx: int, ny: int):
    """Full-sky plate-carree pixel centres; none sits on a pole."""
    xs = (np.arange(nx) + 0.5) * (360.0 / nx)
    ys = -90.0 + (np.arange(ny) + 0.5) * (180.0 / ny)
    lat, lon = np.meshgrid(ys, xs, indexing="ij")
    return lon.ravel().astype(np.float64), lat.ravel().astype(np.float64)


def _flat_gauss(lon, lat, lon_k, lat_k, sigma):
    dx = (lon - lon_k) * math.cos(math.radians(lat_k))
    dy = lat - lat_k
    return np.exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma))


def plain2d(scale: float = 1.0, seed: int | None = None) -> Workload:
    rng = rng_for(1, seed)
    side = 5.0 * math.sqrt(scale)
    n = max(1, int(round(20_000 * scale)))
    lon0, lat0 = 30.0, 0.0
    lon = lon0 + (rng.random(n) - 0.5) * side
    lat = lat0 + (rng.random(n) - 0.5) * side
    sig_src = 6.0 * ARCMIN / math.sqrt(8.0 * math.log(2.0))
    val = rng.normal(0.0, 0.1, n)
    for _ in range(5):
        lk = lon0 + (rng.random() - 0.5) * side
        bk = lat0 + (rng.random() - 0.5) * side
        val += rng.uniform(1.0, 10.0) * _flat_gauss(lon, lat, lk, bk, sig_src)
    npx = max(2, int(round(100 * math.sqrt(scale))))
    lon_t, lat_t = car_grid(lon0, lat0, npx, npx, 3.0 * ARCMIN)
    sigma = 2.5 * ARCMIN
    return Workload("plain2d", lon, lat, val.astype(np.float32)[:, None], None, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": sigma}, 3.0 * sigma, sigma / 2.0,
                    (npx, npx), {"scale": scale})


def _raster(rng, lon_lo, lat_lo, side, n_total, row_step, scan_step, jitter):
    """Basket-weave raster: zig-zag scans along longitude, then along latitude,
    truncated at ``n_total`` samples."""
    nrow = max(1, int(round(side / row_step)))
    nalong = max(1, int(round(side / scan_step)))
    rows = lat_lo + (np.arange(nrow) + 0.5) * row_step
    along = lon_lo + (np.arange(nalong) + 0.5) * scan_step
    # pass 1: scans of constant latitude
    lat1 = np.repeat(rows, nalong)
    lon1 = np.tile(along, nrow).reshape(nrow, nalong)
    lon1[1::2] = lon1[1::2, ::-1]
    lon1 = lon1.ravel()
    # pass 2: scans of constant longitude
    cols = lon_lo + (np.arange(nrow) + 0.5) * row_step
    along2 = lat_lo + (np.arange(nalong) + 0.5) * scan_step
    lon2 = np.repeat(cols, nalong)
    lat2 = np.tile(along2, nrow).reshape(nrow, nalong)
    lat2[1::2] = lat2[1::2, ::-1]
    lat2 = lat2.ravel()
    lon = np.concatenate([lon1, lon2])[:n_total]
    lat = np.concatenate([lat1, lat2])[:n_total]
    lon = lon + rng.normal(0.0, jitter, lon.size)
    lat = lat + rng.normal(0.0, jitter, lat.size)
    return lon, lat


def cube(scale: float = 1.0, seed: int | None = None, n_channels: int = 256) -> Workload:
    rng = rng_for(2, seed)
    side = 10.0 * math.sqrt(scale)
    n = max(1, int(round(1_000_000 * scale)))
    lon_lo, lat_lo = 120.0 - 0.5 * side, 30.0 - 0.5 * side
    lon, lat = _raster(rng, lon_lo, lat_lo, side, n, 1.0 * ARCMIN, 0.5 * ARCMIN,
                       0.2 * ARCMIN)
    C = n_channels
    # spatially smooth line amplitude: a few broad blobs
    amp = np.zeros(lon.size)
    for _ in range(6):
        lk = lon_lo + rng.random() * side
        bk = lat_lo + rng.random() * side
        amp += rng.uniform(1.0, 10.0) * _flat_gauss(lon, lat, lk, bk, 0.15 * side + 0.05)
    chan = np.arange(C, dtype=np.float32)
    sig_ch = 5.0 / math.sqrt(8.0 * math.log(2.0))
    data = rng.standard_normal((lon.size, C), dtype=np.float32)
    for _ in range(3):
        c0 = rng.uniform(0.08 * C, 0.92 * C)
        prof = np.exp(-((chan - c0) ** 2) / (2.0 * sig_ch * sig_ch)).astype(np.float32)
        data += (amp.astype(np.float32) * rng.uniform(0.3, 1.0))[:, None] * prof[None, :]
    npx = max(2, int(round(512 * math.sqrt(scale))))
    lon_t, lat_t = car_grid(120.0, 30.0, npx, npx, side / npx)
    sigma = 3.0 * ARCMIN
    return Workload("cube", lon, lat, data, None, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": sigma}, 3.0 * sigma, sigma / 2.0,
                    (npx, npx), {"scale": scale})


def allsky(scale: float = 1.0, seed: int | None = None, n_channels: int = 32) -> Workload:
    rng = rng_for(3, seed)
    n = max(1, int(round(10_000_000 * scale)))
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 360.0, n)
    lat = np.degrees(np.arcsin(z))
    lon = phi
    C = n_channels
    nb = 16
    bz = rng.uniform(-1.0, 1.0, nb)
    bphi = rng.uniform(0.0, 2.0 * math.pi, nb)
    bs = np.sqrt(1.0 - bz * bz)
    bvec = np.stack([bs * np.cos(bphi), bs * np.sin(bphi), bz], axis=1)      # [nb, 3]
    sig_b = math.radians(5.0) / math.sqrt(8.0 * math.log(2.0))
    kappa = 1.0 / (sig_b * sig_b)
    A = rng.uniform(-5.0, 5.0, (nb, C)).astype(np.float32)
    data = np.empty((n, C), dtype=np.float32)
    step = 1 << 20
    for s in range(0, n, step):
        e = min(n, s + step)
        cz = z[s:e]
        cs = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
        cp = np.radians(phi[s:e])
        u = np.stack([cs * np.cos(cp), cs * np.sin(cp), cz], axis=1)
        B = np.exp(kappa * (u @ bvec.T - 1.0)).astype(np.float32)            # [m, nb]
        data[s:e] = B @ A + rng.normal(0.0, 0.1, (e - s, C)).astype(np.float32)
    nx = max(4, int(round(4096 * math.sqrt(scale))))
    ny = max(2, nx // 2)
    lon_t, lat_t = allsky_car(nx, ny)
    smaj, smin = 10.0 * ARCMIN, 6.0 * ARCMIN
    return Workload("allsky", lon, lat, data, None, lon_t, lat_t,
                    {"type": "gauss2d", "smaj": smaj, "smin": smin, "pa": 30.0},
                    3.0 * smaj, smin / 2.0, (ny, nx), {"scale": scale})


def diff(scale: float = 1.0, seed: int | None = None) -> Workload:
    rng = rng_for(5, seed)
    side = 512.0 * ARCMIN * math.sqrt(scale)
    n = max(1, int(round(200_000 * scale)))
    lon0, lat0 = 200.0, -20.0
    lon = lon0 + (rng.random(n) - 0.5) * side
    lat = lat0 + (rng.random(n) - 0.5) * side
    C = 16
    data = rng.normal(0.0, 1.0, (n, C)).astype(np.float32)
    for _ in range(8):
        lk = lon0 + (rng.random() - 0.5) * side
        bk = lat0 + (rng.random() - 0.5) * side
        prof = _flat_gauss(lon, lat, lk, bk, 10.0 * ARCMIN).astype(np.float32)
        data += prof[:, None] * rng.uniform(1.0, 10.0, C).astype(np.float32)[None, :]
    npx = max(2, int(round(256 * math.sqrt(scale))))
    lon_t, lat_t = car_grid(lon0, lat0, npx, npx, 2.0 * ARCMIN)
    sigma = 4.0 * ARCMIN
    return Workload("diff", lon, lat, data, None, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": sigma}, 3.0 * sigma, sigma / 2.0,
                    (npx, npx), {"scale": scale})


def random_field(cid: int, n: int, n_targets_side: int, C: int, lon0: float, lat0: float,
                 side_deg: float, sigma_deg: float, seed: int | None = None,
                 weights: bool = False) -> Workload:
    """Small generic case for edge tests: uniform samples in a square field."""
    rng = rng_for(cid, seed)
    lon = lon0 + (rng.random(n) - 0.5) * side_deg
    lat = np.clip(lat0 + (rng.random(n) - 0.5) * side_deg, -90.0, 90.0)
    data = rng.normal(0.0, 1.0, (n, C)).astype(np.float32) + 3.0
    om = rng.uniform(0.2, 2.0, n).astype(np.float32) if weights else None
    lon_t, lat_t = car_grid(lon0, lat0, n_targets_side, n_targets_side,
                            side_deg / n_targets_side)
    lat_t = np.clip(lat_t, -90.0, 90.0)
    return Workload("random", lon, lat, data, om, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": sigma_deg}, 3.0 * sigma_deg,
                    sigma_deg / 2.0, (n_targets_side, n_targets_side), {})


# ---------------------------------------------------------------------------
# Batched jobs (many independent gridding problems of uneven size)
# ---------------------------------------------------------------------------
BATCH_CHANNELS = (1, 16, 64, 512)
BATCH_SIDES = (64, 128, 256, 512, 1024)


def batch_specs(n_jobs: int = 64, seed: int | None = None, n_range=(1e4, 1e6),
                channels=BATCH_CHANNELS, sides=BATCH_SIDES) -> list:
    """Job descriptions: sample count log-uniform in n_range, channels and
    target-grid side drawn from the given sets, sigma ~ U[1', 8'], pixel =
    sigma / 2, support 3 sigma, field centre lon ~ U[0, 360), lat ~ U[-60, 60]
    (moved towards the equator when the field would reach |lat| > 88), data
    dtype alternating FP32 / BF16."""
    rng = rng_for(4, seed)
    specs = []
    for j in range(n_jobs):
        n = int(round(10.0 ** rng.uniform(math.log10(n_range[0]), math.log10(n_range[1]))))
        C = int(rng.choice(channels))
        side = int(rng.choice(sides))
        sigma = rng.uniform(1.0, 8.0) * ARCMIN
        step = sigma / 2.0
        half = 0.5 * side * step
        lon0 = rng.uniform(0.0, 360.0)
        lat0 = float(np.clip(rng.uniform(-60.0, 60.0), -88.0 + half, 88.0 - half)) \
            if half < 88.0 else 0.0
        specs.append({"job": j, "n": n, "C": C, "side": side, "sigma": sigma, "step": step,
                      "lon0": lon0, "lat0": lat0, "dtype": "bf16" if j % 2 else "f32",
                      "seed": int(rng.integers(0, 2 ** 31))})
    return specs


def batch_job(spec: dict) -> Workload:
    """A job of batch_specs as a numpy workload: samples uniform in the field,
    data N(0, 1) plus three Gaussian sources (FWHM 4 sigma) with per-channel
    amplitudes U[1, 10]."""
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    n, C, side, step = spec["n"], spec["C"], spec["side"], spec["step"]
    half = 0.5 * side * step
    lon = spec["lon0"] + rng.uniform(-half, half, n)
    lat = spec["lat0"] + rng.uniform(-half, half, n)
    data = rng.standard_normal((n, C), dtype=np.float32)
    fwhm = 4.0 * spec["sigma"]
    for _ in range(3):
        lk = spec["lon0"] + rng.uniform(-half, half)
        bk = spec["lat0"] + rng.uniform(-half, half)
        prof = _flat_gauss(lon, lat, lk, bk, fwhm).astype(np.float32)
        data += prof[:, None] * rng.uniform(1.0, 10.0, C).astype(np.float32)[None, :]
    lon_t, lat_t = car_grid(spec["lon0"], spec["lat0"], side, side, step)
    return Workload("batch%d" % spec["job"], lon, lat, data, None, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": spec["sigma"]}, 3.0 * spec["sigma"],
                    spec["sigma"] / 2.0, (side, side), dict(spec))


def batch_job_device(spec: dict, device, dtype_override=None):
    """batch_job with the channel data generated on the device (seeded torch
    generator; used by the benchmark, where numpy would spend tens of seconds
    on the 3e9 values of a 64-job batch).  Returns (lon_s, lat_s, data[n, C]
    float32 on the device, lon_t, lat_t, spec)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    n, C, side, step = spec["n"], spec["C"], spec["side"], spec["step"]
    half = 0.5 * side * step
    lon = spec["lon0"] + rng.uniform(-half, half, n)
    lat = spec["lat0"] + rng.uniform(-half, half, n)
    gen = torch.Generator(device=device)
    gen.manual_seed(spec["seed"])
    data = torch.randn((n, C), generator=gen, device=device, dtype=torch.float32)
    fwhm = 4.0 * spec["sigma"]
    lon_d = torch.from_numpy(lon).to(device)
    lat_d = torch.from_numpy(lat).to(device)
    for _ in range(3):
        lk = spec["lon0"] + rng.uniform(-half, half)
        bk = spec["lat0"] + rng.uniform(-half, half)
        dx = (lon_d - lk) * math.cos(math.radians(bk))
        dy = lat_d - bk
        prof = torch.exp(-(dx * dx + dy * dy) / (2.0 * fwhm * fwhm)).float()
        amp = torch.from_numpy(rng.uniform(1.0, 10.0, C).astype(np.float32)).to(device)
        data += prof[:, None] * amp[None, :]
    lon_t, lat_t = car_grid(spec["lon0"], spec["lat0"], side, side, step)
    return lon, lat, data, lon_t, lat_t


# ---------------------------------------------------------------------------
# The paper's Example 1 (Sect. 4): random samples onto a 5 x 5 deg field
# ---------------------------------------------------------------------------
ARCSEC = 1.0 / 3600.0


def example1_device(device, n: int = 100_000_000, seed: int | None = None):
    """n samples uniform in a 5 deg x 5 deg field at (30, 0), one channel of
    N(0, 1) noise, gridded onto 200" pixels (90 x 90) with a Gaussian of FWHM
    300" (support 3 sigma, hpx_maxres sigma / 2).  Drawn on the device with a
    seeded torch generator (1e8 samples).  Returns (lon, lat, data[n, 1],
    lon_t, lat_t, kernel dict, support, hpx_maxres)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + 6 if seed is None else seed)
    side, lon0, lat0 = 5.0, 30.0, 0.0
    lon = lon0 + (torch.rand(n, generator=gen, device=device, dtype=torch.float64) - 0.5) * side
    lat = lat0 + (torch.rand(n, generator=gen, device=device, dtype=torch.float64) - 0.5) * side
    data = torch.randn((n, 1), generator=gen, device=device, dtype=torch.float32)
    npx = int(round(side / (200.0 * ARCSEC)))
    lon_t, lat_t = car_grid(lon0, lat0, npx, npx, 200.0 * ARCSEC)
    sigma = 300.0 * ARCSEC / math.sqrt(8.0 * math.log(2.0))
    return lon, lat, data, lon_t, lat_t, {"type": "gauss1d", "sigma": sigma}, 3.0 * sigma, \
        sigma / 2.0


# ---------------------------------------------------------------------------
# Appendix A.1: point sources on the sphere gridded onto HEALPix sight lines
# ---------------------------------------------------------------------------
def healpix_centres(nside: int):
    """Longitude / latitude (degrees) of the RING-scheme pixel centres of a
    HEALPix tessellation (Gorski et al. 2005): rings of constant z, 4 i
    pixels on polar-cap ring i, 4 nside on the equatorial rings, whose
    longitudes start at 0 or half a pixel on alternate rings.  Target
    positions only (input synthesis)."""
    ns = int(nside)
    lon_parts, lat_parts = [], []
    for i in range(1, 4 * ns):
        if i < ns:                      # north cap
            z = 1.0 - i * i / (3.0 * ns * ns)
            m = 4 * i
            phi = (np.arange(m) + 0.5) * (2.0 * math.pi / m)
        elif i <= 3 * ns:               # equatorial belt
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns)
            m = 4 * ns
            s = (i - ns + 1) % 2
            phi = (np.arange(m) + 0.5 * s) * (2.0 * math.pi / m)
        else:                           # south cap
            k = 4 * ns - i
            z = -(1.0 - k * k / (3.0 * ns * ns))
            m = 4 * k
            phi = (np.arange(m) + 0.5) * (2.0 * math.pi / m)
        lon_parts.append(np.degrees(phi))
        lat_parts.append(np.full(m, math.degrees(math.asin(z))))
    return np.concatenate(lon_parts), np.concatenate(lat_parts)


def _unit(lon_deg, lat_deg, xp=np):
    l = lon_deg * (math.pi / 180.0)
    b = lat_deg * (math.pi / 180.0)
    return xp.stack([xp.cos(b) * xp.cos(l), xp.cos(b) * xp.sin(l), xp.sin(b)], -1)


def sightline_device(device, scale: float = 1.0, seed: int | None = None, n_sources: int = 1024):
    """The simulation of Appendix A.1: 1024 point sources at random positions
    on the sphere (amplitudes U[1, 10]) seen through a Gaussian PSF of FWHM
    4 pixel sizes, sampled at 15 x npix random positions uniform on the
    sphere with N(0, 1) noise added to every sample, and gridded onto the
    pixel centres of a HEALPix grid with a Gaussian kernel of half the PSF's
    FWHM (support 3 sigma, hpx_maxres sigma / 2).  nside = 512 at scale 1
    (npix 3,145,728, ~4.7e7 samples, PSF 27.5', kernel 13.7'), nside 512
    sqrt(scale) rounded to a power of two otherwise.  Samples, sources and
    signal are drawn and evaluated on the device (torch, seeded).
    Returns (lon, lat, data[n, 1] float32, lon_t, lat_t, kernel dict,
    support, hpx_maxres, meta)."""
    import torch
    ns = 512
    while ns > 8 and (ns // 2) ** 2 >= 512 * 512 * scale:
        ns //= 2
    npix = 12 * ns * ns
    n = 15 * npix
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE + 7 if seed is None else seed)
    z = torch.rand(n, generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
    lon = torch.rand(n, generator=gen, device=device, dtype=torch.float64) * 360.0
    lat = torch.rad2deg(torch.asin(z))
    zs = torch.rand(n_sources, generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
    ls = torch.rand(n_sources, generator=gen, device=device, dtype=torch.float64) * 360.0
    amp = 1.0 + 9.0 * torch.rand(n_sources, generator=gen, device=device, dtype=torch.float64)
    pix = math.sqrt(4.0 * math.pi / npix)                 # pixel size (rad)
    fwhm_psf = 4.0 * pix
    s2 = 8.0 * math.log(2.0)
    sig_psf = fwhm_psf / math.sqrt(s2)
    vs = _unit(ls, torch.rad2deg(torch.asin(zs)), torch).to(torch.float32)     # [S, 3]
    data = torch.randn((n, 1), generator=gen, device=device, dtype=torch.float32)
    chunk = 1 << 17
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        u = _unit(lon[a:b], lat[a:b], torch).to(torch.float32)                  # [c, 3]
        c2 = (2.0 - 2.0 * (u @ vs.T)).clamp_min(0.0)                           # chord^2
        data[a:b, 0] += (torch.exp(-c2 / (2.0 * sig_psf * sig_psf)) * amp.to(torch.float32)).sum(1)
    lon_t, lat_t = healpix_centres(ns)
    sigma = math.degrees(0.5 * fwhm_psf / math.sqrt(s2))
    meta = {"nside_targets": ns, "npix": npix, "n_samples": n, "fwhm_psf_deg": math.degrees(fwhm_psf),
            "fwhm_kernel_deg": math.degrees(0.5 * fwhm_psf)}
    return lon, lat, data, lon_t, lat_t, {"type": "gauss1d", "sigma": sigma}, 3.0 * sigma, \
        sigma / 2.0, meta


# ---------------------------------------------------------------------------
# Appendix A.2: scan lines of samples, kernel size against aliasing
# ---------------------------------------------------------------------------
def aliasing(f_space: float, f_kernel: float, support_sigmas: float = 5.0,
             seed: int | None = None, side: float = 1.5, psf: float = 0.1,
             pix_div: int = 20, along_div: int = 100, n_sources: int = 2000) -> Workload:
    """The stripe simulation of Appendix A.2: a quasi-continuous field of
    point sources (uniform positions over the field and a margin, amplitudes
    U[0.5, 1.5]) seen through a Gaussian PSF of FWHM ``psf`` deg, sampled on
    horizontal scan lines ``f_space * psf`` apart with ``psf / along_div``
    spacing along them (no noise), gridded onto ``psf / pix_div`` pixels over
    ``side`` x ``side`` deg with a Gaussian kernel of FWHM ``f_kernel * psf``
    and support ``support_sigmas`` sigma.  The samples cover the field plus
    the largest support of the study (5 sigma of a 0.7 psf kernel) and do not
    depend on the kernel.  ``meta`` holds the sources, for aliasing_truth()."""
    lon, lat, val, src, sig_psf = _aliasing_samples(float(f_space), seed, side, psf, along_div,
                                                    n_sources)
    s2 = math.sqrt(8.0 * math.log(2.0))
    sig_k = f_kernel * psf / s2
    npx = int(round(side * pix_div / psf))
    lon_t, lat_t = car_grid(120.0, 30.0, npx, npx, side / npx)
    return Workload("aliasing", lon, lat, val[:, None], None, lon_t, lat_t,
                    {"type": "gauss1d", "sigma": sig_k}, support_sigmas * sig_k, sig_k / 2.0,
                    (npx, npx),
                    {"f_space": f_space, "f_kernel": f_kernel, "support_sigmas": support_sigmas,
                     "sig_psf": sig_psf, "src": src})


_ALIAS_CACHE: dict = {}


def _aliasing_samples(f_space, seed, side, psf, along_div, n_sources):
    key = (f_space, seed, side, psf, along_div, n_sources)
    if key in _ALIAS_CACHE:
        return _ALIAS_CACHE[key]
    rng = rng_for(8, seed)
    lon0, lat0 = 120.0, 30.0
    s2 = math.sqrt(8.0 * math.log(2.0))
    sig_psf = psf / s2
    reach = 5.0 * 0.7 * psf / s2           # largest support of the study
    margin = 6.0 * sig_psf + reach
    span = side + 2.0 * margin
    dl = span / math.cos(math.radians(lat0))
    src_lon = lon0 + (rng.random(n_sources) - 0.5) * dl
    src_lat = lat0 + (rng.random(n_sources) - 0.5) * span
    src_amp = rng.uniform(0.5, 1.5, n_sources)
    ext = side + 2.0 * reach
    n_lines = int(math.floor(ext / (f_space * psf))) + 1
    lats = lat0 - 0.5 * ext + np.arange(n_lines) * (f_space * psf)
    ext_lon = ext / math.cos(math.radians(lat0))
    n_along = int(round(ext * along_div / psf)) + 1
    lons = lon0 - 0.5 * ext_lon + np.arange(n_along) * (ext_lon / (n_along - 1))
    lat, lon = np.meshgrid(lats, lons, indexing="ij")
    lon = lon.ravel().astype(np.float64)
    lat = lat.ravel().astype(np.float64)
    val = _gauss_field(_unit(lon, lat), src_lon, src_lat, src_amp, sig_psf, 1.0).astype(np.float32)
    out = (lon, lat, val, (src_lon, src_lat, src_amp), sig_psf)
    _ALIAS_CACHE.clear()
    _ALIAS_CACHE[key] = out
    return out


def aliasing_truth(wl: Workload) -> np.ndarray:
    """The field of an aliasing() workload convolved with its (unit-integral)
    gridding kernel, at the targets: each PSF-convolved source becomes a
    Gaussian of variance sigma_psf^2 + sigma_k^2 and peak scaled by
    sigma_psf^2 / (sigma_psf^2 + sigma_k^2) (small-field approximation; the
    kernel's truncation at its support is ignored)."""
    src_lon, src_lat, src_amp = wl.meta["src"]
    sp, sk = wl.meta["sig_psf"], wl.kernel["sigma"]
    st2 = sp * sp + sk * sk
    return _gauss_field(_unit(wl.lon_t, wl.lat_t), src_lon, src_lat, src_amp, math.sqrt(st2),
                        sp * sp / st2)


def _gauss_field(u, src_lon, src_lat, src_amp, sig, scale):
    """sum_k scale * amp_k * exp(-d^2 / 2 sig^2) at the unit vectors u
    (sources beyond 8 sig ignored; sig in degrees)."""
    from scipy.spatial import cKDTree
    vs = _unit(src_lon, src_lat)
    reach = 2.0 * math.sin(math.radians(8.0 * sig) / 2.0)
    m = cKDTree(u).sparse_distance_matrix(cKDTree(vs), reach, output_type="coo_matrix")
    d2 = np.degrees(2.0 * np.arcsin(np.minimum(1.0, 0.5 * m.data))) ** 2
    w = scale * src_amp[m.col] * np.exp(-d2 / (2.0 * sig * sig))
    return np.bincount(m.row, weights=w, minlength=u.shape[0])
