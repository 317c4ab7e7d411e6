"""Input synthesis for the paper's Appendix A workloads, and the oracle on
the A.2 scan-line study:

* the HEALPix pixel centres used as sight-line targets (A.1) are the
  oracle's pix2ang of every RING index, in index order;
* the FP64 brute-force oracle reproduces the study's qualitative result
  (A.2): the relative deviation of the gridded map from the kernel-convolved
  field falls as the kernel widens and rises as the scan lines move apart.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from _parity import kernel_of


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_healpix_centres_match_oracle_pix2ang(nside):
    lon, lat = workloads.healpix_centres(nside)
    npix = 12 * nside * nside
    assert lon.size == npix and lat.size == npix
    z, phi = oracle.pix2ang(nside, np.arange(npix))
    assert np.max(np.abs(np.sin(np.radians(lat)) - z)) < 1e-14
    d = np.abs(np.radians(lon) - phi)
    assert np.max(np.minimum(d, 2 * math.pi - d)) < 1e-13


def _dev(fs, fk):
    wl = workloads.aliasing(fs, fk, side=0.2, n_sources=120)
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                 wl.data.astype(np.float64), kernel_of(wl))
    truth = workloads.aliasing_truth(wl)
    return float(np.max(np.abs(ref.out[:, 0] - truth) / truth))


def test_aliasing_trends_oracle():
    # (the wider kernels at close spacing reach the ~1e-4 floor of the
    # small-field model of the convolved field, so only 0.3 vs 0.7 is ranked)
    d = {(fs, fk): _dev(fs, fk) for fs in (0.2, 0.5) for fk in (0.3, 0.7)}
    assert d[(0.5, 0.3)] > d[(0.5, 0.7)]
    assert d[(0.2, 0.3)] > d[(0.2, 0.7)]
    assert d[(0.5, 0.3)] > d[(0.2, 0.3)]
    assert d[(0.5, 0.7)] > d[(0.2, 0.7)]
