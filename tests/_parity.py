"""Shared comparison helpers for the GPU parity tests.

Error metric for maps (signed data can cancel, so a plain relative error is
ill-posed): e_pc = |R_gpu - R_oracle| / S_pc with S_pc = sum |omega w D| / W_p
emitted by the oracle; weights compare by plain relative error.  The support
masks (W > 0) must agree exactly and W = 0 pixels must be NaN.
"""
import numpy as np

import oracle

FP32_TOL = 1e-5


def kernel_of(wl):
    k = wl.kernel
    if k["type"] == "gauss1d":
        return oracle.gauss1d(k["sigma"], wl.support)
    return oracle.gauss2d(k["smaj"], k["smin"], k["pa"], wl.support)


def gpu_kernel_args(wl):
    k = wl.kernel
    if k["type"] == "gauss1d":
        return "gauss1d", (k["sigma"],)
    return "gauss2d", (k["smaj"], k["smin"], k["pa"])


def compare_maps(got, got_w, ref, tol=FP32_TOL, wtol=FP32_TOL, channels=None):
    """got [P][C] float32, got_w [P]; ref = oracle.GridResult (restricted to the
    same targets).  Returns (max map error, max weight error)."""
    got = np.asarray(got, dtype=np.float64)
    got_w = np.asarray(got_w, dtype=np.float64)
    on = ref.wsum > 0
    assert np.array_equal(on, got_w > 0), \
        "support mismatch at %d targets" % int((on != (got_w > 0)).sum())
    assert np.all(np.isnan(got[~on])), "W = 0 targets must be NaN"
    if not on.any():
        return 0.0, 0.0
    werr = np.abs(got_w[on] - ref.wsum[on]) / ref.wsum[on]
    ref_out, sabs = ref.out[on], ref.sabs[on]
    g = got[on]
    if channels is not None:
        ref_out, sabs, g = ref_out[:, channels], sabs[:, channels], g[:, channels]
    scale = np.where(sabs > 0, sabs, 1.0)
    err = np.abs(g - ref_out) / scale
    err = np.where(np.isnan(ref_out) & np.isnan(g), 0.0, err)
    me, mw = float(np.nanmax(err)), float(werr.max())
    assert np.isfinite(err).all(), "non-finite map error"
    assert me <= tol, "map error %.3e > %.1e" % (me, tol)
    assert mw <= wtol, "weight error %.3e > %.1e" % (mw, wtol)
    return me, mw


def _haversine_np(l1, b1, l2, b2):
    b1, b2 = np.radians(b1), np.radians(b2)
    dl = np.radians(np.asarray(l2) - l1)
    h = np.sin(0.5 * (b2 - b1)) ** 2 + np.cos(b1) * np.cos(b2) * np.sin(0.5 * dl) ** 2
    return 2.0 * np.arcsin(np.sqrt(np.minimum(h, 1.0)))


def candidates_near(lon_c, lat_c, lon_s, lat_s, radius_deg, order=None):
    """Indices of the samples within radius_deg of any centre, as a superset
    (radius widened by 1e-6 relative): latitude bands from one sort, then the
    great-circle distance.  Lets the FP64 brute-force oracle evaluate Eq. 1-3
    exactly for a few targets of a large workload."""
    lat_s = np.asarray(lat_s)
    if order is None:
        order = np.argsort(lat_s, kind="stable")
    ls = lat_s[order]
    rad = radius_deg * (1.0 + 1e-6) + 1e-9
    out = []
    for lc, bc in zip(np.atleast_1d(lon_c), np.atleast_1d(lat_c)):
        lo = np.searchsorted(ls, bc - rad, "left")
        hi = np.searchsorted(ls, bc + rad, "right")
        idx = order[lo:hi]
        d = _haversine_np(lc, bc, np.asarray(lon_s)[idx], lat_s[idx])
        out.append(idx[d <= np.radians(rad)])
    return np.unique(np.concatenate(out)) if out else np.zeros(0, dtype=np.int64)


def oracle_on_targets(wl, tsel, k, data=None, omega="wl"):
    """oracle.grid_bruteforce restricted to the targets tsel and to the samples
    that can reach them (exact for those targets)."""
    data = wl.data if data is None else data
    om = wl.omega if isinstance(omega, str) else omega
    cand = candidates_near(wl.lon_t[tsel], wl.lat_t[tsel], wl.lon_s, wl.lat_s, wl.support)
    return oracle.grid_bruteforce(wl.lon_t[tsel], wl.lat_t[tsel], wl.lon_s[cand], wl.lat_s[cand],
                                  np.asarray(data, dtype=np.float64)[cand], k,
                                  None if om is None else np.asarray(om)[cand]), cand
