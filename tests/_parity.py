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
