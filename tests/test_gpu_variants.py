"""Variants of the method through the C-ABI, against the FP64 oracle:

* normalised interpolation (cg_interp): map -> samples, circular and
  elliptical kernels, the NaN pattern of samples with no target in reach,
  and the weight sums;
* one weight per sample and channel (cg_grid_oneshot_pcw): FP32 and BF16
  data, both map layouts, zero weights (their NaN values must not leak),
  and equality with the per-sample weighted one-shot call when every
  channel carries the same weight.
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import FP32_TOL, kernel_of, gpu_kernel_args

pytestmark = pytest.mark.gpu


def _gridder(wl):
    from paper_1604_06667_gb300 import Gridder, _capi
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    kt, kp = gpu_kernel_args(wl)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    return g


def _wl(name, scale, C=None):
    if name == "cube":
        return workloads.cube(scale=scale, n_channels=C or 4)
    if name == "allsky":
        return workloads.allsky(scale=scale, n_channels=C or 3)
    return workloads.plain2d(scale=scale)


@pytest.mark.parametrize("name,scale", [("plain2d", 0.5), ("cube", 0.002), ("allsky", 0.0005)])
def test_interp_against_oracle(name, scale):
    import torch
    wl = _wl(name, scale)
    g = _gridder(wl)
    g.grid_oneshot(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data).cuda())
    rng = np.random.Generator(np.random.PCG64(71))
    y = rng.normal(size=(wl.n_targets, wl.n_channels)).astype(np.float32)
    v = torch.empty(wl.n_samples, device="cuda")
    x = g.interp(torch.from_numpy(y).cuda(), out_weights=v)
    g.sync()
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    g.close()
    xr, vr = oracle.interp_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                      y.astype(np.float64), kernel_of(wl))
    on = vr > 0
    assert np.array_equal(on, v > 0)
    assert np.all(np.isnan(x[~on]))
    assert np.max(np.abs(v[on] - vr[on]) / vr[on]) < FP32_TOL
    # error relative to the mean |y| the sample's neighbourhood carries
    sabs, _ = oracle.interp_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                       np.abs(y).astype(np.float64), kernel_of(wl))
    assert np.max(np.abs(x[on] - xr[on]) / sabs[on]) < FP32_TOL


@pytest.mark.parametrize("bf16,channel_major", [(False, False), (True, True)])
def test_pcw_against_oracle(bf16, channel_major):
    import torch
    wl = _wl("cube", 0.002, C=5)
    rng = np.random.Generator(np.random.PCG64(73 + int(bf16)))
    om = rng.uniform(0.1, 3.0, (wl.n_samples, wl.n_channels)).astype(np.float32)
    om[rng.random(om.shape) < 0.2] = 0.0
    data = wl.data.copy()
    data[om == 0.0] = np.nan          # dropped values must not be read
    d = torch.from_numpy(data).cuda()
    if bf16:
        d = d.to(torch.bfloat16)
    dref = d.to(torch.float32).cpu().numpy().astype(np.float64)
    dref[om == 0.0] = 0.0
    g = _gridder(wl)
    shape = (wl.n_channels, wl.n_targets) if channel_major else (wl.n_targets, wl.n_channels)
    w = torch.empty(shape, device="cuda")
    out = g.grid_oneshot_pcw(wl.lon_s, wl.lat_s, d, torch.from_numpy(om).cuda(), out_weights=w,
                             channel_major=channel_major)
    g.sync()
    out, w = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    if channel_major:
        out, w = out.T, w.T
    R, W, S = oracle.grid_bruteforce_pcw(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref,
                                         kernel_of(wl), om.astype(np.float64))
    on = W > 0
    assert np.array_equal(on, w > 0)
    assert np.all(np.isnan(out[~on]))
    assert np.max(np.abs(w[on] - W[on]) / W[on]) < FP32_TOL
    assert np.max(np.abs(out[on] - R[on]) / S[on]) < FP32_TOL


def test_pcw_uniform_equals_weighted_oneshot():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = _wl("cube", 0.002, C=4)
    rng = np.random.Generator(np.random.PCG64(79))
    om = rng.uniform(0.5, 2.0, wl.n_samples).astype(np.float32)
    d = torch.from_numpy(wl.data).cuda()
    g = _gridder(wl)
    g.set_path(_capi.CG_PATH_FP32)
    w1 = torch.empty(wl.n_targets, device="cuda")
    r1 = g.grid_oneshot(wl.lon_s, wl.lat_s, d, torch.from_numpy(om).cuda(), out_weights=w1)
    g.sync()
    r1, w1 = r1.cpu().numpy(), w1.cpu().numpy()
    pcw = torch.from_numpy(np.repeat(om[:, None], wl.n_channels, 1)).cuda()
    w2 = torch.empty((wl.n_targets, wl.n_channels), device="cuda")
    r2 = g.grid_oneshot_pcw(wl.lon_s, wl.lat_s, d, pcw, out_weights=w2)
    g.sync()
    r2, w2 = r2.cpu().numpy(), w2.cpu().numpy()
    g.close()
    on = w1 > 0
    assert np.array_equal(np.isnan(r1), np.isnan(r2))
    for c in range(wl.n_channels):
        assert np.allclose(w2[on, c], w1[on], rtol=2e-6, atol=0)
    assert np.allclose(r2[on], r1[on], rtol=1e-5, atol=1e-5)


def _tsinc_wl(name, scale, C=None):
    """A workload re-gridded with the tapered sinc: first zero a = 1.2 sigma,
    taper b = 2 sigma, support 3 sigma of the workload's Gaussian."""
    wl = _wl(name, scale, C)
    s = wl.kernel["sigma"]
    wl.kernel = {"type": "tsinc", "a": 1.2 * s, "b": 2.0 * s}
    return wl


def _tsinc_grid(wl, d, path):
    import torch
    from paper_1604_06667_gb300 import Gridder
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("tsinc", (wl.kernel["a"], wl.kernel["b"]), wl.support, wl.hpx_maxres)
    g.set_path(path)
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.grid_oneshot(wl.lon_s, wl.lat_s, d, out_weights=w)
    g.sync()
    res = (out.cpu().numpy(), w.cpu().numpy(), g)
    return res


def _tsinc_check(wl, out, w, data64, tol):
    """Errors relative to sums of magnitudes (the signed weights cancel, so
    R = N / W is ill-conditioned where W << sum |w|): W against
    sum |omega w|, the numerator N = R W against sum |omega w D|."""
    k = oracle.tapered_sinc(wl.kernel["a"], wl.kernel["b"], wl.support)
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, data64, k)
    ones = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                  np.ones((wl.n_samples, 1)), k)
    on = ref.wsum > 0
    assert np.array_equal(on, w > 0)
    assert np.all(np.isnan(out[~on]))
    wabs = ones.sabs[on, 0] * ones.wsum[on]
    assert np.max(np.abs(w[on] - ref.wsum[on]) / wabs) < tol
    num = out[on] * w[on, None]
    nabs = ref.sabs[on] * ref.wsum[on, None]
    assert np.max(np.abs(num - ref.num[on]) / nabs) < tol


def test_tsinc_fp32_against_oracle():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = _tsinc_wl("plain2d", 0.3)
    out, w, g = _tsinc_grid(wl, torch.from_numpy(wl.data).cuda(), _capi.CG_PATH_FP32)
    g.close()
    _tsinc_check(wl, out, w, wl.data.astype(np.float64), FP32_TOL)


def test_tsinc_tensor_cores_against_oracle():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = _tsinc_wl("cube", 0.002, C=16)
    d16 = torch.from_numpy(wl.data).cuda().to(torch.bfloat16)
    out, w, g = _tsinc_grid(wl, d16, _capi.CG_PATH_TC)
    assert g.info()["path"] == _capi.CG_PATH_TC
    g.close()
    _tsinc_check(wl, out, w, d16.to(torch.float32).cpu().numpy().astype(np.float64), 5e-5)


def test_tsinc_interp_against_oracle():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = _tsinc_wl("plain2d", 0.3)
    out, w, g = _tsinc_grid(wl, torch.from_numpy(wl.data).cuda(), _capi.CG_PATH_FP32)
    rng = np.random.Generator(np.random.PCG64(83))
    y = rng.normal(size=(wl.n_targets, 1)).astype(np.float32)
    v = torch.empty(wl.n_samples, device="cuda")
    x = g.interp(torch.from_numpy(y).cuda(), out_weights=v)
    g.sync()
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    g.close()
    k = oracle.tapered_sinc(wl.kernel["a"], wl.kernel["b"], wl.support)
    xr, vr = oracle.interp_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, y.astype(np.float64), k)
    on = vr > 0
    assert np.array_equal(on, v > 0)
    assert np.max(np.abs(v[on] - vr[on]) / vr[on]) < FP32_TOL
    # numerators sum_p w y against sum_p |w| max |y| (the signed weights cancel)
    lt, bt = np.radians(wl.lat_t), np.radians(wl.lon_t)
    vabs = np.empty(wl.n_samples)
    for i0 in range(0, wl.n_samples, 512):
        ls = np.radians(wl.lat_s[i0:i0 + 512])[:, None]
        lo = np.radians(wl.lon_s[i0:i0 + 512])[:, None]
        h = np.sin(0.5 * (lt - ls)) ** 2 + np.cos(lt) * np.cos(ls) * np.sin(0.5 * (bt - lo)) ** 2
        d = np.degrees(2 * np.arcsin(np.sqrt(np.minimum(1.0, h))))
        xx = np.pi * d / wl.kernel["a"]
        wk = np.where(xx > 0, np.sin(xx) / np.where(xx > 0, xx, 1), 1.0) * \
            np.exp(-(d / wl.kernel["b"]) ** 2)
        vabs[i0:i0 + 512] = np.where(d <= wl.support, np.abs(wk), 0.0).sum(1)
    num_err = np.abs(x[on, 0] * v[on] - xr[on, 0] * vr[on]) / (vabs[on] * np.abs(y).max())
    assert np.max(num_err) < FP32_TOL
