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
