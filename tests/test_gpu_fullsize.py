"""Parity at the full workload sizes, on sampled outputs the FP64 oracle
computes one by one (brute force over the samples that can reach each
sampled target, found by a latitude-band prefilter that is a superset):

* spectral cube (1e6 x 256 -> 512^2), in the launch configuration bench.py
  times (BF16 tensor-core one-shot with split weights), plus the exact pair
  count of the whole map against the oracle's stored count;
* plain 2-D (2e4 -> 100^2), the whole map;
* all-sky elliptical (1e7 x 32 -> 4096 x 2048);
* the differentiable workload (2e5 x 16 -> 256^2): forward map, adjoint
  (degridding) on sampled samples, d/dsigma on sampled targets, and a
  non-increasing 50-step map-making loss;
* the paper's Example 1 (1e8 samples) and its Appendix A.1 sight-line
  simulation (4.7e7 samples onto the 3,145,728 pixel centres of an nside-512
  HEALPix grid);
* the bench's 64-job batch, captured fused, every job on sampled targets, in
  the FP32 form and in the mixed form (BF16 tensor cores for C >= 16).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads
from _parity import (FP32_TOL, candidates_near, compare_maps, gpu_kernel_args, kernel_of,
                     oracle_on_targets, _haversine_np)

pytestmark = pytest.mark.gpu
TC_TOL = 5e-5
HERE = os.path.dirname(os.path.abspath(__file__))


def _gridder(wl, path=None):
    from paper_1604_06667_gb300 import Gridder
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    kt, kp = gpu_kernel_args(wl)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    if path is not None:
        g.set_path(path)
    return g


def _sampled_targets(wl, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(wl.n_targets, n, replace=False))


def test_cube_full_tc_bench_configuration():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = workloads.cube(scale=1.0)
    d16 = torch.from_numpy(wl.data).cuda().to(torch.bfloat16)
    g = _gridder(wl, _capi.CG_PATH_TC)
    out = torch.empty((wl.n_targets, wl.n_channels), device="cuda")
    w = torch.empty(wl.n_targets, device="cuda")
    g.grid_oneshot(torch.from_numpy(wl.lon_s).cuda(), torch.from_numpy(wl.lat_s).cuda(), d16,
                   out=out, out_weights=w)
    g.sync()
    info = g.info()
    out_np, w_np = out.cpu().numpy(), w.cpu().numpy()
    dr = d16.float().cpu().numpy()          # the oracle sees the same BF16-rounded data
    g.close()
    gold = json.load(open(os.path.join(HERE, "golden", "pair_counts.json")))["cube_scale1"]
    assert info["n_pairs"] == gold["pairs"]
    tsel = _sampled_targets(wl, 192, 601)
    ref, _ = oracle_on_targets(wl, tsel, kernel_of(wl), data=dr)
    compare_maps(out_np[tsel], w_np[tsel], ref, tol=TC_TOL)


def test_plain2d_full_whole_map():
    import torch
    wl = workloads.plain2d(scale=1.0)
    g = _gridder(wl)
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.grid_oneshot(wl.lon_s, wl.lat_s, wl.data, out_weights=w)
    out_np, w_np = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, wl.data, kernel_of(wl))
    compare_maps(out_np, w_np, ref, tol=FP32_TOL)


def test_allsky_full_elliptical_sampled():
    import torch
    wl = workloads.allsky(scale=1.0)
    g = _gridder(wl)
    w = torch.empty(wl.n_targets, device="cuda")
    d32 = torch.from_numpy(wl.data).cuda()
    out = g.grid_oneshot(torch.from_numpy(wl.lon_s).cuda(), torch.from_numpy(wl.lat_s).cuda(),
                         d32, out_weights=w)
    tsel = np.concatenate([_sampled_targets(wl, 96, 602),
                           np.arange(0, 64),                       # the first row: near a pole
                           np.arange(wl.n_targets - 64, wl.n_targets)])
    tsel = np.unique(tsel)
    got, got_w = out[torch.from_numpy(tsel).cuda()].cpu().numpy(), w.cpu().numpy()[tsel]
    g.close()
    ref, _ = oracle_on_targets(wl, tsel, kernel_of(wl))
    compare_maps(got, got_w, ref, tol=FP32_TOL)


def test_diff_full_forward_adjoint_dsigma_mapmaking():
    import torch
    from paper_1604_06667_gb300 import Gridder, mapmaking
    wl = workloads.diff(scale=1.0)
    k = kernel_of(wl)
    g = _gridder(wl)
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.grid_oneshot(wl.lon_s, wl.lat_s, wl.data, out_weights=w)
    out_np, w_np = out.cpu().numpy(), w.cpu().numpy()
    # forward on sampled targets
    tsel = _sampled_targets(wl, 128, 603)
    ref, cand = oracle_on_targets(wl, tsel, k)
    compare_maps(out_np[tsel], w_np[tsel], ref, tol=FP32_TOL)
    # d/dsigma on the same targets
    dR, _ = g.dsigma(torch.from_numpy(wl.data))
    dref = oracle.dsigma_bruteforce(wl.lon_t[tsel], wl.lat_t[tsel], wl.lon_s[cand], wl.lat_s[cand],
                                    np.asarray(wl.data, dtype=np.float64)[cand], k)
    on = np.isfinite(dref[:, 0])
    got = dR.cpu().numpy()[tsel]
    assert np.max(np.abs(got[on] - dref[on])) <= 1e-4 * np.abs(dref[on]).max()
    # adjoint on sampled samples: x_n = sum_p w_pn y_p / W_p with W_p of the
    # targets within reach, each from the oracle
    rng = np.random.Generator(np.random.PCG64(604))
    y = rng.normal(0, 1, (wl.n_targets, wl.n_channels)).astype(np.float32)
    xg = g.degrid(torch.from_numpy(y), map_weights=w).cpu().numpy()
    nsel = rng.choice(wl.n_samples, 24, replace=False)
    for n in nsel:
        dt = _haversine_np(wl.lon_s[n], wl.lat_s[n], wl.lon_t, wl.lat_t)
        near = np.nonzero(dt <= np.radians(wl.support) * (1 + 1e-6) + 1e-12)[0]
        if near.size == 0:
            assert np.all(xg[n] == 0.0)
            continue
        rw, _ = oracle_on_targets(wl, near, k, data=np.zeros((wl.n_samples, 1)))
        x = np.zeros(wl.n_channels)
        xs = np.zeros(wl.n_channels)
        for j, p in enumerate(near):
            if not rw.wsum[j] > 0:
                continue
            wv = oracle.kernel_value(k, wl.lon_t[p], wl.lat_t[p], wl.lon_s[n], wl.lat_s[n])
            x += wv / rw.wsum[j] * y[p].astype(np.float64)
            xs += wv / rw.wsum[j] * np.abs(y[p].astype(np.float64))
        assert np.all(np.abs(xg[n] - x) <= 2e-5 * xs + 1e-30), (n, xg[n], x)
    g.close()
    # map making at full size: no dense oracle; the loss must not increase
    g2 = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g2.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    _, losses, alpha = mapmaking.gd(g2, wl.lon_s, wl.lat_s, wl.data, steps=50)
    g2.close()
    assert alpha > 0
    assert np.all(np.diff(losses) <= 1e-6 * losses[0])
    assert losses[-1] < losses[0]


def _host_wl(lon, lat, data, lon_t, lat_t, kern, support):
    class W:
        pass
    wl = W()
    wl.lon_s, wl.lat_s = lon.cpu().numpy(), lat.cpu().numpy()
    wl.data = data.cpu().numpy()
    wl.lon_t, wl.lat_t = lon_t, lat_t
    wl.omega, wl.support = None, support
    wl.n_targets = lon_t.size
    return wl


def test_paper_example1_full_sampled():
    """The paper's Example 1 at 1e8 samples (few targets, many samples: the
    FP32 gridder splits each tile's candidates over many CTAs)."""
    import torch
    from paper_1604_06667_gb300 import Gridder
    lon, lat, data, lon_t, lat_t, kern, support, maxres = workloads.example1_device("cuda")
    g = Gridder(lon_t, lat_t, n_channels=1)
    g.set_kernel("gauss1d", (kern["sigma"],), support, maxres)
    w = torch.empty(lon_t.size, device="cuda")
    out = g.grid_oneshot(lon, lat, data, out_weights=w)
    g.sync()
    out_np, w_np = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    wl = _host_wl(lon, lat, data, lon_t, lat_t, kern, support)
    del lon, lat, data
    tsel = np.unique(np.concatenate([_sampled_targets(wl, 24, 607), [0, lon_t.size - 1]]))
    ref, _ = oracle_on_targets(wl, tsel, oracle.gauss1d(kern["sigma"], support))
    compare_maps(out_np[tsel], w_np[tsel], ref, tol=FP32_TOL)


def test_paper_sightline_a1_full_sampled():
    """Appendix A.1 at full size: samples uniform on the sphere onto HEALPix
    sight lines (arbitrary targets, tiles from the k-d tree), sampled targets
    including the first and last pixel (the poles' rings)."""
    import torch
    from paper_1604_06667_gb300 import Gridder
    lon, lat, data, lon_t, lat_t, kern, support, maxres, meta = workloads.sightline_device("cuda")
    assert meta["nside_targets"] == 512 and lon_t.size == 12 * 512 * 512
    g = Gridder(lon_t, lat_t, n_channels=1)
    g.set_kernel("gauss1d", (kern["sigma"],), support, maxres)
    w = torch.empty(lon_t.size, device="cuda")
    out = g.grid_oneshot(lon, lat, data, out_weights=w)
    g.sync()
    out_np, w_np = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    wl = _host_wl(lon, lat, data, lon_t, lat_t, kern, support)
    del lon, lat, data
    tsel = np.unique(np.concatenate([_sampled_targets(wl, 24, 611), [0, lon_t.size - 1]]))
    ref, _ = oracle_on_targets(wl, tsel, oracle.gauss1d(kern["sigma"], support))
    compare_maps(out_np[tsel], w_np[tsel], ref, tol=FP32_TOL)


@pytest.mark.parametrize("form", ["fp32", "mixed"])
def test_batch_config4_fused_every_job(form):
    """The bench's 64-job batch (1.26e7 samples, 3.0e9 channel values, grids
    64^2 .. 1024^2, sigma U[1', 8']) captured fused: every job against the
    FP64 oracle on 24 sampled targets (the samples within reach of them).
    FP32 form: FP32 data on the FP32 gridder, 1e-5 of S.  Mixed form: BF16
    data for C >= 16 on the tensor cores (hi + lo weights), against the
    oracle on the caller's unrounded FP32 data, within the BF16 data-rounding
    bound (unit roundoff 2^-8) plus the 5e-5 of the weights; the C = 1 jobs
    stay FP32 (1e-5)."""
    import torch
    from paper_1604_06667_gb300 import Batch, Gridder, _capi
    dev = torch.device("cuda")
    specs = workloads.batch_specs(64)
    jobs, meta = [], []
    for sp in specs:
        lon, lat, d32, lon_t, lat_t = workloads.batch_job_device(sp, dev)
        g = Gridder(lon_t, lat_t, n_channels=sp["C"], device=dev)
        g.set_kernel("gauss1d", (sp["sigma"],), 3.0 * sp["sigma"], sp["sigma"] / 2.0)
        tc = form == "mixed" and sp["C"] >= 16
        g.set_path(_capi.CG_PATH_TC if tc else _capi.CG_PATH_FP32)
        d = d32.to(torch.bfloat16) if tc else d32
        out = torch.empty((g.n_targets, sp["C"]), device=dev)
        w = torch.empty(g.n_targets, device=dev)
        jobs.append((g, lon, lat, d, out, w))
        meta.append((sp, lon, lat, d32, lon_t, lat_t, tc))
    b = Batch(jobs).set_fused(True).capture()
    b.run()
    b.sync()
    worst = {}
    for j, ((g, _, _, _, out, w), (sp, lon, lat, d32, lon_t, lat_t, tc)) in enumerate(zip(jobs, meta)):
        rng = np.random.Generator(np.random.PCG64(9000 + j))
        tsel = np.sort(rng.choice(lon_t.size, size=min(24, lon_t.size), replace=False))
        sigma = sp["sigma"]
        cand = candidates_near(lon_t[tsel], lat_t[tsel], lon, lat, 3.0 * sigma)
        rows = torch.from_numpy(cand).to(dev)
        dref = d32[rows].double().cpu().numpy()
        ref = oracle.grid_bruteforce(lon_t[tsel], lat_t[tsel], lon[cand], lat[cand], dref,
                                     oracle.gauss1d(sigma, 3.0 * sigma))
        tol = (2.0 ** -8 + 5e-5) if tc else FP32_TOL
        ts = torch.from_numpy(tsel).to(dev)
        me, mw = compare_maps(out[ts].cpu().numpy(), w[ts].cpu().numpy(), ref, tol=tol,
                              wtol=5e-5 if tc else FP32_TOL)
        key = "tc" if tc else "fp32"
        worst[key] = max(worst.get(key, 0.0), me)
    print("batch config 4 (%s form): largest error in units of S by gridder form: %s"
          % (form, {k: "%.2e" % v for k, v in worst.items()}))
    b.close()
    for jb in jobs:
        jb[0].close()
