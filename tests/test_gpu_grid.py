"""GPU gridding (FP32 CUDA-core form) against the FP64 oracle (paper Eq. 1-3).

Small cases run the brute-force or lookup oracle over every target; they span
many tiles and a ragged last tile.  Edge cases: one sample, an empty add,
samples outside every support (NaN map), invalid coordinates, channel counts
that leave ragged channel blocks, per-sample weights, several adds, both
output layouts, BF16 input, nside independence and run-to-run determinism.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, gpu_kernel_args, kernel_of

pytestmark = pytest.mark.gpu

ARCMIN = 1.0 / 60.0


def run_gpu(wl, data=None, weights=None, nside=0, path=None, channel_major=False, adds=1):
    import torch
    from paper_1604_06667_gb300 import Gridder
    data = wl.data if data is None else data
    weights = wl.omega if weights is None else weights
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=data.shape[1])
    kt, kp = gpu_kernel_args(wl)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres, nside=nside)
    if path is not None:
        g.set_path(path)
    n = wl.n_samples
    cuts = np.linspace(0, n, adds + 1).astype(int)
    dt = torch.from_numpy(data) if isinstance(data, np.ndarray) else data
    for a, b in zip(cuts[:-1], cuts[1:]):
        g.grid(wl.lon_s[a:b], wl.lat_s[a:b], dt[a:b],
               None if weights is None else weights[a:b])
    w = torch.empty(wl.n_targets, device="cuda", dtype=torch.float32)
    out = g.get_datacube(channel_major=channel_major, out_weights=w)
    res = (out.cpu().numpy(), w.cpu().numpy(), g.info())
    g.close()
    return res


def ref_of(wl, data=None, weights=None, lookup=True):
    data = wl.data if data is None else data
    weights = wl.omega if weights is None else weights
    d64 = np.asarray(data, dtype=np.float64)
    om = None if weights is None else np.asarray(weights, dtype=np.float64)
    k = kernel_of(wl)
    if lookup:
        ns = oracle.nside_for_resolution(wl.hpx_maxres)
        return oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, d64, k, om)
    return oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, d64, k, om)


def test_plain2d_small_bruteforce():
    wl = workloads.plain2d(scale=0.12)
    out, w, info = run_gpu(wl)
    ref = ref_of(wl, lookup=False)
    assert info["n_tiles"] > 10 and wl.n_targets % info["tile_size"] != 0
    compare_maps(out, w, ref)


@pytest.mark.parametrize("C", [1, 7, 16, 17, 64, 130, 257])
def test_channel_counts(C):
    wl = workloads.random_field(200 + C, 1500, 23, C, 75.0, -30.0, 1.2, 2.0 * ARCMIN)
    out, w, _ = run_gpu(wl)
    compare_maps(out, w, ref_of(wl))


def test_cube_small():
    wl = workloads.cube(scale=0.004)
    assert wl.n_channels == 256
    out, w, _ = run_gpu(wl)
    compare_maps(out, w, ref_of(wl))


def test_elliptical_near_pole_and_wrap():
    # field straddling lon = 0 close to the north pole (paper Fig. 1 scenario)
    rng = np.random.Generator(np.random.PCG64(301))
    n = 6000
    lon = rng.uniform(-30, 30, n) % 360.0
    lat = rng.uniform(87.5, 90.0, n)
    lon_t, lat_t = workloads.car_grid(0.0, 88.6, 40, 25, 0.1)
    lon_t = lon_t % 360.0
    wl = workloads.Workload("pole", lon, lat, rng.normal(0, 1, (n, 3)).astype(np.float32), None,
                            lon_t, np.minimum(lat_t, 90.0),
                            {"type": "gauss2d", "smaj": 0.12, "smin": 0.06, "pa": 45.0},
                            0.36, 0.03)
    out, w, _ = run_gpu(wl)
    compare_maps(out, w, ref_of(wl))


def test_allsky_elliptical_small():
    wl = workloads.allsky(scale=0.004, n_channels=4)
    # widen the kernel so that the sparse small case has pairs everywhere
    wl.kernel = {"type": "gauss2d", "smaj": 1.5, "smin": 0.9, "pa": 30.0}
    wl.support = 4.5
    wl.hpx_maxres = 0.45
    out, w, _ = run_gpu(wl)
    compare_maps(out, w, ref_of(wl))


def test_weights_multi_add_and_layouts():
    wl = workloads.random_field(310, 3000, 30, 5, 200.0, 10.0, 1.5, 2.5 * ARCMIN, weights=True)
    ref = ref_of(wl)
    out, w, _ = run_gpu(wl, adds=3)
    compare_maps(out, w, ref)
    out_cm, w2, _ = run_gpu(wl, adds=1, channel_major=True)
    compare_maps(out_cm.T, w2, ref)


def test_bf16_input_fp32_path():
    import torch
    wl = workloads.random_field(320, 2500, 24, 12, 10.0, 40.0, 1.0, 2.0 * ARCMIN)
    d16 = torch.from_numpy(wl.data).to(torch.bfloat16)
    d_round = d16.to(torch.float32).numpy()
    out, w, _ = run_gpu(wl, data=d16)
    compare_maps(out, w, ref_of(wl, data=d_round))


def test_single_sample_and_empty_and_far():
    import torch
    from paper_1604_06667_gb300 import Gridder
    lon_t, lat_t = workloads.car_grid(50.0, 20.0, 21, 21, 0.01)
    g = Gridder(lon_t, lat_t, n_channels=2)
    g.set_kernel("gauss1d", (0.02,), 0.06, 0.01)
    # empty add is a no-op; everything NaN, W = 0
    g.grid(np.zeros(0), np.zeros(0), torch.zeros((0, 2)))
    w = torch.empty(lon_t.size, device="cuda")
    out = g.get_datacube(out_weights=w).cpu().numpy()
    assert np.all(np.isnan(out)) and np.all(w.cpu().numpy() == 0)
    # one sample far from all targets: still nothing
    g.grid([230.0], [-20.0], torch.tensor([[1.0, 2.0]]))
    out = g.get_datacube(out_weights=w).cpu().numpy()
    assert np.all(np.isnan(out)) and np.all(w.cpu().numpy() == 0)
    # one sample inside: W is the sampled kernel, R the sample's value
    g.reset()
    g.grid([50.013], [20.004], torch.tensor([[1.5, -2.0]]))
    out = g.get_datacube(out_weights=w).cpu().numpy()
    wref = np.array([oracle.kernel_value(oracle.gauss1d(0.02, 0.06), a, b, 50.013, 20.004)
                     for a, b in zip(lon_t, lat_t)])
    wg = w.cpu().numpy()
    on = wref > 0
    assert np.array_equal(on, wg > 0)
    assert np.max(np.abs(wg[on] - wref[on]) / wref[on]) < 1e-5
    assert np.allclose(out[on], [1.5, -2.0], rtol=1e-6)
    g.close()


def test_invalid_samples_reported_and_skipped():
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    wl = workloads.random_field(330, 800, 12, 2, 30.0, 30.0, 1.0, 2.0 * ARCMIN)
    lon, lat = wl.lon_s.copy(), wl.lat_s.copy()
    lat[5] = 95.0
    lon[7] = np.nan
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=2)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    g.grid(lon, lat, torch.from_numpy(wl.data))
    with pytest.raises(_capi.CygridError) as ei:
        g.get_datacube()
    assert ei.value.status == _capi.CG_EINVAL
    # the handle stays usable and the valid samples were gridded
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.get_datacube(out_weights=w).cpu().numpy()
    keep = np.ones(wl.n_samples, bool)
    keep[[5, 7]] = False
    sub = workloads.Workload("v", wl.lon_s[keep], wl.lat_s[keep], wl.data[keep], None, wl.lon_t,
                             wl.lat_t, wl.kernel, wl.support, wl.hpx_maxres)
    compare_maps(out, w.cpu().numpy(), ref_of(sub))
    g.close()


def test_result_independent_of_nside_and_deterministic():
    wl = workloads.random_field(340, 3000, 20, 3, 120.0, -60.0, 1.0, 2.0 * ARCMIN)
    ref = ref_of(wl)
    outs = []
    for ns in (0, 256, 8192):
        out, w, info = run_gpu(wl, nside=ns)
        compare_maps(out, w, ref)
        outs.append(out)
    a, _, _ = run_gpu(wl)
    assert np.array_equal(np.nan_to_num(a, nan=7.0), np.nan_to_num(outs[0], nan=7.0))


def test_bad_arguments():
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    lon_t, lat_t = workloads.car_grid(0.0, 0.0, 4, 4, 0.1)
    with pytest.raises(_capi.CygridError):
        Gridder(np.array([0.0, np.nan]), np.array([0.0, 0.0]))
    g = Gridder(lon_t, lat_t, n_channels=1)
    with pytest.raises(_capi.CygridError) as ei:
        g.grid([0.0], [0.0], torch.ones((1, 1)))
    assert ei.value.status == _capi.CG_ESTATE
    with pytest.raises(_capi.CygridError):
        g.set_kernel("gauss1d", (-1.0,), 0.1, 0.01)
    with pytest.raises(_capi.CygridError):
        g.set_kernel("gauss1d", (0.1,), 0.0, 0.01)
    g.set_kernel("gauss1d", (0.1,), 0.3, 0.05)
    g.close()


def test_stage_timing_and_destroy():
    """Stage timing on, several calls, read, destroy: events are owned once."""
    import torch
    from paper_1604_06667_gb300 import Gridder
    wl = workloads.random_field(350, 2000, 16, 4, 10.0, 10.0, 1.0, 2.0 * ARCMIN)
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=4)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    g.set_timing(True)
    for rep in range(3):
        for _ in range(3):
            g.grid_oneshot(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data))
        t = g.read_timing()
        assert t["grid_launches"] == 3 and t["grid"] > 0 and t["sort"] > 0
    g.grid(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data))
    g.close()


def test_candidate_splits_few_targets():
    """8,100 targets and 3e5 samples: each tile's candidates are shared by
    many CTAs whose partial sums are reduced in a fixed order; sampled
    targets against the brute-force oracle, and repeated calls identical."""
    import torch
    from paper_1604_06667_gb300 import Gridder
    from _parity import oracle_on_targets
    lon, lat, data, lon_t, lat_t, kern, support, maxres = \
        workloads.example1_device("cuda", n=300_000, seed=608)
    data = data.repeat(1, 3) * torch.tensor([1.0, -2.0, 0.5], device="cuda")
    g = Gridder(lon_t, lat_t, n_channels=3)
    g.set_kernel("gauss1d", (kern["sigma"],), support, maxres)
    w = torch.empty(lon_t.size, device="cuda")
    a = g.grid_oneshot(lon, lat, data, out_weights=w).clone()
    b = g.grid_oneshot(lon, lat, data)
    g.sync()
    g.close()
    assert torch.equal(torch.nan_to_num(a, nan=-9.0), torch.nan_to_num(b, nan=-9.0))

    class W:
        pass
    wl = W()
    wl.lon_s, wl.lat_s, wl.data = lon.cpu().numpy(), lat.cpu().numpy(), data.cpu().numpy()
    wl.lon_t, wl.lat_t, wl.omega, wl.support = lon_t, lat_t, None, support
    rng = np.random.Generator(np.random.PCG64(609))
    tsel = np.sort(rng.choice(lon_t.size, 200, replace=False))
    ref, _ = oracle_on_targets(wl, tsel, oracle.gauss1d(kern["sigma"], support))
    compare_maps(a.cpu().numpy()[tsel], w.cpu().numpy()[tsel], ref)
