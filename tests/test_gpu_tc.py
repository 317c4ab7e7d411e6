"""Tensor-core form (BF16 tcgen05, FP32 accumulation in TMEM) against the FP64
oracle run on the same BF16-rounded channel data (paper Eq. 1-3).

CG_PATH_TC stores each weight as a hi + lo pair of BF16 numbers (~16
significant bits); with FP32 accumulation the only difference from the FP64
definition on the same BF16 data is rounding, bound TC_TOL on the
S-normalised map error and the relative weight-map error.  CG_PATH_TC_FAST
keeps single BF16 weights (8 significant bits, each rounded to within
2^-8 of itself) in the numerator while W is summed in FP32 from the
unrounded weights, so the numerator moves by at most 2^-8 sum |omega w D|:
at most 2^-8 of S (bound FAST_TOL).
Also checked: the fused one-shot epilogue, store / add accumulation, several
adds, the channel-major layout, ragged channel counts (padding to the MMA N),
more than 256 channels (several channel slabs), the elliptical kernel and
sample weights, and agreement with the FP32 CUDA-core form.
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, gpu_kernel_args, kernel_of, oracle_on_targets

pytestmark = pytest.mark.gpu

TC_TOL = 5e-5
FAST_TOL = 2.0 ** -8
BF16_TOL = TC_TOL
ARCMIN = 1.0 / 60.0


def bf16_data(wl):
    import torch
    d16 = torch.from_numpy(wl.data).to(torch.bfloat16)
    return d16, d16.to(torch.float32).numpy()


def oracle_ref(wl, data):
    ns = oracle.nside_for_resolution(wl.hpx_maxres)
    om = None if wl.omega is None else wl.omega.astype(np.float64)
    return oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                              data.astype(np.float64), kernel_of(wl), om)


def gridder(wl, path=None):
    from paper_1604_06667_gb300 import Gridder, _capi
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    kt, kp = gpu_kernel_args(wl)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    g.set_path(_capi.CG_PATH_TC if path is None else path)
    return g


def oneshot(wl, d16, path=None, channel_major=False):
    import torch
    g = gridder(wl, path)
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.grid_oneshot(wl.lon_s, wl.lat_s, d16,
                         None if wl.omega is None else wl.omega, out_weights=w,
                         channel_major=channel_major)
    g.sync()
    info = g.info()
    res = out.cpu().numpy(), w.cpu().numpy(), info
    g.close()
    return res


def test_cube_small_oneshot_fused():
    from paper_1604_06667_gb300 import _capi
    wl = workloads.cube(scale=0.004)
    d16, dr = bf16_data(wl)
    out, w, info = oneshot(wl, d16)
    assert info["path"] == _capi.CG_PATH_TC and info["tile_size"] == 128
    ref = oracle_ref(wl, dr)
    me, mw = compare_maps(out, w, ref, tol=BF16_TOL, wtol=BF16_TOL)
    assert info["n_pairs"] == ref.npairs
    print("cube small: map err %.2e, weight err %.2e" % (me, mw))


@pytest.mark.parametrize("C", [8, 24, 64, 200, 256, 264, 512])
def test_channel_counts_tc(C):
    wl = workloads.random_field(400 + C, 1500, 25, C, 33.0, 12.0, 1.2, 2.0 * ARCMIN)
    d16, dr = bf16_data(wl)
    out, w, _ = oneshot(wl, d16)
    compare_maps(out, w, oracle_ref(wl, dr), tol=BF16_TOL, wtol=BF16_TOL)


def test_accumulate_modes_and_layout():
    import torch
    wl = workloads.random_field(450, 4000, 30, 32, 250.0, -45.0, 1.5, 2.5 * ARCMIN, weights=True)
    d16, dr = bf16_data(wl)
    ref = oracle_ref(wl, dr)
    g = gridder(wl)
    cuts = [0, 1000, 2500, 4000]
    for a, b in zip(cuts[:-1], cuts[1:]):
        g.grid(wl.lon_s[a:b], wl.lat_s[a:b], d16[a:b], wl.omega[a:b])
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.get_datacube(out_weights=w)
    compare_maps(out.cpu().numpy(), w.cpu().numpy(), ref, tol=BF16_TOL, wtol=BF16_TOL)
    # finalize is non-destructive; channel-major layout
    out2 = g.get_datacube(channel_major=True)
    compare_maps(out2.cpu().numpy().T, w.cpu().numpy(), ref, tol=BF16_TOL, wtol=BF16_TOL)
    g.close()
    out3, w3, _ = oneshot(wl, d16, channel_major=True)
    compare_maps(out3.T, w3, ref, tol=BF16_TOL, wtol=BF16_TOL)


def test_elliptical_tc():
    wl = workloads.allsky(scale=0.004, n_channels=16)
    wl.kernel = {"type": "gauss2d", "smaj": 1.5, "smin": 0.9, "pa": 30.0}
    wl.support = 4.5
    wl.hpx_maxres = 0.45
    d16, dr = bf16_data(wl)
    out, w, _ = oneshot(wl, d16)
    compare_maps(out, w, oracle_ref(wl, dr), tol=BF16_TOL, wtol=BF16_TOL)


def test_tc_agrees_with_fp32_form():
    from paper_1604_06667_gb300 import _capi
    wl = workloads.random_field(460, 3000, 28, 64, 100.0, 60.0, 1.2, 2.0 * ARCMIN)
    d16, dr = bf16_data(wl)
    a, wa, ia = oneshot(wl, d16, path=_capi.CG_PATH_TC)
    b, wb, ib = oneshot(wl, d16, path=_capi.CG_PATH_FP32)
    assert ia["path"] == _capi.CG_PATH_TC and ib["path"] == _capi.CG_PATH_FP32
    assert ia["n_pairs"] == ib["n_pairs"]
    ref = oracle_ref(wl, dr)
    compare_maps(b, wb, ref)                              # FP32 form: 1e-5
    compare_maps(a, wa, ref, tol=BF16_TOL, wtol=BF16_TOL)  # BF16 form


def test_fast_form_bound():
    from paper_1604_06667_gb300 import _capi
    wl = workloads.allsky(scale=0.004, n_channels=16)
    wl.kernel = {"type": "gauss2d", "smaj": 1.5, "smin": 0.9, "pa": 30.0}
    wl.support = 4.5
    wl.hpx_maxres = 0.45
    d16, dr = bf16_data(wl)
    out, w, info = oneshot(wl, d16, path=_capi.CG_PATH_TC_FAST)
    assert info["path"] == _capi.CG_PATH_TC_FAST
    me, mw = compare_maps(out, w, oracle_ref(wl, dr), tol=FAST_TOL, wtol=FAST_TOL)
    print("fast form: map err %.2e, weight err %.2e" % (me, mw))


def test_persistent_multi_tile_per_cta():
    """More tiles than resident CTAs: each persistent CTA runs several tiles
    (pipeline phases carried across tiles)."""
    wl = workloads.cube(scale=0.2, n_channels=32)
    d16, dr = bf16_data(wl)
    out, w, info = oneshot(wl, d16)
    assert info["n_tiles"] > 2 * 152   # at least two tiles per persistent CTA
    # 512 targets spread over the whole map (so over every CTA's later tiles),
    # each against the brute-force oracle on the samples that can reach it
    rng = np.random.Generator(np.random.PCG64(605))
    tsel = np.sort(rng.choice(wl.n_targets, 512, replace=False))
    ref, _ = oracle_on_targets(wl, tsel, kernel_of(wl), data=dr)
    compare_maps(np.asarray(out)[tsel], np.asarray(w)[tsel], ref, tol=BF16_TOL, wtol=BF16_TOL)


def test_tc_rejects_unsupported_inputs():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = workloads.random_field(470, 200, 8, 6, 10.0, 10.0, 0.5, 2.0 * ARCMIN)
    g = gridder(wl)
    with pytest.raises(_capi.CygridError) as ei:
        g.grid(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data))    # FP32 data, C % 8 != 0
    assert ei.value.status == _capi.CG_EINVAL
    g.close()


def _destination(lon1, lat1, d, beta):
    """Point at great-circle distance d (rad) and bearing beta (rad) from
    (lon1, lat1) in degrees (spherical direct problem, FP64)."""
    b1, l1 = np.radians(lat1), np.radians(lon1)
    b2 = np.arcsin(np.sin(b1) * np.cos(d) + np.cos(b1) * np.sin(d) * np.cos(beta))
    l2 = l1 + np.arctan2(np.sin(beta) * np.sin(d) * np.cos(b1),
                         np.cos(d) - np.sin(b1) * np.sin(b2))
    return np.degrees(l2), np.degrees(b2)


@pytest.mark.parametrize("path", ["fp32", "tc"])
def test_cut_edges_exact(path):
    """Samples placed at d = r (1 + delta) around targets, delta from 1e-8 to
    1e-5 on both sides (chord^2 within and at the edges of the +-1e-5 guard
    band): the pair count equals the FP64 oracle's exactly, on both forms."""
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    ARC = 1.0 / 60.0
    sigma = 3.0 * ARC
    r = 3.0 * sigma
    lon_t, lat_t = workloads.car_grid(140.0, -35.0, 12, 12, sigma / 2.0)
    rng = np.random.Generator(np.random.PCG64(606))
    deltas = np.array([1e-8, 1e-7, 1e-6, 4.9e-6, 4.98e-6, 5.0e-6, 5.02e-6, 5.1e-6, 1e-5])
    deltas = np.concatenate([deltas, -deltas])
    centre = np.nonzero((np.abs(np.arange(144) // 12 - 5.5) < 3) & (np.abs(np.arange(144) % 12 - 5.5) < 3))[0]
    lon_s, lat_s = [], []
    for p in centre:
        for dl in deltas:
            beta = rng.uniform(0, 2 * np.pi, 3)
            lo, la = _destination(lon_t[p], lat_t[p], np.radians(r) * (1.0 + dl), beta)
            lon_s.append(lo)
            lat_s.append(la)
    lon_s, lat_s = np.concatenate(lon_s), np.concatenate(lat_s)
    data = rng.normal(0, 1, (lon_s.size, 16)).astype(np.float32)
    k = oracle.gauss1d(sigma, r)
    g = Gridder(lon_t, lat_t, n_channels=16)
    g.set_kernel("gauss1d", (sigma,), r, sigma / 2.0)
    g.set_path(_capi.CG_PATH_TC if path == "tc" else _capi.CG_PATH_FP32)
    d = torch.from_numpy(data)
    if path == "tc":
        d = d.to(torch.bfloat16)
    w = torch.empty(lon_t.size, device="cuda")
    g.grid_oneshot(lon_s, lat_s, d, out_weights=w)
    g.sync()
    npairs = g.info()["n_pairs"]
    g.close()
    ref = oracle.grid_bruteforce(lon_t, lat_t, lon_s, lat_s, d.float().numpy(), k)
    assert npairs == ref.npairs
    on = ref.wsum > 0
    assert np.array_equal(on, w.cpu().numpy() > 0)
    assert np.max(np.abs(w.cpu().numpy()[on] - ref.wsum[on]) / ref.wsum[on]) < 5e-5
