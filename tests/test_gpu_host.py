"""Host-buffer one-shot calls (cg_grid_oneshot_host).

* a sequence of pipelined calls with different samples and data gives, call
  by call and bit for bit, what cg_grid_oneshot gives on the same inputs in
  device memory (tensor-core and FP32 forms, both map layouts, sample weights,
  the weight map), read after one cg_sync;
* a call with more samples than the staging slots hold regrows them while an
  earlier call may still be in flight;
* one call against the FP64 oracle (the same bound as the device call);
* host tensors on the wrong device are refused before anything runs.
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, kernel_of

pytestmark = pytest.mark.gpu


def _gridder(wl, path):
    from paper_1604_06667_gb300 import Gridder, _capi
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    g.set_path(_capi.CG_PATH_TC if path == "tc" else _capi.CG_PATH_FP32)
    return g


def _inputs(scales, seed0, C, bf16):
    import torch
    out = []
    for i, sc in enumerate(scales):
        wl = workloads.cube(scale=sc, seed=seed0 + i, n_channels=C)
        d = torch.from_numpy(wl.data)
        if bf16:
            d = d.to(torch.bfloat16)
        out.append((wl, d))
    return out


def _device_ref(g, wl, d, weights, channel_major):
    import torch
    w = torch.empty(wl.n_targets, device="cuda")
    o = g.grid_oneshot(wl.lon_s, wl.lat_s, d.cuda(),
                       None if weights is None else weights.cuda(), out_weights=w,
                       channel_major=channel_major)
    g.sync()
    return o.cpu().numpy(), w.cpu().numpy()


@pytest.mark.parametrize("path,bf16,channel_major,with_w", [
    ("tc", True, False, False), ("tc", True, True, True), ("fp32", False, False, True)])
def test_pipelined_calls_equal_device_calls(path, bf16, channel_major, with_w):
    import torch
    # three calls on one target grid (the grid of the first workload)
    ins = _inputs([0.004, 0.004, 0.004], 900, 64, bf16)
    base = ins[0][0]
    g = _gridder(base, path)
    hosts = []
    for k, (wl, d) in enumerate(ins):
        rng = np.random.default_rng(k)
        wts = torch.from_numpy(rng.uniform(0.5, 2.0, wl.n_samples).astype(np.float32)) \
            if with_w else None
        lon = torch.from_numpy(wl.lon_s).pin_memory()
        lat = torch.from_numpy(wl.lat_s).pin_memory()
        hd = d.pin_memory()
        hw = wts.pin_memory() if wts is not None else None
        shape = (base.n_channels, base.n_targets) if channel_major else \
            (base.n_targets, base.n_channels)
        ho = torch.full(shape, -7.0).pin_memory()
        how = torch.full((base.n_targets,), -7.0).pin_memory()
        g.grid_oneshot_host(lon, lat, hd, ho, weights=hw, out_weights=how,
                            channel_major=channel_major)
        hosts.append((wl, d, wts, ho, how))
    g.sync()
    for wl, d, wts, ho, how in hosts:
        ref_o, ref_w = _device_ref(g, wl, d, wts, channel_major)
        assert np.array_equal(ho.numpy(), ref_o, equal_nan=True)
        assert np.array_equal(how.numpy(), ref_w, equal_nan=True)
    g.close()


def test_staging_regrows_between_calls():
    import torch
    ins = _inputs([0.002, 0.006, 0.003], 950, 32, True)
    base = ins[0][0]
    g = _gridder(base, "tc")
    outs = []
    for wl, d in ins:
        ho = torch.empty((base.n_targets, base.n_channels)).pin_memory()
        g.grid_oneshot_host(torch.from_numpy(wl.lon_s).pin_memory(),
                            torch.from_numpy(wl.lat_s).pin_memory(), d.pin_memory(), ho)
        outs.append((wl, d, ho))
    g.sync()
    for wl, d, ho in outs:
        ref_o, _ = _device_ref(g, wl, d, None, False)
        assert np.array_equal(ho.numpy(), ref_o, equal_nan=True)
    g.close()


def test_host_call_against_oracle():
    import torch
    wl = workloads.cube(scale=0.002, seed=990, n_channels=16)
    d16 = torch.from_numpy(wl.data).to(torch.bfloat16)
    g = _gridder(wl, "tc")
    ho = torch.empty((wl.n_targets, wl.n_channels)).pin_memory()
    hw = torch.empty(wl.n_targets).pin_memory()
    g.grid_oneshot_host(torch.from_numpy(wl.lon_s), torch.from_numpy(wl.lat_s), d16, ho,
                        out_weights=hw)
    g.sync()
    ns = oracle.nside_for_resolution(wl.hpx_maxres)
    ref = oracle.grid_lookup(ns, wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                             d16.to(torch.float32).numpy().astype(np.float64), kernel_of(wl))
    compare_maps(ho.numpy(), hw.numpy(), ref, tol=5e-5, wtol=5e-5)
    g.close()


def test_device_tensors_refused():
    import torch
    wl = workloads.cube(scale=0.002, seed=991, n_channels=16)
    g = _gridder(wl, "tc")
    ho = torch.empty((wl.n_targets, wl.n_channels))
    with pytest.raises(ValueError):
        g.grid_oneshot_host(torch.from_numpy(wl.lon_s).cuda(), torch.from_numpy(wl.lat_s),
                            torch.from_numpy(wl.data).to(torch.bfloat16), ho)
    g.close()
