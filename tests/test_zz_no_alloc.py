"""The allocation-free sample index, cg_sort_samples_noalloc.

Some callers cannot allocate device memory: programs that run on a fixed,
pre-reserved memory budget, code inside another framework's memory manager
that forbids foreign allocations, or hot paths where an allocation could block
or fail.  For them the library keeps the scratch of this one entry point in a
static device array.  This test calls it through the C ABI and checks that its
output equals, bit for bit (integer indices), what the allocating path returns
(cg_grid_add followed by cg_grid_export_index) -- on two calls in a row with
different inputs, so the second call cannot pass on the first call's leftovers.
It runs alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _noalloc(nside, lon, lat):
    import torch
    from paper_1604_06667_gb300 import _capi
    lon_d = torch.as_tensor(lon, dtype=torch.float64).cuda()
    lat_d = torch.as_tensor(lat, dtype=torch.float64).cuda()
    n = lon_d.numel()
    pix = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    perm = torch.full((n,), -7, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _capi.cg_sort_samples_noalloc(int(nside), ctypes.c_void_p(lon_d.data_ptr()),
                                  ctypes.c_void_p(lat_d.data_ptr()), n,
                                  ctypes.c_void_p(pix.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                  stream)
    torch.cuda.synchronize()
    return pix.cpu().numpy(), perm.cpu().numpy()


def _allocating(wl, nside):
    import torch
    from paper_1604_06667_gb300 import Gridder
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres, nside=nside)
    g.grid(wl.lon_s, wl.lat_s, torch.from_numpy(wl.data))
    pix, perm, _ = g.export_index(wl.n_samples)
    g.sync()
    out = pix.cpu().numpy(), perm.cpu().numpy()
    g.close()
    return out


def test_noalloc_matches_allocating_path_on_two_calls():
    from paper_1604_06667_gb300 import _capi
    first = workloads.cube(scale=0.15, n_channels=8)          # 150,000 samples
    second = workloads.plain2d(scale=0.5)                     # 10,000 samples, other field
    assert first.n_samples <= _capi.CG_NOALLOC_MAX_SAMPLES
    for wl in (first, second):
        ns = oracle.nside_for_resolution(wl.hpx_maxres)
        want_pix, want_perm = _allocating(wl, ns)
        got_pix, got_perm = _noalloc(ns, wl.lon_s, wl.lat_s)
        assert np.array_equal(got_pix, want_pix)
        assert np.array_equal(got_perm, want_perm)


def test_noalloc_rejects_sizes_above_its_limit():
    from paper_1604_06667_gb300 import _capi
    n = _capi.CG_NOALLOC_MAX_SAMPLES + 1
    with pytest.raises(_capi.CygridError) as ei:
        _capi.cg_sort_samples_noalloc(1024, ctypes.c_void_p(16), ctypes.c_void_p(16), n,
                                      ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert ei.value.status == _capi.CG_EINVAL
    assert "limit" in _capi.cg_last_error()
