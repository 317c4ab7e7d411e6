"""The failure path of the tensor-core gridder's bounded waits, exercised
without any fault: cg_debug_hold makes the producer warps wait for a device
word that nothing sets, with a ~1 ms limit.  The wait runs out, the kernel
records the time-out, every warp role stops, the MMAs complete and the tensor
memory is freed; the next synchronising call reports CG_ETIMEOUT.  The same
handle then grids correctly (against the FP64 oracle on the same BF16 data,
paper Eq. 1-3), twice, so no resource (tensor memory, barrier phase, error
word) was left behind."""
import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, kernel_of

pytestmark = pytest.mark.gpu

ARCMIN = 1.0 / 60.0


def test_bounded_wait_runs_out_and_handle_recovers():
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    wl = workloads.random_field(495, 3000, 30, 32, 140.0, 40.0, 1.5, 2.5 * ARCMIN)
    d16 = torch.from_numpy(wl.data).to(torch.bfloat16)
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                 d16.float().numpy().astype(np.float64), kernel_of(wl))
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    g.set_path(_capi.CG_PATH_TC)
    g.debug_hold(True, 2_000_000)
    with pytest.raises(_capi.CygridError) as ei:
        g.grid_oneshot(wl.lon_s, wl.lat_s, d16)
        g.sync()
    assert ei.value.status == _capi.CG_ETIMEOUT
    g.debug_hold(False)
    for _ in range(2):
        w = torch.empty(wl.n_targets, device="cuda")
        out = g.grid_oneshot(wl.lon_s, wl.lat_s, d16, out_weights=w)
        g.sync()
        compare_maps(out.cpu().numpy(), w.cpu().numpy(), ref, tol=5e-5, wtol=5e-5)
    g.close()
