"""Batches of independent jobs replayed as one CUDA graph (cg_batch_*).

* every job's map and weights equal, bit for bit, a direct one-shot call on
  its handle with the path and FP32 shape the autotuner chose;
* two jobs against the FP64 oracle (FP32 form 1e-5, BF16 tensor-core form
  5e-5 of S);
* the graph reads its inputs by address: doubling a job's data in place
  doubles its map on the next replay; replays are deterministic;
* planner errors: a handle shared by two jobs, a run before the capture.
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, kernel_of

pytestmark = pytest.mark.gpu


def _build(specs):
    import torch
    from paper_1604_06667_gb300 import Gridder
    jobs, wls = [], []
    for sp in specs:
        wl = workloads.batch_job(sp)
        g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
        g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
        d = torch.from_numpy(wl.data).cuda()
        if sp["dtype"] == "bf16":
            d = d.to(torch.bfloat16)
        out = torch.empty((wl.n_targets, wl.n_channels), device="cuda")
        w = torch.empty(wl.n_targets, device="cuda")
        jobs.append((g, wl.lon_s, wl.lat_s, d, out, w))
        wls.append(wl)
    return jobs, wls


def _specs(n=8, seed=700):
    return workloads.batch_specs(n_jobs=n, seed=seed, n_range=(2e3, 2e4), sides=(32, 64, 96))


def test_batch_equals_per_job_and_oracle():
    import torch
    from paper_1604_06667_gb300 import Batch
    jobs, wls = _build(_specs())
    b = Batch(jobs, n_streams=4).autotune(reps=1).capture()
    b.run()
    torch.cuda.synchronize()
    got = [(j[4].clone(), j[5].clone()) for j in jobs]
    ch = b.choices()
    assert b.info()["graph_kernels"] > len(jobs)
    for (g, lon, lat, d, _, _), c, (o, w) in zip(jobs, ch, got):
        g.set_path(c["path"])
        g.set_f32_shape(c["f32_shape"])
        w2 = torch.empty_like(w)
        o2 = g.grid_oneshot(lon, lat, d, out_weights=w2)
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(o, nan=-9.0), torch.nan_to_num(o2, nan=-9.0))
        assert torch.equal(w, w2)
    # the oracle on the first FP32 job and the first BF16 job
    for want in ("f32", "bf16"):
        k = next(i for i, sp in enumerate(_specs()) if sp["dtype"] == want)
        wl = wls[k]
        dref = jobs[k][3].float().cpu().numpy()
        ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
        tol = 1e-5 if ch[k]["path"] == 1 else 5e-5
        compare_maps(got[k][0].cpu().numpy(), got[k][1].cpu().numpy(), ref, tol=tol, wtol=tol)
    b.close()
    for j in jobs:
        j[0].close()


def test_batch_replay_reads_inputs_in_place():
    import torch
    from paper_1604_06667_gb300 import Batch
    jobs, _ = _build(_specs(n=5, seed=701))
    b = Batch(jobs, n_streams=3).capture()
    b.run()
    torch.cuda.synchronize()
    first = [j[4].clone() for j in jobs]
    b.run()
    torch.cuda.synchronize()
    for j, f in zip(jobs, first):
        assert torch.equal(torch.nan_to_num(j[4], nan=-9.0), torch.nan_to_num(f, nan=-9.0))
    jobs[0][3].mul_(2)
    b.run()
    torch.cuda.synchronize()
    a, f = jobs[0][4], first[0]
    on = torch.isfinite(f)
    assert torch.equal(a[on], 2 * f[on])
    b.close()
    for j in jobs:
        j[0].close()


def test_batch_errors():
    import ctypes
    from paper_1604_06667_gb300 import Batch, _capi
    jobs, _ = _build(_specs(n=2, seed=702))
    with pytest.raises(_capi.CygridError) as ei:
        Batch([jobs[0], jobs[0]])
    assert ei.value.status == _capi.CG_EINVAL
    b = Batch(jobs, n_streams=2)
    with pytest.raises(_capi.CygridError) as ei:
        b.run()
    assert ei.value.status == _capi.CG_ESTATE
    b.close()
    for j in jobs:
        j[0].close()
