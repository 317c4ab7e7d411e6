"""Fused batches (cg_batch_set_fused): one sample index for all jobs, one
persistent FP32 gridder launch over every job's (tile, slab, split) items,
one split reduction, fix-up and normalisation; tensor-core jobs on their
segment of the shared index.

* every job against the FP64 brute-force oracle on the whole map: FP32 form
  1e-5 of S (FP32 data, and BF16 data against the oracle on the same
  BF16-rounded values), tensor-core form 5e-5 of S;
* fused results equal the per-job graph's to 1e-6 of S (the candidate
  splits, and so the FP32 summation order, may differ);
* the captured graph holds a fixed handful of kernels, not a pipeline per job;
* replays read their inputs in place and are deterministic;
* a bounded wait that runs out (testing hook) is reported as CG_ETIMEOUT and
  the batch grids correctly afterwards; invalid sample coordinates are
  reported as CG_EINVAL without disturbing the other jobs.
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import compare_maps, kernel_of

pytestmark = pytest.mark.gpu


def _specs(n, seed):
    return workloads.batch_specs(n_jobs=n, seed=seed, n_range=(2e3, 3e4), sides=(32, 64, 96))


def _build(specs, tc_jobs=(), auto=False):
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    jobs, wls = [], []
    for i, sp in enumerate(specs):
        wl = workloads.batch_job(sp)
        g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
        g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
        d = torch.from_numpy(wl.data).cuda()
        if sp["dtype"] == "bf16":
            d = d.to(torch.bfloat16)
        if not auto:
            g.set_path(_capi.CG_PATH_TC if i in tc_jobs else _capi.CG_PATH_FP32)
        out = torch.empty((wl.n_targets, wl.n_channels), device="cuda")
        w = torch.empty(wl.n_targets, device="cuda")
        jobs.append((g, wl.lon_s, wl.lat_s, d, out, w))
        wls.append(wl)
    return jobs, wls


def _close(b, jobs):
    b.close()
    for j in jobs:
        j[0].close()


def _tc_eligible(specs):
    return [i for i, sp in enumerate(specs) if sp["dtype"] == "bf16" and sp["C"] % 8 == 0]


def test_fused_batch_against_oracle():
    import torch
    from paper_1604_06667_gb300 import Batch
    specs = _specs(12, 710)
    tc = _tc_eligible(specs)[:2]
    jobs, wls = _build(specs, tc_jobs=tc)
    b = Batch(jobs).set_fused(True).capture()
    b.run()
    b.sync()
    kernels = b.info()["graph_kernels"]
    for k, (wl, job) in enumerate(zip(wls, jobs)):
        dref = job[3].float().cpu().numpy().astype(np.float64)
        ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
        tol = 5e-5 if k in tc else 1e-5
        me, mw = compare_maps(job[4].cpu().numpy(), job[5].cpu().numpy(), ref, tol=tol, wtol=tol)
        print("job %2d: n %6d C %3d side %3d %s%s: max err %.2e, W %.2e"
              % (k, wl.n_samples, wl.n_channels, wl.grid_shape[0], specs[k]["dtype"],
                 " (tensor cores)" if k in tc else "", me, mw))
    # index (keys, gather, ranges and three kernels per sort pass, at most 8
    # passes of 64-bit keys), per register shape one FP32 group (order,
    # gridder, reduce, fix-up, normalise; 6 shapes) and the tensor-core jobs'
    # own (order, gridder, fix-up): no per-job index or FP32 pipeline
    assert kernels <= 3 + 3 * 8 + 5 * 6 + 3 * len(tc), kernels
    _close(b, jobs)


def test_fused_equals_per_job_graph():
    import torch
    from paper_1604_06667_gb300 import Batch
    specs = _specs(8, 711)
    jobs, wls = _build(specs, auto=True)   # both graphs choose each job's form alike
    b = Batch(jobs, n_streams=4).capture()
    b.run()
    b.sync()
    per_job = [(j[4].clone(), j[5].clone()) for j in jobs]
    b.close()
    b = Batch(jobs).set_fused(True).capture()
    b.run()
    b.sync()
    for (g, _, _, d, o, w), (o1, w1), wl in zip(jobs, per_job, wls):
        on = w1 > 0
        assert torch.equal(on, w > 0)
        assert torch.equal(torch.isnan(o), torch.isnan(o1))
        # scale: the oracle's S is not at hand here; |R| + the data spread
        scale = torch.abs(o1[on]) + d.float().std()
        err = (torch.abs(o[on] - o1[on]) / scale).max().item()
        werr = (torch.abs(w[on] - w1[on]) / w1[on]).max().item()
        assert err <= 1e-6 and werr <= 1e-6, (err, werr)
    _close(b, jobs)


def test_fused_replays_in_place_and_deterministic():
    import torch
    from paper_1604_06667_gb300 import Batch
    jobs, _ = _build(_specs(5, 712))
    b = Batch(jobs).set_fused(True).capture()
    b.run()
    b.sync()
    first = [j[4].clone() for j in jobs]
    b.run()
    b.sync()
    for j, f in zip(jobs, first):
        assert torch.equal(torch.nan_to_num(j[4], nan=-9.0), torch.nan_to_num(f, nan=-9.0))
    jobs[0][3].mul_(2)
    b.run()
    b.sync()
    a, f = jobs[0][4], first[0]
    on = torch.isfinite(f)
    assert torch.equal(a[on], 2 * f[on])
    _close(b, jobs)


def test_fused_timeout_then_recovers():
    import torch
    from paper_1604_06667_gb300 import Batch, _capi
    specs = _specs(4, 713)
    jobs, wls = _build(specs)
    b = Batch(jobs).set_fused(True).debug_hold(True, 2_000_000).capture()
    b.run()
    with pytest.raises(_capi.CygridError) as ei:
        b.sync()
    assert ei.value.status == _capi.CG_ETIMEOUT
    b.debug_hold(False).capture()
    b.run()
    b.sync()
    for wl, job in zip(wls, jobs):
        dref = job[3].float().cpu().numpy().astype(np.float64)
        ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
        compare_maps(job[4].cpu().numpy(), job[5].cpu().numpy(), ref, tol=1e-5, wtol=1e-5)
    _close(b, jobs)


def test_fused_bad_coordinates_reported():
    import torch
    from paper_1604_06667_gb300 import Batch, _capi
    specs = _specs(3, 714)
    jobs, wls = _build(specs)
    lat_bad = wls[1].lat_s.copy()
    lat_bad[7] = np.nan
    g, lon, _, d, o, w = jobs[1]
    jobs[1] = (g, lon, lat_bad, d, o, w)
    b = Batch(jobs).set_fused(True).capture()
    b.run()
    with pytest.raises(_capi.CygridError) as ei:
        b.sync()
    assert ei.value.status == _capi.CG_EINVAL
    # the other jobs are untouched by the skipped sample
    for k in (0, 2):
        wl, job = wls[k], jobs[k]
        dref = job[3].float().cpu().numpy().astype(np.float64)
        ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
        compare_maps(job[4].cpu().numpy(), job[5].cpu().numpy(), ref, tol=1e-5, wtol=1e-5)
    _close(b, jobs)
