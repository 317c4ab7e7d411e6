"""Adjoint (degridding), d/dsigma, autograd and the map-making loop on the GPU
against the FP64 oracle (the normalised operator R = G D of Eq. 1-3,
G[p][n] = omega_n w_pn / W_p).

Bounds: degrid |x_gpu - x_oracle| <= 2e-5 * (G^T |y|) per element (FP32
weights and sums); adjoint identity <G x, y> = <x, G^T y> to 1e-5 relative;
dR/dsigma to 1e-4 of max |dR| (FP32 weights, FP64 epilogue); the 50-step
map-making losses to 1e-4 relative of the oracle's loop on the dense G.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from _parity import gpu_kernel_args, kernel_of

pytestmark = pytest.mark.gpu
ARCMIN = 1.0 / 60.0


def _gridder(wl):
    from paper_1604_06667_gb300 import Gridder
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    kt, kp = gpu_kernel_args(wl)
    g.set_kernel(kt, kp, wl.support, wl.hpx_maxres)
    return g


def _forward(g, wl, data=None):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(wl.data if data is None else data, dtype=np.float32))
    W = torch.empty(wl.n_targets, device="cuda", dtype=torch.float32)
    om = None if wl.omega is None else torch.from_numpy(np.asarray(wl.omega, dtype=np.float32))
    R = g.grid_oneshot(wl.lon_s, wl.lat_s, d, weights=om, out_weights=W)
    return R, W


def _cases():
    return [
        ("diff", workloads.diff(scale=0.01)),
        ("weights", workloads.random_field(401, 1500, 20, 5, 33.0, 47.0, 0.6, 2.0 * ARCMIN,
                                           weights=True)),
        ("elliptical", _elliptical()),
    ]


def _elliptical():
    wl = workloads.random_field(402, 1500, 20, 3, 120.0, -70.0, 0.8, 2.0 * ARCMIN)
    wl.kernel = {"type": "gauss2d", "smaj": 3.0 * ARCMIN, "smin": 1.5 * ARCMIN, "pa": 35.0}
    wl.support = 9.0 * ARCMIN
    wl.hpx_maxres = 0.75 * ARCMIN
    return wl


@pytest.mark.parametrize("name,wl", _cases(), ids=[c[0] for c in _cases()])
def test_degrid_matches_oracle(name, wl):
    import torch
    g = _gridder(wl)
    _, W = _forward(g, wl)
    rng = np.random.Generator(np.random.PCG64(410))
    y = rng.normal(0, 1, (wl.n_targets, wl.n_channels))
    got = g.degrid(torch.from_numpy(y.astype(np.float32)), map_weights=W).cpu().numpy()
    g.close()
    k = kernel_of(wl)
    y32 = y.astype(np.float32).astype(np.float64)
    ref = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, y32, k, wl.omega)
    scale = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, np.abs(y32), k,
                                     wl.omega)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-5 * scale + 1e-30), float((err / np.maximum(scale, 1e-30)).max())
    assert np.count_nonzero(scale) > 0.5 * scale.size


def test_adjoint_identity_larger():
    import torch
    wl = workloads.diff(scale=0.1)          # 20,000 samples, 81 x 81 targets
    g = _gridder(wl)
    rng = np.random.Generator(np.random.PCG64(411))
    x = rng.normal(0, 1, (wl.n_samples, wl.n_channels)).astype(np.float32)
    y = rng.normal(0, 1, (wl.n_targets, wl.n_channels)).astype(np.float32)
    Gx, W = _forward(g, wl, data=x)
    Gty = g.degrid(torch.from_numpy(y), map_weights=W)
    Gx = torch.nan_to_num(Gx, nan=0.0).double().cpu().numpy()
    Gty = Gty.double().cpu().numpy()
    g.close()
    lhs = float(np.sum(Gx * y))
    rhs = float(np.sum(x.astype(np.float64) * Gty))
    mag = float(np.sum(np.abs(Gx * y)))
    assert abs(lhs - rhs) <= 1e-5 * mag, (lhs, rhs, mag)


def test_degrid_uses_accumulated_weights_and_errors():
    import torch
    from paper_1604_06667_gb300 import _capi
    wl = workloads.diff(scale=0.01)
    g = _gridder(wl)
    y = torch.ones((wl.n_targets, wl.n_channels), device="cuda")
    with pytest.raises(_capi.CygridError) as ei:        # no add yet
        g.n_samples = wl.n_samples
        g.degrid(y)
    assert ei.value.status == _capi.CG_ESTATE
    _, W = _forward(g, wl)
    a = g.degrid(y, map_weights=W)
    b = g.degrid(y)                                     # the accumulated weight map
    assert torch.allclose(a, b, rtol=1e-6, atol=1e-7)
    g.reset()
    with pytest.raises(_capi.CygridError) as ei:        # reset: no weight map left
        g.degrid(y)
    assert ei.value.status == _capi.CG_ESTATE
    with pytest.raises(_capi.CygridError) as ei:
        _capi.cg_degrid(g._h, ctypes.c_void_p(y.data_ptr()), None,
                        ctypes.c_void_p(a.data_ptr()), wl.n_samples + 1)
    assert ei.value.status == _capi.CG_EINVAL
    g.close()


def test_reuse_index_equals_fresh_add():
    import torch
    wl = workloads.diff(scale=0.02)
    rng = np.random.Generator(np.random.PCG64(412))
    d2 = rng.normal(0, 1, (wl.n_samples, wl.n_channels)).astype(np.float32)
    g = _gridder(wl)
    _forward(g, wl)
    a = g.grid_oneshot(None, None, torch.from_numpy(d2))
    b = g.grid_oneshot(wl.lon_s, wl.lat_s, torch.from_numpy(d2))
    g.close()
    assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))


def test_dsigma_matches_oracle():
    import torch
    wl = workloads.random_field(413, 1200, 18, 4, 75.0, 10.0, 0.5, 2.0 * ARCMIN, weights=True)
    g = _gridder(wl)
    _forward(g, wl)
    rng = np.random.Generator(np.random.PCG64(414))
    gr = rng.normal(0, 1, (wl.n_targets, wl.n_channels)).astype(np.float32)
    dR, ds = g.dsigma(torch.from_numpy(np.asarray(wl.data, dtype=np.float32)),
                      grad_out=torch.from_numpy(gr))
    dR = dR.double().cpu().numpy()
    ds = float(ds)
    g.close()
    k = kernel_of(wl)
    ref = oracle.dsigma_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                   np.asarray(wl.data, dtype=np.float64), k, wl.omega)
    on = np.isfinite(ref[:, 0])
    assert np.array_equal(on, np.isfinite(dR[:, 0]))
    scale = np.abs(ref[on]).max()
    assert np.max(np.abs(dR[on] - ref[on])) <= 1e-4 * scale
    ref_s = float(np.sum(gr.astype(np.float64)[on] * ref[on]))
    mag = float(np.sum(np.abs(gr.astype(np.float64)[on] * ref[on])))
    assert abs(ds - ref_s) <= 1e-4 * mag, (ds, ref_s)


def test_autograd_gradients():
    import torch
    from paper_1604_06667_gb300 import Gridder, autograd
    wl = workloads.diff(scale=0.01)
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    sigma = torch.tensor(wl.kernel["sigma"], device="cuda", requires_grad=True)
    data = torch.from_numpy(np.asarray(wl.data, dtype=np.float32)).cuda().requires_grad_(True)
    rng = np.random.Generator(np.random.PCG64(415))
    gr = torch.from_numpy(rng.normal(0, 1, (wl.n_targets, wl.n_channels)).astype(np.float32)).cuda()
    R = autograd.grid(g, wl.lon_s, wl.lat_s, data, sigma, wl.support, wl.hpx_maxres)
    loss = torch.nansum(R * gr)
    loss.backward()
    k = kernel_of(wl)
    ref_gd = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                      gr.double().cpu().numpy(), k, None)
    got_gd = data.grad.double().cpu().numpy()
    scale = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                     np.abs(gr.double().cpu().numpy()), k, None)
    assert np.all(np.abs(got_gd - ref_gd) <= 2e-5 * scale + 1e-30)
    dref = oracle.dsigma_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s,
                                    np.asarray(wl.data, dtype=np.float64), k, None)
    on = np.isfinite(dref[:, 0])
    ref_s = float(np.sum(gr.double().cpu().numpy()[on] * dref[on]))
    mag = float(np.sum(np.abs(gr.double().cpu().numpy()[on] * dref[on])))
    assert abs(float(sigma.grad) - ref_s) <= 1e-4 * mag, (float(sigma.grad), ref_s)
    g.close()


def test_mapmaking_loop_matches_oracle():
    from paper_1604_06667_gb300 import Gridder, mapmaking
    wl = workloads.diff(scale=0.01)          # 2,000 samples, 26 x 26 targets, 16 channels
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    m, losses, alpha = mapmaking.gd(g, wl.lon_s, wl.lat_s, wl.data, steps=50)
    g.close()
    k = kernel_of(wl)
    G = oracle.operator_matrix(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, k)
    D32 = np.asarray(wl.data, dtype=np.float32).astype(np.float64)
    mref, lref, aref = oracle.mapmaking_gd(G, D32, 50)
    assert abs(alpha - aref) <= 1e-5 * aref
    assert np.all(np.diff(losses) <= 1e-6 * losses[0])
    assert np.allclose(losses, lref, rtol=1e-4, atol=0), np.max(np.abs(losses / lref - 1))
    mm = m.double().cpu().numpy()
    assert np.max(np.abs(mm - mref)) <= 1e-4 * np.max(np.abs(mref))


def test_mapmaking_steps_in_library():
    """cg_md_residual / cg_md_update: r <- r - D with 1/2 |r|^2 in FP64 (fixed
    order: repeated calls agree bit for bit), m <- m - alpha g with NaN g as 0,
    against numpy in FP64; argument errors."""
    import ctypes
    import torch
    from paper_1604_06667_gb300 import Gridder, _capi
    rng = np.random.Generator(np.random.PCG64(4242))
    g = Gridder(np.array([1.0, 2.0]), np.array([0.0, 0.5]), n_channels=1)
    n = 300_001                      # several blocks and a ragged tail
    r0 = rng.standard_normal(n).astype(np.float32)
    d = rng.standard_normal(n).astype(np.float32)
    r = torch.from_numpy(r0).cuda()
    dd = torch.from_numpy(d).cuda()
    loss = torch.zeros(2, dtype=torch.float64, device="cuda")
    _capi.cg_md_residual(g._h, r.data_ptr(), dd.data_ptr(), n, loss.data_ptr())
    g.sync()
    want = (r0 - d).astype(np.float32)          # one FP32 subtraction per value
    assert np.array_equal(r.cpu().numpy(), want)
    ref = 0.5 * np.sum(want.astype(np.float64) ** 2)
    got = float(loss[0])
    assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    # the same residual again from the same inputs: the same bits
    r2 = torch.from_numpy(r0).cuda()
    _capi.cg_md_residual(g._h, r2.data_ptr(), dd.data_ptr(), n, loss[1:].data_ptr())
    g.sync()
    assert float(loss[1]) == got
    # update with NaN gradient entries
    m0 = rng.standard_normal(n).astype(np.float32)
    gr = rng.standard_normal(n).astype(np.float32)
    gr[::97] = np.nan
    m = torch.from_numpy(m0).cuda()
    grd = torch.from_numpy(gr).cuda()
    alpha = 0.37
    _capi.cg_md_update(g._h, m.data_ptr(), grd.data_ptr(), alpha, n)
    g.sync()
    g0 = np.where(np.isnan(gr), 0.0, gr).astype(np.float64)
    mref = m0.astype(np.float64) - np.float64(np.float32(alpha)) * g0
    assert np.max(np.abs(m.cpu().numpy() - mref)) <= 1e-6 * (1 + np.max(np.abs(mref)))
    assert np.array_equal(m.cpu().numpy()[::97], m0[::97])
    # errors
    with pytest.raises(_capi.CygridError) as ei:
        _capi.cg_md_update(g._h, m.data_ptr(), grd.data_ptr(), float("nan"), n)
    assert ei.value.status == _capi.CG_EINVAL
    with pytest.raises(_capi.CygridError) as ei:
        _capi.cg_md_residual(g._h, None, dd.data_ptr(), n, loss.data_ptr())
    assert ei.value.status == _capi.CG_EINVAL
    g.close()
