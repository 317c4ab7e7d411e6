"""Non-finite channel values reach only the targets within the sample's support
(paper Eq. 1-2: the sums run over the pairs with d <= r only).

One sample carries a NaN in some channels, another +Inf and a third -Inf in
the same channel as the second.  Against the FP64 brute-force oracle fed the
same values: every (target, channel) the oracle computes finite must match it
(1e-5 of S for the FP32 form, the BF16 bounds of the tensor-core forms on the
BF16-rounded data), every one the oracle computes non-finite must come out
non-finite of the same kind (NaN, or Inf of the same sign), and the weight
maps must agree everywhere.  Covered: the tensor-core form with hi + lo and
with single BF16 weights, the FP32 form with candidate splits (few tiles), in
one channel slab and in six (4-channel register shape), and without splits
(many tiles); each as a one-shot call and as an accumulation over two adds
(the second add carries the bad samples and must leave the first add's sums
intact elsewhere).
"""
import numpy as np
import pytest

import oracle
import workloads
from _parity import kernel_of

pytestmark = pytest.mark.gpu

ARCMIN = 1.0 / 60.0

# (form, targets per side, FP32 register shape or None for the default)
CASES = [
    ("tc", 28, None),
    ("fast", 28, None),
    ("fp32", 28, None),     # 13 tiles: candidate splits, one slab
    ("fp32", 28, 0),        # candidate splits, 4 channels per slab
    ("fp32", 280, None),    # 1,225 tiles: no splits
]


def _bad_field(C, side=28):
    wl = workloads.random_field(490 + C, 2500, side, C, 75.0, -15.0, 1.3, 2.0 * ARCMIN)
    d = wl.data.copy()
    centre = np.argmin((wl.lon_s - 75.0) ** 2 + (wl.lat_s + 15.0) ** 2)
    far = np.argmin((wl.lon_s - 75.4) ** 2 + (wl.lat_s + 15.3) ** 2)
    # ~8' away: their 6' supports overlap in part (Inf - Inf = NaN there)
    near = np.argmin((wl.lon_s - 75.535) ** 2 + (wl.lat_s + 15.3) ** 2)
    d[centre, 3] = np.nan
    d[centre, C - 1] = np.nan
    d[far, 5] = np.inf
    d[near, 5] = -np.inf
    wl.data = d
    return wl


def _check(got, got_w, ref, tol):
    got = np.asarray(got, dtype=np.float64)
    got_w = np.asarray(got_w, dtype=np.float64)
    on = ref.wsum > 0
    assert np.array_equal(on, got_w > 0)
    assert np.max(np.abs(got_w[on] - ref.wsum[on]) / ref.wsum[on]) <= max(tol, 5e-5)
    r = ref.out[on]
    g = got[on]
    bad = ~np.isfinite(r)
    assert bad.any(), "the planted values must reach some targets"
    # non-finite where the oracle is, of the same kind
    assert np.array_equal(np.isnan(g[bad]), np.isnan(r[bad]))
    inf = np.isinf(r)
    assert np.array_equal(np.sign(g[inf]), np.sign(r[inf]))
    # finite and within tolerance everywhere else
    ok = ~bad
    assert np.isfinite(g[ok]).all(), "a non-finite value leaked beyond the support"
    sabs = ref.sabs[on][ok]
    err = np.abs(g[ok] - r[ok]) / np.where(sabs > 0, sabs, 1.0)
    assert err.max() <= tol, err.max()
    return int(bad.sum()), float(err.max())


def _gridder(wl, form, shape):
    from paper_1604_06667_gb300 import Gridder, _capi
    g = Gridder(wl.lon_t, wl.lat_t, n_channels=wl.n_channels)
    g.set_kernel("gauss1d", (wl.kernel["sigma"],), wl.support, wl.hpx_maxres)
    g.set_path({"fp32": _capi.CG_PATH_FP32, "tc": _capi.CG_PATH_TC,
                "fast": _capi.CG_PATH_TC_FAST}[form])
    if shape is not None:
        g.set_f32_shape(shape)
    return g


def _data(wl, form):
    """The data the gridder gets, the data the oracle gets, the tolerance."""
    import torch
    if form == "fp32":
        return torch.from_numpy(wl.data), wl.data.astype(np.float64), 1e-5
    d16 = torch.from_numpy(wl.data).to(torch.bfloat16)
    return d16, d16.float().numpy().astype(np.float64), (5e-5 if form == "tc" else 2.0 ** -8)


@pytest.mark.parametrize("form,side,shape", CASES)
def test_nonfinite_stays_in_support(form, side, shape):
    import torch
    wl = _bad_field(24, side)
    data, dref, tol = _data(wl, form)
    g = _gridder(wl, form, shape)
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.grid_oneshot(wl.lon_s, wl.lat_s, data, out_weights=w)
    g.sync()
    got, got_w = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
    nbad, me = _check(got, got_w, ref, tol)
    print("%s/%d/%s: %d non-finite results where the oracle has them, max err %.2e"
          % (form, side, shape, nbad, me))


@pytest.mark.parametrize("form,side,shape", [c for c in CASES if c[0] != "fast"])
def test_nonfinite_accumulating_adds(form, side, shape):
    import torch
    wl = _bad_field(16, side)
    data, dref, tol = _data(wl, form)
    bad = ~np.isfinite(wl.data).all(axis=1)
    first = np.nonzero(~bad)[0][: wl.n_samples // 2]
    second = np.setdiff1d(np.arange(wl.n_samples), first)
    g = _gridder(wl, form, shape)
    for part in (first, second):
        g.grid(wl.lon_s[part], wl.lat_s[part], data[torch.from_numpy(part)])
    w = torch.empty(wl.n_targets, device="cuda")
    out = g.get_datacube(out_weights=w)
    g.sync()
    got, got_w = out.cpu().numpy(), w.cpu().numpy()
    g.close()
    ref = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, dref, kernel_of(wl))
    _check(got, got_w, ref, tol)
