"""FP64 CPU oracle for convolution-based gridding -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code, header, table or constant generator with it.

The arithmetic lives in ``cg_oracle.c`` (plain C, binary64, no FMA
contraction); this module is argument marshalling through ctypes plus a few
plain-numpy helpers that follow the paper's definitions:

* Eq. 1-3 (Sect. 2.1): ``grid_bruteforce`` -- every sample against every target.
* Sect. 2.2 steps 1-3c and Sect. 3.3-3.4: ``grid_lookup`` -- the HEALPix
  lookup scheme (optionally with the ring-shifted disc of Eq. 4-5).
* Sect. 3.5: ``nside_for_resolution`` -- the hpx-max-resolution rule.
* Adjoint and d/dsigma of the normalised operator: ``degrid_bruteforce``,
  ``dsigma_bruteforce``; the dense operator ``operator_matrix`` and the
  gradient-descent map-making loop ``mapmaking_gd`` built on them.
* Variants: normalised interpolation map -> samples (``interp_bruteforce``)
  and one weight per sample and channel (``grid_bruteforce_pcw``).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)


class Kernel(ctypes.Structure):
    """Kernel description (degrees), mirrors ``or_kernel`` in cg_oracle.c."""
    _fields_ = [("type", ctypes.c_int32), ("sigma_deg", _dbl), ("smaj_deg", _dbl),
                ("smin_deg", _dbl), ("pa_deg", _dbl), ("support_deg", _dbl)]


def gauss1d(sigma_deg: float, support_deg: float) -> Kernel:
    return Kernel(0, sigma_deg, 0.0, 0.0, 0.0, support_deg)


def gauss2d(smaj_deg: float, smin_deg: float, pa_deg: float, support_deg: float) -> Kernel:
    return Kernel(1, 0.0, smaj_deg, smin_deg, pa_deg, support_deg)


def tapered_sinc(a_deg: float, b_deg: float, support_deg: float) -> Kernel:
    """w(d) = sin(pi d / a) / (pi d / a) * exp(-d^2 / b^2): the sin(x)/x kernel
    the paper names (App. A.1), tapered so that a finite support suffices."""
    return Kernel(2, b_deg, a_deg, 0.0, 0.0, support_deg)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_ang2pix_ring.restype = _i64
        L.or_ang2pix_ring.argtypes = [_i64, _dbl, _dbl]
        L.or_ang2pix_ring_many.restype = None
        L.or_ang2pix_ring_many.argtypes = [_i64, _i64, _pd, _pd, _pi64]
        L.or_ang2pix_margin.restype = _dbl
        L.or_ang2pix_margin.argtypes = [_i64, _dbl, _dbl]
        L.or_ring_info.restype = None
        L.or_ring_info.argtypes = [_i64, _i64, _pi64, _pi64, _pd, _pd]
        L.or_pix2ring.restype = _i64
        L.or_pix2ring.argtypes = [_i64, _i64]
        L.or_pix2ang_ring.restype = None
        L.or_pix2ang_ring.argtypes = [_i64, _i64, _pd, _pd]
        L.or_haversine.restype = _dbl
        L.or_haversine.argtypes = [_dbl] * 4
        L.or_bearing.restype = _dbl
        L.or_bearing.argtypes = [_dbl] * 4
        L.or_kernel_value.restype = _dbl
        L.or_kernel_value.argtypes = [ctypes.POINTER(Kernel)] + [_dbl] * 4
        L.or_lon_fold_deg.restype = _dbl
        L.or_lon_fold_deg.argtypes = [_dbl]
        grid_args = [_i64, _pd, _pd, _i64, _pd, _pd, _i32, _pd, _pd, ctypes.POINTER(Kernel),
                     _pd, _pd, _pd, _pd, _pi64]
        L.or_grid_bruteforce.restype = ctypes.c_int
        L.or_grid_bruteforce.argtypes = grid_args
        L.or_grid_lookup.restype = ctypes.c_int
        L.or_grid_lookup.argtypes = [_i64, _i32] + grid_args
        L.or_query_disc.restype = _i64
        L.or_query_disc.argtypes = [_i64, _dbl, _dbl, _dbl, _pi64, _i64]
        L.or_query_disc_shifted.restype = _i64
        L.or_query_disc_shifted.argtypes = [_i64, _dbl, _dbl, _dbl, _pi64, _i64]
        L.or_sort_stable.restype = None
        L.or_sort_stable.argtypes = [_i64, _pi64, _pi64]
        L.or_csr.restype = _i64
        L.or_csr.argtypes = [_i64, _pi64, _pi64, _pi64]
        L.or_ring_offsets.restype = None
        L.or_ring_offsets.argtypes = [_i64, _i64, _pi64, _pi64]
        L.or_degrid_bruteforce.restype = ctypes.c_int
        L.or_degrid_bruteforce.argtypes = [_i64, _pd, _pd, _i64, _pd, _pd, _i32, _pd,
                                           ctypes.POINTER(Kernel), _pd, _pd]
        L.or_interp_bruteforce.restype = ctypes.c_int
        L.or_interp_bruteforce.argtypes = [_i64, _pd, _pd, _i64, _pd, _pd, _i32,
                                           ctypes.POINTER(Kernel), _pd, _pd, _pd]
        L.or_dsigma_bruteforce.restype = ctypes.c_int
        L.or_dsigma_bruteforce.argtypes = [_i64, _pd, _pd, _i64, _pd, _pd, _i32, _pd, _pd,
                                           ctypes.POINTER(Kernel), _pd]
        _lib = L
    return _lib


def _d(a):
    """Contiguous float64 array and its ctypes pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_pd)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_pi64)


# --------------------------------------------------------------------------
# HEALPix (Gorski et al. 2005; paper Sect. 2.2, 3.2)
# --------------------------------------------------------------------------

def nside_for_resolution(hpx_maxres_deg: float) -> int:
    """Sect. 3.5 hpx-max-resolution: the smallest power-of-two nside whose
    pixel size sqrt(pi/3)/nside (radians) does not exceed ``hpx_maxres``."""
    target = math.radians(hpx_maxres_deg)
    ns = 1
    while math.sqrt(math.pi / 3.0) / ns > target:
        ns *= 2
    return ns


def ang2pix(nside: int, lon_deg, lat_deg) -> np.ndarray:
    lon, plon = _d(lon_deg)
    lat, plat = _d(lat_deg)
    out = np.empty(lon.shape, dtype=np.int64)
    lib().or_ang2pix_ring_many(nside, lon.size, plon, plat, out.ctypes.data_as(_pi64))
    return out


def ang2pix_margin(nside: int, lon_deg, lat_deg) -> np.ndarray:
    L = lib()
    lon = np.ascontiguousarray(lon_deg, dtype=np.float64).ravel()
    lat = np.ascontiguousarray(lat_deg, dtype=np.float64).ravel()
    return np.array([L.or_ang2pix_margin(nside, a, b) for a, b in zip(lon, lat)])


def ring_info(nside: int, ring: int):
    """(count, first pixel, z, phase) of ring ``ring`` (1..4nside-1)."""
    c, f = _i64(), _i64()
    z, ph = _dbl(), _dbl()
    lib().or_ring_info(nside, ring, ctypes.byref(c), ctypes.byref(f), ctypes.byref(z),
                       ctypes.byref(ph))
    return c.value, f.value, z.value, ph.value


def pix2ring(nside: int, pix: int) -> int:
    return lib().or_pix2ring(nside, int(pix))


def pix2ang(nside: int, pix):
    """Pixel centre: (z, phi radians) arrays."""
    pix = np.atleast_1d(np.asarray(pix, dtype=np.int64))
    z = np.empty(pix.shape)
    phi = np.empty(pix.shape)
    L = lib()
    zz, pp = _dbl(), _dbl()
    for k, p in enumerate(pix.ravel()):
        L.or_pix2ang_ring(nside, int(p), ctypes.byref(zz), ctypes.byref(pp))
        z.flat[k] = zz.value
        phi.flat[k] = pp.value
    return z, phi


def query_disc(nside: int, lon_deg: float, lat_deg: float, radius_rad: float,
               shifted: bool = False) -> np.ndarray:
    L = lib()
    fn = L.or_query_disc_shifted if shifted else L.or_query_disc
    cap = 1 << 12
    while True:
        out = np.empty(cap, dtype=np.int64)
        n = fn(nside, lon_deg, lat_deg, radius_rad, out.ctypes.data_as(_pi64), cap)
        if n <= cap:
            return np.unique(out[:n])
        cap = int(n)


def haversine(lon1, lat1, lon2, lat2) -> float:
    return lib().or_haversine(lon1, lat1, lon2, lat2)


def bearing(lon1, lat1, lon2, lat2) -> float:
    return lib().or_bearing(lon1, lat1, lon2, lat2)


def kernel_value(k: Kernel, lon_t, lat_t, lon_s, lat_s) -> float:
    return lib().or_kernel_value(ctypes.byref(k), lon_t, lat_t, lon_s, lat_s)


# --------------------------------------------------------------------------
# Sort / CSR (the sorted replacement for the paper's hash tables, Sect. 3.4)
# --------------------------------------------------------------------------

def sort_stable(keys) -> np.ndarray:
    k, pk = _i(keys)
    perm = np.empty(k.size, dtype=np.int64)
    lib().or_sort_stable(k.size, pk, perm.ctypes.data_as(_pi64))
    return perm


def csr(sorted_keys):
    k, pk = _i(sorted_keys)
    uniq = np.empty(k.size, dtype=np.int64)
    off = np.empty(k.size + 1, dtype=np.int64)
    u = lib().or_csr(k.size, pk, uniq.ctypes.data_as(_pi64), off.ctypes.data_as(_pi64))
    return uniq[:u].copy(), off[:u + 1].copy()


def ring_offsets(nside: int, sorted_keys) -> np.ndarray:
    k, pk = _i(sorted_keys)
    out = np.empty(4 * nside + 1, dtype=np.int64)
    lib().or_ring_offsets(nside, k.size, pk, out.ctypes.data_as(_pi64))
    return out


# --------------------------------------------------------------------------
# Gridding (Eq. 1-3)
# --------------------------------------------------------------------------

class GridResult:
    """num = Eq. 1 numerator, wsum = Eq. 2 weight map, out = Eq. 3 map
    (NaN where wsum == 0), sabs = sum |w D| / wsum, npairs = #pairs d <= r."""

    def __init__(self, num, wsum, out, sabs, npairs):
        self.num, self.wsum, self.out, self.sabs, self.npairs = num, wsum, out, sabs, npairs


def _grid_common(fn, pre, lon_t, lat_t, lon_s, lat_s, data, omega, k):
    lt, plt = _d(lon_t)
    bt, pbt = _d(lat_t)
    ls, pls = _d(lon_s)
    bs, pbs = _d(lat_s)
    P, N = lt.size, ls.size
    data = np.asarray(data, dtype=np.float64)
    if data.ndim == 1:
        data = data[:, None]
    C = data.shape[1]
    dd, pdd = _d(data)
    if omega is None:
        pom = None
    else:
        om, pom = _d(omega)
    num = np.empty((P, C))
    wsum = np.empty(P)
    out = np.empty((P, C))
    sabs = np.empty((P, C))
    npairs = _i64()
    rc = fn(*pre, P, plt, pbt, N, pls, pbs, C, pdd, pom, ctypes.byref(k),
            num.ctypes.data_as(_pd), wsum.ctypes.data_as(_pd), out.ctypes.data_as(_pd),
            sabs.ctypes.data_as(_pd), ctypes.byref(npairs))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return GridResult(num, wsum, out, sabs, npairs.value)


def grid_bruteforce(lon_t, lat_t, lon_s, lat_s, data, k: Kernel, omega=None) -> GridResult:
    """Eq. 1-3 by brute force: every target against every sample."""
    return _grid_common(lib().or_grid_bruteforce, (), lon_t, lat_t, lon_s, lat_s, data,
                        omega, k)


def grid_lookup(nside: int, lon_t, lat_t, lon_s, lat_s, data, k: Kernel, omega=None,
                shifted: bool = False) -> GridResult:
    """Sect. 2.2 HEALPix lookup: target index table, per-sample query-disc,
    exact cut d <= r.  ``shifted`` uses the per-ring disc of Eq. 4-5."""
    return _grid_common(lib().or_grid_lookup, (nside, 1 if shifted else 0), lon_t, lat_t,
                        lon_s, lat_s, data, omega, k)


def degrid_bruteforce(lon_t, lat_t, lon_s, lat_s, y, k: Kernel, omega=None) -> np.ndarray:
    """Adjoint of the normalised gridding operator: xhat = G^T y."""
    lt, plt = _d(lon_t)
    bt, pbt = _d(lat_t)
    ls, pls = _d(lon_s)
    bs, pbs = _d(lat_s)
    y = np.asarray(y, dtype=np.float64)
    if y.ndim == 1:
        y = y[:, None]
    C = y.shape[1]
    yy, py = _d(y)
    pom = None if omega is None else _d(omega)[1]
    om_keep = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
    if om_keep is not None:
        pom = om_keep.ctypes.data_as(_pd)
    out = np.empty((ls.size, C))
    rc = lib().or_degrid_bruteforce(lt.size, plt, pbt, ls.size, pls, pbs, C, pom,
                                    ctypes.byref(k), py, out.ctypes.data_as(_pd))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def interp_bruteforce(lon_t, lat_t, lon_s, lat_s, y, k: Kernel):
    """Normalised interpolation of the map y [P, C] at the samples:
    xhat[n] = sum_p w_pn y_p / V_n, V_n = sum_p w_pn (d_pn <= r); NaN where
    V_n = 0.  Returns (xhat [N, C], V [N])."""
    lt, plt = _d(lon_t)
    bt, pbt = _d(lat_t)
    ls, pls = _d(lon_s)
    bs, pbs = _d(lat_s)
    y = np.asarray(y, dtype=np.float64)
    if y.ndim == 1:
        y = y[:, None]
    C = y.shape[1]
    yy, py = _d(y)
    out = np.empty((ls.size, C))
    v = np.empty(ls.size)
    rc = lib().or_interp_bruteforce(lt.size, plt, pbt, ls.size, pls, pbs, C, ctypes.byref(k), py,
                                    out.ctypes.data_as(_pd), v.ctypes.data_as(_pd))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out, v


def grid_bruteforce_pcw(lon_t, lat_t, lon_s, lat_s, data, k: Kernel, omega_pc):
    """Eq. 1-3 with one weight per sample and channel (omega_pc [N, C]):
    N_pc = sum_n omega_nc w_pn D_nc, W_pc = sum_n omega_nc w_pn, R = N / W
    (NaN where W_pc = 0), channel by channel through grid_bruteforce.
    Returns (R [P, C], W [P, C], S [P, C])."""
    data = np.asarray(data, dtype=np.float64)
    om = np.asarray(omega_pc, dtype=np.float64)
    P, C = np.asarray(lon_t).size, data.shape[1]
    R, W, S = np.empty((P, C)), np.empty((P, C)), np.empty((P, C))
    for c in range(C):
        res = grid_bruteforce(lon_t, lat_t, lon_s, lat_s, data[:, c:c + 1], k, om[:, c])
        R[:, c], W[:, c], S[:, c] = res.out[:, 0], res.wsum, res.sabs[:, 0]
    return R, W, S


def dsigma_bruteforce(lon_t, lat_t, lon_s, lat_s, data, k: Kernel, omega=None) -> np.ndarray:
    """d R / d sigma (per target, channel; sigma in degrees; support fixed)."""
    lt, plt = _d(lon_t)
    bt, pbt = _d(lat_t)
    ls, pls = _d(lon_s)
    bs, pbs = _d(lat_s)
    data = np.asarray(data, dtype=np.float64)
    if data.ndim == 1:
        data = data[:, None]
    C = data.shape[1]
    dd, pdd = _d(data)
    om_keep = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
    pom = None if om_keep is None else om_keep.ctypes.data_as(_pd)
    out = np.empty((lt.size, C))
    rc = lib().or_dsigma_bruteforce(lt.size, plt, pbt, ls.size, pls, pbs, C, pdd, pom,
                                    ctypes.byref(k), out.ctypes.data_as(_pd))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


# ---------------------------------------------------------------------------
# Map making by gradient descent on the adjoint (plain numpy, FP64)
# ---------------------------------------------------------------------------
def operator_matrix(lon_t, lat_t, lon_s, lat_s, k: Kernel, omega=None) -> np.ndarray:
    """Dense normalised gridding operator G [P, N] with R = G D (Eq. 3):
    G[p, n] = omega_n w_pn / W_p, zero rows where W_p = 0.  Built by gridding
    the identity (data = the N x N unit matrix), so it is the brute-force
    gridder's own operator.  Small problems only (N channels)."""
    N = np.asarray(lon_s).size
    res = grid_bruteforce(lon_t, lat_t, lon_s, lat_s, np.eye(N), k, omega)
    return np.nan_to_num(res.out, nan=0.0)


def mapmaking_gd(G: np.ndarray, data, steps: int, alpha: float | None = None):
    """Gradient descent on L(m) = 1/2 ||G^T m - D||^2 (the map m [P, C] whose
    adjoint interpolation G^T m reproduces the samples D [N, C]).

    Step alpha = 1 / max_n sum_p G[p, n] (the largest column sum of G): with
    unit row sums (Eq. 3 normalisation) ||G G^T||_2 <= ||G||_inf ||G||_1 =
    max column sum, so the loss cannot increase.  Starts from m = 0.
    Returns (m, losses[steps + 1]) with losses[k] the loss before step k."""
    G = np.asarray(G, dtype=np.float64)
    D = np.asarray(data, dtype=np.float64)
    if D.ndim == 1:
        D = D[:, None]
    if alpha is None:
        alpha = 1.0 / G.sum(axis=0).max()
    m = np.zeros((G.shape[0], D.shape[1]))
    losses = []
    for _ in range(steps):
        r = G.T @ m - D
        losses.append(0.5 * float(np.sum(r * r)))
        m = m - alpha * (G @ r)
    r = G.T @ m - D
    losses.append(0.5 * float(np.sum(r * r)))
    return m, np.array(losses), alpha
