"""Python front end in the shape of the paper's Listing 1 (Sect. 3.5):

    g = Gridder(lon_t, lat_t, n_channels)              # SlGrid: target sight lines
    g.set_kernel("gauss1d", (sigma,), support, hpx_maxres)
    g.grid(lon, lat, data)                             # accumulate (Eq. 1-2)
    cube = g.get_datacube()                            # normalise (Eq. 3)

Tensors are torch CUDA tensors (torch provides device memory and the stream);
all arithmetic runs in the CUDA library behind the C ABI.
"""
from __future__ import annotations

import ctypes

import torch

from . import _capi as C

_KERNELS = {"gauss1d": C.CG_GAUSS1D, "gauss2d": C.CG_GAUSS2D, "tsinc": C.CG_TSINC}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev_f64(x, device):
    # build non-tensor inputs directly in float64 (torch would otherwise turn
    # Python floats into float32 and round the coordinates)
    t = x if isinstance(x, torch.Tensor) else torch.as_tensor(x, dtype=torch.float64)
    return t.to(device=device, dtype=torch.float64).contiguous()


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Gridder:
    """Convolution gridder onto a fixed list of target directions (degrees)."""

    def __init__(self, lon_t, lat_t, n_channels: int = 1, device="cuda", stream=None):
        self.device = torch.device(device)
        self.lon_t = _dev_f64(lon_t, self.device)
        self.lat_t = _dev_f64(lat_t, self.device)
        self.n_targets = int(self.lon_t.numel())
        self.n_channels = int(n_channels)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            C.cg_grid_create(ctypes.byref(h), _ptr(self.lon_t), _ptr(self.lat_t), self.n_targets,
                             self.n_channels, _stream_handle(self.stream))
        self._h = h

    # -- kernel ---------------------------------------------------------
    def set_kernel(self, kernel_type: str, kernel_params, support: float,
                   hpx_maxres: float | None = None, nside: int = 0):
        params = (ctypes.c_double * 3)(*([float(p) for p in kernel_params] + [0.0] * 3)[:3])
        C.cg_set_kernel(self._h, _KERNELS[kernel_type], params, len(kernel_params),
                        float(support), int(nside), float(hpx_maxres or 0.0))
        return self

    def set_path(self, path: int):
        C.cg_set_path(self._h, int(path))
        return self

    def set_f32_shape(self, shape: int):
        C.cg_set_f32_shape(self._h, int(shape))
        return self

    # -- gridding -------------------------------------------------------
    @staticmethod
    def _data_dtype(data):
        if data.dtype == torch.float32:
            return C.CG_F32
        if data.dtype == torch.bfloat16:
            return C.CG_BF16
        raise TypeError("data must be float32 or bfloat16")

    def _prep(self, lon, lat, data, weights):
        """lon = lat = None: the samples of the previous add (its index is reused)."""
        data = torch.as_tensor(data, device=self.device)
        if data.dtype not in (torch.float32, torch.bfloat16):
            data = data.to(torch.float32)
        if lon is None and lat is None:
            data = data.reshape(-1, self.n_channels).contiguous()
            return None, None, data, weights, int(data.shape[0])
        lon = _dev_f64(lon, self.device)
        lat = _dev_f64(lat, self.device)
        data = data.reshape(lon.numel(), self.n_channels).contiguous()
        if weights is not None:
            weights = torch.as_tensor(weights, device=self.device, dtype=torch.float32).contiguous()
        self.index_gen = getattr(self, "index_gen", 0) + 1
        self.n_samples = int(lon.numel())
        return lon, lat, data, weights, int(lon.numel())

    def grid(self, lon, lat, data, weights=None):
        """Accumulate (Eq. 1-2).  lon = lat = None grids new data for the samples
        of the previous add, reusing its sample index."""
        lon, lat, data, weights, n = self._prep(lon, lat, data, weights)
        C.cg_grid_add(self._h, _ptr(lon), _ptr(lat), _ptr(data), self._data_dtype(data),
                      _ptr(weights), n)
        self._keep = (lon, lat, data, weights)   # alive until the stream has consumed them
        return self

    def get_datacube(self, channel_major: bool = False, out=None, out_weights=None):
        shape = (self.n_channels, self.n_targets) if channel_major else \
            (self.n_targets, self.n_channels)
        if out is None:
            out = torch.empty(shape, device=self.device, dtype=torch.float32)
        C.cg_grid_finalize(self._h, _ptr(out), 1 if channel_major else 0, _ptr(out_weights))
        return out

    def get_weights(self):
        w = torch.empty(self.n_targets, device=self.device, dtype=torch.float32)
        tmp = torch.empty((self.n_targets, self.n_channels), device=self.device,
                          dtype=torch.float32)
        C.cg_grid_finalize(self._h, _ptr(tmp), 0, _ptr(w))
        return w

    def grid_oneshot(self, lon, lat, data, weights=None, out=None, out_weights=None,
                     channel_major: bool = False):
        lon, lat, data, weights, n = self._prep(lon, lat, data, weights)
        shape = (self.n_channels, self.n_targets) if channel_major else \
            (self.n_targets, self.n_channels)
        if out is None:
            out = torch.empty(shape, device=self.device, dtype=torch.float32)
        C.cg_grid_oneshot(self._h, _ptr(lon), _ptr(lat), _ptr(data), self._data_dtype(data),
                          _ptr(weights), n, _ptr(out), 1 if channel_major else 0,
                          _ptr(out_weights))
        self._keep = (lon, lat, data, weights)
        return out

    def grid_oneshot_host(self, lon, lat, data, out, weights=None, out_weights=None,
                          channel_major: bool = False):
        """One-shot gridding of samples in host memory into the host array
        ``out`` (cg_grid_oneshot_host): inputs are copied in, the map is
        copied back.  CPU tensors, contiguous (page-locked ones let
        consecutive calls overlap their copies with the computation); they
        must stay alive and unmodified until ``sync()``."""
        def host(t, dtype=None):
            t = torch.as_tensor(t)
            if t.device.type != "cpu":
                raise ValueError("grid_oneshot_host takes host (CPU) tensors")
            if dtype is not None and t.dtype != dtype:
                raise ValueError("expected %s, got %s" % (dtype, t.dtype))
            if not t.is_contiguous():
                raise ValueError("host tensors must be contiguous")
            return t
        lon, lat = host(lon, torch.float64), host(lat, torch.float64)
        data = host(data)
        if data.dtype not in (torch.float32, torch.bfloat16):
            raise ValueError("data must be float32 or bfloat16")
        n = int(lon.numel())
        if lat.numel() != n or data.numel() != n * self.n_channels:
            raise ValueError("lon, lat and data disagree in the sample count")
        out = host(out, torch.float32)
        if out.numel() != self.n_targets * self.n_channels:
            raise ValueError("out must hold n_targets x n_channels floats")
        if weights is not None:
            weights = host(weights, torch.float32)
        if out_weights is not None:
            out_weights = host(out_weights, torch.float32)
        C.cg_grid_oneshot_host(self._h, _ptr(lon), _ptr(lat), _ptr(data), self._data_dtype(data),
                               _ptr(weights), n, _ptr(out), 1 if channel_major else 0,
                               _ptr(out_weights))
        self._keep_host = getattr(self, "_keep_host", [])[-3:] + [(lon, lat, data, weights, out,
                                                                    out_weights)]
        self.index_gen = getattr(self, "index_gen", 0) + 1
        self.n_samples = n
        return out

    def grid_oneshot_pcw(self, lon, lat, data, pc_weights, out=None, out_weights=None,
                         channel_major: bool = False):
        """Eq. 1-3 with one weight per sample and channel (cg_grid_oneshot_pcw):
        pc_weights [N, C] float32 >= 0.  Returns the map; out_weights (same
        shape as the map) receives W_pc."""
        lon, lat, data, _, n = self._prep(lon, lat, data, None)
        pcw = torch.as_tensor(pc_weights, device=self.device, dtype=torch.float32)
        pcw = pcw.reshape(n, self.n_channels).contiguous()
        shape = (self.n_channels, self.n_targets) if channel_major else \
            (self.n_targets, self.n_channels)
        if out is None:
            out = torch.empty(shape, device=self.device, dtype=torch.float32)
        C.cg_grid_oneshot_pcw(self._h, _ptr(lon), _ptr(lat), _ptr(data), self._data_dtype(data),
                              _ptr(pcw), n, _ptr(out), 1 if channel_major else 0,
                              _ptr(out_weights))
        self._keep = (lon, lat, data, pcw)
        return out

    def interp(self, ymap, out=None, out_weights=None):
        """Normalised interpolation of ymap [P, C] at the samples of the last
        add (cg_interp): out[n] = sum_p w_pn y_p / sum_p w_pn, NaN where no
        target is within the support; out_weights [N] receives the sums."""
        y = torch.as_tensor(ymap, device=self.device, dtype=torch.float32)
        y = y.reshape(self.n_targets, self.n_channels).contiguous()
        n = int(self.n_samples)
        if out is None:
            out = torch.empty((n, self.n_channels), device=self.device, dtype=torch.float32)
        C.cg_interp(self._h, _ptr(y), _ptr(out), _ptr(out_weights), n)
        self._keep_map = y
        return out

    # -- adjoint and kernel-width derivative ------------------------------
    def degrid(self, ymap, map_weights=None, out=None):
        """G^T y: the adjoint of the normalised gridding of the last add's
        samples (ymap [P, C] float32; map_weights = W_p of that gridding, or
        None for the accumulated weight map).  Returns [N, C] float32."""
        ymap = torch.as_tensor(ymap, device=self.device, dtype=torch.float32)
        ymap = ymap.reshape(self.n_targets, self.n_channels).contiguous()
        if map_weights is not None:
            map_weights = torch.as_tensor(map_weights, device=self.device,
                                          dtype=torch.float32).contiguous()
        n = int(getattr(self, "n_samples", 0))
        if out is None:
            out = torch.empty((n, self.n_channels), device=self.device, dtype=torch.float32)
        C.cg_degrid(self._h, _ptr(ymap), _ptr(map_weights), _ptr(out), n)
        self._keep_d = (ymap, map_weights)
        return out

    def dsigma(self, data, grad_out=None, want_dR: bool = True):
        """d R / d sigma (gauss1d, support fixed; sigma in degrees) for the last
        add's samples with channel data `data`.  Returns (dR [P, C] or None,
        sum(grad_out * dR) as a 0-d float64 device tensor or None)."""
        data = torch.as_tensor(data, device=self.device)
        if data.dtype not in (torch.float32, torch.bfloat16):
            data = data.to(torch.float32)
        data = data.reshape(-1, self.n_channels).contiguous()
        dR = torch.empty((self.n_targets, self.n_channels), device=self.device,
                         dtype=torch.float32) if want_dR else None
        ds = None
        if grad_out is not None:
            grad_out = torch.as_tensor(grad_out, device=self.device, dtype=torch.float32)
            grad_out = grad_out.reshape(self.n_targets, self.n_channels).contiguous()
            ds = torch.empty((), device=self.device, dtype=torch.float64)
        C.cg_grid_dsigma(self._h, _ptr(data), self._data_dtype(data), _ptr(grad_out), _ptr(dR),
                         _ptr(ds))
        self._keep_s = (data, grad_out)
        return dR, ds

    def debug_hold(self, enable: bool = True, wait_cycles: int = 0):
        """Testing hook (cg_debug_hold): tensor-core launches time out on
        purpose until disabled; the next sync raises CG_ETIMEOUT."""
        C.cg_debug_hold(self._h, 1 if enable else 0, int(wait_cycles))
        return self

    def reset(self):
        C.cg_grid_reset(self._h)

    def sync(self):
        C.cg_sync(self._h)

    def info(self) -> dict:
        inf = C.CgInfo()
        C.cg_get_info(self._h, ctypes.byref(inf))
        return {f: getattr(inf, f) for f, _ in C.CgInfo._fields_}

    def export_index(self, n: int):
        """(sorted RING indices, permutation, ring offsets) of the last add."""
        pix = torch.empty(n, device=self.device, dtype=torch.int64)
        perm = torch.empty(n, device=self.device, dtype=torch.int64)
        ring = torch.empty(4 * self.info()["nside"] + 1, device=self.device, dtype=torch.int64)
        C.cg_grid_export_index(self._h, _ptr(pix), _ptr(perm), _ptr(ring), int(n))
        return pix, perm, ring

    def set_timing(self, enable: bool = True):
        C.cg_set_timing(self._h, 1 if enable else 0)

    def read_timing(self) -> dict:
        """Summed ms per stage since the previous read, and the gridder launch count."""
        ms = (ctypes.c_double * C.CG_N_STAGES)()
        n = ctypes.c_int64()
        C.cg_read_timing(self._h, ms, ctypes.byref(n))
        out = {name: ms[i] for i, name in enumerate(C.STAGE_NAMES)}
        out["grid_launches"] = n.value
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            C.cg_grid_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unit_vectors(lon, lat, stream=None):
    """Unit vectors [n, 3] (float64) of directions, as the gridder evaluates them."""
    lon = _dev_f64(lon, "cuda")
    lat = _dev_f64(lat, "cuda")
    out = torch.empty((lon.numel(), 3), device=lon.device, dtype=torch.float64)
    C.cg_unit_vectors(_ptr(lon), _ptr(lat), int(lon.numel()), _ptr(out), _stream_handle(stream))
    return out


def ang2pix_ring(nside: int, lon, lat, stream=None):
    """RING HEALPix index of each direction (int64 tensor, -1 if invalid)."""
    lon = _dev_f64(lon, "cuda")
    lat = _dev_f64(lat, "cuda")
    pix = torch.empty(lon.numel(), device=lon.device, dtype=torch.int64)
    C.cg_ang2pix_ring(int(nside), _ptr(lon), _ptr(lat), int(lon.numel()), _ptr(pix),
                      _stream_handle(stream))
    return pix
