"""Many gridding jobs as one CUDA graph (cg_batch_* of the C ABI).

    b = Batch([(gridder, lon, lat, data, out, out_weights), ...], n_streams=16)
    b.autotune(reps=2)          # per job: FP32 register-blocking shape or BF16 tensor cores
    b.set_fused(True)           # optional: one index and one gridder launch for all jobs
    b.capture()                 # one graph (per-job branches, or the fused pipeline)
    b.run()                     # one launch per replay
    b.sync()                    # wait; raises on the jobs' device errors

Each job needs its own Gridder (targets, kernel, channel count).  The tensors
must stay alive and in place while the batch is used: the graph reads and
writes them by address.
"""
from __future__ import annotations

import ctypes

import torch

from . import _capi as C
from .gridder import _dev_f64, _ptr, _stream_handle


class Batch:
    def __init__(self, jobs, n_streams: int = 16):
        self._keep = []
        descs = (C.CgJob * len(jobs))()
        for i, job in enumerate(jobs):
            g, lon, lat, data = job[:4]
            out = job[4] if len(job) > 4 else None
            out_w = job[5] if len(job) > 5 else None
            weights = job[6] if len(job) > 6 else None
            lon = _dev_f64(lon, g.device)
            lat = _dev_f64(lat, g.device)
            data = data.reshape(lon.numel(), g.n_channels).contiguous()
            if out is None:
                out = torch.empty((g.n_targets, g.n_channels), device=g.device)
            self._keep.append((g, lon, lat, data, out, out_w, weights))
            d = descs[i]
            d.grid = g._h.value
            d.lon_deg, d.lat_deg, d.data = lon.data_ptr(), lat.data_ptr(), data.data_ptr()
            d.data_dtype = g._data_dtype(data)
            d.weights = weights.data_ptr() if weights is not None else None
            d.n_samples = lon.numel()
            d.out = out.data_ptr()
            d.layout_channel_major = 0
            d.out_weights = out_w.data_ptr() if out_w is not None else None
        h = ctypes.c_void_p()
        C.cg_batch_create(ctypes.byref(h), descs, len(jobs), int(n_streams))
        self._h = h
        self.n_jobs = len(jobs)

    @property
    def outputs(self):
        return [k[4] for k in self._keep]

    def autotune(self, reps: int = 2, allow_tc: bool = True):
        C.cg_batch_autotune(self._h, int(reps), 1 if allow_tc else 0)
        return self

    def capture(self, stream=None):
        C.cg_batch_capture(self._h, _stream_handle(stream))
        return self

    def run(self, stream=None):
        C.cg_batch_run(self._h, _stream_handle(stream))

    def set_fused(self, fused: bool = True):
        C.cg_batch_set_fused(self._h, 1 if fused else 0)
        return self

    def sync(self):
        C.cg_batch_sync(self._h)

    def debug_hold(self, enable: bool = True, wait_cycles: int = 0):
        """Testing hook: the fused FP32 gridder waits for a word nothing
        sets, gives up and reports a time-out at sync()."""
        C.cg_batch_debug_hold(self._h, 1 if enable else 0, int(wait_cycles))
        return self

    def choices(self):
        out = []
        for j in range(self.n_jobs):
            p, s, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            ms = ctypes.c_double()
            C.cg_batch_get_choice(self._h, j, ctypes.byref(p), ctypes.byref(s), ctypes.byref(ms),
                                  ctypes.byref(st))
            out.append({"path": p.value, "f32_shape": s.value, "ms": ms.value,
                        "stream": st.value})
        return out

    def info(self):
        k, n = ctypes.c_int64(), ctypes.c_int32()
        C.cg_batch_info(self._h, ctypes.byref(k), ctypes.byref(n))
        return {"graph_kernels": k.value, "n_streams": n.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            C.cg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
