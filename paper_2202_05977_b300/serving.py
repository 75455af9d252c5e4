"""Python handle of the library's serving loop (wskpn_serve_*): argument
marshalling only; scheduling, batching and graph replay run in libwskpn."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _frames, _lib, default_config


class Server:
    """Continuous-batching denoise server on the current CUDA device."""

    def __init__(self, weights, precision="bf16", max_hw=(1440, 2560), n_workers=4, max_batch=4,
                 max_queue=8192, mem_budget=8 << 30, use_graphs=True, batch_window_us=200, temporal=None,
                 **cfg_kw):
        self._lib = _lib.load()
        cfg = default_config(precision, max_batch=max_batch, max_hw=max_hw, **cfg_kw)
        sc = _lib.ServeConfig()
        _lib.check(self._lib.wskpn_serve_config_default(ctypes.byref(sc)))
        sc.n_workers, sc.max_batch, sc.max_queue = n_workers, max_batch, max_queue
        sc.mem_budget, sc.use_graphs, sc.batch_window_us = mem_budget, int(use_graphs), batch_window_us
        for k, v in (temporal or {}).items():  # alpha_min, tau_pos, tau_normal, min_weight
            setattr(sc.temporal, k, float(v))
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).ravel())
        h = ctypes.c_void_p()
        _lib.check(self._lib.wskpn_serve_start(ctypes.byref(cfg), w.ctypes.data, w.size, ctypes.byref(sc),
                                               ctypes.byref(h)))
        self._h = h

    def submit(self, stream_id, radiance, albedo, normal, depth, out):
        """Queue one frame ([1, C, H, W] or [C, H, W] device tensors) -> ticket.
        Raises WskpnError(EBUSY) when refused."""
        sq = lambda t: t if t.dim() == 4 else t.unsqueeze(0)
        fr, B, H, W = _frames(sq(radiance), sq(albedo), sq(normal), sq(depth))
        if B != 1:
            raise ValueError("one frame per request")
        t = ctypes.c_uint64()
        s = self._lib.wskpn_serve_submit(self._h, int(stream_id), fr, H, W, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.byref(t))
        if s != _lib.OK:
            raise _lib.WskpnError(s, "submit refused")
        return t.value

    def submit_temporal(self, stream_id, radiance, albedo, normal, depth, position, motion, out, reset=False):
        """Queue one frame with temporal accumulation (Sec. 4.3) against the
        history the server keeps for `stream_id`; position [3,H,W] and motion
        [2,H,W] float32 device tensors -> ticket."""
        sq = lambda t: t if t.dim() == 4 else t.unsqueeze(0)
        fr, B, H, W = _frames(sq(radiance), sq(albedo), sq(normal), sq(depth))
        if B != 1:
            raise ValueError("one frame per request")
        for name, t, c in (("position", position, 3), ("motion", motion, 2)):
            if tuple(t.shape[-3:]) != (c, H, W) or not t.is_contiguous() or not t.is_cuda:
                raise ValueError(f"{name} must be a contiguous CUDA tensor [{c},{H},{W}]")
        t = ctypes.c_uint64()
        s = self._lib.wskpn_serve_submit_temporal(self._h, int(stream_id), fr, ctypes.c_void_p(position.data_ptr()),
                                                  ctypes.c_void_p(motion.data_ptr()), int(bool(reset)), H, W,
                                                  ctypes.c_void_p(out.data_ptr()), ctypes.byref(t))
        if s != _lib.OK:
            raise _lib.WskpnError(s, "submit refused")
        return t.value

    def try_submit(self, *a):
        """submit that returns the status instead of raising: (status, ticket)."""
        try:
            return _lib.OK, self.submit(*a)
        except _lib.WskpnError as e:
            return e.status, None

    def wait(self, ticket, timeout_ms=-1):
        """Status of the ticket (OK, ETIMEOUT, ...)."""
        return self._lib.wskpn_serve_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms))

    def wait_info(self, ticket, timeout_ms=-1):
        """(status, timeline dict) of the ticket: h, w, worker, batch and
        submit / dispatch / done times in ms since the server started (the
        dict is None unless delivered)."""
        info = _lib.ServeTicketInfo()
        s = self._lib.wskpn_serve_wait_info(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(info))
        if s in (_lib.ETIMEOUT, _lib.EINVAL):
            return s, None
        return s, {f: getattr(info, f) for f, _ in _lib.ServeTicketInfo._fields_}

    def pause(self, paused=True):
        _lib.check(self._lib.wskpn_serve_pause(self._h, int(paused)))

    def stats(self) -> dict:
        st = _lib.ServeStats()
        _lib.check(self._lib.wskpn_serve_stats_get(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _lib.ServeStats._fields_}

    def stop(self):
        if getattr(self, "_h", None):
            self._lib.wskpn_serve_stop(self._h)
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
