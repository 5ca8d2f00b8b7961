"""Python front-end of the native fit server (scatman_server_* in the C ABI).

``Server`` marshals requests into the library's scheduler, which admits them
onto its CUDA streams under the device-memory budget.  ``run_stream`` replays
a Poisson arrival sequence (submitting each request at its arrival time from
a feeder thread) and reports throughput and submit-to-result latency.
"""
from __future__ import annotations

import ctypes
import threading
import time
from typing import Dict, List, Optional

import numpy as np

from . import _lib
from .api import ScatmanError, make_config, make_shape
from .types import n_params


class Server:
    def __init__(self, budget_bytes: int, slots: int = 8, precision="tc_bf16_split", soft_width: float = 0.5):
        lib = _lib.load()
        cfg = _lib.scatman_server_config()
        cfg.hbm_budget_bytes = int(budget_bytes)
        cfg.slots = int(slots)
        cfg.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.soft_width = float(soft_width)
        out = ctypes.c_void_p()
        code = lib.scatman_server_create(ctypes.byref(cfg), ctypes.byref(out))
        if code != 0:
            raise ScatmanError(code, "scatman_server_create failed")
        self.ptr = out
        self.precision = cfg.precision
        self._live: Dict[int, tuple] = {}
        self._lock = threading.Lock()

    def submit(self, geometry, shape, target: np.ndarray, want_gradient: bool = True, want_I: bool = False):
        """Queues one fit request; returns (ticket, result dict filled on completion)."""
        lib = _lib.load()
        req = _lib.scatman_request()
        cfg, _ = make_config(geometry, self.precision)
        req.geometry = cfg
        st, alm = make_shape(shape)
        req.shape = st
        tgt = np.ascontiguousarray(target, dtype=np.float32)
        req.target = tgt.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        req.want_gradient = int(want_gradient)
        res = {"loss": np.zeros(1), "grad": np.zeros(n_params(shape)),
               "I": np.zeros(geometry.n_pix, dtype=np.float32) if want_I else None}
        req.grad_out = res["grad"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        req.loss_out = res["loss"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if want_I:
            req.I_out = res["I"].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        t = ctypes.c_longlong()
        code = lib.scatman_server_submit(self.ptr, ctypes.byref(req), ctypes.byref(t))
        if code != 0:
            raise ScatmanError(code, "scatman_server_submit")
        with self._lock:
            self._live[t.value] = (res, alm, tgt)      # outputs must outlive the request
        return t.value, res

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """Returns (status, latency_s)."""
        lib = _lib.load()
        st = ctypes.c_int()
        lat = ctypes.c_double()
        code = lib.scatman_server_wait(self.ptr, ticket, timeout_s, ctypes.byref(st), ctypes.byref(lat))
        if code != 0:
            raise ScatmanError(code, "scatman_server_wait")
        with self._lock:
            self._live.pop(ticket, None)
        return st.value, lat.value

    def cancel(self, ticket: int) -> bool:
        """Cancels a queued request: True if it will not run (its wait then
        reports ERR_CANCELLED), False if it was already admitted."""
        code = _lib.load().scatman_server_cancel(self.ptr, ticket)
        if code == _lib.SCATMAN_ERR_STATE:
            return False
        if code != 0:
            raise ScatmanError(code, "scatman_server_cancel")
        return True

    def stats(self) -> dict:
        s = _lib.scatman_server_stats()
        _lib.load().scatman_server_stats_get(self.ptr, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if self.ptr:
            _lib.load().scatman_server_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint_bytes(geometry, precision) -> int:
    cfg, _ = make_config(geometry, precision)
    return int(_lib.load().scatman_footprint_bytes(ctypes.byref(cfg)))


def run_stream(server: Server, requests: List, targets: List[np.ndarray], time_scale: float = 1.0,
               want_I: bool = False, wait_timeout_s: float = 120.0):
    """Submits request i at requests[i].arrival_s * time_scale (seconds after
    start) and waits for all; a request that has not finished `wait_timeout_s`
    after its turn to be collected raises ScatmanError (SCATMAN_ERR_TIMEOUT)
    instead of blocking forever.  Returns (results, latencies_s, status, wall_s)."""
    n = len(requests)
    tickets: List[Optional[int]] = [None] * n
    results: List[Optional[dict]] = [None] * n
    errors = []
    t0 = time.perf_counter()

    def feeder():
        try:
            for i, r in enumerate(requests):
                delay = r.arrival_s * time_scale - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets[i], results[i] = server.submit(r.geometry, r.shape, targets[i], want_I=want_I)
        except Exception as e:          # surfaced after the join
            errors.append(e)

    th = threading.Thread(target=feeder)
    th.start()
    lat = [0.0] * n
    status = [0] * n
    for i in range(n):
        while tickets[i] is None and th.is_alive():
            time.sleep(1e-4)
        if tickets[i] is None:
            break
        status[i], lat[i] = server.wait(tickets[i], timeout_s=wait_timeout_s)
    th.join()
    wall = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return results, lat, status, wall
