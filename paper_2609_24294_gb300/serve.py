"""Python side of the serving engine (zfpx_server_*): argument marshalling and
the arrival-driven request loop.

The engine itself (admission by HBM budget, batching, streams, completion)
is native; this module feeds it requests at their arrival times, pumps and
polls it, and records each request's latency from arrival to the moment the
host sees it finished.
"""
import ctypes
import time

import numpy as np
import torch

from . import zfpx as z


class Server:
    def __init__(self, row_len, arena_bytes, nstreams=4, max_batch=64):
        self.row_len = [int(v) for v in row_len]
        arr = (ctypes.c_int64 * len(self.row_len))(*self.row_len)
        h = ctypes.c_void_p()
        z._check(z.lib().zfpx_server_create(ctypes.byref(h), arr, len(self.row_len), int(arena_bytes), nstreams,
                                            max_batch), "zfpx_server_create")
        self._h = h
        self._buf = (ctypes.c_int64 * 4096)()

    def set_launch(self, warps_per_cta, ctas_per_sm=0):
        z._check(z.lib().zfpx_server_set_launch(self._h, warps_per_cta, ctas_per_sm), "zfpx_server_set_launch")

    def set_unit_blocks(self, blocks_per_lane_1d):
        z._check(z.lib().zfpx_server_set_unit_blocks(self._h, blocks_per_lane_1d), "zfpx_server_set_unit_blocks")

    def set_batching(self, min_requests=1, max_wait_us=0.0):
        """Batching window: launch once min_requests wait or the oldest has waited max_wait_us."""
        z._check(z.lib().zfpx_server_set_batching(self._h, int(min_requests), float(max_wait_us)),
                 "zfpx_server_set_batching")

    def set_claim_units(self, units_per_claim):
        z._check(z.lib().zfpx_server_set_claim_units(self._h, units_per_claim), "zfpx_server_set_claim_units")

    def submit(self, src, lev_stride, nlev, dims, rate, row0, row1):
        """src: device pointer (int) of level 0, first point of row row0."""
        f = z.Field()
        f.d_src = src
        f.d_dst = None
        f.lev_stride = lev_stride
        f.dst_lev_stride = 0
        f.nlev, f.dims, f.rate, f.row0, f.row1, f.reserved = nlev, dims, rate, row0, row1, 0
        rid = ctypes.c_int64()
        rc = z.lib().zfpx_server_submit(self._h, ctypes.byref(f), ctypes.byref(rid))
        if rc:
            raise z.ZfpxError(rc, "zfpx_server_submit")
        return rid.value

    def pump(self):
        n = ctypes.c_int()
        z._check(z.lib().zfpx_server_pump(self._h, ctypes.byref(n)), "zfpx_server_pump")
        return n.value

    def poll(self):
        n = ctypes.c_int()
        z._check(z.lib().zfpx_server_poll(self._h, self._buf, len(self._buf), ctypes.byref(n)), "zfpx_server_poll")
        return [self._buf[i] for i in range(n.value)]

    def result(self, rid):
        """(stream bytes as a uint8 numpy array, decoded values as float32 numpy) -- copies."""
        ds, sb, dv, vb = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_void_p(), ctypes.c_size_t()
        z._check(z.lib().zfpx_server_result(self._h, rid, ctypes.byref(ds), ctypes.byref(sb), ctypes.byref(dv),
                                            ctypes.byref(vb)), "zfpx_server_result")
        s = np.empty(sb.value, dtype=np.uint8)
        v = np.empty(vb.value // 4, dtype=np.float32)
        z._check(z.lib().zfpx_server_copy_result(self._h, rid, s.ctypes.data_as(ctypes.c_void_p), s.nbytes,
                                                 v.ctypes.data_as(ctypes.c_void_p), v.nbytes),
                 "zfpx_server_copy_result")
        return s, v

    def release(self, rid):
        z._check(z.lib().zfpx_server_release(self._h, rid), "zfpx_server_release")

    def stats(self):
        out = (ctypes.c_int64 * 6)()
        z._check(z.lib().zfpx_server_stats(self._h, out), "zfpx_server_stats")
        keys = ("queued", "streams_busy", "arena_used", "arena_bytes", "batches", "finished_unpolled")
        return dict(zip(keys, list(out)))

    def close(self):
        if getattr(self, "_h", None) is not None and z._lib is not None:
            z._lib.zfpx_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_requests_native(server, requests, arrivals=None):
    """The same loop as run_requests, run inside the library (zfpx_server_run):
    no Python between arrivals, results released as they finish.  Returns
    per-request latency (s; NaN for refused requests), the wall time from the
    first arrival to the last completion, the most streams busy at once and
    the number of batches."""
    n = len(requests)
    arr = (z.Field * max(n, 1))()
    for k, r in enumerate(requests):
        f = arr[k]
        f.d_src = r["src"]
        f.d_dst = None
        f.lev_stride = r["lev_stride"]
        f.dst_lev_stride = 0
        f.nlev, f.dims, f.rate, f.row0, f.row1, f.reserved = r["nlev"], r["dims"], r["rate"], r["row0"], r["row1"], 0
    a = None if arrivals is None else np.ascontiguousarray(arrivals, dtype=np.float64)
    t_done = np.empty(max(n, 1), dtype=np.float64)
    info = np.zeros(4, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    z._check(z.lib().zfpx_server_run(server._h, arr, n, None if a is None else a.ctypes.data_as(dp),
                                     t_done.ctypes.data_as(dp), info.ctypes.data_as(dp)), "zfpx_server_run")
    t_done = t_done[:n]
    base = np.zeros(n) if a is None else a
    lat = np.where(t_done >= 0, t_done - base, np.nan)
    return lat, float(info[0]), int(info[2]), int(info[1])


def run_requests(server, requests, arrivals=None, keep_results=False, max_inflight_results=None):
    """Submits request i at arrivals[i] seconds after the start (all at once
    if arrivals is None), pumping and polling until every request finished.
    requests: list of kwargs for Server.submit.  Returns per-request latency
    (s), the wall time from first arrival to last completion, the largest
    number of streams seen busy, and (optionally) every result."""
    n = len(requests)
    arrivals = np.zeros(n) if arrivals is None else np.asarray(arrivals, dtype=np.float64)
    t_done = np.full(n, np.nan)
    idx_of = {}
    results = [None] * n if keep_results else None
    i = done = 0
    busy_max = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i] <= now:
            rid = server.submit(**requests[i])
            idx_of[rid] = i
            i += 1
        server.pump()
        busy_max = max(busy_max, server.stats()["streams_busy"])
        for rid in server.poll():
            k = idx_of.pop(rid)
            t_done[k] = time.perf_counter() - t0
            if keep_results:
                results[k] = server.result(rid)
            server.release(rid)
            done += 1
    lat = t_done - arrivals
    wall = float(np.nanmax(t_done) - arrivals.min())
    return lat, wall, busy_max, results
