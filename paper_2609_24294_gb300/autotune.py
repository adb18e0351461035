"""Launch-shape autotuner for the persistent kernels.

The kernels' results never depend on the launch shape; only their speed
does.  The tuner times a small set of candidate shapes on the real workload
(CUDA events on the launching stream, after a warm-up, median of a few
repetitions) and keeps the fastest.  Choices are cached in a JSON file keyed
by the workload's signature, the GPU name and its SM count, so a workload is
tuned once per machine type.

Candidates: warps per CTA (4 or 8: the per-warp shared-memory tiles and the
scheduling granularity) x CTAs per SM (1..as many as fit: fewer CTAs leave
more L1 per block, more CTAs hide latency).
"""
import hashlib
import json
import os
import statistics

import torch

CACHE = os.environ.get("ZFPX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "zfpx", "tune.json"))

BATCH_CANDIDATES = [(4, 0), (4, 3), (4, 2), (8, 0), (8, 1)]


def _device_key():
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except Exception:
        pass


def batch_signature(batch, specs):
    h = hashlib.sha1()
    h.update(json.dumps([list(batch.row_len), [list(s) for s in specs]]).encode())
    return "batch:" + h.hexdigest()[:16]


def time_call(fn, reps=3, warmup=1, stream=None):
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_batch(batch, specs, out, candidates=None, reps=3, use_cache=True):
    """Picks (warps per CTA, CTAs per SM) for batch encode + decode; returns
    (choice, {choice: ms})."""
    key = batch_signature(batch, specs) + "@" + _device_key()
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        w, c = cache[key]["choice"]
        batch.set_launch(w, c)
        return (w, c), cache[key].get("timings", {})
    timings = {}
    for (w, c) in (candidates or BATCH_CANDIDATES):
        batch.set_launch(w, c)
        ms = time_call(lambda: (batch.encode(out), batch.decode(out)), reps=reps)
        timings["%d,%d" % (w, c)] = ms
    best = min(timings, key=timings.get)
    w, c = (int(v) for v in best.split(","))
    batch.set_launch(w, c)
    if use_cache:
        cache[key] = {"choice": [w, c], "timings": timings}
        _store(cache)
    return (w, c), timings
