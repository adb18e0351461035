"""Launch-shape autotuner for the persistent kernels.

The kernels' results never depend on the launch shape; only their speed
does.  The tuner times a small set of candidate shapes on the real workload
(CUDA events on the launching stream, after a warm-up, median of a few
repetitions) and keeps the fastest.  Choices are cached in a JSON file keyed
by the workload's signature, the GPU name and its SM count, so a workload is
tuned once per machine type.

Candidates:
* batched ragged kernels: warps per CTA (2, 3, 4 or 8: the per-warp
  shared-memory tiles and the scheduling granularity) x CTAs per SM (1..as many as fit: fewer
  CTAs leave more L1 per block, more CTAs hide latency); then, for batches
  with 1-D fields, the 1-D blocks each lane codes per work unit (fewer claims
  and searches per block against balance on short batches); then the work
  units a warp claims at a time (fewer atomics against a shorter tail);
* plan codec kernels (3-D blocks): consecutive 32-block units per warp (the
  blocks-per-warp knob; each CTA of the grid codes units-per-warp x warps
  units, so it also sets the grid size), per direction and rate.
"""
import hashlib
import json
import os
import statistics

import torch

CACHE = os.environ.get("ZFPX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "zfpx", "tune.json"))

BATCH_CANDIDATES = [(3, 0), (2, 0), (4, 0), (3, 3), (8, 0)]
LB1_DEFAULT = 16
LB1_CANDIDATES = (2, 4, 8, 16, 32)
UPC_DEFAULT = 4
UPC_CANDIDATES = (1, 2, 4, 8)
UPW_CANDIDATES = (1, 2, 3, 4, 8)


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


def tune_batch(batch, specs, out, candidates=None, lb1_candidates=None, reps=3, use_cache=True):
    """Picks (warps per CTA, CTAs per SM) for batch encode + decode, then the
    1-D blocks per lane if any spec (nlev, dims, rate) has dims 1, then the
    units per claim; returns ((warps, ctas, blocks_per_lane_1d,
    units_per_claim), {candidate: ms})."""
    key = batch_signature(batch, specs) + "@" + _device_key()
    cache = _load() if use_cache else {}
    if use_cache and key in cache and len(cache[key]["choice"]) == 4:
        w, c, l1, uc = cache[key]["choice"]
        batch.set_launch(w, c)
        batch.set_unit_blocks(l1)
        batch.set_claim_units(uc)
        return (w, c, l1, uc), cache[key].get("timings", {})
    timings = {}
    both = lambda: (batch.encode(out), batch.decode(out))
    batch.set_unit_blocks(LB1_DEFAULT)
    batch.set_claim_units(UPC_DEFAULT)
    for (w, c) in (candidates or BATCH_CANDIDATES):
        batch.set_launch(w, c)
        timings["%d,%d" % (w, c)] = time_call(both, reps=reps)
    best = min(timings, key=timings.get)
    w, c = (int(v) for v in best.split(","))
    batch.set_launch(w, c)
    l1, best_ms = LB1_DEFAULT, timings[best]
    if any(s[1] == 1 for s in specs):
        for cand in (lb1_candidates or LB1_CANDIDATES):
            if cand == LB1_DEFAULT:
                continue
            batch.set_unit_blocks(cand)
            ms = time_call(both, reps=reps)
            timings["%d,%d,lb%d" % (w, c, cand)] = ms
            if ms < best_ms:
                l1, best_ms = cand, ms
        batch.set_unit_blocks(l1)
    uc = UPC_DEFAULT
    for cand in UPC_CANDIDATES:
        if cand == UPC_DEFAULT:
            continue
        batch.set_claim_units(cand)
        ms = time_call(both, reps=reps)
        timings["%d,%d,lb%d,upc%d" % (w, c, l1, cand)] = ms
        if ms < best_ms:
            uc, best_ms = cand, ms
    batch.set_claim_units(uc)
    if use_cache:
        cache[key] = {"choice": [w, c, l1, uc], "timings": timings}
        _store(cache)
    return (w, c, l1, uc), timings


def plan_signature(plan, rate):
    return "codec:%s/%s/%s/%d,%d,%d,%d/r%d" % (tuple(plan.n), tuple(plan.src_strides), tuple(plan.dst_strides),
                                              plan.pr, plan.pc, plan.transposition, plan.dims, rate)


def tune_codec(plan, rate, src, buf, dst, candidates=None, reps=3, use_cache=True):
    """Picks units per warp for the plan's pack+compress and decompress+unpack
    at `rate` (3-D blocks) and sets them; returns ({"encode": upw, "decode":
    upw}, {direction: {upw: ms}})."""
    from . import zfpx as z
    key = plan_signature(plan, rate) + "@" + _device_key()
    cache = _load() if use_cache else {}
    if use_cache and key in cache:
        ch = cache[key]["choice"]
        z.zfpx_set_units_per_warp(True, rate, ch["encode"])
        z.zfpx_set_units_per_warp(False, rate, ch["decode"])
        return ch, cache[key].get("timings", {})
    calls = {"encode": lambda: z.zfpx_pack_compress(plan, rate, src, buf),
             "decode": lambda: z.zfpx_decompress_unpack(plan, rate, buf, dst, layout=z.LAYOUT_SEND)}
    choice, timings = {}, {}
    for d, fn in calls.items():
        timings[d] = {}
        for u in (candidates or UPW_CANDIDATES):
            z.zfpx_set_units_per_warp(d == "encode", rate, u)
            timings[d][str(u)] = time_call(fn, reps=reps)
        best = min(timings[d], key=timings[d].get)
        choice[d] = int(best)
        z.zfpx_set_units_per_warp(d == "encode", rate, choice[d])
    if use_cache:
        cache[key] = {"choice": choice, "timings": timings}
        _store(cache)
    return choice, timings
