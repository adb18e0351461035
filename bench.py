"""Benchmark of the fused pencil-transposition pack + ZFP fixed-rate path.

Workload (one GPU): a 1280 x 640 x 137 float32 field (T639 power-law
spectrum, unit RMS per level plus 0.01 white noise, seed 1) held in HBM,
planned over an 8 x 8 grid of simulated ranks for the z -> lambda
transposition (512 messages of 160 x 80 x 17/18 values).  One step =
for rate in (8, 16): fused pack+compress -> device-local all-to-all ->
fused decompress+unpack.  The metric is GB/s of float32 through the codec
passes: 4 passes x 449 MB per step (compress reads the field, decompress
writes it, at each rate), divided by the step time.  The comparators (plain
float32 and float16-cast pack -> all-to-all -> unpack) are timed the same
way on the same field and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl zfpx|reference]
Under torchrun every rank runs its own field (weak scaling, no data-path
collective); rank 0 prints one JSON line.
"""
import argparse
import glob
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time
from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fused pack+ZFP rate-8/16 GB/s (fp32 in) vs HBM roofline & fp16-cast pack"
SHAPE = (137, 640, 1280)                    # [lev][lat][lon]
PR = PC = 8
RATES = (8, 16)
WORKLOAD = ("1280x640x137 float32 T639 (l+1)^-1.5 field + 0.01 noise (seed 1), "
            "z->lambda over 8x8 simulated ranks (512 messages), ZFP 3-D rates 8 and 16: "
            "pack+compress, device-local all-to-all, decompress+unpack")
FALLBACK_HBM = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    from paper_2609_24294_gb300 import multirank
    return multirank.env()


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


CODEC_SOURCES = ("codec.cu", "zfpx_block.cuh", "zfpx_enc3.cuh", "zfpx_internal.h", "zfpx_smem.cuh")


def kernel_source_sha():
    """Hash of the sources that define the plan codec kernels."""
    h = hashlib.sha256()
    for name in CODEC_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2609_24294_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def recorded_pipes(kernel_key, sha):
    """ALU-pipe, issue-slot and DRAM utilisation (% of peak) from a committed ncu summary
    of the same sources: the codec kernels' limiting unit."""
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(f):
            m = re.match(r"^pipes:\s*kernel=(\S+)\s+alu_pct=([\d.]+)\s+issue_pct=([\d.]+)\s+dram_pct=([\d.]+)"
                         r"\s+source_sha=(\w+)", line.strip())
            if m and m.group(1) == kernel_key and m.group(5) == sha:
                return {"unit": "alu pipe (integer)", "alu_pct_of_peak": float(m.group(2)),
                        "issue_slots_pct": float(m.group(3)), "dram_pct_of_peak": float(m.group(4)),
                        "source": "ncu --set full, profiles/" + os.path.basename(f)}
    return None


def recorded_traffic(kernel_key, sha):
    """DRAM bytes per launch from a committed ncu summary of the same sources."""
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(f):
            m = re.match(r"^traffic:\s*kernel=(\S+)\s+bytes_per_launch=(\d+)\s+source_sha=(\w+)", line.strip())
            if m and m.group(1) == kernel_key and m.group(3) == sha:
                return int(m.group(2))
    return None


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(x, max_seconds, max_messages=None, threads=None):
    """Runs the oracle over messages of the same plan (both rates, compress and
    decompress) on `threads` host cores (default all) until max_seconds or the
    whole field is done.  Returns (f32 bytes processed, seconds, threads, messages)."""
    from oracle import codec as oc
    from oracle import plan as opl
    nz, ny, nx = x.shape
    plan = opl.Plan(nx, ny, nz, PR, PC, 0, 3)
    msgs = plan.messages[: max_messages or len(plan.messages)]
    threads = threads or os.cpu_count() or 1

    def one(m):
        box = x[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx]
        out = np.empty(box.shape, dtype=np.float32)
        for r in RATES:
            s = oc.encode_array(3, r, box)
            oc.decode_array(3, r, s, out)
        return 4 * 4 * m.nvals          # f32 bytes through 4 codec passes

    done_bytes, done = 0, 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        it = iter(msgs)
        pending = set()
        for _ in range(2 * threads):
            m = next(it, None)
            if m is not None:
                pending.add(ex.submit(one, m))
        while pending:
            finished, pending = wait(pending, return_when=FIRST_COMPLETED)
            for f in finished:                   # refill as soon as any message is done
                done_bytes += f.result()
                done += 1
                if time.perf_counter() - t0 < max_seconds:
                    m = next(it, None)
                    if m is not None:
                        pending.add(ex.submit(one, m))
    return done_bytes, time.perf_counter() - t0, threads, done


def field_errors(x, y):
    """Errors of y against x (float32 tensors on the device), in FP64: global relative L2,
    max |error|, mean |error| / |x| over x != 0, and the relative L2 error of each 4x4x4
    block (lon, lat, lev; levels past the last multiple of 4 left out; blocks of zeros
    skipped): mean and quantiles."""
    import torch
    x64 = x.double()
    d = y.double() - x64
    ax = x64.abs()
    nz = ax > 0
    res = {"rel_l2": float(d.norm() / x64.norm()), "max_abs": float(d.abs().max()),
           "mean_rel": float((d.abs()[nz] / ax[nz]).mean())}
    L = (x.shape[0] // 4) * 4

    def blocks(t):
        t = t[:L]
        Z, Y, X = t.shape
        return t.reshape(Z // 4, 4, Y // 4, 4, X // 4, 4).permute(0, 2, 4, 1, 3, 5).reshape(-1, 64)
    bx = blocks(x64).norm(dim=1)
    bd = blocks(d).norm(dim=1)
    keep = bx > 0
    eb = bd[keep] / bx[keep]
    qs = torch.quantile(eb, torch.tensor([0.5, 0.9, 0.99], dtype=torch.float64, device=eb.device))
    res["block"] = {"mean": float(eb.mean()), "p50": float(qs[0]), "p90": float(qs[1]),
                    "p99": float(qs[2]), "max": float(eb.max()), "blocks": int(keep.sum())}
    del x64, d, ax, nz, bx, bd
    return res


def reconstruction_errors(z, plan, x, decoded=None):
    """ZFP rates 8 and 16 (decoded[r] if given, else coded here) and the float16 cast,
    round to nearest and toward zero, through the same plan."""
    import torch
    out = {}
    y = torch.empty_like(x)
    for r in RATES:
        if decoded is not None:
            out["r%d" % r] = field_errors(x, decoded[r])
            continue
        sb = torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        z.zfpx_pack_compress(plan, r, x, sb)
        z.zfpx_permute(plan, r, sb, rb)
        z.zfpx_decompress_unpack(plan, r, rb, y)
        out["r%d" % r] = field_errors(x, y)
        del sb, rb
    for label, mode in (("fp16_rn", z.ROUND_NEAREST), ("fp16_rz", z.ROUND_ZERO)):
        sb = torch.zeros(plan.buffer_bytes(z.RATE_F16), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        z.zfpx_cast_fp16_pack(plan, mode, x, sb)
        z.zfpx_permute(plan, z.RATE_F16, sb, rb)
        z.zfpx_fp16_unpack(plan, rb, y)
        out[label] = field_errors(x, y)
        del sb, rb
    return out


def make_field():
    import fieldgen
    return fieldgen.t639_field()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    x = make_field()
    nbytes, secs = [], []
    for i in range(args.warmup + args.steps):
        b, s, threads, done = oracle_sample(x, args.ref_seconds)
        if i >= args.warmup:
            nbytes.append(b)
            secs.append(s)
    value = sum(nbytes) / sum(secs) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(secs) / len(secs), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": "per step: messages of the same plan for ~%.0f s (4 codec passes each)"
                                   % args.ref_seconds},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ other workloads (reported beside the headline)
def _events_ms(fn, reps, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _octahedral_fields():
    import torch
    from fieldgen import octahedral as og
    fields = []
    for i, (nlev, kind, dims, rate) in enumerate(og.O1280_TEN_FIELDS):
        src = og.octahedral_field(1280, nlev, 300 + i, kind=kind, device="cuda")
        fields.append((src, torch.empty_like(src), dims, rate))
    return og.row_lengths(1280), fields


def extra_small_latency(z):
    """The 64 x 32 x 8 T21 field (64 KiB, 256 blocks) over 2 x 2 ranks: latency of one
    pack+compress -> all-to-all -> decompress+unpack at rates 16 and 8 (median of 50)."""
    import torch
    import fieldgen
    x = torch.from_numpy(fieldgen.t21_field()).cuda()
    plan = z.Plan.for_fields(x, 2, 2, 0, 3)
    res = {"workload": "64x32x8 f32 (64 KiB) T21, 2x2 ranks"}
    st = torch.cuda.current_stream()
    for r in (16, 8):
        plan.prepare(r)
        sb = torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        y = torch.empty_like(x)

        def once():
            z.zfpx_pack_compress(plan, r, x, sb)
            z.zfpx_permute(plan, r, sb, rb)
            z.zfpx_decompress_unpack(plan, r, rb, y)
        for _ in range(5):
            once()
        ts = []
        for _ in range(50):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            once()
            b.record(st)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        res["r%d_us" % r] = 1e3 * float(np.median(ts))
    return res


def extra_batched(z, reps, peak, lens, fields):
    """Ten fields on the O1280 octahedral grid (levels 137,137,137,137,1,137,
    91,60,30,1; 1-D blocks for the single-level fields, 3-D row-quads for the
    rest; rates 8 and 16 alternating): one persistent launch encodes them all,
    one decodes them all; autotuned launch shape; against the float32 and
    float16 packs of the same fields."""
    import torch
    from paper_2609_24294_gb300 import autotune
    npts = int(lens.sum())
    specs = [(f[0].shape[0], f[2], f[3]) for f in fields]
    batch = z.Batch(lens, fields)
    out = torch.empty(batch.nbytes(), dtype=torch.uint8, device="cuda")
    choice, timings = autotune.tune_batch(batch, specs, out, use_cache=False)
    f32_bytes = sum(4 * f[0].numel() for f in fields)
    enc_ms = _events_ms(lambda: batch.encode(out), reps)
    dec_ms = _events_ms(lambda: batch.decode(out), reps)
    moved = f32_bytes + batch.nbytes()
    err = {}
    for i, (src, dst, dims, rate) in enumerate(fields):
        d = (dst.double() - src.double())
        err["field%d_r%d_d%d" % (i, rate, dims)] = float(d.norm() / src.double().norm())
    comp = {}
    plans = [z.Plan((npts, 1, f[0].shape[0]), 1, 1, 0, 3) for f in fields]
    for label, rate in (("float32", z.RATE_F32), ("float16_rn", z.RATE_F16)):
        bufs = [torch.empty(p.buffer_bytes(rate), dtype=torch.uint8, device="cuda") for p in plans]
        views = [f[0].view(f[0].shape[0], 1, npts) for f in fields]

        def pk():
            for p, v, bb in zip(plans, views, bufs):
                if rate == z.RATE_F32:
                    z.zfpx_pack(p, v, bb)
                else:
                    z.zfpx_cast_fp16_pack(p, z.ROUND_NEAREST, v, bb)
        ms = _events_ms(pk, reps)
        comp[label] = {"pack_f32_GBps": f32_bytes / (ms / 1e3) / 1e9, "ms": ms}
        del bufs
    res = {"workload": "O1280 octahedral, 10 fields, 868 levels, 5.73e9 values (22.9 GB), rates 8/16, dims 1/3",
           "launch": {"warps_per_cta": choice[0], "ctas_per_sm": choice[1], "blocks_per_lane_1d": choice[2],
                      "units_per_claim": choice[3], "tuned_ms": timings},
           "encode_ms": enc_ms, "decode_ms": dec_ms,
           "encode_f32_GBps": f32_bytes / (enc_ms / 1e3) / 1e9, "decode_f32_GBps": f32_bytes / (dec_ms / 1e3) / 1e9,
           "encode_frac_of_measured_hbm": moved / (enc_ms / 1e3) / 1e9 / peak,
           "decode_frac_of_measured_hbm": moved / (dec_ms / 1e3) / 1e9 / peak,
           "stream_bytes": batch.nbytes(), "comparators": comp, "rel_l2_error": err}
    batch.close()
    return res


def extra_serving(z, peak, lens, fields, n=2000, rate_hz=50e3, arena=40 << 30):
    """Request loop: n messages (row x level slabs of the resident O1280
    fields, sizes lognormal around 1 MiB clipped to 16 KiB..64 MiB), Poisson
    arrivals at rate_hz, rates 8 / 16, admitted into a 40 GB arena, batched
    continuously over 8 streams; p50 / p99 latency from arrival to completion
    seen by the host, sustained GB/s; beside float32 / float16 pack+unpack of
    the same slabs."""
    import torch
    from fieldgen import octahedral as og
    from paper_2609_24294_gb300 import serve
    reqs = og.serving_requests(n, [f[0].shape[0] for f in fields], [f[2] for f in fields], 5, lens)
    offs = np.concatenate([[0], np.cumsum(lens)])
    calls = []
    for r in reqs:
        f = fields[r["field"]][0]
        ptr = f.data_ptr() + 4 * (r["z0"] * f.stride(0) + int(offs[r["row0"]]))
        calls.append(dict(src=ptr, lev_stride=f.stride(0), nlev=r["nz"], dims=r["dims"], rate=r["rate"],
                          row0=r["row0"], row1=r["row1"]))
    # engine settings from a sweep on these slabs (max batch 32 .. 2048, 1 .. 8 streams, 1-D unit
    # sizes 4 .. 16): 512 requests per batch at most, 8 streams, 8 1-D blocks per lane
    srv = serve.Server(lens, arena_bytes=arena, nstreams=8, max_batch=512)
    srv.set_unit_blocks(8)
    serve.run_requests_native(srv, calls[:50])                            # warm-up
    arrivals = np.cumsum(np.random.default_rng(5).exponential(1.0 / rate_hz, n))
    lat, wall, busy_max, nbatch = serve.run_requests_native(srv, calls, arrivals=arrivals)
    total = float(sum(r["bytes"] for r in reqs))
    res = {"workload": "%d O1280 slabs, lognormal sizes (median %.2f MB, max %.1f MB), Poisson %.0f/s, rates 8/16, "
                       "40 GB arena, 8 streams, at most 512 requests per batch, request loop in the library" % (
                           n, np.median([r["bytes"] for r in reqs]) / 1e6, max(r["bytes"] for r in reqs) / 1e6,
                           rate_hz),
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "wall_ms": wall * 1e3, "f32_GBps_sustained": total / wall / 1e9,
           "offered_GBps": total * rate_hz / n / 1e9, "batches": nbatch, "requests_per_batch": n / max(nbatch, 1),
           "max_streams_busy": busy_max}
    # the same arrivals with a batching window (launch at 8 waiting requests or after 200 us)
    srv.set_batching(8, 200.0)
    lat_w, wall_w, _, nb_w = serve.run_requests_native(srv, calls, arrivals=arrivals)
    srv.set_batching(1, 0.0)
    res["window_8_or_200us"] = {"p50_ms": float(np.percentile(lat_w, 50) * 1e3),
                                "p99_ms": float(np.percentile(lat_w, 99) * 1e3),
                                "f32_GBps_sustained": total / wall_w / 1e9, "batches": nb_w,
                                "requests_per_batch": n / max(nb_w, 1)}
    # capacity: every request submitted at once, the engine batching as fast as it can
    _, wall_cap, _, nb_cap = serve.run_requests_native(srv, calls)
    res["capacity_f32_GBps"] = total / wall_cap / 1e9
    res["capacity_requests_per_batch"] = n / max(nb_cap, 1)
    # the same loop driven from Python (ctypes per submit, pump and poll), for comparison
    _, wall_py, _, _ = serve.run_requests(srv, calls)
    res["capacity_f32_GBps_python_loop"] = total / wall_py / 1e9
    srv.close()
    # comparators: the same slabs through float32 / float16 pack + unpack, back to back, replayed
    # from a CUDA graph (one launch per slab and direction would otherwise be host-bound)
    plans, views, outs = [], [], []
    for r in reqs:
        f = fields[r["field"]][0]
        span = int(offs[r["row1"]] - offs[r["row0"]])
        v = f[r["z0"]:r["z0"] + r["nz"], int(offs[r["row0"]]):int(offs[r["row0"]]) + span].unsqueeze(1)
        p = z.Plan.for_fields(v, 1, 1, 0, 3, dst=torch.empty((r["nz"], 1, span), device="cuda"))
        plans.append(p)
        views.append(v)
    for label, rate in (("float32", z.RATE_F32), ("float16_rn", z.RATE_F16)):
        bufs = [torch.empty(p.buffer_bytes(rate), dtype=torch.uint8, device="cuda") for p in plans]
        dsts = [torch.empty((v.shape[0], 1, v.shape[2]), device="cuda") for v in views]
        for p in plans:
            p.prepare(rate)

        def run():
            for p, v, bb, d in zip(plans, views, bufs, dsts):
                if rate == z.RATE_F32:
                    z.zfpx_pack(p, v, bb)
                    z.zfpx_unpack(p, bb, d)
                else:
                    z.zfpx_cast_fp16_pack(p, z.ROUND_NEAREST, v, bb)
                    z.zfpx_fp16_unpack(p, bb, d)
        cs = torch.cuda.Stream()
        graph = z.capture(run, cs)
        with torch.cuda.stream(cs):
            ms = _events_ms(lambda: graph.launch(cs), 3, warmup=1)
        res["comparator_" + label] = {"f32_GBps": total / (ms / 1e3) / 1e9, "ms_all": ms,
                                      "launches": graph.num_kernels()}
        graph.close()
        del bufs, dsts
    return res


def extra_pair(z, reps, peak):
    """2560 x 1280 x 137 float32 (T1279 power-law field), z->lambda then
    lambda->theta over 8 x 8 ranks at rate 8, with the all-to-all, as one
    CUDA graph; against the same pair with float32 and float16 messages."""
    import torch
    from fieldgen.sht_torch import sht_field_torch
    x = sht_field_torch(2560, 1280, 137, 1279, seed=2, device="cuda")
    mid = torch.empty_like(x)
    dst = torch.empty_like(x)
    p1 = z.Plan.for_fields(x, 8, 8, 0, 3, dst=mid)
    p2 = z.Plan.for_fields(mid, 8, 8, 1, 3, dst=dst)
    fbytes = 4 * x.numel()
    res = {"workload": "2560x1280x137 f32 (1.8 GB) T1279, z->lambda then lambda->theta, 8x8 ranks, CUDA graph"}
    for rate in (8, 16):
        nb = max(p1.buffer_bytes(rate), p2.buffer_bytes(rate))
        send = torch.empty(nb, dtype=torch.uint8, device="cuda")
        recv = torch.empty(nb, dtype=torch.uint8, device="cuda")
        g = z.PairGraph(p1, p2, rate, x, mid, dst, send, recv)
        ms = _events_ms(lambda: g.launch(), reps)
        rel = float((dst.double() - x.double()).norm() / x.double().norm())
        res["r%d" % rate] = {"ms_per_pair": ms, "kernels": g.num_kernels(),
                             "f32_GBps_through_codec": 4 * fbytes / (ms / 1e3) / 1e9, "rel_l2_error_after_pair": rel}
        g.close()
        del send, recv
    s = torch.cuda.Stream()
    for label, rate in (("float32", z.RATE_F32), ("float16_rn", z.RATE_F16)):
        nb = max(p1.buffer_bytes(rate), p2.buffer_bytes(rate))
        send = torch.empty(nb, dtype=torch.uint8, device="cuda")
        recv = torch.empty(nb, dtype=torch.uint8, device="cuda")
        for p in (p1, p2):
            p.prepare(rate)

        def run():
            for p, a, b in ((p1, x, mid), (p2, mid, dst)):
                if rate == z.RATE_F32:
                    z.zfpx_pack(p, a, send, stream=s)
                    z.zfpx_permute(p, rate, send, recv, stream=s)
                    z.zfpx_unpack(p, recv, b, stream=s)
                else:
                    z.zfpx_cast_fp16_pack(p, z.ROUND_NEAREST, a, send, stream=s)
                    z.zfpx_permute(p, rate, send, recv, stream=s)
                    z.zfpx_fp16_unpack(p, recv, b, stream=s)
        graph = z.capture(run, s)
        with torch.cuda.stream(s):
            ms = _events_ms(lambda: graph.launch(s), reps)
        res[label] = {"ms_per_pair": ms, "f32_GBps": 4 * fbytes / (ms / 1e3) / 1e9}
        graph.close()
        del send, recv
    del x, mid, dst
    return res


def extra_blocks_2d(z, xd, reps, peak):
    """The benchmark field and plan (1280 x 640 x 137, 8 x 8 ranks, z->lambda) coded
    with 2-D blocks (4 x 4 values of one level, the block shape for single-level
    fields) instead of 3-D blocks: per-kernel time, throughput and error."""
    import torch
    plan = z.Plan.for_fields(xd, PR, PC, 0, 2)
    fbytes = 4 * xd.numel()
    x64 = xd.double()
    res = {"workload": "1280x640x137 f32, 8x8 ranks, z->lambda, 2-D blocks (each level on its own)"}
    for r in RATES:
        plan.prepare(r)
        send = torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        out = torch.empty_like(xd)
        tc = _events_ms(lambda: z.zfpx_pack_compress(plan, r, xd, send), reps)
        td = _events_ms(lambda: z.zfpx_decompress_unpack(plan, r, send, out, layout=z.LAYOUT_SEND), reps)
        moved = fbytes + plan.buffer_bytes(r)
        res["r%d" % r] = {"compress_ms": tc, "decompress_ms": td,
                          "compress_f32_GBps": fbytes / (tc / 1e3) / 1e9,
                          "decompress_f32_GBps": fbytes / (td / 1e3) / 1e9,
                          "compress_frac_of_measured_hbm": moved / (tc / 1e3) / 1e9 / peak,
                          "decompress_frac_of_measured_hbm": moved / (td / 1e3) / 1e9 / peak,
                          "rel_l2": float((out.double() - x64).norm() / x64.norm())}
        del send, out
    plan.close()
    return res


def extra_float64(z, xd, reps, peak):
    """The benchmark field held as float64 (the precision the paper's fields come in)
    and coded with the float64 fixed-rate 3-D codec on one array: per rate the
    encode / decode times, throughput of float64 values, the fraction of the
    measured copy bandwidth (float64 array plus stream) and the error."""
    import torch
    x64 = xd.double()
    n = tuple(reversed(x64.shape))
    fbytes = 8 * x64.numel()
    res = {"workload": "1280x640x137 f64 (the f32 field widened) as one array, 3-D blocks, fixed rate"}
    out = torch.empty_like(x64)
    for r in (8, 16, 32):
        nb = z.zfpx_stream_bytes_f64(r, n)
        st = torch.empty(nb, dtype=torch.uint8, device="cuda")
        te = _events_ms(lambda: z.zfpx_encode_f64(r, x64, st), reps)
        td = _events_ms(lambda: z.zfpx_decode_f64(r, st, out), reps)
        moved = fbytes + nb
        res["r%d" % r] = {"encode_ms": te, "decode_ms": td,
                          "encode_f64_GBps": fbytes / (te / 1e3) / 1e9, "decode_f64_GBps": fbytes / (td / 1e3) / 1e9,
                          "encode_frac_of_measured_hbm": moved / (te / 1e3) / 1e9 / peak,
                          "decode_frac_of_measured_hbm": moved / (td / 1e3) / 1e9 / peak,
                          "rel_l2": float((out - x64).norm() / x64.norm()),
                          "max_abs_error": float((out - x64).abs().max())}
        del st
    del x64, out
    return res


# dense TF32 tensor peak: the measured dense BF16 peak (MEASURED_PEAKS.json) times
# the nominal TF32 / BF16 ratio of GB300 (1.1 / 2.25 PFLOP/s dense)
TF32_OVER_BF16 = 1.1 / 2.25


def tf32_peak_tflops():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["bf16_tflops"]) * TF32_OVER_BF16, "measured bf16 x 1.1/2.25"
    except Exception:
        return 1900.0 * TF32_OVER_BF16, "fallback bf16 x 1.1/2.25"


def legendre_mma_flops(nlat, T, nlev):
    """Flops the tensor cores execute for the Legendre transform: every
    128-row x nt-column tile of every (order, parity) block runs K rounded up
    to 32 in 8-deep steps, three TF32 products per step (hi x hi, hi x lo,
    lo x hi)."""
    nh = nlat // 2
    N = 2 * nlev
    ntiles = (N + 255) // 256
    nt = ((N + ntiles - 1) // ntiles + 15) // 16 * 16
    kp = (nh + 31) // 32 * 32
    tiles = 0
    for m in range(T + 1):
        for p in range(2):
            cnt = (T - m - p) // 2 + 1 if T - m - p >= 0 else 0
            tiles += (cnt + 127) // 128
    return 3 * 2.0 * 128 * nt * kp * tiles * ntiles


def extra_sht_fourier(z, xd, reps, peak):
    """The spectral transform around the compressed transpositions, on the
    benchmark field over 8 x 8 ranks: the longitude FFT of every 1280-point row
    (K = 640 wavenumbers, T639), the second transposition (lambda -> theta) on
    the real and imaginary wavenumber fields (split over m), and the Legendre
    transform to the T639 coefficients.  Times and roofline fractions of the two
    transforms; relative L2 errors of the spectra and of the coefficients with
    the first transposition compressed, the second, and both, against the same
    transforms of the uncompressed field."""
    import torch
    nz, ny, nx = xd.shape
    K = nx // 2
    T = K - 1
    re = torch.empty((nz, ny, K), device="cuda")
    im = torch.empty_like(re)
    t = _events_ms(lambda: z.zfpx_rfft_lon(xd, re, im), reps)
    moved = 4 * xd.numel() + 8 * re.numel()
    res = {"workload": "1280x640x137 f32, rows of 1280 longitudes -> 640 wavenumbers -> T639 coefficients; 8x8 ranks",
           "fft_ms": t, "fft_GBps": moved / (t / 1e3) / 1e9,
           "fft_frac_of_measured_hbm": moved / (t / 1e3) / 1e9 / peak}
    # the decode fused with the FFT against decompress+unpack then FFT, from the
    # received streams of the benchmark plan
    fplan = z.Plan.for_fields(xd, PR, PC, 0, 3)
    dec = torch.empty_like(xd)
    fre, fim = torch.empty_like(re), torch.empty_like(im)
    work = None
    for r in RATES:
        recv = torch.zeros(fplan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        z.zfpx_pack_compress(fplan, r, xd, recv, z.LAYOUT_RECV)
        work = z.zfpx_decompress_rfft(fplan, r, recv, fre, fim, work=work)

        def sep():
            z.zfpx_decompress_unpack(fplan, r, recv, dec)
            z.zfpx_rfft_lon(dec, re, im)
        t_sep = _events_ms(sep, reps)
        t_fus = _events_ms(lambda: z.zfpx_decompress_rfft(fplan, r, recv, fre, fim, work=work), reps)
        torch.cuda.synchronize()
        same = bool(torch.equal(fre.view(torch.int32), re.view(torch.int32)) and
                    torch.equal(fim.view(torch.int32), im.view(torch.int32)))
        moved = recv.numel() + 8 * re.numel()                 # streams in, wavenumbers out
        res["decode_fft_r%d" % r] = {"separate_ms": t_sep, "fused_ms": t_fus, "identical": same,
                                     "fused_GBps_f32_equiv": 4 * xd.numel() / (t_fus / 1e3) / 1e9,
                                     "fused_frac_of_measured_hbm": moved / (t_fus / 1e3) / 1e9 / peak}
        del recv
    del dec, fre, fim, work
    fplan.close()
    z.zfpx_rfft_lon(xd, re, im)                              # the spectra of the uncompressed field again
    leg = z.Legendre(ny, T)
    a_re = torch.empty((nz, leg.ncoeffs), device="cuda")
    a_im = torch.empty_like(a_re)
    tl = _events_ms(lambda: leg.forward(re, im, a_re, a_im), reps)
    nh = ny // 2
    flops = 2.0 * 2 * nz * nh * leg.ncoeffs                   # folded: nh multiply-adds per coefficient and part
    leg.status()
    tpk, tpk_kind = tf32_peak_tflops()
    mma = legendre_mma_flops(ny, T, nz)
    res.update({"legendre_ms": tl, "legendre_TFLOPs": flops / (tl / 1e3) / 1e12,
                "legendre_tensor_TFLOPs": mma / (tl / 1e3) / 1e12,
                "legendre_frac_of_tf32_peak": mma / (tl / 1e3) / 1e12 / tpk,
                "tf32_peak_TFLOPs": tpk, "tf32_peak_kind": tpk_kind,
                "legendre_note": "fold + tcgen05 kernel; TFLOPs = useful folded flops / time; tensor_TFLOPs = the "
                                 "three-term TF32 products the tensor cores execute (tiles padded to 128 rows, "
                                 "K to 32) / time"})
    exact = torch.complex(re.double(), im.double())
    enorm = float(exact.norm())
    a_exact = torch.complex(a_re.double(), a_im.double())
    anorm = float(a_exact.norm())
    b_re, b_im = torch.empty_like(a_re), torch.empty_like(a_im)

    def coeff_err(fre, fim):
        leg.forward(fre, fim, b_re, b_im)
        return float((torch.complex(b_re.double(), b_im.double()) - a_exact).norm()) / anorm

    dre, dim_ = torch.empty_like(re), torch.empty_like(im)
    plan1 = z.Plan.for_fields(xd, PR, PC, 0, 3)
    plan2 = z.Plan.for_fields(re, PR, PC, 1, 3)
    plang = z.Plan.for_fields(xd, PR, PC, 1, 3)
    x64 = xd.double()
    for r in RATES:
        out = {}
        # transposition 1 coded at rate r, then the FFT of the decoded pencil
        plan1.prepare(r)
        sb = torch.zeros(plan1.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        dec = torch.empty_like(xd)
        z.zfpx_pack_compress(plan1, r, xd, sb)
        z.zfpx_permute(plan1, r, sb, rb)
        z.zfpx_decompress_unpack(plan1, r, rb, dec)
        z.zfpx_rfft_lon(dec, dre, dim_)
        out["t1_spectrum_rel_l2"] = float((torch.complex(dre.double(), dim_.double()) - exact).norm()) / enorm
        out["t1_coeff_rel_l2"] = coeff_err(dre, dim_)
        del sb, rb, dec
        # transposition 2 on the wavenumber fields
        plan2.prepare(r)
        sb = torch.zeros(plan2.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        ore, oim = torch.empty_like(re), torch.empty_like(im)

        def t2(fre, fim):
            for f, o in ((fre, ore), (fim, oim)):
                z.zfpx_pack_compress(plan2, r, f, sb)
                z.zfpx_permute(plan2, r, sb, rb)
                z.zfpx_decompress_unpack(plan2, r, rb, o)
        out["t2_wavenumber_ms"] = _events_ms(lambda: t2(re, im), reps)
        out["t2_wavenumber_rel_l2"] = float((torch.complex(ore.double(), oim.double()) - exact).norm()) / enorm
        out["t2_coeff_rel_l2"] = coeff_err(ore, oim)
        t2(dre, dim_)                                            # both transpositions compressed
        out["t1_t2_coeff_rel_l2"] = coeff_err(ore, oim)
        del sb, rb, ore, oim
        # the same transposition on the grid-point field, for comparison
        plang.prepare(r)
        sb = torch.zeros(plang.buffer_bytes(r), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        og = torch.empty_like(xd)

        def tg():
            z.zfpx_pack_compress(plang, r, xd, sb)
            z.zfpx_permute(plang, r, sb, rb)
            z.zfpx_decompress_unpack(plang, r, rb, og)
        out["t2_grid_ms"] = _events_ms(tg, reps)
        out["t2_grid_rel_l2"] = float((og.double() - x64).norm() / x64.norm())
        del sb, rb, og
        res["r%d" % r] = out
    for p in (plan1, plan2, plang):
        p.close()
    leg.close()
    del exact, a_exact, x64, re, im, dre, dim_, a_re, a_im, b_re, b_im
    return res


def extra_accuracy(z, xd, reps, peak):
    """The accuracy mode (variable rate to an absolute tolerance, 3-D blocks) on the
    benchmark field as one array: per tolerance the bits per value, the errors
    against the float32 input, and the encode / decode times (the rate-16 codec plus
    the per-block bit counts, the scan and the bit-level pack / unpack)."""
    import torch
    n = tuple(reversed(xd.shape))
    nblk = ((n[0] + 3) // 4) * ((n[1] + 3) // 4) * ((n[2] + 3) // 4)
    lengths = torch.zeros(nblk, dtype=torch.int16, device="cuda")
    payload = torch.zeros(z.zfpx_accuracy_max_payload_bytes(n), dtype=torch.uint8, device="cuda")
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    work = torch.zeros(z.zfpx_accuracy_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(xd)
    fbytes = 4 * xd.numel()
    x64 = xd.double()
    res = {"workload": "1280x640x137 f32 (unit RMS per level) as one array, 3-D blocks, absolute tolerances"}
    for tol in (1e-2, 1e-3, 1e-4):
        te = _events_ms(lambda: z.zfpx_encode_accuracy(xd, tol, lengths, payload, total, work), reps)
        bits = int(total.item())
        used = payload[:max(8, 8 * ((bits + 63) // 64))]
        td = _events_ms(lambda: z.zfpx_decode_accuracy(lengths, used, out, work), reps)
        d = (out.double() - x64).abs()
        cut = int((lengths >= 1024).sum())
        res["tol_%g" % tol] = {"bits_per_value": bits / xd.numel(), "max_abs_error": float(d.max()),
                               "rel_l2": float((out.double() - x64).norm() / x64.norm()),
                               "blocks_cut_at_1024_bits": cut, "blocks": nblk,
                               "encode_ms": te, "decode_ms": td,
                               "encode_f32_GBps": fbytes / (te / 1e3) / 1e9, "decode_f32_GBps": fbytes / (td / 1e3) / 1e9}
    del lengths, payload, work, out
    # the same field over the 8 x 8 plan: variable-size messages and the all-to-all-v
    plan = z.Plan.for_fields(xd, PR, PC, 0, 3)
    acc = z.AccuracyTransposition(plan)
    for tol in (1e-2, 1e-3):
        tc = _events_ms(lambda: acc.compress(xd, tol), reps)
        tx = _events_ms(lambda: acc.exchange(), reps)
        res.setdefault("plan_8x8", {})
        out2 = torch.empty_like(xd)
        td = _events_ms(lambda: acc.decompress(out2), reps)
        w = acc.words.cpu().numpy()
        res["plan_8x8"]["tol_%g" % tol] = {
            "compress_ms": tc, "exchange_ms": tx, "decompress_ms": td,
            "message_bytes_min_median_max": [int(8 * w.min()), int(8 * np.median(w)), int(8 * w.max())],
            "bits_per_value": float(64 * w.sum()) / xd.numel(),
            "max_abs_error": float((out2.double() - x64).abs().max())}
        del out2
    del acc
    plan.close()
    return res


def _flushed_ms(fn, reps, flush):
    """Mean device time of fn, each repetition after an L2 flush (a write larger
    than L2), timed with events around fn alone."""
    import torch
    fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.fill_(1)
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / reps


PIECES = (1, 2, 4, 8)


def _strategy_fns(z, plan, s, r, pen, buf, out):
    if s == "float32":
        return (lambda: z.zfpx_pack(plan, pen, buf)), (lambda: z.zfpx_unpack(plan, buf, out))
    if s == "float16":
        return (lambda: z.zfpx_cast_fp16_pack(plan, z.ROUND_NEAREST, pen, buf),
                lambda: z.zfpx_fp16_unpack(plan, buf, out))
    return (lambda: z.zfpx_pack_compress(plan, r, pen, buf)), (lambda: z.zfpx_decompress_unpack(plan, r, buf, out))


def extra_network_model(z, xd, reps):
    """The row transposition of the 2560 x 1280 x 137 grid at the node counts of
    Table 1: one rank's pack-side and unpack-side kernels timed on this GPU on
    that rank's z-pencil (lon/p x lat/p x 137, cut from the benchmark field, rows
    padded to a multiple of 4 values, L2 flushed before each launch), the Table 1 message sizes from the plan, and
    the communication-time model of netmodel (Dragonfly, 200 Gb/s, 1 us per
    hop), serial as in the paper and pipelined per piece.  For the pipelined
    figure the pencil is also cut into k = 2, 4, 8 longitude pieces (starts on
    multiples of 4 values), each piece's kernels timed alone, and the measured
    pieces flow through the three-stage model."""
    import torch
    from paper_2609_24294_gb300 import netmodel as nm
    sizes = nm.message_sizes()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")     # 256 MB > L2
    per_rank, per_pieces = {}, {}
    for N in nm.TABLE1_N:
        p = nm.grid_side(N)
        nlat, nlon = 1280 // p, 2560 // p
        pitch = (nlon + 3) // 4 * 4                  # rows start on 16 bytes, as an FFT-ready pencil would
        pen = torch.empty(137, nlat, pitch, device="cuda")[:, :, :nlon]
        pen.copy_(xd[:, :nlat, :nlon])
        out = torch.empty(137, nlat, pitch, device="cuda")[:, :, :nlon]
        t, tk = {}, {}
        for s in nm.STRATEGIES:
            r = nm.RATE_OF[s]
            tk[s] = {}
            for k in PIECES:
                cuts = [min(nlon, (nlon * i // k + 3) // 4 * 4) for i in range(k)] + [nlon]
                meas = []
                for a, b in zip(cuts[:-1], cuts[1:]):
                    if b <= a:
                        continue
                    plan = z.Plan.for_fields(pen[:, :, a:b], 1, 1, 0, 3, dst=out[:, :, a:b])
                    plan.prepare(r)
                    buf = torch.empty(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
                    fp, fu = _strategy_fns(z, plan, s, r, pen[:, :, a:b], buf, out[:, :, a:b])
                    meas.append((_flushed_ms(fp, reps, flush) / 1e3, _flushed_ms(fu, reps, flush) / 1e3))
                    plan.close()
                    del buf
                tk[s][len(meas)] = meas
            t[s] = tk[s][1][0]
        per_rank[N] = t
        per_pieces[N] = tk
        del pen, out
    del flush
    res = nm.model(nm.TABLE1_N, sizes, per_rank, per_rank_pieces=per_pieces)
    table = {}
    for N in nm.TABLE1_N:
        table[N] = {s: {"MiB": round(res[N][s]["message_bytes"] / 2 ** 20, 2),
                        "pack_us": round(1e6 * res[N][s]["pack_s"], 1),
                        "comm_us": round(1e6 * res[N][s]["comm_s"], 1),
                        "unpack_us": round(1e6 * res[N][s]["unpack_s"], 1),
                        "speedup_serial": round(res[N][s]["speedup_serial"], 3),
                        "speedup_pipelined": round(res[N][s]["speedup_pipelined"], 3),
                        "pieces": res[N][s]["pieces"],
                        "piece_pack_us": {k: [round(1e6 * a, 1) for a, _ in v] for k, v in per_pieces[N][s].items()
                                          if k > 1}} for s in nm.STRATEGIES}
    return {"workload": "row transposition of 2560x1280x137 f32 at N = 4..121 (p x p ranks); per-rank "
                        "kernels timed on one rank's lon/p x lat/p x 137 pencil (row pitch a multiple of 4), L2 flushed; alpha-beta "
                        "Dragonfly model (200 Gb/s links, 1 us/hop, injection-bound, no contention); pipelined = "
                        "measured pieces (1, 2, 4, 8 longitude cuts) through a three-stage flow shop",
            "per_N": table,
            "paper_speedup_N121": nm.PAPER_SPEEDUP_N121}


def extra_pipeline(z, xd, plan, reps):
    """The benchmark plan (1280 x 640 x 137, 8 x 8 ranks) transposed by the
    per-piece pipeline on this GPU (compress, all-to-all and decompress of
    successive pieces on three streams) against the same three kernels in
    series: device time per transposition, and the pipeline's result checked
    byte for byte against the serial one."""
    import torch
    res = {}
    for rate in RATES:
        nb = plan.buffer_bytes(rate)
        send = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        out = torch.empty_like(xd)

        def serial():
            z.zfpx_pack_compress(plan, rate, xd, send)
            z.zfpx_permute(plan, rate, send, recv)
            z.zfpx_decompress_unpack(plan, rate, recv, out)
        ser = _events_ms(serial, reps, warmup=3)
        ref = (recv.clone(), out.clone())
        row = {"serial_ms": round(ser, 4)}
        for k in PIECES[1:]:
            pl = z.Pipeline(plan, rate, k)
            send.zero_()
            recv.zero_()
            out.fill_(float("nan"))
            ms = _events_ms(lambda: pl.run(xd, send, recv, out), reps, warmup=3)
            torch.cuda.synchronize()
            same = bool(torch.equal(recv, ref[0]) and torch.equal(out.view(torch.int32), ref[1].view(torch.int32)))
            row["pieces_%d" % pl.pieces] = {"ms": round(ms, 4), "vs_serial": round(ser / ms, 3), "identical": same}
            pl.close()
        res["rate_%d" % rate] = row
        del send, recv, out
    return {"workload": "1280x640x137 f32, 8x8 ranks, z->lambda: pack+compress, all-to-all, decompress+unpack; "
                        "pieces by destination peer on three streams vs serial",
            "per_rate": res}


def extra_sht_step(net, sht):
    """One forward spectral-transform step of the Table 1 grid (2560 x 1280 x 137,
    T1279) at the node counts of Table 1, from this run's measurements: the row
    transposition's per-rank kernel times and modelled exchange (extras
    network_model), the column transposition taken to cost the same, and one
    rank's FFT and Legendre shares at the rates measured on the 1280 x 640 x 137
    field (extras sht_fourier; values per second for the FFT, folded flops per
    second for the Legendre transform).  Serial, as the paper's model."""
    from paper_2609_24294_gb300 import netmodel as nm
    fft_rate = 1280 * 640 * 137 / (sht["fft_ms"] / 1e3)
    leg_rate = 2.0 * 2 * 137 * 320 * 640 * 641 / 2 / (sht["legendre_ms"] / 1e3)
    tr, fft_s, leg_s = {}, {}, {}
    for N in nm.TABLE1_N:
        row = net["per_N"][N]
        tr[N] = {s: (row[s]["pack_us"] / 1e6, row[s]["comm_us"] / 1e6, row[s]["unpack_us"] / 1e6)
                 for s in nm.STRATEGIES}
        fft_s[N] = nm.fft_values_per_rank(N) / fft_rate
        leg_s[N] = nm.legendre_flops_per_rank(N) / leg_rate
    res = nm.sht_step(nm.TABLE1_N, tr, fft_s, leg_s)
    table = {}
    for N in nm.TABLE1_N:
        table[N] = {"fft_us": round(1e6 * fft_s[N], 1), "legendre_us": round(1e6 * leg_s[N], 1)}
        for s in nm.STRATEGIES:
            table[N][s] = {"step_us": round(1e6 * res[N][s]["step_s"], 1),
                           "speedup_step": round(res[N][s]["speedup_step"], 3),
                           "speedup_transposition": round(res[N][s]["speedup_transposition"], 3)}
    return {"workload": "forward SHT step of 2560x1280x137 (T1279) at N = 4..121: row transposition, FFT, "
                        "column transposition (taken equal to the row one), Legendre; serial; compute scaled "
                        "from the rates measured on the 1280x640x137 field",
            "per_N": table}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    from paper_2609_24294_gb300 import multirank
    ws, rank, local = multirank.env()
    torch.cuda.set_device(local)
    multirank.init()
    from paper_2609_24294_gb300 import build, zfpx as z
    build.build()
    z.lib()

    x = make_field()
    nz, ny, nx = x.shape
    nvals = x.size
    field_bytes = 4 * nvals
    xd = torch.from_numpy(x).cuda()
    plan = z.Plan.for_fields(xd, PR, PC, 0, 3)
    for r in RATES + (z.RATE_F32, z.RATE_F16):
        plan.prepare(r)
    send = {r: torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda") for r in RATES}
    recv = {r: torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda") for r in RATES}
    outs = {r: torch.empty_like(xd) for r in RATES}
    stream = torch.cuda.current_stream()

    names = []
    for r in RATES:
        names += ["compress_r%d" % r, "permute_r%d" % r, "decompress_r%d" % r]

    # launch shape of the codec kernels (units per warp) picked by the autotuner on
    # this plan, before any timing; results do not depend on it
    from paper_2609_24294_gb300 import autotune
    tuned = {}
    for r in RATES:
        choice, _ = autotune.tune_codec(plan, r, xd, send[r], outs[r], use_cache=False)
        tuned["r%d" % r] = choice

    def step(ev=None):
        k = 0
        for r in RATES:
            if ev is not None:
                ev[k].record(stream)
            z.zfpx_pack_compress(plan, r, xd, send[r])
            if ev is not None:
                ev[k + 1].record(stream)
            z.zfpx_permute(plan, r, send[r], recv[r])
            if ev is not None:
                ev[k + 2].record(stream)
            z.zfpx_decompress_unpack(plan, r, recv[r], outs[r])
            k += 3
        if ev is not None:
            ev[k].record(stream)

    barrier = multirank.barrier

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = z.zfpx_launch_count()
    per_kernel = {n: 0.0 for n in names}
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(args.steps)]
    t_start.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = z.zfpx_launch_count() - launches0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    for i in range(args.steps):
        for j, n in enumerate(names):
            per_kernel[n] += evs[i][j].elapsed_time(evs[i][j + 1])
    barrier()
    total_ms = multirank.max_over_ranks(total_ms, device="cuda")
    ms_per_step = total_ms / args.steps
    pass_bytes = 2 * len(RATES) * field_bytes            # f32 bytes through the codec passes
    value = ws * pass_bytes * args.steps / (total_ms / 1e3) / 1e9

    # per-kernel figures (algorithmic bytes = f32 side + compressed stream actually written/read)
    peak, peak_kind = measured_peak()
    kern = {}
    for r in RATES:
        cbytes = plan.buffer_bytes(r)
        for n, moved in (("compress_r%d" % r, field_bytes + cbytes), ("permute_r%d" % r, 2 * cbytes),
                         ("decompress_r%d" % r, cbytes + field_bytes)):
            ms = per_kernel[n] / args.steps
            kern[n] = {"ms": ms, "algorithmic_bytes": moved, "GBps": moved / (ms / 1e3) / 1e9,
                       "f32_GBps": (field_bytes / (ms / 1e3) / 1e9) if "permute" not in n else None,
                       "frac_of_measured_hbm": moved / (ms / 1e3) / 1e9 / peak}
    dom = max((n for n in names if "permute" not in n), key=lambda n: kern[n]["ms"])
    sha = kernel_source_sha()
    kkey = {"compress_r8": "encode3_r8", "compress_r16": "encode3_r16", "decompress_r8": "decode3_r8",
            "decompress_r16": "decode3_r16"}[dom]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["GBps"], "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": kern[dom]["GBps"] / peak,
                "traffic": recorded_traffic(kkey, sha), "source_sha": sha,
                "limiter": recorded_pipes(kkey, sha)}

    # comparators on the same field: float32 and float16 (RN) pack -> all-to-all -> unpack
    comp = {}
    for label, rate in (("float32", z.RATE_F32), ("float16_rn", z.RATE_F16)):
        sb = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
        rb = torch.zeros_like(sb)
        o = torch.empty_like(xd)

        def cstep():
            if rate == z.RATE_F32:
                z.zfpx_pack(plan, xd, sb)
                z.zfpx_permute(plan, rate, sb, rb)
                z.zfpx_unpack(plan, rb, o)
            else:
                z.zfpx_cast_fp16_pack(plan, z.ROUND_NEAREST, xd, sb)
                z.zfpx_permute(plan, rate, sb, rb)
                z.zfpx_fp16_unpack(plan, rb, o)
        for _ in range(args.warmup):
            cstep()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ms = [0.0, 0.0, 0.0]
        for _ in range(args.steps):
            e[0].record(stream)
            if rate == z.RATE_F32:
                z.zfpx_pack(plan, xd, sb)
            else:
                z.zfpx_cast_fp16_pack(plan, z.ROUND_NEAREST, xd, sb)
            e[1].record(stream)
            z.zfpx_permute(plan, rate, sb, rb)
            e[2].record(stream)
            if rate == z.RATE_F32:
                z.zfpx_unpack(plan, rb, o)
            else:
                z.zfpx_fp16_unpack(plan, rb, o)
            e[3].record(stream)
            torch.cuda.synchronize()
            for j in range(3):
                ms[j] += e[j].elapsed_time(e[j + 1])
        bb = plan.buffer_bytes(rate)
        comp[label] = {"pack_f32_GBps": field_bytes / (ms[0] / args.steps / 1e3) / 1e9,
                       "unpack_f32_GBps": field_bytes / (ms[2] / args.steps / 1e3) / 1e9,
                       "pack_frac_of_measured_hbm": (field_bytes + bb) / (ms[0] / args.steps / 1e3) / 1e9 / peak,
                       "roundtrip_ms": sum(ms) / args.steps, "message_bytes_total": bb}
        del sb, rb, o

    # reconstruction error (FP64 against the float32 input, off the timed path): the timed
    # outputs, the float16 cast both ways, and the same for the temperature-like field
    err = {"unit_rms_field": reconstruction_errors(z, plan, xd, outs),
           "temperature_like": reconstruction_errors(z, plan, (250.0 + 20.0 * xd.double()).float())}

    # end to end through the public API: pinned host field in, decoded fields out.  Every step
    # copies its field in and both decoded fields out; the copies run on their own streams,
    # double-buffered, so step i+1's input and step i's outputs cross the host link while the
    # codec works.
    hx = torch.from_numpy(x).pin_memory()
    hout = {r: torch.empty(SHAPE, dtype=torch.float32).pin_memory() for r in RATES}
    xin = [torch.empty_like(xd) for _ in range(2)]
    dout = {r: [torch.empty_like(xd) for _ in range(2)] for r in RATES}
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]                 # input b is on the device
    ev_used = [torch.cuda.Event() for _ in range(2)]               # the codec has read input b
    ev_done = {r: [torch.cuda.Event() for _ in range(2)] for r in RATES}   # output (r, b) written
    ev_read = {r: [torch.cuda.Event() for _ in range(2)] for r in RATES}   # output (r, b) copied out
    for e in ev_used + [ev_read[r][k] for r in RATES for k in range(2)]:
        e.record(stream)

    def e2e_steps(n):
        for i in range(n):
            k = i % 2
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_used[k])
                xin[k].copy_(hx, non_blocking=True)
                ev_in[k].record(s_in)
            stream.wait_event(ev_in[k])
            for j, r in enumerate(RATES):
                stream.wait_event(ev_read[r][k])
                z.zfpx_pack_compress(plan, r, xin[k], send[r])
                if j == len(RATES) - 1:
                    ev_used[k].record(stream)
                z.zfpx_permute(plan, r, send[r], recv[r])
                z.zfpx_decompress_unpack(plan, r, recv[r], dout[r][k])
                ev_done[r][k].record(stream)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_done[r][k])
                    hout[r].copy_(dout[r][k], non_blocking=True)
                    ev_read[r][k].record(s_out)
        tail = torch.cuda.Event()
        tail.record(s_out)
        stream.wait_event(tail)
        tail_in = torch.cuda.Event()
        tail_in.record(s_in)
        stream.wait_event(tail_in)
    e2e_steps(args.warmup)
    torch.cuda.synchronize()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s_in.wait_stream(stream)
    s_out.wait_stream(stream)
    e2e_steps(args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = multirank.max_over_ranks(a.elapsed_time(b), device="cuda")
    e2e_value = ws * pass_bytes * args.steps / (e2e_ms / 1e3) / 1e9

    extras = {}
    if not args.no_extras:
        reps = max(3, args.steps // 2)
        try:
            extras["small_field_latency"] = extra_small_latency(z)
        except Exception as e:
            extras["small_field_latency"] = {"error": repr(e)}
        try:
            extras["transposition_pair"] = extra_pair(z, reps, peak)
        except Exception as e:              # reported, never silently dropped
            extras["transposition_pair"] = {"error": repr(e)}
        try:
            extras["network_model"] = extra_network_model(z, xd, reps)
        except Exception as e:
            extras["network_model"] = {"error": repr(e)}
        try:
            extras["pipeline"] = extra_pipeline(z, xd, plan, reps)
        except Exception as e:
            extras["pipeline"] = {"error": repr(e)}
        try:
            extras["blocks_2d"] = extra_blocks_2d(z, xd, reps, peak)
        except Exception as e:
            extras["blocks_2d"] = {"error": repr(e)}
        try:
            extras["accuracy_mode"] = extra_accuracy(z, xd, reps, peak)
        except Exception as e:
            extras["accuracy_mode"] = {"error": repr(e)}
        try:
            extras["float64"] = extra_float64(z, xd, reps, peak)
        except Exception as e:
            extras["float64"] = {"error": repr(e)}
        try:
            extras["sht_fourier"] = extra_sht_fourier(z, xd, reps, peak)
        except Exception as e:
            extras["sht_fourier"] = {"error": repr(e)}
        try:
            extras["sht_step_model"] = extra_sht_step(extras["network_model"], extras["sht_fourier"])
        except Exception as e:
            extras["sht_step_model"] = {"error": repr(e)}
        torch.cuda.empty_cache()
        try:
            lens, ofields = _octahedral_fields()
            try:
                extras["batched_ragged"] = extra_batched(z, reps, peak, lens, ofields)
            except Exception as e:
                extras["batched_ragged"] = {"error": repr(e)}
            try:
                extras["serving"] = extra_serving(z, peak, lens, ofields)
            except Exception as e:
                extras["serving"] = {"error": repr(e)}
            del ofields
        except Exception as e:
            extras["octahedral_fields"] = {"error": repr(e)}
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        b_, s_, threads, done = oracle_sample(x, args.cpu_seconds)
        b1, s1, _, done1 = oracle_sample(x, max(1.0, args.cpu_seconds / 4), threads=1)
        cpu = {"value": b_ / s_ / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": "%d of 512 messages of this plan, each through r8 and r16 compress+decompress "
                         "(%.1f s on %d threads)" % (done, s_, threads),
               "single_thread": {"value": b1 / s1 / 1e9, "unit": "GB/s",
                                 "sample": "%d messages in %.1f s on 1 thread" % (done1, s1)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (449 MB field, 0.9 GB moved per pass)",
                       "ranks": "8x8", "rates": list(RATES), "parallelism": "independent field per GPU",
                       "units_per_warp": tuned},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": field_bytes,
                    "d2h_bytes_per_step": len(RATES) * field_bytes},
            "gpu_launches": int(launches),
            "clocks": clk,
            "kernels": kern,
        }
        detail = dict(line, comparators=comp, error=err, extras=extras)
        emit(line, detail, args.detail_file)
    multirank.finalize()
    return 0


HEADLINE_MAX_BYTES = 3800


def _round_floats(o, digits=4):
    if isinstance(o, float):
        return float("%.*g" % (digits, o))
    if isinstance(o, dict):
        return {k: _round_floats(v, digits) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_round_floats(v, digits) for v in o]
    return o


def headline(line, detail_file):
    """The one-line result: the headline keys with floats kept to four significant
    digits, the per-kernel table reduced to ms / GB/s / fraction, and the name of the
    file that holds the full record (comparators, errors, extras)."""
    out = dict(line)
    if out.get("kernels"):
        out["kernels"] = {k: {"ms": v["ms"], "GBps": v["GBps"], "frac": v["frac_of_measured_hbm"]}
                          for k, v in out["kernels"].items()}
    out["detail_file"] = detail_file
    out = _round_floats(out)
    s = json.dumps(out, separators=(",", ":"))
    if len(s) > HEADLINE_MAX_BYTES:          # keep the parseable line short whatever it holds
        out.pop("kernels", None)
        if isinstance(out.get("roofline"), dict):
            out["roofline"].pop("limiter", None)
        s = json.dumps(out, separators=(",", ":"))
    return s


def emit(line, detail, detail_file):
    """Writes the full record to `detail_file` and to stderr, then prints the compact
    headline as the last line of stdout."""
    full = json.dumps(detail, indent=1, default=str)
    try:
        with open(detail_file, "w") as f:
            f.write(full + "\n")
    except OSError as e:
        log("could not write %s: %r" % (detail_file, e))
    log(full)
    print(headline(line, detail_file), flush=True)


def run_profile_case(args):
    """A workload for an ncu capture of kernels the headline step does not run, or whose
    benchmark workload is too large to capture in full.  `batch`: the ten O1280 fields
    with every level count divided by 16 (at least 1; 51 levels, 337 M values, 1.35 GB
    of float32), one batch encode and one decode launch per repetition.  `blocks12`: the
    benchmark field and plan (1280 x 640 x 137, 8 x 8 ranks) coded with 2-D and then
    1-D blocks, rates 8 and 16, pack+compress and decompress+unpack per repetition.
    `sht`: the benchmark field's longitude FFT (1280 -> 640 wavenumbers) and the T639
    Legendre transform of its wavenumber fields, one of each per repetition.
    `f64`: the benchmark field widened to float64 (898 MB) as one array, the
    float64 3-D codec at rates 8 and 16, one encode and one decode per rate and
    repetition.  Prints one line; times nothing."""
    import torch
    from paper_2609_24294_gb300 import build, zfpx as z
    build.build()
    z.lib()
    if args.profile_case == "blocks12":
        xd = torch.from_numpy(make_field()).cuda()
        n = 0
        for _ in range(max(1, args.steps)):
            for dims in (2, 1):
                plan = z.Plan.for_fields(xd, PR, PC, 0, dims)
                for r in RATES:
                    send = torch.zeros(plan.buffer_bytes(r), dtype=torch.uint8, device="cuda")
                    out = torch.empty_like(xd)
                    z.zfpx_pack_compress(plan, r, xd, send)
                    z.zfpx_decompress_unpack(plan, r, send, out, layout=z.LAYOUT_SEND)
                    n += 2
                plan.close()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "values": xd.numel(), "launches": n}))
        return 0
    if args.profile_case == "f64":
        x64 = torch.from_numpy(make_field()).cuda().double()
        n = tuple(reversed(x64.shape))
        out = torch.empty_like(x64)
        launches = 0
        for _ in range(max(1, args.steps)):
            for r in RATES:
                st = torch.empty(z.zfpx_stream_bytes_f64(r, n), dtype=torch.uint8, device="cuda")
                z.zfpx_encode_f64(r, x64, st)
                z.zfpx_decode_f64(r, st, out)
                launches += 2
                del st
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "values": x64.numel(), "launches": launches}))
        return 0
    if args.profile_case == "sht":
        xd = torch.from_numpy(make_field()).cuda()
        nz, ny, nx = xd.shape
        re = torch.empty((nz, ny, nx // 2), device="cuda")
        im = torch.empty_like(re)
        leg = z.Legendre(ny, nx // 2 - 1)
        a_re = torch.empty((nz, leg.ncoeffs), device="cuda")
        a_im = torch.empty_like(a_re)
        for _ in range(max(1, args.steps)):
            z.zfpx_rfft_lon(xd, re, im)
            leg.forward(re, im, a_re, a_im)
        torch.cuda.synchronize()
        leg.close()
        print(json.dumps({"profile_case": args.profile_case, "values": xd.numel(), "launches": 3 * max(1, args.steps)}))
        return 0
    from fieldgen import octahedral as og
    fields = []
    for i, (nlev, kind, dims, rate) in enumerate(og.O1280_TEN_FIELDS):
        lev = max(1, nlev // 16)
        src = og.octahedral_field(1280, lev, 300 + i, kind=kind, device="cuda")
        fields.append((src, torch.empty_like(src), dims if lev > 1 else 1, rate))
    lens = og.row_lengths(1280)
    batch = z.Batch(lens, fields)
    out = torch.empty(batch.nbytes(), dtype=torch.uint8, device="cuda")
    for _ in range(max(1, args.steps)):
        batch.encode(out)
        batch.decode(out)
    torch.cuda.synchronize()
    nvals = sum(f[0].numel() for f in fields)
    print(json.dumps({"profile_case": args.profile_case, "values": nvals, "stream_bytes": batch.nbytes(),
                      "launches": 2 * max(1, args.steps)}))
    batch.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zfpx", choices=["zfpx", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--detail-file", default="bench_detail.json",
                    help="where the full record (comparators, errors, extras) is written")
    ap.add_argument("--profile-case", choices=["batch", "blocks12", "sht", "f64"], default=None,
                    help="run a reduced workload for an ncu capture and exit")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
