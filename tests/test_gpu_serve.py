"""The serving engine: admission by the arena (HBM budget), continuous
batching over several streams, and the result of every request the same
whether it ran alone or in the mix (tolerance 0: the codec is deterministic
per block).  A sample is also checked against the oracle."""
import numpy as np
import pytest
import torch

from fieldgen import octahedral as og
from oracle import batch as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _setup(N=24):
    lens = og.row_lengths(N)
    specs = [(13, "temperature", 3), (1, "humidity", 1), (9, "power", 3), (2, "power", 1)]
    fields = [og.octahedral_field(N, nlev, 50 + i, kind=kind).cuda() for i, (nlev, kind, _) in enumerate(specs)]
    reqs = og.serving_requests(60, [s[0] for s in specs], [s[2] for s in specs], 7, lens,
                               min_bytes=256, max_bytes=48 << 10, median_bytes=4 << 10)
    offs = np.concatenate([[0], np.cumsum(lens)])
    calls = []
    for r in reqs:
        f = fields[r["field"]]
        ptr = f.data_ptr() + 4 * (r["z0"] * f.stride(0) + int(offs[r["row0"]]))
        calls.append(dict(src=ptr, lev_stride=f.stride(0), nlev=r["nz"], dims=r["dims"], rate=r["rate"],
                          row0=r["row0"], row1=r["row1"]))
    return lens, specs, fields, reqs, calls


def test_alone_equals_mix_and_oracle(z):
    from paper_2609_24294_gb300 import serve
    lens, specs, fields, reqs, calls = _setup()
    srv = serve.Server(lens, arena_bytes=64 << 20, nstreams=4, max_batch=16)
    alone = []
    for c in calls:                                   # one request at a time
        _, _, _, res = serve.run_requests(srv, [c], keep_results=True)
        alone.append(res[0])
    st0 = srv.stats()
    assert st0["batches"] == len(calls)
    rng = np.random.default_rng(1)
    arrivals = np.cumsum(rng.exponential(20e-6, len(calls)))       # 50k requests/s
    lat, wall, busy_max, mixed = serve.run_requests(srv, calls, arrivals=arrivals, keep_results=True)
    st1 = srv.stats()
    assert st1["batches"] - st0["batches"] < len(calls)             # requests shared batches
    for i, ((sa, va), (sm, vm)) in enumerate(zip(alone, mixed)):
        assert sa.tobytes() == sm.tobytes(), i
        assert np.array_equal(va.view(np.uint32), vm.view(np.uint32)), i
    assert np.all(lat > 0) and st1["arena_used"] == 0 and st1["queued"] == 0
    # another 1-D work-unit size changes nothing either
    srv.set_unit_blocks(2)
    _, _, _, mixed2 = serve.run_requests(srv, calls, arrivals=arrivals, keep_results=True)
    for i, ((sa, va), (sm, vm)) in enumerate(zip(alone, mixed2)):
        assert sa.tobytes() == sm.tobytes(), i
        assert np.array_equal(va.view(np.uint32), vm.view(np.uint32)), i
    # oracle on a sample of requests
    offs = np.concatenate([[0], np.cumsum(lens)])
    for i in range(0, len(calls), 7):
        r = reqs[i]
        f = fields[r["field"]].cpu().numpy()
        sub = f[r["z0"]:r["z0"] + r["nz"], offs[r["row0"]]:offs[r["row1"]]]
        ref = ob.encode_field(np.ascontiguousarray(sub), lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        assert alone[i][0].tobytes() == ref.tobytes(), i
        dec = ob.decode_field(ref, sub.shape, lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        assert np.array_equal(alone[i][1].view(np.uint32), dec.reshape(-1).view(np.uint32)), i
    srv.close()


def test_admission_waits_for_memory_and_refuses_oversize(z):
    from paper_2609_24294_gb300 import serve
    lens, specs, fields, reqs, calls = _setup()
    need = max(r["bytes"] for r in reqs)
    # an arena that holds only a couple of requests at a time: everything still finishes
    srv = serve.Server(lens, arena_bytes=3 * need, nstreams=2, max_batch=8)
    lat, wall, busy_max, res = serve.run_requests(srv, calls, keep_results=False)
    assert np.all(np.isfinite(lat)) and srv.stats()["arena_used"] == 0
    # a request larger than the whole arena is refused at submission
    small = serve.Server(lens, arena_bytes=8192, nstreams=1, max_batch=1)
    big = max(calls, key=lambda c: c["nlev"] * (c["row1"] - c["row0"]))
    with pytest.raises(z.ZfpxError) as e:
        small.submit(**big)
    assert e.value.code == -5
    srv.close()
    small.close()


def test_native_loop_matches_python_loop(z):
    """zfpx_server_run (the request loop inside the library) finishes every
    request, refuses what cannot fit, and leaves results identical to the
    submit / pump / poll path (checked on a request kept afterwards)."""
    from fieldgen import octahedral as og
    from paper_2609_24294_gb300 import serve
    lens = og.row_lengths(64)
    f = og.octahedral_field(64, 9, 77, device="cuda")
    offs = np.concatenate([[0], np.cumsum(lens)])
    calls = []
    for k in range(40):
        r0 = 4 * (k % 28)
        r1 = min(len(lens), r0 + 4 * (1 + k % 5))
        calls.append(dict(src=f.data_ptr() + 4 * int(offs[r0]), lev_stride=f.stride(0), nlev=1 + k % 9,
                          dims=3 if k % 3 else 1, rate=8 if k % 2 else 16, row0=r0, row1=r1))
    srv = serve.Server(lens, arena_bytes=1 << 24, nstreams=3, max_batch=8)
    arrivals = np.cumsum(np.full(len(calls), 2e-5))
    lat, wall, busy, nb = serve.run_requests_native(srv, calls, arrivals=arrivals)
    assert np.all(np.isfinite(lat)) and np.all(lat >= 0) and wall > 0 and 1 <= busy <= 3 and nb >= 1
    lat2, _, _, _ = serve.run_requests_native(srv, calls)                  # all at once
    assert np.all(np.isfinite(lat2))
    _, _, _, kept = serve.run_requests(srv, calls[:3], keep_results=True)
    _, _, _, again = serve.run_requests(srv, calls[:3], keep_results=True)
    for a, b in zip(kept, again):
        assert a[0].tobytes() == b[0].tobytes() and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    srv.close()
    # a request larger than the arena is refused, the others still finish
    small = serve.Server(lens, arena_bytes=4096, nstreams=1, max_batch=4)
    big = dict(calls[0], nlev=9, row0=0, row1=len(lens))
    lat3, _, _, _ = serve.run_requests_native(small, [big])
    assert np.isnan(lat3).all()
    small.close()


def test_batching_window(z):
    """With a batching window (launch at 6 waiting requests or after 300 us)
    requests share batches at an arrival rate the device outpaces, every one
    finishes, and each result is the one the default mode gives."""
    from paper_2609_24294_gb300 import serve
    lens, specs, fields, reqs, calls = _setup()
    srv = serve.Server(lens, arena_bytes=64 << 20, nstreams=4, max_batch=16)
    _, _, _, plain = serve.run_requests(srv, calls, keep_results=True)
    b0 = srv.stats()["batches"]
    srv.set_batching(6, 300.0)
    arrivals = np.cumsum(np.full(len(calls), 20e-6))                # 50k requests/s
    lat, wall, busy, nb = serve.run_requests_native(srv, calls, arrivals=arrivals)
    assert np.all(np.isfinite(lat)) and nb >= 1
    assert len(calls) / nb >= 3                                      # batches are shared
    _, _, _, windowed = serve.run_requests(srv, calls, keep_results=True)
    for (sa, va), (sb, vb) in zip(plain, windowed):
        assert sa.tobytes() == sb.tobytes() and np.array_equal(va.view(np.uint32), vb.view(np.uint32))
    with pytest.raises(z.ZfpxError):
        srv.set_batching(17, 0.0)                                    # above max_batch
    with pytest.raises(z.ZfpxError):
        srv.set_batching(1, -1.0)
    srv.set_batching(1, 0.0)
    assert srv.stats()["batches"] > b0
    srv.close()
