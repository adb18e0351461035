"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times:

* the transposition pair on 2560 x 1280 x 137 (T1279 field, 8 x 8 ranks) as
  one CUDA graph, rates 8 and 16: every value of the final field against the
  oracle chained through both transpositions (Sec. II-B, II-C), run over all
  host cores;
* the ten-field O1280 batch (22.9 GB, one launch each way): every byte of
  every field's stream and every decoded value against the oracle, 3-D
  row-quads and 1-D rows, and the other launch shape the tuner picks between
  giving the same bytes and values;
* the serving loop on 2000 requests over the same fields: every request's
  stream and values against the oracle, and a sample of requests run alone
  against the same requests in the mix.
"""
import numpy as np
import pytest
import torch

from fieldgen import octahedral as og
from oracle import batch as ob
from oracle import codec as oc
from oracle import plan as opl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


# ---------------------------------------------------------------- transposition pair
def _oracle_transposition(msgs, rate, src, dst):
    """One transposition by the oracle: every message box of src coded at `rate`
    and decoded into the same box of dst, messages spread over all host cores
    (the boxes partition the field, so the threads write disjoint regions)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    def one(m):
        if m.nx * m.ny * m.nz == 0:
            return
        box = src[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx]
        s = oc.encode_array(3, rate, box)
        oc.decode_array(3, rate, s, dst[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx])

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        list(ex.map(one, msgs))


@pytest.mark.parametrize("rate", [8, 16])
def test_pair_full_size(z, rate):
    from fieldgen.sht_torch import sht_field_torch
    x = sht_field_torch(2560, 1280, 137, 1279, seed=2, device="cuda")
    nz, ny, nx = x.shape
    mid = torch.empty_like(x)
    dst = torch.full_like(x, float("nan"))
    p1 = z.Plan.for_fields(x, 8, 8, 0, 3, dst=mid)
    p2 = z.Plan.for_fields(mid, 8, 8, 1, 3, dst=dst)
    nb = max(p1.buffer_bytes(rate), p2.buffer_bytes(rate))
    send = torch.empty(nb, dtype=torch.uint8, device="cuda")
    recv = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = z.PairGraph(p1, p2, rate, x, mid, dst, send, recv)
    g.launch()
    g.launch()                                    # a replay gives the same field
    torch.cuda.synchronize()
    hx = x.cpu().numpy()
    got = dst.cpu().numpy()
    g.close()
    del x, mid, dst, send, recv
    torch.cuda.empty_cache()
    # the oracle through both transpositions, every value
    omid = np.full_like(hx, np.nan)
    _oracle_transposition(opl.Plan(nx, ny, nz, 8, 8, 0, 3).messages, rate, hx, omid)
    assert np.isfinite(omid).all()
    want = np.full_like(hx, np.nan)
    _oracle_transposition(opl.Plan(nx, ny, nz, 8, 8, 1, 3).messages, rate, omid, want)
    diff = got.view(np.uint32) != want.view(np.uint32)
    assert not diff.any(), "%d of %d values differ, first at %s" % (diff.sum(), diff.size, np.argwhere(diff)[0])


# ---------------------------------------------------------------- batched O1280 and serving
@pytest.fixture(scope="module")
def o1280():
    lens = og.row_lengths(1280)
    fields = []
    for i, (nlev, kind, dims, rate) in enumerate(og.O1280_TEN_FIELDS):
        src = og.octahedral_field(1280, nlev, 300 + i, kind=kind, device="cuda")
        fields.append((src, torch.empty_like(src), dims, rate))
    yield lens, fields
    del fields
    torch.cuda.empty_cache()


def _pool():
    import os
    from concurrent.futures import ThreadPoolExecutor
    return ThreadPoolExecutor(max_workers=os.cpu_count() or 1)


def _oracle_field(f_np, lens, dims, rate):
    """The field's stream and decoded values by the oracle, one item (level
    quad, or level for dims 1) per task over all host cores: an item's
    stream is that of the field cut to the item's levels."""
    items = ob.field_items(lens, f_np.shape[0], dims)

    def enc(it):
        z0, nz = it
        return ob.encode_field(np.ascontiguousarray(f_np[z0:z0 + nz]), lens, dims, rate)

    with _pool() as ex:
        parts = list(ex.map(enc, items))
    dec = np.empty_like(f_np)

    def dcd(k):
        z0, nz = items[k]
        dec[z0:z0 + nz] = ob.decode_field(parts[k], (nz, f_np.shape[1]), lens, dims, rate)

    with _pool() as ex:
        list(ex.map(dcd, range(len(items))))
    return np.concatenate(parts), dec


def test_batched_full_size(z, o1280):
    """The ten O1280 fields (22.9 GB) in one encode and one decode launch: every
    byte of every field's stream and every decoded value against the oracle
    (field by field, so the host holds one field at a time); the other launch
    shape the tuner picks between gives the same bytes and values."""
    lens, fields = o1280
    spec = [(f[0].shape[0], f[2], f[3]) for f in fields]
    offs, total = ob.layout(lens, spec)
    outs = []
    for warps in (4, 8):
        batch = z.Batch(lens, fields)
        batch.set_launch(warps, 0)
        assert batch.nbytes() == total
        out = torch.empty(batch.nbytes(), dtype=torch.uint8, device="cuda")
        for _, dst, _, _ in fields:
            dst.fill_(float("nan"))
        batch.encode(out)
        batch.decode(out)
        torch.cuda.synchronize()
        for fi in range(len(fields)):
            assert batch.field_offset(fi) == offs[fi]
        batch.close()
        if outs:
            assert torch.equal(out, outs[0])
            for fi, (_, dst, _, _) in enumerate(fields):
                assert torch.equal(dst.view(torch.int32), outs[1][fi].view(torch.int32)), fi
            break
        outs = [out, [f[1].clone() for f in fields]]
    out, decoded = outs
    for fi, (src, _, dims, rate) in enumerate(fields):
        f_np = src.cpu().numpy()
        want_s, want_v = _oracle_field(f_np, lens, dims, rate)
        got_s = out[offs[fi]:offs[fi] + want_s.size].cpu().numpy()
        assert got_s.tobytes() == want_s.tobytes(), fi
        got_v = decoded[fi].cpu().numpy()
        diff = got_v.view(np.uint32) != want_v.view(np.uint32)
        assert not diff.any(), (fi, int(diff.sum()))
        del f_np, want_s, want_v, got_s, got_v


def test_serving_full_size(z, o1280):
    """2000 requests at Poisson arrivals through the serving loop: every
    request's stream and values against the oracle (over all host cores), and
    a sample of requests run alone against the same requests in the mix."""
    from paper_2609_24294_gb300 import serve
    lens, fields = o1280
    reqs = og.serving_requests(2000, [f[0].shape[0] for f in fields], [f[2] for f in fields], 5, lens)
    offs = np.concatenate([[0], np.cumsum(lens)])
    calls = []
    for r in reqs:
        f = fields[r["field"]][0]
        ptr = f.data_ptr() + 4 * (r["z0"] * f.stride(0) + int(offs[r["row0"]]))
        calls.append(dict(src=ptr, lev_stride=f.stride(0), nlev=r["nz"], dims=r["dims"], rate=r["rate"],
                          row0=r["row0"], row1=r["row1"]))
    srv = serve.Server(lens, arena_bytes=40 << 30, nstreams=4, max_batch=64)
    arrivals = np.cumsum(np.random.default_rng(5).exponential(1.0 / 50e3, len(calls)))
    lat, wall, busy, mixed = serve.run_requests(srv, calls, arrivals=arrivals, keep_results=True)
    assert np.all(lat > 0)
    picks = [i for i in range(0, len(calls), 50) if reqs[i]["bytes"] < (4 << 20)][:16]
    for i in picks:
        _, _, _, alone = serve.run_requests(srv, [calls[i]], keep_results=True)
        assert alone[0][0].tobytes() == mixed[i][0].tobytes(), i
        assert np.array_equal(alone[0][1].view(np.uint32), mixed[i][1].view(np.uint32)), i
    srv.close()
    host_fields = {}

    def check(i):
        r = reqs[i]
        f = host_fields[r["field"]]
        sub = np.ascontiguousarray(f[r["z0"]:r["z0"] + r["nz"], int(offs[r["row0"]]):int(offs[r["row1"]])])
        ref = ob.encode_field(sub, lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        if mixed[i][0].tobytes() != ref.tobytes():
            return (i, "bytes")
        dec = ob.decode_field(ref, sub.shape, lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        if not np.array_equal(mixed[i][1].view(np.uint32), dec.reshape(-1).view(np.uint32)):
            return (i, "values")
        return None

    bad = []
    for fi in range(len(fields)):                 # one field on the host at a time
        host_fields = {fi: fields[fi][0].cpu().numpy()}
        ids = [i for i in range(len(reqs)) if reqs[i]["field"] == fi]
        with _pool() as ex:
            bad += [b for b in ex.map(check, ids) if b is not None]
    assert not bad, "%d of %d requests differ from the oracle, first %s" % (len(bad), len(reqs), bad[0])
