"""Parity at the benchmark's full sizes, on sampled outputs the oracle computes
one by one, in the launch configurations bench.py times:

* the transposition pair on 2560 x 1280 x 137 (T1279 field, 8 x 8 ranks) as
  one CUDA graph, rates 8 and 16: sampled blocks of the final field against
  the oracle chained through both transpositions (Sec. II-B, II-C);
* the ten-field O1280 batch (22.9 GB, one launch each way): sampled blocks'
  bytes and decoded values, 3-D row-quads and 1-D rows, at both launch
  shapes the tuner picks between;
* the serving loop on 2000 requests over the same fields: sampled requests
  against the oracle, and alone against in the mix.
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
def _box_of(msgs, z, y, x):
    for m in msgs:
        if m.z0 <= z < m.z0 + m.nz and m.y0 <= y < m.y0 + m.ny and m.x0 <= x < m.x0 + m.nx:
            return m
    raise AssertionError("point outside every message")


def _block_points(m, bz, by, bx):
    """Global (z, y, x) of the 64 block positions, clamped to the message box."""
    return [(m.z0 + min(4 * bz + k, m.nz - 1), m.y0 + min(4 * by + j, m.ny - 1), m.x0 + min(4 * bx + i, m.nx - 1))
            for k in range(4) for j in range(4) for i in range(4)]


def _coded(values, rate):
    s = oc.encode_block(3, rate, np.asarray(values, dtype=np.float32))
    return oc.decode_block(3, rate, s)


@pytest.mark.parametrize("rate", [8, 16])
def test_pair_full_size_sampled(z, rate):
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
    assert not torch.isnan(dst).any()
    m1s = opl.Plan(nx, ny, nz, 8, 8, 0, 3).messages
    m2s = opl.Plan(nx, ny, nz, 8, 8, 1, 3).messages
    rng = np.random.default_rng(rate)
    cache = {}

    def mid_value(pz, py, px):                    # the first transposition, by the oracle
        m = _box_of(m1s, pz, py, px)
        key = (m.z0, m.y0, m.x0, (pz - m.z0) // 4, (py - m.y0) // 4, (px - m.x0) // 4)
        if key not in cache:
            pts = _block_points(m, *key[3:])
            idx = torch.tensor(pts, device="cuda")
            src = x[idx[:, 0], idx[:, 1], idx[:, 2]].cpu().numpy()
            cache[key] = _coded(src, rate)
        lz, ly, lx = (pz - m.z0) % 4, (py - m.y0) % 4, (px - m.x0) % 4
        return cache[key][16 * lz + 4 * ly + lx]

    for _ in range(24):
        m = m2s[int(rng.integers(len(m2s)))]
        bz = int(rng.integers((m.nz + 3) // 4))
        by = int(rng.integers((m.ny + 3) // 4))
        bx = int(rng.integers((m.nx + 3) // 4))
        pts = _block_points(m, bz, by, bx)
        want = _coded([mid_value(*p) for p in pts], rate)
        for t, (pz, py, px) in enumerate(pts):
            k, j, i = t // 16, (t // 4) % 4, t % 4
            if 4 * bz + k < m.nz and 4 * by + j < m.ny and 4 * bx + i < m.nx:   # not a padding copy
                got = float(dst[pz, py, px])
                assert np.float32(got).view(np.uint32) == want[t].view(np.uint32), (m.z0, m.y0, m.x0, t)
    g.close()
    del x, mid, dst, send, recv
    torch.cuda.empty_cache()


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


def _sample_blocks(f_np, lens, dims, rate, rng, n):
    """(byte offset in the field's stream, expected block bytes, expected values,
    [(level, point)] of the block's real values) for n sampled blocks."""
    nlev = f_np.shape[0]
    offs = ob.row_offsets(lens)
    out = []
    if dims == 3:
        qb = ob.quad_blocks(lens)
        qpre = np.concatenate([[0], np.cumsum(qb)])
        per_item = int(qpre[-1])
        items = ob.field_items(lens, nlev, dims)
        picks = [(len(items) - 1, len(qb) - 1, int(qb[-1]) - 1)]          # last item, last quad, row end
        while len(picks) < n:
            it = int(rng.integers(len(items)))
            q = int(rng.integers(len(qb)))
            picks.append((it, q, int(rng.integers(int(qb[q])))))
        for it, q, bx in picks:
            z0, nz = items[it]
            box = ob._quad_box(f_np, lens, offs, q, z0, nz)[:, :, 4 * bx:4 * bx + 4]
            s = oc.encode_array(3, rate, np.ascontiguousarray(box))
            vals = oc.decode_block(3, rate, s)
            pts = []
            for k in range(nz):
                for j in range(min(4, len(lens) - 4 * q)):
                    r = 4 * q + j
                    for i in range(4):
                        if 4 * bx + i < lens[r]:
                            pts.append((16 * k + 4 * j + i, z0 + k, int(offs[r]) + 4 * bx + i))
            out.append(((it * per_item + int(qpre[q]) + bx) * 8 * rate, s, vals, pts))
    else:
        rpre = np.concatenate([[0], np.cumsum((np.asarray(lens) + 3) // 4)])
        per_item = int(rpre[-1])
        for _ in range(n):
            r = int(rng.integers(len(lens)))
            bx = int(rng.integers((int(lens[r]) + 3) // 4))
            row = f_np[0, int(offs[r]):int(offs[r]) + int(lens[r])]
            seg = np.array([row[min(4 * bx + i, int(lens[r]) - 1)] for i in range(4)], dtype=np.float32)
            s = oc.encode_array(1, rate, seg.reshape(1, 1, 4))
            vals = oc.decode_block(1, rate, s)
            pts = [(i, 0, int(offs[r]) + 4 * bx + i) for i in range(4) if 4 * bx + i < lens[r]]
            out.append(((int(rpre[r]) + bx) * rate // 2, s, vals, pts))
    return out


@pytest.mark.parametrize("warps", [4, 8])
def test_batched_full_size_sampled(z, o1280, warps):
    lens, fields = o1280
    batch = z.Batch(lens, fields)
    batch.set_launch(warps, 0)
    out = torch.empty(batch.nbytes(), dtype=torch.uint8, device="cuda")
    for _, dst, _, _ in fields:
        dst.fill_(float("nan"))
    batch.encode(out)
    batch.decode(out)
    torch.cuda.synchronize()
    spec = [(f[0].shape[0], f[2], f[3]) for f in fields]
    offs, total = ob.layout(lens, spec)
    assert batch.nbytes() == total
    rng = np.random.default_rng(warps)
    for fi, (src, dst, dims, rate) in enumerate(fields):
        assert batch.field_offset(fi) == offs[fi]
        assert not torch.isnan(dst).any()
        f_np = src.cpu().numpy()
        for off, s, vals, pts in _sample_blocks(f_np, lens, dims, rate, rng, 6):
            a = offs[fi] + off
            got = out[a:a + s.size].cpu().numpy()
            assert got.tobytes() == s.tobytes(), (fi, off)
            for t, lev, p in pts:
                assert np.float32(float(dst[lev, p])).view(np.uint32) == vals[t].view(np.uint32), (fi, lev, p)
        del f_np
    batch.close()


def test_serving_full_size_sampled(z, o1280):
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
        r = reqs[i]
        _, _, _, alone = serve.run_requests(srv, [calls[i]], keep_results=True)
        assert alone[0][0].tobytes() == mixed[i][0].tobytes(), i
        assert np.array_equal(alone[0][1].view(np.uint32), mixed[i][1].view(np.uint32)), i
        sub = fields[r["field"]][0][r["z0"]:r["z0"] + r["nz"], int(offs[r["row0"]]):int(offs[r["row1"]])]
        sub = np.ascontiguousarray(sub.cpu().numpy())
        ref = ob.encode_field(sub, lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        assert mixed[i][0].tobytes() == ref.tobytes(), i
        dec = ob.decode_field(ref, sub.shape, lens[r["row0"]:r["row1"]], r["dims"], r["rate"])
        assert np.array_equal(mixed[i][1].view(np.uint32), dec.reshape(-1).view(np.uint32)), i
    srv.close()
