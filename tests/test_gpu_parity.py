"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact everywhere: compressed bytes (Sec. II-C fixed-rate streams, at
their fixed offsets), decompressed float32 values compared as bit patterns,
float16 casts and the permutation (Sec. II-B).
"""
import numpy as np
import pytest
import torch

import fieldgen
from oracle import codec as oc
from oracle import packs as op
from oracle import plan as opl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def same_bits(a, b):
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    assert a.shape == b.shape
    diff = a.view(np.uint32) != b.view(np.uint32)
    assert not diff.any(), "%d of %d values differ, first at %s" % (diff.sum(), diff.size, np.argwhere(diff)[0])


def smooth_field(shape, seed, offset=0.0):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    x = np.linspace(0, 2 * np.pi, nx)[None, None, :]
    y = np.linspace(0, np.pi, ny)[None, :, None]
    zz = np.linspace(0, 1, nz)[:, None, None]
    f = np.sin(3 * x + zz) * np.cos(2 * y) + 0.3 * np.sin(7 * x * y + 2 * zz) + 0.01 * rng.standard_normal(shape)
    return (offset + f).astype(np.float32)


# ---------------------------------------------------------------- raw arrays
@pytest.mark.parametrize("dims", [3, 2, 1])
@pytest.mark.parametrize("rate", [16, 8])
def test_t21_field_raw_codec(z, dims, rate):
    f = fieldgen.t21_field()                   # 64 lon x 32 lat x 8 levels
    n = (64, 32, 8)
    nb = z.zfpx_stream_bytes(dims, rate, n)
    out = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    z.zfpx_encode(dims, rate, dev(f), out)
    ref = oc.encode_array(dims, rate, f)
    g = host(out)
    assert g.tobytes() == ref.tobytes(), "first differing byte %d" % int(np.argmax(g != ref))
    dec = torch.full_like(dev(f), float("nan"))
    z.zfpx_decode(dims, rate, out, dec)
    rdec = np.empty_like(f)
    oc.decode_array(dims, rate, ref, rdec)
    same_bits(host(dec), rdec)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 5), (7, 5, 3), (2, 9, 33), (17, 6, 130)])
@pytest.mark.parametrize("dims", [3, 2, 1])
def test_small_and_ragged_arrays(z, shape, dims):
    x = smooth_field(shape, 3, offset=10.0)
    n = tuple(reversed(shape))
    for rate in (8, 16):
        out = torch.zeros(z.zfpx_stream_bytes(dims, rate, n), dtype=torch.uint8, device="cuda")
        z.zfpx_encode(dims, rate, dev(x), out)
        ref = oc.encode_array(dims, rate, x)
        assert host(out).tobytes() == ref.tobytes()
        dec = torch.full(shape, float("nan"), device="cuda")
        z.zfpx_decode(dims, rate, out, dec)
        rdec = np.empty_like(x)
        oc.decode_array(dims, rate, ref, rdec)
        same_bits(host(dec), rdec)


def _special_values(shape, seed):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(shape) * 10.0 ** rng.integers(-40, 38, shape)).astype(np.float32)
    nz, ny, nx = shape
    x[0:4, 0:4, 0:4] = 0.0                               # zero block
    x[0:4, 0:4, 4:8] = -0.0
    x[0:4, 4:8, 0:4] = 3.25                              # constant block
    x[0:4, 4:8, 4:8] = np.float32(2e-39)                 # subnormal, above 2^-127
    x[4:8, 0:4, 0:4] = np.float32(5e-40)                 # subnormal, below 2^-127
    x[4:8, 0:4, 4:8] = np.float32(3.4e38) * np.sign(rng.standard_normal((4, 4, 4))).astype(np.float32)
    x[4:8, 4:8, 0:4] = rng.standard_normal((4, 4, 4)).astype(np.float32)
    x[5, 5, 1] = np.inf                                  # non-finite blocks
    x[4:8, 4:8, 4:8] = rng.standard_normal((4, 4, 4)).astype(np.float32)
    x[6, 6, 6] = np.nan
    x[0:4, 8:12, 0:4] = 1e-30 * rng.standard_normal((4, 4, 4)).astype(np.float32)   # small e_max
    return x


def test_special_values(z):
    x = _special_values((8, 12, 16), 5)
    n = (16, 12, 8)
    for dims in (3, 2, 1):
        for rate in (8, 16):
            out = torch.zeros(z.zfpx_stream_bytes(dims, rate, n), dtype=torch.uint8, device="cuda")
            z.zfpx_encode(dims, rate, dev(x), out)
            ref = oc.encode_array(dims, rate, x)
            assert host(out).tobytes() == ref.tobytes()
            dec = torch.empty_like(dev(x))
            z.zfpx_decode(dims, rate, out, dec)
            rdec = np.empty_like(x)
            oc.decode_array(dims, rate, ref, rdec)
            same_bits(host(dec), rdec)


def test_graded_spectrum_blocks(z):
    # many planes with newly significant coefficients (the coder's per-plane
    # bookkeeping beyond its first ten such planes), 3 warps of blocks + tail
    x = fieldgen.graded_blocks(100, 9)
    n = (x.shape[2], 4, 4)
    for rate in (8, 16):
        out = torch.zeros(z.zfpx_stream_bytes(3, rate, n), dtype=torch.uint8, device="cuda")
        z.zfpx_encode(3, rate, dev(x), out)
        ref = oc.encode_array(3, rate, x)
        assert host(out).tobytes() == ref.tobytes()
        dec = torch.empty_like(dev(x))
        z.zfpx_decode(3, rate, out, dec)
        rdec = np.empty_like(x)
        oc.decode_array(3, rate, ref, rdec)
        same_bits(host(dec), rdec)


def _stream_budget_on_group_bit(rate):
    """A 3-D stream whose budget ends exactly on a set group bit while 63
    coefficients are significant: only coefficient 63 is left, and its one
    is implied without another bit.  Built plane by plane: 5 empty planes,
    one making coefficients 0..49 significant, one making 50..62
    significant, planes of 63 verbatim bits and an empty group, and a last
    plane whose group bit is the stream's final bit."""
    rng = np.random.default_rng(rate)
    bits = [1] + [int(b) for b in np.binary_repr(130, 8)[::-1]]          # block flag, exponent
    bits += [0] * 5
    bits += [1] + [1, 1] * 49 + [1, 0]                                    # coefficients 0..49
    bits += list(rng.integers(0, 2, 50)) + [1] + [1, 1] * 12 + [1, 0]     # 50..62
    m = (64 * rate - 64 - len(bits)) // 64
    for _ in range(m):
        bits += list(rng.integers(0, 2, 63)) + [0]
    bits += list(rng.integers(0, 2, 63)) + [1]
    assert len(bits) == 64 * rate
    return np.packbits(np.array(bits, dtype=np.uint8), bitorder="little")


def test_budget_ends_on_group_bit_with_implied_one(z):
    for rate in (8, 16):
        s = _stream_budget_on_group_bit(rate)
        dec = torch.empty((4, 4, 4), device="cuda")
        z.zfpx_decode(3, rate, dev(s), dec)
        rdec = np.empty((4, 4, 4), dtype=np.float32)
        oc.decode_array(3, rate, s, rdec)
        same_bits(host(dec), rdec)


def test_random_streams_decode_like_oracle(z):
    # the decoder is defined on any byte stream
    rng = np.random.default_rng(11)
    n = (32, 8, 8)
    for dims in (3, 2, 1):
        for rate in (8, 16):
            nb = z.zfpx_stream_bytes(dims, rate, n)
            s = rng.integers(0, 256, nb, dtype=np.uint8)
            dec = torch.empty((8, 8, 32), device="cuda")
            z.zfpx_decode(dims, rate, dev(s), dec)
            rdec = np.empty((8, 8, 32), dtype=np.float32)
            oc.decode_array(dims, rate, s, rdec)
            same_bits(host(dec), rdec)


def test_repeated_launches_reuse_work_counters(z):
    # the 3-D kernels hand out work through counters that each launch leaves
    # at zero: every launch of a run must code every block
    x = smooth_field((24, 40, 72), 3, offset=250.0)
    nz, ny, nx = x.shape
    xd = dev(x)
    plan = z.Plan.for_fields(xd, 2, 3, 0, 3)
    for rate in (8, 16):
        outs = []
        for _ in range(4):
            buf = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
            z.zfpx_pack_compress(plan, rate, xd, buf)
            outs.append(buf)
        for buf in outs[1:]:
            assert torch.equal(buf, outs[0])
        decs = []
        for _ in range(4):
            d = torch.full_like(xd, float("nan"))
            z.zfpx_decompress_unpack(plan, rate, outs[0], d, layout=z.LAYOUT_SEND)
            decs.append(d)
        for d in decs[1:]:
            same_bits(host(d), host(decs[0]))
        assert not torch.isnan(decs[0]).any()                       # every value written


# ---------------------------------------------------------------- plans
# the last three leave messages empty (more ranks than levels, points or rows on an axis)
PLANS = [((17, 23, 37), 3, 2), ((8, 32, 64), 2, 2), ((5, 9, 11), 2, 3), ((20, 16, 48), 1, 4),
         ((3, 8, 8), 2, 4), ((1, 1, 1), 3, 3), ((2, 2, 5), 3, 3)]


@pytest.mark.parametrize("t", [0, 1])
@pytest.mark.parametrize("dims", [3, 2, 1])
@pytest.mark.parametrize("shape,pr,pc", PLANS)
def test_pack_compress_permute_decompress(z, t, dims, shape, pr, pc):
    x = smooth_field(shape, 7, offset=250.0)
    nz, ny, nx = shape
    xd = dev(x)
    oplan = opl.Plan(nx, ny, nz, pr, pc, t, dims)
    # destination with a padded row pitch (e.g. room for an in-place real FFT)
    dst_store = torch.full((nz, ny, nx + 6), float("nan"), device="cuda")
    dst = dst_store[:, :, :nx]
    plan = z.Plan.for_fields(xd, pr, pc, t, dims, dst=dst)
    for rate in (8, 16):
        ref_send = op.pack(oplan, rate, x, which="send")
        ref_recv = op.permute(oplan, rate, ref_send)
        send = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
        z.zfpx_pack_compress(plan, rate, xd, send, z.LAYOUT_SEND)
        assert host(send).tobytes() == ref_send.tobytes()
        recv = torch.zeros_like(send)
        z.zfpx_permute(plan, rate, send, recv)
        assert host(recv).tobytes() == ref_recv.tobytes()
        folded = torch.zeros_like(send)
        z.zfpx_pack_compress(plan, rate, xd, folded, z.LAYOUT_RECV)
        assert torch.equal(folded, recv)
        dst.fill_(float("nan"))
        z.zfpx_decompress_unpack(plan, rate, recv, dst, z.LAYOUT_RECV)
        rdst = np.full_like(x, np.nan)
        op.unpack(oplan, rate, ref_recv, rdst)
        same_bits(host(dst), rdst)
        # padding columns untouched
        assert torch.isnan(dst_store[:, :, nx:]).all()


@pytest.mark.parametrize("t", [0, 1])
def test_comparator_packs(z, t):
    rng = np.random.default_rng(9)
    shape = (13, 10, 22)
    x = (rng.standard_normal(shape) * 10.0 ** rng.integers(-9, 6, shape)).astype(np.float32)
    x.reshape(-1)[:6] = [65504.0, 65520.0, -1e6, 6e-8, np.inf, -np.inf]
    nz, ny, nx = shape
    xd = dev(x)
    oplan = opl.Plan(nx, ny, nz, 2, 3, t, 3)
    plan = z.Plan.for_fields(xd, 2, 3, t, 3)
    # float32
    send = torch.zeros(plan.buffer_bytes(z.RATE_F32) // 4, dtype=torch.float32, device="cuda")
    z.zfpx_pack(plan, xd, send)
    ref = op.pack(oplan, 0, x)
    assert host(send).view(np.uint8).tobytes() == ref.tobytes()
    recv = torch.zeros_like(send)
    z.zfpx_permute(plan, z.RATE_F32, send, recv)
    assert host(recv).view(np.uint8).tobytes() == op.permute(oplan, 0, ref).tobytes()
    out = torch.full_like(xd, float("nan"))
    z.zfpx_unpack(plan, recv, out)
    same_bits(host(out), x)
    # float16, both roundings
    for mode, name in ((z.ROUND_NEAREST, "rn"), (z.ROUND_ZERO, "rz")):
        h = torch.zeros(plan.buffer_bytes(z.RATE_F16) // 2, dtype=torch.int16, device="cuda")
        z.zfpx_cast_fp16_pack(plan, mode, xd, h)
        ref = op.pack(oplan, -16, x, round_mode=name)
        assert host(h).view(np.uint8).tobytes() == ref.tobytes(), name
        hr = torch.zeros_like(h)
        z.zfpx_permute(plan, z.RATE_F16, h, hr)
        out = torch.full_like(xd, float("nan"))
        z.zfpx_fp16_unpack(plan, hr, out)
        rout = np.full_like(x, np.nan)
        op.unpack(oplan, -16, op.permute(oplan, -16, ref), rout)
        same_bits(host(out), rout)


def test_strided_sources(z):
    rng = np.random.default_rng(12)
    big = smooth_field((12, 20, 48), 4)
    # unaligned x offset: vector loads off
    src = dev(big)[1:10, 2:19, 3:40]
    x = np.ascontiguousarray(big[1:10, 2:19, 3:40])
    # longitude not the fastest axis: [lev][lon][lat] storage viewed as [lev][lat][lon]
    alt_store = dev(np.ascontiguousarray(np.transpose(x, (0, 2, 1))))
    alt = alt_store.permute(0, 2, 1)
    for s in (src, alt):
        nz, ny, nx = x.shape
        for dims in (3, 2):
            oplan = opl.Plan(nx, ny, nz, 2, 2, 0, dims)
            plan = z.Plan.for_fields(s, 2, 2, 0, dims)
            for rate in (8, 16):
                send = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
                z.zfpx_pack_compress(plan, rate, s, send)
                assert host(send).tobytes() == op.pack(oplan, rate, x).tobytes()
    del rng


def test_random_views_fuzz(z):
    """Random small fields, views of larger arrays (offsets, padded pitches,
    longitude not always fastest), block shapes 1-D / 2-D / 3-D and both rates,
    raw codec against the oracle; the decoder on the oracle's stream."""
    rng = np.random.default_rng(31)
    for it in range(40):
        nz, ny, nx = (int(v) for v in rng.integers(1, 19, 3))
        big = (rng.standard_normal((nz + 3, ny + 5, nx + 9)) * 10.0 ** rng.uniform(-20, 20)).astype(np.float32)
        if it % 4 == 0:
            big += np.float32(rng.uniform(-300, 300))
        oz, oy, ox = (int(rng.integers(0, m)) for m in (3, 5, 9))
        x = big[oz:oz + nz, oy:oy + ny, ox:ox + nx]
        bd = dev(big)
        src = bd[oz:oz + nz, oy:oy + ny, ox:ox + nx]
        if it % 3 == 1:                                   # [lev][lon][lat] storage viewed as [lev][lat][lon]
            alt = dev(np.ascontiguousarray(np.transpose(x, (0, 2, 1))))
            src = alt.permute(0, 2, 1)
        dims, rate = (1, 2, 3)[it % 3], (8, 16)[(it // 3) % 2]
        n = (nx, ny, nz)
        out = torch.zeros(z.zfpx_stream_bytes(dims, rate, n), dtype=torch.uint8, device="cuda")
        z.zfpx_encode(dims, rate, src, out)
        ref = oc.encode_array(dims, rate, np.ascontiguousarray(x))
        assert host(out).tobytes() == ref.tobytes(), (it, dims, rate, x.shape)
        dec = torch.full((nz, ny, nx), float("nan"), device="cuda")
        z.zfpx_decode(dims, rate, out, dec)
        rdec = np.empty_like(x)
        oc.decode_array(dims, rate, ref, rdec)
        same_bits(host(dec), rdec)


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def t639():
    return fieldgen.t639_field()


def _all_messages(oplan, rate, dims, x, hs, so, ho):
    """Every message of the plan through the oracle on all host cores (the C
    oracle releases the GIL): its stream must equal the GPU's bytes at the
    message's offset, and its decoded box the GPU's values.  Returns the
    mismatching messages."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    def one(m):
        nb = opl.message_bytes(m, rate, dims)
        if nb == 0:
            return None
        ref = op.message_stream(oplan, rate, x, m)
        o = so[(m.src, m.dst)]
        if hs[o:o + nb].tobytes() != ref.tobytes():
            return (m.src, m.dst, "bytes")
        box = np.empty((m.nz, m.ny, m.nx), dtype=np.float32)
        oc.decode_array(dims, rate, ref, box)
        got = ho[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx]
        if not np.array_equal(got.view(np.uint32), box.view(np.uint32)):
            return (m.src, m.dst, "values")
        return None

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return [r for r in ex.map(one, oplan.messages) if r is not None]


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("rate", [8, 16])
def test_t639_field_full_size(z, t639, rate, dims):
    """1280 x 640 x 137, 8 x 8 ranks, z->lambda: the launches the benchmark
    times, every one of the 512 messages compared with the oracle -- the
    compressed bytes at their offsets and the decoded values as bit
    patterns -- and the folded receive layout equal to the permutation."""
    x = t639
    xd = dev(x)
    nz, ny, nx = x.shape
    plan = z.Plan.for_fields(xd, 8, 8, 0, dims)
    oplan = opl.Plan(nx, ny, nz, 8, 8, 0, dims)
    send = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
    z.zfpx_pack_compress(plan, rate, xd, send)
    recv = torch.zeros_like(send)
    z.zfpx_permute(plan, rate, send, recv)
    folded = torch.zeros_like(send)
    z.zfpx_pack_compress(plan, rate, xd, folded, z.LAYOUT_RECV)
    assert torch.equal(folded, recv)
    out = torch.full_like(xd, float("nan"))
    z.zfpx_decompress_unpack(plan, rate, recv, out)
    so, ro, total = oplan.layout(rate)
    hs = host(send)
    ho = host(out)
    assert len(oplan.messages) == 512
    bad = _all_messages(oplan, rate, dims, x, hs, so, ho)
    assert not bad, "%d of 512 messages differ from the oracle, first %s" % (len(bad), bad[0])
    assert np.isfinite(ho).all()
