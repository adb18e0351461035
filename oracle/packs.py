"""Pack, all-to-all permutation and unpack over a plan (test infrastructure; oracle side).

The paper's per-rank sequence (Sec. I; Sec. IV-D): pack each destination's
sub-block of the outgoing pencil, compress it (ZFP fixed rate) or cast it
(float16) or leave it (float32), exchange the fixed-size messages with an
all-to-all, then decompress / cast back and unpack into the next pencil.  On
one device the exchange is the permutation recv[dst][src] <- send[src][dst].

A message is the box of the plan (see ``plan``) read in raster order, lon
fastest.  Fields are float32 numpy arrays indexed [lev][lat][lon] and may be
strided views; buffers are uint8 arrays laid out by ``Plan.layout``.

Parity: pinned by invariants in tests/test_oracle_packs.py (every value sent
exactly once, in raster order; unpack(permute(pack(x))) == x for float32).
"""
import numpy as np

from . import codec, fp16
from .plan import message_bytes


def _box(field, m):
    return field[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx]


def pack(plan, rate, field, round_mode="rn", which="send"):
    """Pack every message of ``plan`` into a send (or, with which='recv', a
    receive-layout) buffer.  rate 0 float32, -16 float16, 8/16/... ZFP."""
    send_off, recv_off, total = plan.layout(rate)
    offs = send_off if which == "send" else recv_off
    buf = np.zeros(total, dtype=np.uint8)
    for m in plan.messages:
        nb = message_bytes(m, rate, plan.dims)
        o = offs[(m.src, m.dst)]
        box = _box(field, m)
        if rate == 0:
            data = np.ascontiguousarray(box, dtype=np.float32).view(np.uint8).reshape(-1)
        elif rate == -16:
            conv = fp16.to_f16_rn if round_mode == "rn" else fp16.to_f16_rz
            data = conv(np.ascontiguousarray(box)).view(np.uint8).reshape(-1)
        else:
            data = codec.encode_array(plan.dims, rate, box)
        assert data.size == nb
        buf[o:o + nb] = data
    return buf


def permute(plan, rate, send):
    """The all-to-all on one device: message (src, dst) moves from its send
    slot to its receive slot."""
    send_off, recv_off, total = plan.layout(rate)
    recv = np.zeros(total, dtype=np.uint8)
    for m in plan.messages:
        nb = message_bytes(m, rate, plan.dims)
        a, b = send_off[(m.src, m.dst)], recv_off[(m.src, m.dst)]
        recv[b:b + nb] = send[a:a + nb]
    return recv


def unpack(plan, rate, recv, out, which="recv"):
    """Inverse of ``pack``: write every message's values into the field ``out``."""
    send_off, recv_off, total = plan.layout(rate)
    offs = recv_off if which == "recv" else send_off
    for m in plan.messages:
        nb = message_bytes(m, rate, plan.dims)
        o = offs[(m.src, m.dst)]
        box = _box(out, m)
        data = recv[o:o + nb]
        if rate == 0:
            box[...] = data.view(np.float32).reshape(box.shape)
        elif rate == -16:
            box[...] = fp16.from_f16(data.view(np.uint16)).reshape(box.shape)
        else:
            codec.decode_array(plan.dims, rate, data, box)
    return out


def message_stream(plan, rate, field, m):
    """The bytes of one message alone (used for sampled checks at full size)."""
    box = _box(field, m)
    if rate == 0:
        return np.ascontiguousarray(box, dtype=np.float32).view(np.uint8).reshape(-1)
    if rate == -16:
        return fp16.to_f16_rn(np.ascontiguousarray(box)).view(np.uint8).reshape(-1)
    return codec.encode_array(plan.dims, rate, box)
