"""The transposition pipelined per piece (Sec. III-E, Sec. V-B): compression,
all-to-all and decompression of successive pieces overlap on three streams, and
the send buffer, receive buffer and output field are byte for byte those of the
serial calls (which the parity tests tie to the oracle)."""
import numpy as np
import pytest
import torch

import fieldgen
from oracle import packs as op
from oracle import plan as opl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _serial(z, plan, rate, x):
    nb = plan.buffer_bytes(rate)
    send = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    out = torch.full_like(x, float("nan"))
    z.zfpx_pack_compress(plan, rate, x, send)
    z.zfpx_permute(plan, rate, send, recv)
    z.zfpx_decompress_unpack(plan, rate, recv, out)
    torch.cuda.synchronize()
    return send, recv, out


@pytest.mark.parametrize("rate", [8, 16])
@pytest.mark.parametrize("case", [((37, 100, 212), 3, 2, 0), ((24, 64, 96), 4, 4, 1), ((8, 32, 64), 2, 2, 0)])
def test_pipeline_equals_serial(z, rate, case):
    shape, pr, pc, t = case
    rng = np.random.default_rng(sum(shape) + rate)
    x = torch.from_numpy((250.0 + np.cumsum(rng.standard_normal(shape), axis=2) / 10).astype(np.float32)).cuda()
    plan = z.Plan.for_fields(x, pr, pc, t, 3)
    ref = _serial(z, plan, rate, x)
    for pieces in (1, 2, 3, 8, 100):
        pl = z.Pipeline(plan, rate, pieces)
        assert 1 <= pl.pieces <= min(pieces, max(pr, pc))
        nb = plan.buffer_bytes(rate)
        send = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        out = torch.full_like(x, float("nan"))
        for _ in range(2):                           # a second run over the same buffers
            pl.run(x, send, recv, out)
        torch.cuda.synchronize()
        assert torch.equal(send, ref[0]) and torch.equal(recv, ref[1]), pieces
        assert torch.equal(out.view(torch.int32), ref[2].view(torch.int32)), pieces
        pl.close()


def test_pipeline_t21_against_oracle(z):
    x = fieldgen.t21_field()
    xd = torch.from_numpy(x).cuda()
    plan = z.Plan.for_fields(xd, 2, 2, 0, 3)
    oplan = opl.Plan(64, 32, 8, 2, 2, 0, 3)
    for rate in (8, 16):
        pl = z.Pipeline(plan, rate, 2)
        assert pl.pieces == 2
        nb = plan.buffer_bytes(rate)
        send = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        out = torch.full_like(xd, float("nan"))
        pl.run(xd, send, recv, out)
        torch.cuda.synchronize()
        ref_send = op.pack(oplan, rate, x)
        ref_recv = op.permute(oplan, rate, ref_send)
        ref_out = np.full_like(x, np.nan)
        op.unpack(oplan, rate, ref_recv, ref_out)
        assert send.cpu().numpy().tobytes() == ref_send.tobytes()
        assert recv.cpu().numpy().tobytes() == ref_recv.tobytes()
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref_out.view(np.uint32))
        pl.close()


def test_pipeline_in_a_graph_and_after_other_work(z):
    # the pipeline's streams wait for what the caller's stream had enqueued, and a
    # capture of the run replays to the same result
    shape = (20, 48, 80)
    rng = np.random.default_rng(9)
    x = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    plan = z.Plan.for_fields(x, 2, 4, 0, 3)
    plan.prepare(8)
    ref = _serial(z, plan, 8, x)
    pl = z.Pipeline(plan, 8, 4)
    nb = plan.buffer_bytes(8)
    send = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    out = torch.full_like(x, float("nan"))
    s = torch.cuda.Stream()
    y = torch.zeros_like(x)
    with torch.cuda.stream(s):
        torch.cuda._sleep(20_000_000)                # the caller's earlier work: y <- x after a delay
        y.copy_(x)
        pl.run(y, send, recv, out, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), ref[2].view(torch.int32))
    out.fill_(float("nan"))
    recv.zero_()
    g = z.capture(lambda: pl.run(x, send, recv, out, stream=s), s)
    g.launch(s)
    torch.cuda.synchronize()
    assert torch.equal(recv, ref[1]) and torch.equal(out.view(torch.int32), ref[2].view(torch.int32))
    g.close()
    pl.close()


def test_pipeline_rejects_bad_arguments(z):
    x = torch.zeros((8, 16, 16), device="cuda")
    plan = z.Plan.for_fields(x, 2, 2, 0, 3)
    with pytest.raises(z.ZfpxError):
        z.Pipeline(plan, 12, 2)
    with pytest.raises(z.ZfpxError):
        z.Pipeline(plan, 8, 0)
    pl = z.Pipeline(plan, 8, 2)
    nb = plan.buffer_bytes(8)
    small = torch.zeros(nb - 16, dtype=torch.uint8, device="cuda")
    buf = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(z.ZfpxError):
        pl.run(x, small, buf, x.clone())
    with pytest.raises(z.ZfpxError):
        pl.run(x, buf, buf, x.clone())                # send and receive overlap
    pl.close()
