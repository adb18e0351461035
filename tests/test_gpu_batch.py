"""Batched ragged-row fields in one persistent launch against the oracle
(ZFP fixed rate, Sec. II-C, on an octahedral reduced Gaussian grid)."""
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


SPECS = [(9, "temperature", 3, 8), (6, "power", 3, 16), (1, "humidity", 1, 8), (5, "humidity", 3, 8),
         (2, "power", 1, 16), (3, "temperature", 3, 16)]


# (grid N, warps per CTA, CTAs per SM, 1-D blocks per lane, units per claim); one CTA per SM on the
# N = 96 grid gives fewer warps than work units, so warps claim their units from the queues
@pytest.mark.parametrize("N,warps,ctas,lb1,upc", [(6, 4, 0, 8, 4), (13, 8, 0, 8, 1), (13, 4, 0, 1, 3),
                                                  (13, 4, 0, 3, 64), (6, 8, 0, 64, 2), (13, 2, 0, 16, 4),
                                                  (96, 2, 1, 4, 3), (96, 3, 1, 1, 1), (96, 2, 1, 2, 8)])
def test_batch_matches_oracle(z, N, warps, ctas, lb1, upc):
    lens = og.row_lengths(N)
    if N == 13:
        lens = lens[:-2]                         # a partial last row-quad
    npts = int(lens.sum())
    host, srcs, dsts, specs = [], [], [], []
    for i, (nlev, kind, dims, rate) in enumerate(SPECS):
        full = og.octahedral_field(N, nlev, 100 + i, kind=kind)
        f = full[:, :npts].contiguous().numpy()
        host.append(f)
        srcs.append(torch.from_numpy(f).cuda())
        dsts.append(torch.full_like(srcs[-1], float("nan")))
        specs.append((nlev, dims, rate))
    b = z.Batch(lens, [(s, d, dims, rate) for s, d, (_, dims, rate) in zip(srcs, dsts, specs)])
    b.set_launch(warps, ctas)
    b.set_unit_blocks(lb1)                      # 1-D blocks per lane of a work unit
    b.set_claim_units(upc)                      # work units per claim
    ref = ob.encode_batch(host, lens, specs)
    assert b.nbytes() == ref.size
    out = torch.zeros(b.nbytes(), dtype=torch.uint8, device="cuda")
    before = z.zfpx_launch_count()
    b.encode(out)
    torch.cuda.synchronize()
    assert z.zfpx_launch_count() - before == 1          # one launch for every field
    got = out.cpu().numpy()
    offs, _ = ob.layout(lens, specs)
    for i, o in enumerate(offs):
        assert b.field_offset(i) == o
        nb = ob.field_bytes(lens, *specs[i])
        assert got[o:o + nb].tobytes() == ref[o:o + nb].tobytes(), "field %d" % i
    b.decode(out)
    torch.cuda.synchronize()
    for i, (nlev, dims, rate) in enumerate(specs):
        o = offs[i]
        nb = ob.field_bytes(lens, nlev, dims, rate)
        rdec = ob.decode_field(ref[o:o + nb], host[i].shape, lens, dims, rate)
        assert np.array_equal(dsts[i].cpu().numpy().view(np.uint32), rdec.view(np.uint32)), "field %d" % i


def test_batch_graph_capture(z):
    lens = og.row_lengths(8)
    f = og.octahedral_field(8, 7, 3, kind="temperature").cuda()
    g1 = og.octahedral_field(8, 1, 4).cuda()
    d = torch.zeros_like(f)
    d1 = torch.zeros_like(g1)
    b = z.Batch(lens, [(f, d, 3, 16), (g1, d1, 1, 8)])
    out = torch.zeros(b.nbytes(), dtype=torch.uint8, device="cuda")
    b.encode(out)
    b.decode(out)
    torch.cuda.synchronize()
    ref_out, ref_d = out.clone(), d.clone()
    out.zero_()
    d.zero_()
    s = torch.cuda.Stream()
    graph = z.capture(lambda: (b.encode(out, s), b.decode(out, s)), s)
    assert graph.num_kernels() == 2
    assert out.abs().sum().item() == 0                  # recorded, not run
    graph.launch(s)
    s.synchronize()
    assert torch.equal(out, ref_out) and torch.equal(d, ref_d)
