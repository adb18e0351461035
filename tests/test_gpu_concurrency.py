"""The codec keeps no state on the device between launches: launches of one plan on
two streams at once, and every launch shape (units per warp), give the bytes and
values of an ordered single-stream run (which the parity tests tie to the oracle)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _field(shape, seed, offset=0.0):
    rng = np.random.default_rng(seed)
    f = offset + np.cumsum(rng.standard_normal(shape), axis=2) / 30.0
    return torch.from_numpy(f.astype(np.float32)).cuda()


@pytest.mark.parametrize("rate", [8, 16])
def test_two_streams_one_plan(z, rate):
    shape = (67, 256, 512)                       # 8.8 M values, ~2 ms of work per pair of launches
    xs = [_field(shape, 11, 0.0), _field(shape, 12, 250.0)]
    plan = z.Plan.for_fields(xs[0], 4, 4, 0, 3)
    plan.prepare(rate)
    nb = plan.buffer_bytes(rate)
    # ordered reference on one stream
    ref_b, ref_v = [], []
    for x in xs:
        b = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        v = torch.full_like(x, float("nan"))
        z.zfpx_pack_compress(plan, rate, x, b)
        z.zfpx_decompress_unpack(plan, rate, b, v, layout=z.LAYOUT_SEND)
        ref_b.append(b)
        ref_v.append(v)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    bufs = [torch.zeros(nb, dtype=torch.uint8, device="cuda") for _ in range(2)]
    outs = [torch.full_like(x, float("nan")) for x in xs]
    torch.cuda.synchronize()
    for _ in range(4):                           # the same plan, rate and direction on both streams at once
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                z.zfpx_pack_compress(plan, rate, xs[i], bufs[i])
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                z.zfpx_decompress_unpack(plan, rate, bufs[i], outs[i], layout=z.LAYOUT_SEND)
    torch.cuda.synchronize()
    for i in range(2):
        assert torch.equal(bufs[i], ref_b[i])
        assert torch.equal(outs[i].view(torch.int32), ref_v[i].view(torch.int32))


def test_units_per_warp_does_not_change_results(z):
    x = _field((37, 100, 212), 13, 5.0)
    plan = z.Plan.for_fields(x, 3, 2, 0, 3)
    try:
        for rate in (8, 16):
            nb = plan.buffer_bytes(rate)
            got = []
            for upw in (0, 1, 3, 64, 4096):
                z.zfpx_set_units_per_warp(True, rate, upw)
                z.zfpx_set_units_per_warp(False, rate, upw)
                assert z.zfpx_get_units_per_warp(True, rate) == (upw or z.zfpx_get_units_per_warp(True, rate))
                b = torch.zeros(nb, dtype=torch.uint8, device="cuda")
                v = torch.full_like(x, float("nan"))
                z.zfpx_pack_compress(plan, rate, x, b)
                z.zfpx_decompress_unpack(plan, rate, b, v, layout=z.LAYOUT_SEND)
                torch.cuda.synchronize()
                got.append((b, v))
            for b, v in got[1:]:
                assert torch.equal(b, got[0][0])
                assert torch.equal(v.view(torch.int32), got[0][1].view(torch.int32))
    finally:
        for rate in (8, 16):
            z.zfpx_set_units_per_warp(True, rate, 0)
            z.zfpx_set_units_per_warp(False, rate, 0)
    with pytest.raises(z.ZfpxError):
        z.zfpx_set_units_per_warp(True, 12, 1)
    with pytest.raises(z.ZfpxError):
        z.zfpx_set_units_per_warp(True, 8, 4097)


def test_autotuner_picks_a_candidate_and_results_stay(z):
    from paper_2609_24294_gb300 import autotune
    x = _field((37, 96, 200), 14, 2.0)
    plan = z.Plan.for_fields(x, 2, 2, 0, 3)
    try:
        for rate in (8, 16):
            nb = plan.buffer_bytes(rate)
            b0 = torch.zeros(nb, dtype=torch.uint8, device="cuda")
            z.zfpx_pack_compress(plan, rate, x, b0)
            b, v = torch.zeros_like(b0), torch.empty_like(x)
            choice, timings = autotune.tune_codec(plan, rate, x, b, v, candidates=(1, 2, 5), reps=1, use_cache=False)
            assert choice["encode"] in (1, 2, 5) and choice["decode"] in (1, 2, 5)
            assert set(timings) == {"encode", "decode"} and all(len(t) == 3 for t in timings.values())
            assert z.zfpx_get_units_per_warp(True, rate) == choice["encode"]
            b.zero_()
            z.zfpx_pack_compress(plan, rate, x, b)
            torch.cuda.synchronize()
            assert torch.equal(b, b0)
    finally:
        for rate in (8, 16):
            z.zfpx_set_units_per_warp(True, rate, 0)
            z.zfpx_set_units_per_warp(False, rate, 0)
