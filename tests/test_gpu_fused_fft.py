"""Decompression fused with the longitude FFT (Sec. II-A; Sec. VI): the received
streams of a z -> lambda transposition go straight to wavenumbers.  The result
must equal, bit for bit, decompress+unpack followed by the longitude FFT on the
GPU, and it must sit within the FFT's float32 bound of the float64 oracle's
transform of the oracle-decoded field (the bound of tests/test_gpu_fourier.py)."""
import math

import numpy as np
import pytest
import torch

import fieldgen
from oracle import fourier as of
from oracle import packs as op
from oracle import plan as opl

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _both(z, plan, rate, xd, K):
    nb = plan.buffer_bytes(rate)
    recv = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    z.zfpx_pack_compress(plan, rate, xd, recv, z.LAYOUT_RECV)
    nz, ny, _ = xd.shape
    re = torch.full((nz, ny, K), float("nan"), device="cuda")
    im = torch.full_like(re, float("nan"))
    work = z.zfpx_decompress_rfft(plan, rate, recv, re, im)
    dec = torch.full_like(xd, float("nan"))
    z.zfpx_decompress_unpack(plan, rate, recv, dec)
    sre, sim = torch.full_like(re, float("nan")), torch.full_like(im, float("nan"))
    z.zfpx_rfft_lon(dec, sre, sim)
    # a second call over the same workspace gives the same values
    re2, im2 = torch.full_like(re, float("nan")), torch.full_like(im, float("nan"))
    z.zfpx_decompress_rfft(plan, rate, recv, re2, im2, work=work)
    torch.cuda.synchronize()
    assert torch.equal(re.view(torch.int32), re2.view(torch.int32)) and torch.equal(im.view(torch.int32), im2.view(torch.int32))
    return recv, re, im, sre, sim


def _same(a, b):
    assert torch.equal(a.view(torch.int32), b.view(torch.int32)), int((a.view(torch.int32) != b.view(torch.int32)).sum())


@pytest.mark.parametrize("rate", [16, 8])
def test_t21_field_against_the_oracle(z, rate):
    x = fieldgen.t21_field()                                 # [8 lev][32 lat][64 lon]
    xd = torch.from_numpy(x).cuda()
    nz, ny, nx = x.shape
    plan = z.Plan.for_fields(xd, 2, 2, 0, 3)
    K = 22
    recv, re, im, sre, sim = _both(z, plan, rate, xd, K)
    _same(re, sre)
    _same(im, sim)
    # the oracle: its transposition of the field, then its float64 transform
    oplan = opl.Plan(nx, ny, nz, 2, 2, 0, 3)
    assert recv.cpu().numpy().tobytes() == op.permute(oplan, rate, op.pack(oplan, rate, x)).tobytes()
    dec = np.full_like(x, np.nan)
    op.unpack(oplan, rate, op.permute(oplan, rate, op.pack(oplan, rate, x)), dec)
    rre, rim = of.rfft_lon(dec, K)
    err = np.sqrt((re.cpu().numpy() - rre) ** 2 + (im.cpu().numpy() - rim) ** 2).reshape(-1, K)
    rows = dec.reshape(-1, nx).astype(np.float64)
    bound = 16 * math.log2(nx) * U * np.linalg.norm(rows, axis=1) / math.sqrt(nx) + 1e-30
    assert np.all(np.linalg.norm(err, axis=1) <= bound)


@pytest.mark.parametrize("shape,pr,pc,K", [((37, 30, 96), 2, 3, 49), ((9, 20, 60), 3, 2, 31), ((5, 12, 40), 1, 1, 7)])
def test_odd_shapes_equal_the_separate_path(z, shape, pr, pc, K):
    rng = np.random.default_rng(sum(shape))
    x = (np.cumsum(rng.standard_normal(shape), axis=2) / 10 + 5.0).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    plan = z.Plan.for_fields(xd, pr, pc, 0, 3)
    for rate in (8, 16):
        _, re, im, sre, sim = _both(z, plan, rate, xd, K)
        _same(re, sre)
        _same(im, sim)


def test_benchmark_field_equals_the_separate_path(z):
    x = fieldgen.t639_field()                                # 1280 x 640 x 137
    xd = torch.from_numpy(x).cuda()
    plan = z.Plan.for_fields(xd, 8, 8, 0, 3)
    for rate in (8, 16):
        _, re, im, sre, sim = _both(z, plan, rate, xd, 640)
        _same(re, sre)
        _same(im, sim)


def test_rejects_other_plans(z):
    x = torch.zeros((8, 16, 16), device="cuda")
    plan = z.Plan.for_fields(x, 2, 2, 1, 3)                  # lambda -> theta: rows are not longitude rows
    recv = torch.zeros(plan.buffer_bytes(8), dtype=torch.uint8, device="cuda")
    re = torch.zeros((8, 16, 8), device="cuda")
    with pytest.raises(z.ZfpxError):
        z.zfpx_decompress_rfft(plan, 8, recv, re, re.clone())
    plan0 = z.Plan.for_fields(x, 2, 2, 0, 3)
    with pytest.raises(z.ZfpxError):
        z.zfpx_decompress_rfft(plan0, 12, recv, re, re.clone())
