"""GPU parity of the longitude transform (the FFT after the first
transposition, Sec. II-A/B) through the C ABI against the float64 oracle, and
the second transposition run in wavenumber space (Sec. II-B's lambda -> theta
all-to-all on the Fourier coefficients) against the codec oracle.

Tolerance.  The GPU computes in float32 with twiddles rounded once from
double: a radix-p Stockham stage is sqrt(p) times a unitary map and adds at
most about (p + 3) u of the norm of its input in rounding (u = 2^-24), so
over the log2 N levels of radix 2..5 stages plus the real split the error of
a row's coefficients stays below 16 log2(N) u ||F|| with ||F|| <= ||x|| /
sqrt(N) (Parseval for the 1/N-scaled transform).  The test takes that bound
per row."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

import fieldgen
from oracle import fourier as of
from oracle import codec as oc

U = 2.0 ** -24


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _gpu(z, src, K):
    nz, ny, _ = src.shape
    re = torch.full((nz, ny, K), float("nan"), device="cuda")
    im = torch.full((nz, ny, K), float("nan"), device="cuda")
    z.zfpx_rfft_lon(src, re, im)
    torch.cuda.synchronize()
    return re.cpu().numpy().astype(np.float64), im.cpu().numpy().astype(np.float64)


def _check(x, re, im, K):
    N = x.shape[-1]
    rre, rim = of.rfft_lon(x, K)
    err = np.sqrt((re - rre) ** 2 + (im - rim) ** 2).reshape(-1, K)
    rows = x.reshape(-1, N).astype(np.float64)
    bound = 16 * math.log2(N) * U * np.linalg.norm(rows, axis=1) / math.sqrt(N) + 1e-30
    row_err = np.linalg.norm(err, axis=1)
    assert np.all(row_err <= bound), float((row_err / bound).max())
    return float((row_err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("N", [2, 4, 6, 10, 12, 30, 40, 90, 160, 640, 1280, 2560, 8192])
def test_rows_match_the_oracle(z, N):
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((3, 5, N)) * 10.0 ** rng.uniform(-3, 3, (3, 5, 1))).astype(np.float32)
    for K in sorted({1, N // 2, N // 2 + 1}):
        re, im = _gpu(z, torch.from_numpy(x).cuda(), K)
        _check(x, re, im, K)


def test_special_rows(z):
    N = 1280
    lam = 2.0 * np.pi * np.arange(N) / N
    x = np.zeros((2, 4, N), np.float32)
    x[0, 0] = 3.5                                          # constant: F_0 = 3.5 only
    x[0, 2] = np.cos(7 * lam + 0.3)                        # a tone: F_7 = e^{0.3 i} / 2
    x[1, 1] = np.cos(np.pi * np.arange(N))                 # the Nyquist tone
    x[1, 3, 17] = 1.0                                      # an impulse: |F_m| = 1/N
    re, im = _gpu(z, torch.from_numpy(x).cuda(), N // 2 + 1)
    _check(x, re, im, N // 2 + 1)
    assert not np.isnan(re).any() and not re[0, 1].any() and not im[0, 1].any()   # the zero row
    assert abs(re[0, 0, 0] - 3.5) < 1e-6 and np.abs(re[0, 0, 1:]).max() < 1e-6
    assert abs(re[1, 1, N // 2] - 1.0) < 1e-6


def test_views(z):
    rng = np.random.default_rng(5)
    big = rng.standard_normal((9, 14, 2 * 640 + 6)).astype(np.float32)
    src = torch.from_numpy(big).cuda()[2:8, 1:13:2, 4:4 + 1280]       # even offsets and strides
    x = big[2:8, 1:13:2, 4:4 + 1280]
    K = 640
    store_re = torch.full((6, 6, K + 3), float("nan"), device="cuda")
    store_im = torch.full((6, 6, K + 3), float("nan"), device="cuda")
    re, im = store_re[:, :, 1:1 + K], store_im[:, :, 1:1 + K]
    z.zfpx_rfft_lon(src, re, im)
    torch.cuda.synchronize()
    _check(x, re.cpu().numpy().astype(np.float64), im.cpu().numpy().astype(np.float64), K)
    assert torch.isnan(store_re[:, :, 0]).all() and torch.isnan(store_re[:, :, 1 + K:]).all()


def test_benchmark_field_full_size(z):
    x = fieldgen.t639_field()                                          # 137 x 640 x 1280
    re, im = _gpu(z, torch.from_numpy(x).cuda(), 640)
    _check(x, re, im, 640)


def test_errors(z):
    ok = torch.zeros((2, 2, 16), device="cuda")
    out = torch.zeros((2, 2, 9), device="cuda")
    for shape in [(2, 2, 7), (2, 2, 14), (2, 2, 16386)]:                # odd N; N/2 = 7; N too large
        s = torch.zeros(shape, device="cuda")
        with pytest.raises(z.ZfpxError):
            z.zfpx_rfft_lon(s, torch.zeros((2, 2, 1), device="cuda"), torch.zeros((2, 2, 1), device="cuda"))
    with pytest.raises(z.ZfpxError):
        z.zfpx_rfft_lon(ok, torch.zeros((2, 2, 10), device="cuda"), torch.zeros((2, 2, 10), device="cuda"))  # K > N/2 + 1
    with pytest.raises(z.ZfpxError):
        z.zfpx_rfft_lon(ok.transpose(1, 2).contiguous().transpose(1, 2), out, out.clone())   # rows not contiguous
    with pytest.raises(z.ZfpxError):
        z.zfpx_rfft_lon(torch.zeros((2, 2, 17), device="cuda")[:, :, 1:], out, out.clone())  # rows off 8 bytes


# ------------------------------------------------- the second transposition in wavenumber space
@pytest.mark.parametrize("rate", [8, 16])
def test_second_transposition_on_wavenumber_fields(z, rate):
    """lambda -> theta on the wavenumber fields: each rank's pencil of F_m
    (real and imaginary parts as two [lev][lat][m] fields, split over m
    instead of longitude), compressed, moved and decompressed bit-exactly as
    the codec oracle codes the same boxes."""
    from oracle import plan as opl
    x = fieldgen.t21_field()                                          # 8 x 32 x 64
    K = x.shape[-1] // 2
    rre, rim = of.rfft_lon(x, K)
    for f in (rre.astype(np.float32), rim.astype(np.float32)):
        nz, ny, nx = f.shape
        fd = torch.from_numpy(f).cuda()
        plan = z.Plan.for_fields(fd, 2, 2, 1, 3)
        plan.prepare(rate)
        send = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
        out = torch.full_like(fd, float("nan"))
        z.zfpx_pack_compress(plan, rate, fd, send)
        z.zfpx_decompress_unpack(plan, rate, send, out, layout=z.LAYOUT_SEND)
        torch.cuda.synchronize()
        want = np.full_like(f, np.nan)
        for m in opl.Plan(nx, ny, nz, 2, 2, 1, 3).messages:
            if m.nx * m.ny * m.nz == 0:
                continue
            box = np.ascontiguousarray(f[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx])
            d = np.empty_like(box)
            oc.decode_array(3, rate, oc.encode_array(3, rate, box), d)
            want[m.z0:m.z0 + m.nz, m.y0:m.y0 + m.ny, m.x0:m.x0 + m.nx] = d
        assert out.cpu().numpy().view(np.uint32).tobytes() == want.view(np.uint32).tobytes()
        plan.close()
