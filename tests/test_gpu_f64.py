"""GPU parity of the float64 fixed-rate codec (3-D blocks; the float64 fields
of Sec. III) through the C ABI against the CPU oracle: streams bit-exact,
decoded values bit-exact (sign of zero, subnormal results and overflow
included), on ragged and strided arrays, and the GPU decoder on the oracle's
own streams."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from oracle import codec as oc


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _gpu_roundtrip(z, rate, src):
    n = tuple(reversed(src.shape))
    nbytes = z.zfpx_stream_bytes_f64(rate, n)
    out = torch.full((nbytes + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    z.zfpx_encode_f64(rate, src, out[:nbytes])
    dec = torch.full(src.shape, float("nan"), dtype=torch.float64, device="cuda")
    z.zfpx_decode_f64(rate, out[:nbytes], dec)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert (o[nbytes:] == 0xA5).all()                       # nothing past the stream
    return o[:nbytes], dec.cpu().numpy()


def _check(z, rate, x, src):
    s, d = _gpu_roundtrip(z, rate, src)
    ref = oc.encode_array_f64(rate, x)
    assert s.tobytes() == ref.tobytes()
    rd = np.empty(x.shape, np.float64)
    oc.decode_array_f64(rate, ref, rd)
    assert d.view(np.uint64).tobytes() == rd.view(np.uint64).tobytes()


def _smooth(shape, seed, scale):
    rng = np.random.default_rng(seed)
    g = np.cumsum(np.cumsum(rng.standard_normal(shape), axis=2), axis=1)
    return (250.0 + g) * scale


@pytest.mark.parametrize("rate", [1, 4, 8, 16, 23, 32])
@pytest.mark.parametrize("shape", [(1, 1, 1), (4, 4, 4), (7, 5, 3), (9, 13, 22), (17, 26, 37)])
def test_small_arrays(z, shape, rate):
    x = _smooth(shape, sum(shape) + rate, 10.0 ** (rate - 16))
    _check(z, rate, x, torch.from_numpy(x).cuda())


def test_special_values_and_views(z):
    rng = np.random.default_rng(9)
    big = rng.standard_normal((12, 20, 44)) * 10.0 ** rng.integers(-300, 300, (12, 20, 44))
    big[0:4, 0:4, 0:4] = 0.0
    big[0:4, 4:8, 0:4] = -0.0
    big[0:4, 8:12, 0:4] = 3.25
    big[4:8, 0:4, 0:4] = 5e-310                                      # below 2^-1023: a zero block
    big[4:8, 4:8, 0:4] = rng.standard_normal((4, 4, 4)) * 3e-308      # subnormal results on decode
    big[4:8, 8:12, 0:4] = rng.uniform(-1.7, 1.7, (4, 4, 4)) * 1e308   # near the top exponent
    big[8:12, 0:4, 4:8] = 1.7e308                                     # may round up to inf
    big[5, 5, 9] = np.inf
    big[9, 9, 9] = np.nan
    big[10, 17, 30] = -np.inf
    x = big[1:11, 2:19, 3:41]                                         # unaligned, strided view
    src = torch.from_numpy(big).cuda()[1:11, 2:19, 3:41]
    for rate in (2, 8, 16, 32):
        _check(z, rate, big, torch.from_numpy(big).cuda())
        _check(z, rate, x, src)


def test_transposed_view(z):
    x = _smooth((20, 24, 28), 5, 1e-3)
    src = torch.from_numpy(x).cuda().permute(2, 0, 1)                 # x fastest is now the outer axis
    _check(z, 12, np.transpose(x, (2, 0, 1)), src)


@pytest.mark.parametrize("rate", [8, 16])
def test_gpu_decodes_the_oracle_stream(z, rate):
    x = _smooth((13, 30, 50), 11, 1e-200)
    ref = oc.encode_array_f64(rate, x)
    s = torch.from_numpy(ref).cuda()
    dec = torch.empty(x.shape, dtype=torch.float64, device="cuda")
    z.zfpx_decode_f64(rate, s, dec)
    torch.cuda.synchronize()
    rd = np.empty_like(x)
    oc.decode_array_f64(rate, ref, rd)
    assert dec.cpu().numpy().view(np.uint64).tobytes() == rd.view(np.uint64).tobytes()


def test_field_sized_case(z):
    # 40 levels of a 320 x 160 grid: 2M values, 32K blocks over many persistent units
    x = _smooth((40, 160, 320), 13, 1.0)
    _check(z, 16, x, torch.from_numpy(x).cuda())


def test_errors(z):
    x = torch.zeros((4, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    for bad in (0, 33):
        with pytest.raises(z.ZfpxError):
            z.zfpx_encode_f64(bad, x, out)
    with pytest.raises(z.ZfpxError):
        z.zfpx_encode_f64(16, x, out[:127])                          # one byte short
    with pytest.raises(z.ZfpxError):
        z.zfpx_decode_f64(16, out[:127], x)
    with pytest.raises(z.ZfpxError):
        z.zfpx_encode_f64(16, x, out[1:1 + 128])                     # misaligned stream
