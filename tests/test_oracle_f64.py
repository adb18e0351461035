"""Pins of the oracle's float64 codec (3-D blocks; the paper cites float64
CAMS fields, Sec. III): the same method with the double format's sizes.  The
int64 transform is tied to the pinned int32 one, the stream to budget and
embedding invariants, the reconstruction to a near-lossless bound, and every
bit to the plain-Python second statement."""
import numpy as np
import pytest

import fieldgen
from oracle import codec

import zfp_prose as zp


def _smooth(shape, seed, scale=1.0, offset=0.0):
    rng = np.random.default_rng(seed)
    g = np.cumsum(np.cumsum(rng.standard_normal(shape), axis=2), axis=1)
    return (offset + scale * g).astype(np.float64)


def test_int64_transform_agrees_with_the_pinned_int32_transform():
    rng = np.random.default_rng(61)
    for _ in range(500):
        q = rng.integers(-2 ** 29, 2 ** 29, 64)
        f32 = codec.xform_forward(3, q.astype(np.int32)).astype(np.int64)
        np.testing.assert_array_equal(codec.xform_forward_i64(q), f32)
        # the inverse on transformed blocks (whose inverse stays inside int32)
        i32 = codec.xform_inverse(3, f32.astype(np.int32)).astype(np.int64)
        np.testing.assert_array_equal(codec.xform_inverse_i64(f32), i32)


def test_int64_transform_no_overflow_below_2_62():
    rng = np.random.default_rng(62)
    codec.overflow_reset()
    for _ in range(300):
        q = rng.integers(-2 ** 62 + 1, 2 ** 62, 64)
        q[rng.random(64) < 0.3] = rng.choice([-(2 ** 62) + 1, 2 ** 62 - 1])
        codec.xform_inverse_i64(codec.xform_forward_i64(q))
    assert codec.overflow_count() == 0


def test_special_blocks_and_budget():
    rng = np.random.default_rng(63)
    for v in [np.zeros(64), -np.zeros(64), np.full(64, 1e-309), np.full(64, np.inf)]:
        s = codec.encode_block_f64(16, v)
        assert not s.any() and not codec.decode_block_f64(16, s).any()
    for c in [1.0, -0.5, 250.0, 1e300, np.pi, 2.0 ** -1000]:
        v = np.full(64, c)
        for r in (4, 8, 16, 32):
            np.testing.assert_array_equal(codec.decode_block_f64(r, codec.encode_block_f64(r, v)), v)
    for r in range(1, 65):
        v = rng.standard_normal(64)
        s = codec.encode_block_f64(r, v)
        assert s.size == 8 * r
    assert codec.stream_bytes_f64(16, (9, 6, 5)) == 3 * 2 * 2 * 8 * 16


def test_embedded_prefix_and_error_monotone():
    rng = np.random.default_rng(64)
    rates = [2, 4, 8, 16, 24, 32, 48, 64]
    for _ in range(100):
        v = np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-100, 100)
        st = {r: np.unpackbits(codec.encode_block_f64(r, v), bitorder="little") for r in rates}
        for a, b in zip(rates, rates[1:]):
            np.testing.assert_array_equal(st[a][:64 * a], st[b][:64 * b][:64 * a])
    x = _smooth((8, 16, 24), 65, offset=250.0)
    prev = np.inf
    for r in (4, 8, 12, 16, 24, 32, 48):
        out = np.empty_like(x)
        codec.decode_array_f64(r, codec.encode_array_f64(r, x), out)
        e = np.linalg.norm(out - x) / np.linalg.norm(x)
        assert e <= prev
        prev = e
    assert prev < 1e-12


def test_rate64_near_lossless_bound():
    # every plane coded: truncation to a 62-bit integer (< 1 unit of 2^(emax-62)),
    # the transform round trip (<= 38 units, as for the int32 transform) and the
    # final rounding to float64 (half an ulp of the result)
    rng = np.random.default_rng(66)
    for _ in range(300):
        v = np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-50, 50)
        emax = np.frexp(np.max(np.abs(v)))[1]
        d = codec.decode_block_f64(64, codec.encode_block_f64(64, v))
        unit = 2.0 ** (emax - 62)
        assert np.all(np.abs(d - v) <= 39 * unit + np.spacing(np.abs(d)) / 2)


def test_partial_blocks_are_edge_replicated():
    x = _smooth((5, 6, 9), 67)
    p = np.pad(x, ((0, 3), (0, 2), (0, 3)), mode="edge")
    for r in (8, 16):
        assert codec.encode_array_f64(r, x).tobytes() == codec.encode_array_f64(r, p).tobytes()


@pytest.mark.parametrize("rate", [4, 16, 33, 64])
def test_second_statement_agrees(rate):
    rng = np.random.default_rng(68 + rate)
    blocks = [np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-300, 300) for _ in range(6)]
    blocks += [np.full(64, 250.0), np.zeros(64), np.full(64, 3e-308) * rng.standard_normal(64),
               fieldgen.t21_field()[:4, :4, :4].astype(np.float64).reshape(-1)]
    for v in blocks:
        ref = codec.encode_block_f64(rate, v)
        bits = zp.encode_block_f64(rate, v)
        assert np.packbits(np.array(bits, np.uint8), bitorder="little").tobytes() == ref.tobytes()
        d = codec.decode_block_f64(rate, ref)
        assert zp.decode_block_f64(rate, bits).tobytes() == d.tobytes()
