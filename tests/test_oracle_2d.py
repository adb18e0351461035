"""Pins of the oracle's 2-D blocks (4 x 4 values of one level, for single-level
fields): the same method as the 3-D blocks (Sec. II-C; Lindstrom 2014) with
two transform axes and 16 coefficients.  Each pin ties the 2-D code to
something fixed independently of it: the already pinned 3-D transform and
order, the published matrix, numpy edge padding, the budget arithmetic, and
the plain-Python second statement of the method (tests/zfp_prose.py)."""
import numpy as np
import pytest

import fieldgen
from oracle import codec

import zfp_prose as zp

M = np.array([[4, 4, 4, 4], [5, 1, -1, -5], [-4, 4, 4, -4], [-2, 6, -6, 2]]) / 16.0


def test_order_is_the_3d_order_restricted_to_one_level():
    o3 = [int(t) for t in codec.sequency_order(3) if t < 16]    # k = 0 coefficients, in 3-D order
    o2 = [int(t) for t in codec.sequency_order(2)]
    assert o2 == o3
    assert sorted(o2) == list(range(16))
    seq = [(t & 3) + (t >> 2) for t in o2]
    assert seq == sorted(seq)
    assert [seq.count(s) for s in range(7)] == [1, 2, 3, 4, 3, 2, 1]


def test_transform_is_a_slice_of_the_3d_transform():
    # A 3-D block constant along k is one 2-D block repeated; the integer lift
    # maps a constant line (c, c, c, c) to exactly (c, 0, 0, 0), so the 3-D
    # transform holds the 2-D transform in slice k = 0 and zeros elsewhere.
    rng = np.random.default_rng(21)
    for _ in range(2000):
        q2 = rng.integers(-2 ** 29, 2 ** 29, 16).astype(np.int32)
        q3 = np.tile(q2, 4)
        f3 = codec.xform_forward(3, q3)
        np.testing.assert_array_equal(f3[:16], codec.xform_forward(2, q2))
        assert not f3[16:].any()
        i3 = codec.xform_inverse(3, np.concatenate([q2, np.zeros(48, np.int32)]))
        i2 = codec.xform_inverse(2, q2)
        for k in range(4):
            np.testing.assert_array_equal(i3[16 * k:16 * (k + 1)], i2)


def test_transform_close_to_the_separable_matrix():
    # integer lifting = M (x) M up to the floor halvings: impulses scaled by 2^20
    for idx in range(16):
        q = np.zeros(16, np.int32)
        q[idx] = 1 << 20
        got = codec.xform_forward(2, q).astype(np.float64).reshape(4, 4)     # [j][i]
        want = (M @ q.astype(np.float64).reshape(4, 4).T @ M.T).T            # rows along i, then j
        assert np.max(np.abs(got - want)) <= 4.0


def test_zero_constant_and_budget():
    rng = np.random.default_rng(22)
    for v in [np.zeros(16), np.full(16, 1e-40), -np.zeros(16)]:
        s = codec.encode_block(2, 8, np.asarray(v, np.float32))
        assert not s.any() and not codec.decode_block(2, 8, s).any()
    # a constant codes into at most 2 bits per plane after its first: 65 < 16 r - 9 for r >= 5
    for c in [1.0, -0.5, 250.0, 3.0e38, np.float32(np.pi)] + list(rng.standard_normal(100) * 1e5):
        v = np.full(16, c, dtype=np.float32)
        for r in (6, 8, 16, 32):
            np.testing.assert_array_equal(codec.decode_block(2, r, codec.encode_block(2, r, v)), v)
    for r in range(1, 33):
        v = rng.standard_normal(16).astype(np.float32)
        s = codec.encode_block(2, r, v)
        assert s.size == 2 * r
        assert codec.stream_bytes(2, r, (9, 6, 3)) == 3 * 2 * 3 * 2 * r      # 3 x 2 blocks per level, 3 levels


def test_embedded_prefix_property():
    rng = np.random.default_rng(23)
    rates = [1, 2, 4, 8, 12, 16, 24, 32]
    for _ in range(200):
        v = (np.cumsum(rng.standard_normal(16)) * 10.0 ** rng.uniform(-5, 5)).astype(np.float32)
        streams = {r: np.unpackbits(codec.encode_block(2, r, v), bitorder="little") for r in rates}
        for a, b in zip(rates, rates[1:]):
            np.testing.assert_array_equal(streams[a][:16 * a], streams[b][:16 * a])


def test_partial_blocks_and_raster_order():
    rng = np.random.default_rng(24)
    for shape in [(3, 5, 7), (1, 1, 1), (2, 8, 12), (4, 6, 17)]:
        a = rng.standard_normal(shape).astype(np.float32)
        nz, ny, nx = shape
        padded = np.pad(a, ((0, 0), (0, (-ny) % 4), (0, (-nx) % 4)), mode="edge")
        for r in (8, 16):
            s = codec.encode_array(2, r, a)
            assert s.tobytes() == codec.encode_array(2, r, padded).tobytes()
            # block (bx, by) of level z is block number bx + BX (by + BY z)
            BY, BX = padded.shape[1] // 4, padded.shape[2] // 4
            for z in range(nz):
                for by in range(BY):
                    for bx in range(BX):
                        b = bx + BX * (by + BY * z)
                        blk = padded[z, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
                        assert s[2 * r * b:2 * r * (b + 1)].tobytes() == codec.encode_block(2, r, blk).tobytes()
            out = np.full(shape, np.nan, dtype=np.float32)
            codec.decode_array(2, r, s, out)
            full = np.full(padded.shape, np.nan, dtype=np.float32)
            codec.decode_array(2, r, s, full)
            np.testing.assert_array_equal(out, full[:, :ny, :nx])


def test_error_non_increasing_with_rate_and_better_than_1d():
    f = fieldgen.t21_field()
    for g in (f, fieldgen.temperature_like(f)):
        x = g.astype(np.float64)
        prev = np.inf
        for r in (4, 6, 8, 12, 16, 24, 32):
            out = np.empty_like(g)
            codec.decode_array(2, r, codec.encode_array(2, r, g), out)
            err = np.linalg.norm(out - x) / np.linalg.norm(x)
            assert err <= prev, r
            prev = err
            if r in (8, 16):
                o1 = np.empty_like(g)
                codec.decode_array(1, r, codec.encode_array(1, r, g), o1)
                assert err < np.linalg.norm(o1 - x) / np.linalg.norm(x)     # two decorrelated axes beat one
        assert prev < 1e-6


@pytest.mark.parametrize("rate", [4, 8, 13, 16, 32])
def test_second_statement_agrees(rate):
    rng = np.random.default_rng(25 + rate)
    arrays = [np.ascontiguousarray(fieldgen.t21_field()[:2, :16, :32])]
    arrays += [(rng.standard_normal(s) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
               for s in [(1, 1, 1), (2, 5, 7), (3, 6, 9)]]
    arrays += [np.full((1, 4, 4), 250.0, np.float32), np.zeros((1, 3, 5), np.float32)]
    for a in arrays:
        ref = codec.encode_array(2, rate, a)
        got = zp.encode_array(2, rate, a)
        assert got[:ref.size].tobytes() == ref.tobytes() and not got[ref.size:].any()
        dec = np.empty_like(a)
        codec.decode_array(2, rate, ref, dec)
        assert zp.decode_array(2, rate, ref, a.shape).view(np.uint32).tobytes() == dec.view(np.uint32).tobytes()
