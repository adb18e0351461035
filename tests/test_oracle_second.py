"""The C oracle against a second, independent plain-Python reference
(tests/zfp_prose.py): the same readings of Sec. II-C written twice, in
different ways, must give the same bytes and the same floats."""
import numpy as np
import pytest

import fieldgen
from oracle import codec as oc

import zfp_prose as zp


def _check(dims, rate, a):
    ref = oc.encode_array(dims, rate, a)
    got = zp.encode_array(dims, rate, a)
    assert got[:ref.size].tobytes() == ref.tobytes()
    assert not got[ref.size:].any()                       # only whole-word padding differs
    dec = np.empty_like(a)
    oc.decode_array(dims, rate, ref, dec)
    back = zp.decode_array(dims, rate, ref, a.shape)
    assert back.view(np.uint32).tobytes() == dec.view(np.uint32).tobytes()


@pytest.mark.parametrize("dims,rate", [(3, 16), (3, 8), (1, 16), (1, 8)])
def test_t21_field(dims, rate):
    x = fieldgen.t21_field()
    part = x[:, :, :32] if dims == 3 else x[:2]           # keep the pure-Python side fast
    _check(dims, rate, np.ascontiguousarray(part))


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 7), (5, 6, 9), (2, 3, 13)])
@pytest.mark.parametrize("rate", [4, 8, 13, 16, 24])
def test_small_odd_arrays(shape, rate):
    rng = np.random.default_rng(sum(shape) * 31 + rate)
    a = (rng.standard_normal(shape) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
    for dims in (3, 1):
        _check(dims, rate, a)


def test_special_blocks():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((4, 4, 28)).astype(np.float32)
    a[:, :, 0:4] = 0.0
    a[:, :, 4:8] = 3.25
    a[:, :, 8:12] = np.float32(2e-39)                     # subnormal, above 2^-127
    a[:, :, 12:16] = np.float32(5e-40)                    # subnormal, below 2^-127
    a[:, :, 16:20] *= np.float32(1e37)
    a[1, 1, 21] = np.inf
    a[:, :, 24:28] = fieldgen.graded_blocks(1, 3)
    for rate in (8, 16):
        _check(3, rate, a)


def test_near_lossless_rate_reaches_the_last_planes():
    # at rate 32 a 3-D block codes every plane but part of the last, so the
    # transforms' low bits show in the stream
    rng = np.random.default_rng(9)
    a = (rng.standard_normal((4, 8, 8)) * 7.0).astype(np.float32)
    _check(3, 32, a)
    _check(1, 32, a[:1, :2])


def test_transform_order_and_negabinary_pieces():
    rng = np.random.default_rng(10)
    for _ in range(2000):
        v = [int(t) for t in rng.integers(-(1 << 30), 1 << 30, 4)]
        assert zp._fwd4(v) == [int(t) for t in oc.lift_forward(v)]
        assert zp._inv4(v) == [int(t) for t in oc.lift_inverse(v)]
    q = rng.integers(-(1 << 30), 1 << 30, 64).astype(np.int32)
    ours = [int(t) for t in q]
    for axis in zp._lines(3):
        for line in axis:
            out = zp._fwd4([ours[t] for t in line])
            for t, val in zip(line, out):
                ours[t] = val
    assert ours == [int(t) for t in oc.xform_forward(3, q)]
    assert zp._order(3) == [int(t) for t in oc.sequency_order(3)]
