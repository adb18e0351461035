"""Pins of the oracle's block transform, ordering and negabinary steps.

The decorrelating transform is the published non-orthogonal 4-point
transform of ZFP (Lindstrom 2014, the method the paper uses in Sec. II-C):
(1/16) [[4,4,4,4],[5,1,-1,-5],[-4,4,4,-4],[-2,6,-6,2]] applied separably.
"""
import itertools

import numpy as np
import pytest

from oracle import codec

# The published transform matrix (Lindstrom 2014), typed from the paper, not
# from the oracle.
M = np.array([[4, 4, 4, 4], [5, 1, -1, -5], [-4, 4, 4, -4], [-2, 6, -6, 2]], dtype=np.float64) / 16.0


def test_exact_lifting_equals_published_matrix():
    # With exact halving, the oracle's five lifting steps must be M exactly.
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1.0
        np.testing.assert_array_equal(codec.lift_forward_exact(e), M[:, i])
    rng = np.random.default_rng(0)
    for _ in range(200):
        v = rng.integers(-1000, 1000, 4).astype(np.float64)
        np.testing.assert_allclose(codec.lift_forward_exact(v), M @ v, rtol=0, atol=1e-12)


def test_exact_inverse_lifting_inverts_matrix():
    Minv = np.linalg.inv(M)
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1.0
        np.testing.assert_allclose(codec.lift_inverse_exact(e), Minv[:, i], rtol=0, atol=1e-12)


def test_integer_lifting_brute_force_bounds():
    # All 17^4 integer vectors in [-8, 8]^4: the floor-halving integer lifting
    # stays within 1.5 of M v, and inverse(forward(v)) within 2 of v (bounds
    # found by this brute force and frozen).
    worst_fwd = 0.0
    worst_rt = 0
    for v in itertools.product(range(-8, 9), repeat=4):
        f = codec.lift_forward(v)
        worst_fwd = max(worst_fwd, float(np.abs(f - M @ np.array(v, dtype=np.float64)).max()))
        r = codec.lift_inverse(f)
        worst_rt = max(worst_rt, int(np.abs(r.astype(np.int64) - np.array(v)).max()))
    assert worst_fwd <= 1.5
    assert worst_rt <= 2


def test_integer_lifting_large_values_no_overflow():
    rng = np.random.default_rng(1)
    codec.overflow_reset()
    lim = 2 ** 30 - 1
    cases = [np.full(64, lim), np.full(64, -lim), np.tile([lim, -lim], 32),
             np.tile([lim, lim, -lim, -lim], 16), np.tile([-lim, lim, lim, -lim], 16)]
    cases += [rng.integers(-lim, lim + 1, 64) for _ in range(2000)]
    cases += [rng.choice([-lim, lim, 0], 64) for _ in range(2000)]
    for q in cases:
        f = codec.xform_forward(3, q.astype(np.int32))
        codec.xform_inverse(3, f)
        g = codec.xform_forward(1, q[:4].astype(np.int32))
        codec.xform_inverse(1, g)
    assert codec.overflow_count() == 0


def test_constant_block_transforms_to_dc_only():
    for c in [0, 1, -1, 12345, -(2 ** 29), 2 ** 30 - 1]:
        f = codec.xform_forward(3, np.full(64, c, dtype=np.int32))
        assert f[0] == c and np.all(f[1:] == 0)
        f1 = codec.xform_forward(1, np.full(4, c, dtype=np.int32))
        assert f1[0] == c and np.all(f1[1:] == 0)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_3d_transform_axis_order_and_strides(axis):
    # A block that varies along one axis only: the 3-D transform must equal
    # the 1-D integer transform of that profile, placed on that axis, with all
    # other coefficients zero (constant lines map to (c,0,0,0) exactly).
    rng = np.random.default_rng(2 + axis)
    prof = rng.integers(-(2 ** 20), 2 ** 20, 4).astype(np.int32)
    q = np.zeros((4, 4, 4), dtype=np.int32)        # [k][j][i]
    for t in range(4):
        if axis == 0:
            q[:, :, t] = prof[t]
        elif axis == 1:
            q[:, t, :] = prof[t]
        else:
            q[t, :, :] = prof[t]
    f = codec.xform_forward(3, q.reshape(-1)).reshape(4, 4, 4)
    ref = codec.lift_forward(prof)
    expect = np.zeros((4, 4, 4), dtype=np.int64)
    for t in range(4):
        if axis == 0:
            expect[0, 0, t] = ref[t]
        elif axis == 1:
            expect[0, t, 0] = ref[t]
        else:
            expect[t, 0, 0] = ref[t]
    np.testing.assert_array_equal(f, expect)
    back = codec.xform_inverse(3, f.reshape(-1)).reshape(4, 4, 4)
    assert np.abs(back.astype(np.int64) - q).max() <= 2


def test_3d_round_trip_bound():
    rng = np.random.default_rng(7)
    worst = 0
    for _ in range(3000):
        q = rng.integers(-(2 ** 29), 2 ** 29, 64).astype(np.int32)
        r = codec.xform_inverse(3, codec.xform_forward(3, q))
        worst = max(worst, int(np.abs(r.astype(np.int64) - q).max()))
    # each 1-D round trip is within 2, and the later inverse passes carry an
    # earlier pass's error through M^-1 (row sums of |M^-1| reach 3.75):
    # 2 + 3.75 * (2 + 3.75 * 2) = 37.6 bounds it (25 observed).
    assert worst <= 38


def test_sequency_order_properties():
    o = codec.sequency_order(3)
    assert sorted(o.tolist()) == list(range(64))
    i, j, k = o & 3, (o >> 2) & 3, o >> 4
    seq = i + j + k
    assert np.all(np.diff(seq) >= 0)
    # number of (i,j,k) in [0,3]^3 with i+j+k = s
    counts = [int(np.sum(seq == s)) for s in range(10)]
    assert counts == [1, 3, 6, 10, 12, 12, 10, 6, 3, 1]
    sq = i * i + j * j + k * k
    for s in range(10):
        sel = seq == s
        assert np.all(np.diff(sq[sel]) >= 0)
    assert o[0] == 0 and o[-1] == 63
    np.testing.assert_array_equal(codec.sequency_order(1), [0, 1, 2, 3])


def _negabinary_value(u):
    return sum(((u >> k) & 1) * (-2) ** k for k in range(32))


def test_negabinary_digit_weights():
    rng = np.random.default_rng(3)
    qs = [0, 1, -1, 2, -2, 3, 2 ** 29, -(2 ** 29), 2 ** 30 - 1, -(2 ** 30) + 1]
    qs += [int(x) for x in rng.integers(-(2 ** 31) + 1, 2 ** 30, 5000)]
    lo = -sum(2 ** k for k in range(1, 32, 2))     # most negative 32-digit negabinary
    hi = sum(2 ** k for k in range(0, 32, 2))
    for q in qs:
        if not (lo <= q <= hi):
            continue
        u = codec.to_negabinary(q)
        assert _negabinary_value(u) == q
        assert codec.from_negabinary(u) == q


def test_negabinary_bijection_sample():
    rng = np.random.default_rng(4)
    for u in list(range(0, 1 << 12)) + [int(x) for x in rng.integers(0, 2 ** 32, 20000, dtype=np.uint64)]:
        q = codec.from_negabinary(u)
        assert codec.to_negabinary(q) == u
