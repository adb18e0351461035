"""Pins of the oracle's embedded coder and block/array codec.

ZFP fixed-rate mode (paper Sec. II-C, Sec. IV-B): every 4^d block takes
exactly 4^d * r bits; the coder sends bit planes from the most significant
down with group testing and stops at the budget (Lindstrom 2014).
"""
import os
import re

import numpy as np
import pytest

from oracle import codec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_blocks.txt")


# ------------------------------------------------------------------ plane cost
def closed_form_plane_cost(S, X, n):
    """Bits one plane costs and the new n, from counting alone:
    n verbatim bits; then per set bit p >= n: one group bit plus the bits
    n..p (the last coefficient's bit is implied); a final 0 group bit when
    coefficients remain."""
    if n >= S:
        return S, S
    rest = X >> n
    c = bin(rest).count("1")
    if c == 0:
        return n + 1, n
    j = rest.bit_length() - 1 + n
    cost = j + 1 + c + (1 if j < S - 1 else 0) - (1 if j == S - 1 else 0)
    return cost, j + 1


@pytest.mark.parametrize("S", [4, 16, 64])
def test_plane_cost_matches_closed_form(S):
    rng = np.random.default_rng(S)
    for trial in range(20000):
        density = rng.choice([0.02, 0.1, 0.5, 0.9])
        bits = rng.random(S) < density
        X = int(sum(1 << i for i in range(S) if bits[i]))
        n = int(rng.integers(0, S + 1))
        got_bits, got_n = codec.plane_bits(S, X, n)
        exp_bits, exp_n = closed_form_plane_cost(S, X, n)
        assert (got_bits, got_n) == (exp_bits, exp_n), (S, hex(X), n)


def _plane(u, k):
    return int(sum(((int(u[i]) >> k) & 1) << i for i in range(len(u))))


def _random_coeffs(rng, S):
    # magnitudes falling with index, like transformed smooth data
    scale = 2.0 ** (29 - 0.4 * np.arange(S) * (64 / S) * rng.uniform(0.2, 1.0))
    q = (rng.standard_normal(S) * scale).astype(np.int64)
    q = np.clip(q, -(2 ** 30) + 1, 2 ** 30 - 1)
    return np.array([codec.to_negabinary(int(v)) for v in q], dtype=np.uint32)


@pytest.mark.parametrize("S", [4, 64])
def test_planes_round_trip_and_truncation(S):
    rng = np.random.default_rng(10 + S)
    for trial in range(400):
        u = _random_coeffs(rng, S)
        # cumulative closed-form cost per plane
        n, costs = 0, []
        for k in range(31, -1, -1):
            c, n = closed_form_plane_cost(S, _plane(u, k), n)
            costs.append(c)
        total = sum(costs)
        # unlimited budget: exact
        stream, used = codec.encode_planes(u, total + 100)
        assert used == total
        dec, used_d = codec.decode_planes(S, stream, total + 100)
        assert used_d == total
        np.testing.assert_array_equal(dec, u)
        # truncated budget
        B = int(rng.integers(1, total + 1))
        stream, used = codec.encode_planes(u, B)
        assert used == B
        # nothing written beyond the budget
        allbits = np.unpackbits(stream, bitorder="little")
        assert not allbits[B:].any()
        dec, _ = codec.decode_planes(S, stream, B)
        spent, k = 0, 31
        for c in costs:
            if spent + c > B:
                break
            spent += c
            k -= 1
        for kk in range(31, k, -1):          # fully coded planes: exact
            assert _plane(dec, kk) == _plane(u, kk)
        if k >= 0:                           # the partial plane: no false ones
            assert _plane(dec, k) & ~_plane(u, k) == 0
            for kk in range(k - 1, -1, -1):  # below: nothing
                assert _plane(dec, kk) == 0


def test_embedded_prefix_property():
    rng = np.random.default_rng(5)
    for dims in (1, 3):
        S = 4 ** dims
        rates = [3, 4, 6, 8, 12, 16, 24, 32] if dims == 1 else [1, 2, 4, 8, 12, 16, 24, 32]
        for _ in range(150):
            v = (rng.standard_normal(S) * 10.0 ** rng.uniform(-5, 5)).astype(np.float32)
            if dims == 3:
                v = (np.cumsum(v) + rng.standard_normal() * 100).astype(np.float32)
            streams = {r: np.unpackbits(codec.encode_block(dims, r, v), bitorder="little") for r in rates}
            for a, b in zip(rates, rates[1:]):
                na = S * a
                np.testing.assert_array_equal(streams[a][:na], streams[b][:na])


# ------------------------------------------------------------------ golden
def _parse_values(s):
    out = []
    for part in s.split(","):
        if "*" in part:
            v, n = part.split("*")
            out += [float(v)] * int(n)
        else:
            out.append(float(part))
    return np.array(out, dtype=np.float32)


def _golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = dict(kv.split("=", 1) for kv in line.split()[1:])
        cases.append((line.split()[0], int(f["dims"]), int(f["rate"]), _parse_values(f["values"]),
                      bytes.fromhex(f["stream"]), _parse_values(f["decoded"])))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_hand_derived_streams(case):
    name, dims, rate, values, stream, decoded = case
    assert len(stream) * 8 == (4 ** dims) * rate
    got = codec.encode_block(dims, rate, values)
    assert got.tobytes() == stream
    dec = codec.decode_block(dims, rate, np.frombuffer(stream, dtype=np.uint8))
    np.testing.assert_array_equal(dec, decoded)
    # +0.0, not -0.0, for zero blocks
    assert np.all(np.signbit(dec) == np.signbit(decoded))


# ------------------------------------------------------------------ invariants
def test_zero_and_subnormal_blocks_are_zero():
    for dims in (1, 3):
        S = 4 ** dims
        for v in [np.zeros(S), -np.zeros(S), np.full(S, 1e-40), np.full(S, -3e-45)]:
            s = codec.encode_block(dims, 16, np.asarray(v, dtype=np.float32))
            assert not s.any()
            d = codec.decode_block(dims, 16, s)
            assert np.all(d == 0) and not np.any(np.signbit(d))


def test_constant_blocks_exact_3d():
    rng = np.random.default_rng(6)
    consts = [1.0, -1.0, 0.5, 250.0, 3.0e38, -1.1754944e-38, np.float32(np.pi)]
    consts += list((rng.standard_normal(300) * 10.0 ** rng.uniform(-30, 30, 300)))
    for c in consts:
        v = np.full(64, c, dtype=np.float32)
        for r in (2, 4, 8, 16, 32):
            d = codec.decode_block(3, r, codec.encode_block(3, r, v))
            np.testing.assert_array_equal(d, v)


def test_constant_blocks_1d_exact_iff_they_fit():
    # 1-D budget is 4r - 9 bits; a constant codes into 1 + 2 bits per plane
    # after its leading digit, so exactness depends on the mantissa length.
    seen = set()
    for c in [1.0, 0.5, 250.0, 0.1, -3.7, 1.0e-3]:
        v = np.full(4, c, dtype=np.float32)
        for r in (8, 16):
            s = codec.encode_block(1, r, v)
            d = codec.decode_block(1, r, s)
            q = int(np.float64(np.float32(c)) * 2.0 ** (30 - np.frexp(np.float64(np.float32(c)))[1]))
            u = codec.to_negabinary(q)
            n, need = 0, 0
            for k in range(31, -1, -1):
                cost, n = closed_form_plane_cost(4, (u >> k) & 1, n)
                need += cost
                if (u & ((1 << k) - 1)) == 0:
                    break                      # lower planes are all zero
            fits = need <= 4 * r - 9
            seen.add(fits)
            if fits:
                np.testing.assert_array_equal(d, v)
    assert seen == {True, False}


def test_budget_exact_for_every_rate():
    rng = np.random.default_rng(8)
    for dims in (1, 3):
        for r in range(3 if dims == 1 else 1, 33):
            v = rng.standard_normal(4 ** dims).astype(np.float32)
            s = codec.encode_block(dims, r, v)
            bits = (4 ** dims) * r
            assert s.size == (bits + 7) // 8
            assert not np.unpackbits(s, bitorder="little")[bits:].any()


# ------------------------------------------------------------------ arrays
def test_partial_blocks_are_edge_replicated():
    rng = np.random.default_rng(9)
    for shape in [(5, 6, 17), (1, 1, 1), (3, 5, 7), (18, 4, 9), (17, 2, 160)]:
        a = rng.standard_normal(shape).astype(np.float32)   # [z][y][x]
        nz, ny, nx = shape
        pz, py, px = (-nz) % 4, (-ny) % 4, (-nx) % 4
        padded = np.pad(a, ((0, pz), (0, py), (0, px)), mode="edge")
        for r in (8, 16):
            s1 = codec.encode_array(3, r, a)
            s2 = codec.encode_array(3, r, padded)
            assert s1.tobytes() == s2.tobytes()
            out = np.full(shape, np.nan, dtype=np.float32)
            codec.decode_array(3, r, s1, out)
            full = np.full(padded.shape, np.nan, dtype=np.float32)
            codec.decode_array(3, r, s2, full)
            np.testing.assert_array_equal(out, full[:nz, :ny, :nx])
        # 1-D blocks along x
        p1 = np.pad(a, ((0, 0), (0, 0), (0, px)), mode="edge")
        for r in (8, 16):
            assert codec.encode_array(1, r, a).tobytes() == codec.encode_array(1, r, p1).tobytes()


def test_block_raster_order():
    # block (bx, by, bz) of an array is the block stream at index
    # bx + BX*(by + BY*bz): encode each 4^3 block alone and compare.
    rng = np.random.default_rng(11)
    a = rng.standard_normal((8, 12, 16)).astype(np.float32)
    s = codec.encode_array(3, 8, a)
    BX, BY, BZ = 4, 3, 2
    for bz in range(BZ):
        for by in range(BY):
            for bx in range(BX):
                blk = a[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
                b = bx + BX * (by + BY * bz)
                np.testing.assert_array_equal(s[64 * b:64 * (b + 1)], codec.encode_block(3, 8, blk))


def test_strided_views_equal_contiguous():
    rng = np.random.default_rng(12)
    big = rng.standard_normal((20, 30, 50)).astype(np.float32)
    view = big[3:14, 5:22, 7:40]
    cont = np.ascontiguousarray(view)
    for dims in (1, 3):
        assert codec.encode_array(dims, 16, view).tobytes() == codec.encode_array(dims, 16, cont).tobytes()


def test_error_non_increasing_with_rate():
    import fieldgen
    f = fieldgen.t21_field()
    fields = [f, fieldgen.temperature_like(f)]
    x64 = [g.astype(np.float64) for g in fields]
    for g, x in zip(fields, x64):
        prev_glob, prev_mean = np.inf, np.inf
        for r in (4, 6, 8, 12, 16, 24, 32):
            out = np.empty_like(g)
            codec.decode_array(3, r, codec.encode_array(3, r, g), out)
            err = out.astype(np.float64) - x
            glob = np.linalg.norm(err) / np.linalg.norm(x)
            blocks = err.reshape(2, 4, 8, 4, 16, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)
            xb = x.reshape(2, 4, 8, 4, 16, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)
            mean_rel = np.mean(np.linalg.norm(blocks, axis=1) / np.linalg.norm(xb, axis=1))
            assert glob <= prev_glob and mean_rel <= prev_mean, r
            prev_glob, prev_mean = glob, mean_rel
        assert prev_glob < 1e-6


def test_rate32_near_lossless_bound():
    # With every plane coded only three things remain: truncation to a 30-bit
    # integer (< 1 unit of 2^(emax-30)), the transform round trip (<= 38
    # units, test_3d_round_trip_bound) and the final rounding to float32
    # (half an ulp of the result).
    rng = np.random.default_rng(13)
    for _ in range(300):
        v = (np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-3, 3)).astype(np.float32)
        emax = np.frexp(np.max(np.abs(v.astype(np.float64))))[1]
        d = codec.decode_block(3, 32, codec.encode_block(3, 32, v))
        unit = 2.0 ** (emax - 30)
        half_ulp = np.spacing(np.abs(d)).astype(np.float64) / 2
        assert np.all(np.abs(d.astype(np.float64) - v) <= 39 * unit + half_ulp)
