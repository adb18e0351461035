"""Pins of the oracle's accuracy and precision modes (variable-rate coding to an absolute
error tolerance, 3-D blocks; the mode the paper names and leaves for future
work, Sec. II-C).  Each pin ties it to something fixed independently: the
error bound the plane cut-off is chosen for, the embedded property of the
pinned fixed-rate coder (a block's accuracy bits are a prefix of its rate-16
bits), monotonicity in the tolerance, and the plain-Python second statement."""
import numpy as np
import pytest

import fieldgen
from oracle import codec

import zfp_prose as zp


def _blocks(a):
    """[z][y][x] array -> its 4x4x4 blocks (edge-replicated), raster order."""
    nz, ny, nx = a.shape
    p = np.pad(a, ((0, (-nz) % 4), (0, (-ny) % 4), (0, (-nx) % 4)), mode="edge")
    Z, Y, X = (d // 4 for d in p.shape)
    return p.reshape(Z, 4, Y, 4, X, 4).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 64)


def _fields():
    rng = np.random.default_rng(41)
    f = fieldgen.t21_field()
    out = [f, fieldgen.temperature_like(f)]
    for _ in range(4):
        g = np.cumsum(np.cumsum(rng.standard_normal((9, 13, 22)), axis=2), axis=1)
        out.append((g * 10.0 ** rng.uniform(-6, 6)).astype(np.float32))
    return out


def test_minexp_and_kmin():
    for tol, want in [(1.0, 0), (0.75, -1), (0.5, -1), (0.49, -2), (1e-3, -10), (3.0, 1)]:
        assert codec.accuracy_minexp(tol) == want, tol
    assert codec.accuracy_kmin(5, -10) == 7
    assert codec.accuracy_kmin(40, -10) == 0
    assert codec.accuracy_kmin(-30, 0) == 32


def test_error_within_tolerance_unless_cut_or_clamped():
    for a in _fields():
        x = a.astype(np.float64)
        amax = np.abs(x).max()
        for rel in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
            tol = rel * amax
            L, P, bits = codec.encode_accuracy(a, tol)
            assert bits == int(L.astype(np.int64).sum())
            out = np.empty_like(a)
            codec.decode_accuracy(L, P, out)
            err = _blocks(np.abs(out.astype(np.float64) - x))
            blk = _blocks(x)
            minexp = codec.accuracy_minexp(tol)
            for b in range(blk.shape[0]):
                m = np.abs(blk[b]).max()
                if m == 0.0:
                    assert L[b] == 1
                    continue
                emax = np.frexp(m)[1]
                if L[b] < 1024 and minexp - emax + 22 >= 0:
                    assert err[b].max() <= tol, (rel, b)


def test_prefix_of_the_fixed_rate_stream_and_monotone():
    rng = np.random.default_rng(42)
    for _ in range(300):
        v = (np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-8, 8)).astype(np.float32)
        fixed = np.unpackbits(codec.encode_block(3, 16, v), bitorder="little")
        prev = None
        for tol in 10.0 ** np.arange(4, -12, -1.0) * np.abs(v).max():
            L, P, bits = codec.encode_accuracy(v.reshape(4, 4, 4), tol)
            acc = np.unpackbits(P, bitorder="little")[:bits]
            np.testing.assert_array_equal(acc, fixed[:bits])           # embedded coding: a prefix
            if prev is not None:
                assert bits >= prev                                      # finer tolerance, more bits
            prev = bits


def test_special_blocks():
    z = np.zeros((4, 4, 4), np.float32)
    L, P, bits = codec.encode_accuracy(z, 1e-3)
    assert bits == 1 and L[0] == 1 and not P.any()
    tiny = np.full((4, 4, 4), 1e-9, np.float32)          # far below the tolerance: header only
    L, P, bits = codec.encode_accuracy(tiny, 1.0)
    assert bits == 9
    out = np.ones_like(tiny)
    codec.decode_accuracy(L, P, out)
    assert not out.any()
    const = np.full((4, 4, 4), 250.0, np.float32)        # a constant: exact at any tolerance
    L, P, bits = codec.encode_accuracy(const, 1e-6)
    out = np.empty_like(const)
    codec.decode_accuracy(L, P, out)
    np.testing.assert_array_equal(out, const)


@pytest.mark.parametrize("rel", [1e-1, 1e-3, 1e-5])
def test_second_statement_agrees(rel):
    rng = np.random.default_rng(43)
    for a in [fieldgen.t21_field()[:4, :8, :16]] + [
            (rng.standard_normal(s) * 10.0 ** rng.uniform(-5, 5)).astype(np.float32) for s in [(4, 4, 4), (5, 7, 9)]]:
        a = np.ascontiguousarray(a)
        tol = rel * float(np.abs(a).max())
        L, P, bits = codec.encode_accuracy(a, tol)
        stream = []
        for blk in _blocks(a.astype(np.float64)).astype(np.float32):
            stream += zp.encode_block_accuracy(blk, tol)
        assert [int(l) for l in L] == [len(zp.encode_block_accuracy(b, tol))
                                      for b in _blocks(a.astype(np.float64)).astype(np.float32)]
        np.testing.assert_array_equal(np.unpackbits(P, bitorder="little")[:bits], np.array(stream, np.uint8))


# ---------------------------------------------------------------- precision mode
def test_precision_error_bound_prefix_and_monotone():
    # planes 31 .. 32 - p kept: by the same argument as the accuracy cut-off the
    # error of an uncut block stays below 2^(e_max - p + 9); the bits are a prefix
    # of the rate-16 stream and grow with p
    for a in _fields():
        x = a.astype(np.float64)
        blk = _blocks(x)
        prev_bits, prev_err = 0, np.inf
        for p in (2, 6, 10, 14, 18, 24):
            L, P, bits = codec.encode_precision(a, p)
            out = np.empty_like(a)
            codec.decode_accuracy(L, P, out)
            err = _blocks(np.abs(out.astype(np.float64) - x))
            for b in range(blk.shape[0]):
                m = np.abs(blk[b]).max()
                if m > 0 and L[b] < 1024:
                    assert err[b].max() <= 2.0 ** (np.frexp(m)[1] - p + 9), (p, b)
            assert bits >= prev_bits
            e = np.linalg.norm(out - x)
            assert e <= prev_err
            prev_bits, prev_err = bits, e
    rng = np.random.default_rng(44)
    for _ in range(100):
        v = (np.cumsum(rng.standard_normal(64)) * 10.0 ** rng.uniform(-8, 8)).astype(np.float32)
        fixed = np.unpackbits(codec.encode_block(3, 16, v), bitorder="little")
        for p in (1, 5, 11, 17, 32):
            L, P, bits = codec.encode_precision(v.reshape(4, 4, 4), p)
            np.testing.assert_array_equal(np.unpackbits(P, bitorder="little")[:bits], fixed[:bits])


@pytest.mark.parametrize("p", [3, 12, 20])
def test_precision_second_statement_agrees(p):
    rng = np.random.default_rng(45 + p)
    a = np.ascontiguousarray((rng.standard_normal((5, 7, 9)) * 10.0 ** rng.uniform(-5, 5)).astype(np.float32))
    L, P, bits = codec.encode_precision(a, p)
    stream, lens = [], []
    for blk in _blocks(a.astype(np.float64)).astype(np.float32):
        bb = zp._code(3, blk, 1024 - 9, lambda e: 32 - p)
        stream += bb
        lens.append(len(bb))
    assert [int(l) for l in L] == lens
    np.testing.assert_array_equal(np.unpackbits(P, bitorder="little")[:bits], np.array(stream, np.uint8))
