"""Pins of the oracle's pack / permute / unpack and float16 casts.

Pack and all-to-all as in the paper's per-rank sequence (Sec. I; Sec. IV-D);
float16 cast comparator (Sec. I; Sec. IV-F).
"""
import numpy as np
import pytest

from oracle import packs, fp16
from oracle.plan import Plan, message_bytes


def _ids(shape):
    return np.arange(np.prod(shape), dtype=np.float32).reshape(shape)   # exact below 2^24


@pytest.mark.parametrize("t", [0, 1])
def test_f32_pack_sends_every_value_once_in_raster_order(t):
    shape = (9, 10, 14)                      # [lev][lat][lon]
    plan = Plan(14, 10, 9, 3, 2, transposition=t)
    x = _ids(shape)
    send = packs.pack(plan, 0, x)
    so, _, _ = plan.layout(0)
    seen = []
    for m in plan.messages:
        v = send[so[(m.src, m.dst)]:so[(m.src, m.dst)] + 4 * m.nvals].view(np.float32).astype(np.int64)
        z, rem = np.divmod(v, shape[1] * shape[2])
        y, xx = np.divmod(rem, shape[2])
        # inside the box, raster order lon fastest
        assert np.all((xx >= m.x0) & (xx < m.x0 + m.nx) & (y >= m.y0) & (y < m.y0 + m.ny)
                      & (z >= m.z0) & (z < m.z0 + m.nz))
        key = (z - m.z0) * m.ny * m.nx + (y - m.y0) * m.nx + (xx - m.x0)
        np.testing.assert_array_equal(key, np.arange(m.nvals))
        seen.append(v)
    np.testing.assert_array_equal(np.sort(np.concatenate(seen)), np.arange(x.size))


@pytest.mark.parametrize("t", [0, 1])
def test_f32_round_trip_through_permutation(t):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((17, 12, 20)).astype(np.float32)
    plan = Plan(20, 12, 17, 2, 3, transposition=t)
    recv = packs.permute(plan, 0, packs.pack(plan, 0, x))
    out = np.full_like(x, np.nan)
    packs.unpack(plan, 0, recv, out)
    np.testing.assert_array_equal(out, x)
    # the permutation equals packing straight into the receive layout
    np.testing.assert_array_equal(recv, packs.pack(plan, 0, x, which="recv"))


def test_zfp_pack_messages_are_independent_streams():
    rng = np.random.default_rng(1)
    x = np.cumsum(rng.standard_normal((18, 16, 24)), axis=2).astype(np.float32)
    plan = Plan(24, 16, 18, 2, 2, transposition=0)
    for r in (8, 16):
        send = packs.pack(plan, r, x)
        so, _, total = plan.layout(r)
        for m in plan.messages:
            nb = message_bytes(m, r)
            o = so[(m.src, m.dst)]
            np.testing.assert_array_equal(send[o:o + nb], packs.message_stream(plan, r, x, m))
        out = np.full_like(x, np.nan)
        packs.unpack(plan, r, packs.permute(plan, r, send), out)
        assert np.all(np.isfinite(out))
        assert np.linalg.norm(out - x) / np.linalg.norm(x) < (5e-2 if r == 8 else 1e-3)


def _f16_neighbours(h):
    b = h.view(np.uint16).astype(np.int32)
    return [(b + d).astype(np.uint16).view(np.float16) for d in (-1, 1)]


def test_fp16_rn_definition():
    # nearest float16; ties to the even significand; beyond the largest
    # finite half (65504) + half an ulp (16) overflow to inf
    rng = np.random.default_rng(2)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32) * np.float32(10.0) ** rng.integers(-9, 6, 200000).astype(np.float32),
        np.array([65504.0, 65519.99, 65520.0, -65520.0, 6e-8, 2.98e-8, 5.96e-8, 1e-10, 0.0, -0.0], np.float32),
    ])
    h = fp16.to_f16_rn(x).view(np.float16)
    finite = np.isfinite(h)
    hx = h.astype(np.float64)
    err = np.abs(hx - x)
    lo, hi = _f16_neighbours(h)
    for nb in (lo, hi):
        ok = np.isfinite(nb) & finite
        e2 = np.abs(nb.astype(np.float64) - x)
        assert np.all(err[ok] <= e2[ok])
        tie = ok & (err == e2) & (err > 0)
        assert np.all(h.view(np.uint16)[tie] % 2 == 0)
    big = np.abs(x.astype(np.float64)) >= 65520.0
    assert np.all(np.isinf(h[big])) and np.all(finite[~big])


def test_fp16_rz_definition():
    rng = np.random.default_rng(3)
    x = np.concatenate([
        rng.standard_normal(200000).astype(np.float32) * np.float32(10.0) ** rng.integers(-9, 6, 200000).astype(np.float32),
        np.array([65504.0, 65535.0, 1e6, -1e6, 6e-8, 1e-10, -1e-10, 0.0], np.float32),
        np.array([np.inf, -np.inf], np.float32),
    ])
    h = fp16.to_f16_rz(x).view(np.float16)
    fin = np.isfinite(x)
    hx = h.astype(np.float64)
    ax = np.abs(x.astype(np.float64))
    assert np.all(np.abs(hx[fin]) <= ax[fin])
    assert np.all(np.signbit(h[fin & (x != 0)]) == np.signbit(x[fin & (x != 0)]))
    # the next float16 away from zero is already beyond |x| (or x is past the range)
    up = (np.abs(h).view(np.uint16).astype(np.int32) + 1).astype(np.uint16).view(np.float16).astype(np.float64)
    inrange = fin & (ax < 65520.0)
    assert np.all(up[inrange] > ax[inrange])
    assert np.all(np.abs(hx[fin & (ax >= 65504)]) == 65504.0)
    assert np.all(np.isinf(h[~fin]))
