"""Pins of the batched ragged-row oracle (oracle/batch.py) against things other than
itself: hand-written index tables and byte offsets for a tiny ragged grid, the C
oracle's own raster block order and edge replication on regular arrays built with
numpy.pad, exact reconstruction of constant fields (which zero padding would break),
and the padding bound of the octahedral grid.  Planted mistakes (zero padding, the
wrong row replicated, an unaligned field offset, rows out of order) are each caught."""
import numpy as np
import pytest

from fieldgen import octahedral as og
from oracle import batch, codec

# tiny ragged grid: 6 rows -> row-quads {0..3} and {4, 5} (two rows missing)
LENS = np.array([4, 8, 12, 4, 8, 4], dtype=np.int64)
_QUAD_BOX = batch._quad_box


def _ident_field(nlev, lens):
    """f[z, p] = 1000 z + p: every value names its level and point."""
    return (1000.0 * np.arange(nlev)[:, None] + np.arange(int(lens.sum()))[None, :]).astype(np.float32)


# the padded row-quad boxes of LENS, written out by hand: point index of every (row, x)
HAND_BOX_POINTS = {
    0: [[0, 1, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3],              # row 0, length 4, edge-replicated to 12
        [4, 5, 6, 7, 8, 9, 10, 11, 11, 11, 11, 11],        # row 1, length 8
        [12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23],  # row 2, length 12 (the quad's longest)
        [24, 25, 26, 27, 27, 27, 27, 27, 27, 27, 27, 27]],  # row 3, length 4
    1: [[28, 29, 30, 31, 32, 33, 34, 35],                  # row 4, length 8
        [36, 37, 38, 39, 39, 39, 39, 39],                  # row 5, length 4
        [36, 37, 38, 39, 39, 39, 39, 39],                  # rows 6 and 7 do not exist: they
        [36, 37, 38, 39, 39, 39, 39, 39]],                 # repeat row 5, the last one
}


def check_quad_box(quad_box):
    nlev = 6
    f = _ident_field(nlev, LENS)
    offs = batch.row_offsets(LENS)
    for q, pts in HAND_BOX_POINTS.items():
        for z0, nz in ((0, 4), (4, 2)):
            box = quad_box(f, LENS, offs, q, z0, nz)
            want = 1000.0 * np.arange(z0, z0 + nz)[:, None, None] + np.array(pts, dtype=np.float64)[None]
            assert box.shape == want.shape
            np.testing.assert_array_equal(box, want.astype(np.float32))


def test_quad_box_hand_table():
    check_quad_box(batch._quad_box)


def test_quad_box_is_numpy_edge_pad():
    rng = np.random.default_rng(3)
    lens = rng.integers(1, 30, size=11)
    f = rng.standard_normal((3, int(lens.sum()))).astype(np.float32)
    offs = batch.row_offsets(lens)
    for q in range((len(lens) + 3) // 4):
        rows = [f[:, offs[r]:offs[r] + lens[r]] for r in range(4 * q, min(4 * q + 4, len(lens)))]
        mx = max(r.shape[1] for r in rows)
        rows = [np.pad(r, ((0, 0), (0, mx - r.shape[1])), mode="edge") for r in rows]
        want = np.pad(np.stack(rows, axis=1), ((0, 0), (0, 4 - len(rows)), (0, 0)), mode="edge")
        np.testing.assert_array_equal(batch._quad_box(f, lens, offs, q, 0, 3), want)


def check_layout(layout):
    fields = [(5, 3, 8), (1, 1, 16), (3, 3, 16)]
    # field 0: 2 level quads x (3 + 2 blocks) x 64 B = 640 -> next field at 768
    # field 1: 1 level x (1 + 2 + 3 + 1 + 2 + 1 blocks) x 8 B = 80 -> 848 -> next at 1024
    # field 2: 1 level quad x 5 blocks x 128 B = 640 -> 1664 -> total 1792
    offs, total = layout(LENS, fields)
    assert list(offs) == [0, 768, 1024] and total == 1792


def test_layout_hand_offsets():
    check_layout(batch.layout)


def test_layout_alignment_random():
    rng = np.random.default_rng(4)
    lens = rng.integers(1, 40, size=13)
    fields = [(int(rng.integers(1, 9)), int(rng.choice([1, 3])), int(rng.choice([8, 16]))) for _ in range(9)]
    offs, total = batch.layout(lens, fields)
    ends = [o + batch.field_bytes(lens, *fl) for o, fl in zip(offs, fields)]
    assert all(o % 256 == 0 for o in offs) and total % 256 == 0
    assert all(e <= o2 for e, o2 in zip(ends, offs[1:] + [total]))
    assert all(o2 - e < 256 for e, o2 in zip(ends, offs[1:] + [total]))


def test_octahedral_padding_at_most_12_points_per_row():
    lens = og.row_lengths(1280)
    qb = batch.quad_blocks(lens)
    pad = np.array([4 * qb[r // 4] - lens[r] for r in range(len(lens))])
    assert pad.min() >= 0 and pad.max() <= 12
    assert len(lens) == 2560 and int(lens.sum()) == 6_599_680 and int(lens.max()) == 5136


def check_encode_field(encode_field):
    rng = np.random.default_rng(5)
    # equal rows: the item / row-quad / x order is the raster block order of the regular array
    for nrows, L, nlev in ((7, 12, 6), (8, 8, 4), (5, 20, 1)):
        lens = np.full(nrows, L, dtype=np.int64)
        f = rng.standard_normal((nlev, nrows * L)).astype(np.float32)
        reg = f.reshape(nlev, nrows, L)
        for dims in (3, 1):
            for rate in (8, 16):
                np.testing.assert_array_equal(encode_field(f, lens, dims, rate),
                                              codec.encode_array(dims, rate, reg))
    # ragged rows whose quads share one longest row: the item box of the whole field is a
    # regular array built by numpy edge padding (short rows to the longest, the missing
    # last row repeating row 6)
    lens = np.array([8, 4, 8, 6, 8, 8, 5], dtype=np.int64)
    offs = batch.row_offsets(lens)
    f = rng.standard_normal((6, int(lens.sum()))).astype(np.float32)
    rows = [np.pad(f[:, offs[r]:offs[r] + lens[r]], ((0, 0), (0, 8 - lens[r])), mode="edge") for r in range(7)]
    reg = np.pad(np.stack(rows, axis=1), ((0, 0), (0, 1), (0, 0)), mode="edge")
    for rate in (8, 16):
        np.testing.assert_array_equal(encode_field(f, lens, 3, rate), codec.encode_array(3, rate, reg))
    return reg


def test_encode_field_is_raster_order_of_padded_array():
    check_encode_field(batch.encode_field)


def test_decode_field_crops_the_padded_array():
    rng = np.random.default_rng(6)
    lens = np.array([8, 4, 8, 6, 8, 8, 5], dtype=np.int64)
    offs = batch.row_offsets(lens)
    f = rng.standard_normal((6, int(lens.sum()))).astype(np.float32)
    rows = [np.pad(f[:, offs[r]:offs[r] + lens[r]], ((0, 0), (0, 8 - lens[r])), mode="edge") for r in range(7)]
    reg = np.pad(np.stack(rows, axis=1), ((0, 0), (0, 1), (0, 0)), mode="edge")
    for dims, rate in ((3, 8), (3, 16), (1, 8), (1, 16)):
        s = batch.encode_field(f, lens, dims, rate)
        got = batch.decode_field(s, f.shape, lens, dims, rate)
        if dims == 3:
            dec = codec.decode_array(3, rate, s, np.empty_like(reg))
            want = np.concatenate([dec[:, r, :lens[r]] for r in range(7)], axis=1)
        else:
            want = np.concatenate([codec.decode_array(1, rate, codec.encode_array(1, rate, f[:, None, o:o + L]),
                                                      np.empty((6, 1, L), np.float32))[:, 0]
                                   for o, L in zip(offs, lens)], axis=1)
        np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))


def check_constant_exact(encode_field, decode_field):
    # a constant field: with edge replication every 3-D box is constant, which decodes
    # exactly at any rate >= 2 (one significant coefficient)
    lens = LENS
    for c in (1.0, -3.75, 250.0, 1e-3):
        f = np.full((5, int(lens.sum())), c, dtype=np.float32)
        for rate in (2, 8, 16):
            s = encode_field(f, lens, 3, rate)
            np.testing.assert_array_equal(decode_field(s, f.shape, lens, 3, rate), f)


def test_constant_fields_exact():
    check_constant_exact(batch.encode_field, batch.decode_field)


# ---- planted mistakes: each one fails a pin above
def _quad_box_zero_pad(f, lens, offs, q, z0, nz):
    box = _QUAD_BOX(f, lens, offs, q, z0, nz)
    for j in range(4):
        r = min(4 * q + j, len(lens) - 1)
        box[:, j, int(lens[r]):] = 0.0
    return box


def _quad_box_wrong_row(f, lens, offs, q, z0, nz):
    box = _QUAD_BOX(f, lens, offs, q, z0, nz)
    nrows = min(4, len(lens) - 4 * q)
    if nrows < 4:
        box[:, nrows:, :] = box[:, :1, :]        # repeats the quad's first row, not its last
    return box


def _layout_unaligned(lens, fields):
    offs, o = [], 0
    for fl in fields:
        offs.append(o)
        o += batch.field_bytes(lens, *fl)
    return offs, o


def _encode_rows_reversed(f, lens, dims, rate):
    if dims != 1:
        return batch.encode_field(f, lens, dims, rate)
    offs = batch.row_offsets(lens)
    parts = []
    for z in range(f.shape[0]):
        for r in reversed(range(len(lens))):
            parts.append(codec.encode_array(1, rate, f[z:z + 1, offs[r]:offs[r] + lens[r]].reshape(1, 1, -1)))
    return np.concatenate(parts)


@pytest.mark.parametrize("mut", ["zero_pad", "wrong_row"])
def test_planted_quad_box_mistakes_caught(monkeypatch, mut):
    bad = {"zero_pad": _quad_box_zero_pad, "wrong_row": _quad_box_wrong_row}[mut]
    with pytest.raises(AssertionError):
        check_quad_box(bad)
    monkeypatch.setattr(batch, "_quad_box", bad)
    with pytest.raises(AssertionError):
        check_encode_field(batch.encode_field)
    if mut == "zero_pad":
        with pytest.raises(AssertionError):
            check_constant_exact(batch.encode_field, batch.decode_field)


def test_planted_layout_and_order_mistakes_caught():
    with pytest.raises(AssertionError):
        check_layout(_layout_unaligned)
    with pytest.raises(AssertionError):
        check_encode_field(_encode_rows_reversed)
