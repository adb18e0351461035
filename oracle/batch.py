"""Batched ragged-row compression (test infrastructure; oracle side).

Fields on a grid of ragged rows (rows back to back, row r holding len[r]
points; the octahedral reduced Gaussian grid is the case in view), stored
[level][point].  A field is coded with either
  * dims 1: blocks of 4 consecutive points of one row of one level, or
  * dims 3: blocks of 4 points x 4 consecutive rows x 4 consecutive levels.
    A row-quad spans rows 4q..4q+3; its blocks cover x = 0 .. max len - 1 of
    the quad, each shorter row repeating its last point (edge replication),
    a missing last row / level repeating the last one.
Stream of a field: items in level order (dims 3: level quads; dims 1:
levels), inside an item the blocks in row (row-quad) order, then along x.
Every field starts at a multiple of 256 bytes.  Each item is exactly the
stream that codec.encode_array gives for the padded item box, which is how
this module computes it (ZFP fixed-rate, paper Sec. II-C).
"""
import numpy as np

from . import codec

ALIGN = 256


def _align(v):
    return (v + ALIGN - 1) // ALIGN * ALIGN


def row_offsets(lens):
    return np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)


def quad_blocks(lens):
    """Blocks along x of every row-quad: ceil(max len in the quad / 4)."""
    nq = (len(lens) + 3) // 4
    return np.array([(int(max(lens[4 * q:4 * q + 4])) + 3) // 4 for q in range(nq)], dtype=np.int64)


def field_items(lens, nlev, dims):
    """(level start, levels) of each item."""
    if dims == 3:
        return [(z, min(4, nlev - z)) for z in range(0, nlev, 4)]
    return [(z, 1) for z in range(nlev)]


def item_blocks(lens, dims):
    if dims == 3:
        return int(quad_blocks(lens).sum())
    return int(sum((int(L) + 3) // 4 for L in lens))


def field_bytes(lens, nlev, dims, rate):
    per_block = 8 * rate if dims == 3 else rate // 2
    return item_blocks(lens, dims) * len(field_items(lens, nlev, dims)) * per_block


def layout(lens, fields):
    """Byte offset of every field's stream, and the total."""
    offs, o = [], 0
    for (nlev, dims, rate) in fields:
        offs.append(o)
        o = _align(o + field_bytes(lens, nlev, dims, rate))
    return offs, o


def _quad_box(f, lens, offs, q, z0, nz):
    """Padded box [nz][rows 4][max len] of row-quad q (edge replication)."""
    nrows = len(lens)
    rows = [min(4 * q + j, nrows - 1) for j in range(4)]
    mx = int(max(lens[r] for r in rows[: min(4, nrows - 4 * q)]))
    box = np.empty((nz, 4, mx), dtype=np.float32)
    for j, r in enumerate(rows):
        x = np.minimum(np.arange(mx), int(lens[r]) - 1)
        box[:, j, :] = f[z0:z0 + nz, int(offs[r]) + x]
    return box


def encode_field(f, lens, dims, rate):
    """Stream of one field (numpy [nlev][points])."""
    nlev = f.shape[0]
    offs = row_offsets(lens)
    parts = []
    for z0, nz in field_items(lens, nlev, dims):
        if dims == 3:
            for q in range((len(lens) + 3) // 4):
                parts.append(codec.encode_array(3, rate, _quad_box(f, lens, offs, q, z0, nz)))
        else:
            for r, L in enumerate(lens):
                row = f[z0:z0 + 1, int(offs[r]):int(offs[r]) + int(L)].reshape(1, 1, -1)
                parts.append(codec.encode_array(1, rate, row))
    return np.concatenate(parts)


def decode_field(stream, shape, lens, dims, rate):
    nlev, npts = shape
    out = np.zeros(shape, dtype=np.float32)
    offs = row_offsets(lens)
    pos = 0
    for z0, nz in field_items(lens, nlev, dims):
        if dims == 3:
            qb = quad_blocks(lens)
            for q in range(len(qb)):
                nb = int(qb[q]) * 8 * rate
                mx = int(qb[q]) * 4
                box = np.empty((nz, 4, mx), dtype=np.float32)
                codec.decode_array(3, rate, stream[pos:pos + nb], box)
                pos += nb
                for j in range(min(4, len(lens) - 4 * q)):
                    r = 4 * q + j
                    out[z0:z0 + nz, int(offs[r]):int(offs[r]) + int(lens[r])] = box[:, j, :int(lens[r])]
        else:
            for r, L in enumerate(lens):
                nb = ((int(L) + 3) // 4) * rate // 2
                row = np.empty((1, 1, int(L)), dtype=np.float32)
                codec.decode_array(1, rate, stream[pos:pos + nb], row)
                pos += nb
                out[z0, int(offs[r]):int(offs[r]) + int(L)] = row[0, 0]
    return out


def encode_batch(fields_data, lens, fields):
    """fields_data: list of numpy [nlev][points]; fields: list of (nlev, dims, rate)."""
    offs, total = layout(lens, fields)
    buf = np.zeros(total, dtype=np.uint8)
    for f, (nlev, dims, rate), o in zip(fields_data, fields, offs):
        s = encode_field(f, lens, dims, rate)
        buf[o:o + s.size] = s
    return buf
