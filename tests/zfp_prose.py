"""A second, independent CPU reference of ZFP fixed-rate coding, in plain
Python (test infrastructure; slow, for small inputs only).

It follows the method as the paper outlines it (Sec. II-C; Lindstrom 2014)
step by step, written a different way from the C oracle: bits are Python
lists, the coefficient order is computed by sorting, and the bit planes are
coded by the literal group-testing procedure (one emitted bit at a time,
with the budget counted down), not by a state machine or closed forms.  The
readings (zero-block threshold, truncating quantisation, edge-replicated
partial blocks, LSB-first bit order) are the repository's, as stated in its
design notes.  Shares no code with oracle/ or the CUDA path.
"""
import math

import numpy as np


def _wrap(v):
    """int32 ring value of a Python int."""
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v & 0x80000000 else v


def _wrap64(v):
    """int64 ring value of a Python int."""
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >> 63 else v


def _fwd4(v, _wrap=_wrap):
    """Integer lifting of one 4-vector; halvings are floor shifts."""
    x, y, z, w = v
    x = _wrap(x + w) >> 1
    w = _wrap(w - x)
    z = _wrap(z + y) >> 1
    y = _wrap(y - z)
    x = _wrap(x + z) >> 1
    z = _wrap(z - x)
    w = _wrap(w + y) >> 1
    y = _wrap(y - w)
    w = _wrap(w + (y >> 1))
    y = _wrap(y - (w >> 1))
    return [x, y, z, w]


def _inv4(v, _wrap=_wrap):
    """The steps of _fwd4 undone in reverse order (a halving undone by a doubling)."""
    x, y, z, w = v
    y = _wrap(y + (w >> 1))
    w = _wrap(w - (y >> 1))
    y = _wrap(y + w)
    w = _wrap(2 * w - y)
    z = _wrap(z + x)
    x = _wrap(2 * x - z)
    y = _wrap(y + z)
    z = _wrap(2 * z - y)
    w = _wrap(w + x)
    x = _wrap(2 * x - w)
    return [x, y, z, w]


def _lines(dims):
    """Index lines of a block along axis 0, then 1, then 2 (index i + 4j + 16k)."""
    if dims == 1:
        return [[[0, 1, 2, 3]]]
    size = 4 ** dims
    axes = []
    for stride in (1, 4, 16)[:dims]:
        lines = []
        for base in range(size):
            if (base // stride) % 4 == 0:
                lines.append([base + stride * t for t in range(4)])
        axes.append(lines)
    return axes


def _order(dims):
    """Coefficients by total sequency, then i^2+j^2+k^2, then index (k = 0 in 2-D)."""
    if dims == 1:
        return [0, 1, 2, 3]
    keys = []
    for idx in range(4 ** dims):
        i, j, k = idx % 4, (idx // 4) % 4, idx // 16
        keys.append((i + j + k, i * i + j * j + k * k, idx))
    return [key[2] for key in sorted(keys)]


def encode_block(dims, rate, values):
    """Bits (list of 0/1) of one block of 4^dims float32 values."""
    maxbits = (4 ** dims) * rate
    bits = _code(dims, values, maxbits - 9, lambda e: 0)
    return bits + [0] * (maxbits - len(bits))


def encode_block_accuracy(values, tol):
    """Bits of one 3-D block in the accuracy mode: planes from 31 down to
    kmin = minexp - e_max + 22 (clamped to 0..32, minexp = floor(log2 tol)),
    at most 1024 bits, no fill."""
    minexp = math.frexp(tol)[1] - 1
    return _code(3, values, 1024 - 9, lambda e: min(32, max(0, minexp - e + 22)))


# the two value formats: exponent bias and bits, integer precision, planes
F32 = dict(dtype=np.float32, bias=127, ebits=8, intprec=30, planes=32, wrap=_wrap)
F64 = dict(dtype=np.float64, bias=1023, ebits=11, intprec=62, planes=64, wrap=_wrap64)


def _code(dims, values, budget, kstop_of, fmt=F32):
    """Header and planes (top) .. kstop_of(e_max) of one block, at most budget
    bits after the header; a zero block is the single bit 0."""
    size = 4 ** dims
    vals = [float(v) for v in np.asarray(values, dtype=fmt["dtype"]).reshape(-1)]
    big = max(abs(v) for v in vals)
    if not math.isfinite(big) or big == 0.0:
        return [0]
    e = math.frexp(big)[1]
    if e + fmt["bias"] <= 0:
        return [0]
    bits = [1] + [(e + fmt["bias"]) >> b & 1 for b in range(fmt["ebits"])]
    kstop = kstop_of(e)
    q = [int(math.trunc(math.ldexp(v, fmt["intprec"] - e))) for v in vals]
    for axis in _lines(dims):
        for line in axis:
            out = _fwd4([q[t] for t in line], fmt["wrap"])
            for t, val in zip(line, out):
                q[t] = val
    P = fmt["planes"]
    nega = int("10" * (P // 2), 2)
    u = [(fmt["wrap"](q[idx]) + nega & ((1 << P) - 1)) ^ nega for idx in _order(dims)]
    n = 0
    for k in range(P - 1, kstop - 1, -1):
        if budget <= 0:
            break
        plane = [c >> k & 1 for c in u]
        for i in range(n):                           # significant coefficients: verbatim
            if budget == 0:
                break
            bits.append(plane[i])
            budget -= 1
        while n < size and budget > 0:               # group tests
            g = 1 if any(plane[n:]) else 0
            bits.append(g)
            budget -= 1
            if not g:
                break
            j = n
            while True:
                if j == size - 1:                    # the last one is implied
                    n = size
                    break
                if budget == 0:
                    break
                bits.append(plane[j])
                budget -= 1
                if plane[j]:
                    n = j + 1
                    break
                j += 1
            if budget == 0:
                break
    return bits


def decode_block(dims, rate, bits):
    """float32 values of one block from its maxbits bits."""
    size = 4 ** dims
    maxbits = size * rate
    bits = list(bits)[:maxbits]
    if not bits[0]:
        return np.zeros(size, dtype=np.float32)
    e = sum(bits[1 + b] << b for b in range(8)) - 127
    pos = 9
    budget = maxbits - 9
    u = [0] * size
    n = 0
    for k in range(31, -1, -1):
        if budget <= 0:
            break
        for i in range(n):
            if budget == 0:
                break
            u[i] |= bits[pos] << k
            pos += 1
            budget -= 1
        while n < size and budget > 0:
            g = bits[pos]
            pos += 1
            budget -= 1
            if not g:
                break
            j = n
            while True:
                if j == size - 1:
                    u[j] |= 1 << k
                    n = size
                    break
                if budget == 0:
                    break
                b = bits[pos]
                pos += 1
                budget -= 1
                if b:
                    u[j] |= 1 << k
                    n = j + 1
                    break
                j += 1
            if budget == 0:
                break
    q = [0] * size
    for idx, c in zip(_order(dims), u):
        q[idx] = _wrap((c ^ 0xAAAAAAAA) - 0xAAAAAAAA)
    for axis in reversed(_lines(dims)):
        for line in axis:
            out = _inv4([q[t] for t in line])
            for t, val in zip(line, out):
                q[t] = val
    return np.array([np.float32(float(v) * 2.0 ** (e - 30)) for v in q], dtype=np.float32)


def _blocks(dims, shape):
    nz, ny, nx = shape
    if dims == 1:
        return [(z, y, x) for z in range(nz) for y in range(ny) for x in range(0, nx, 4)]
    if dims == 2:
        return [(z, y, x) for z in range(nz) for y in range(0, ny, 4) for x in range(0, nx, 4)]
    return [(z, y, x) for z in range(0, nz, 4) for y in range(0, ny, 4) for x in range(0, nx, 4)]


def _gather(dims, a, z, y, x):
    nz, ny, nx = a.shape
    if dims == 1:
        return [a[z, y, min(x + i, nx - 1)] for i in range(4)]
    if dims == 2:
        return [a[z, min(y + j, ny - 1), min(x + i, nx - 1)] for j in range(4) for i in range(4)]
    return [a[min(z + k, nz - 1), min(y + j, ny - 1), min(x + i, nx - 1)]
            for k in range(4) for j in range(4) for i in range(4)]


def encode_array(dims, rate, a):
    """Bytes of a [z][y][x] float32 array: blocks in raster order (x fastest),
    partial blocks edge-replicated, bit p of the stream = bit p % 8 of byte p / 8."""
    bits = []
    for z, y, x in _blocks(dims, a.shape):
        bits += encode_block(dims, rate, _gather(dims, a, z, y, x))
    bits += [0] * (-len(bits) % 8)
    return np.packbits(np.array(bits, dtype=np.uint8), bitorder="little")


def decode_array(dims, rate, stream, shape):
    bits = np.unpackbits(np.asarray(stream, dtype=np.uint8), bitorder="little").tolist()
    out = np.zeros(shape, dtype=np.float32)
    nz, ny, nx = shape
    per = (4 ** dims) * rate
    for b, (z, y, x) in enumerate(_blocks(dims, shape)):
        vals = decode_block(dims, rate, bits[b * per:(b + 1) * per])
        if dims == 1:
            for i in range(4):
                if x + i < nx:
                    out[z, y, x + i] = vals[i]
        elif dims == 2:
            for j in range(4):
                for i in range(4):
                    if y + j < ny and x + i < nx:
                        out[z, y + j, x + i] = vals[4 * j + i]
        else:
            for k in range(4):
                for j in range(4):
                    for i in range(4):
                        if z + k < nz and y + j < ny and x + i < nx:
                            out[z + k, y + j, x + i] = vals[16 * k + 4 * j + i]
    return out


def encode_block_f64(rate, values):
    """Bits of one 3-D block of float64 values at rate bits per value."""
    maxbits = 64 * rate
    bits = _code(3, values, maxbits - 12, lambda e: 0, F64)
    return bits + [0] * (maxbits - len(bits))


def decode_block_f64(rate, bits):
    """float64 values of one 3-D block from its 64 rate bits (the plane loop of
    decode_block with 64 planes, an 11-bit exponent and int64 coefficients)."""
    size, maxbits = 64, 64 * rate
    bits = list(bits)[:maxbits]
    if not bits[0]:
        return np.zeros(size)
    e = sum(bits[1 + b] << b for b in range(11)) - 1023
    pos, budget, n = 12, maxbits - 12, 0
    u = [0] * size
    for k in range(63, -1, -1):
        if budget <= 0:
            break
        for i in range(n):
            if budget == 0:
                break
            u[i] |= bits[pos] << k
            pos += 1
            budget -= 1
        while n < size and budget > 0:
            g = bits[pos]
            pos += 1
            budget -= 1
            if not g:
                break
            j = n
            while True:
                if j == size - 1:
                    u[j] |= 1 << k
                    n = size
                    break
                if budget == 0:
                    break
                b = bits[pos]
                pos += 1
                budget -= 1
                if b:
                    u[j] |= 1 << k
                    n = j + 1
                    break
                j += 1
            if budget == 0:
                break
    nega = int("10" * 32, 2)
    q = [0] * size
    for idx, c in zip(_order(3), u):
        q[idx] = _wrap64((c ^ nega) - nega)
    for axis in reversed(_lines(3)):
        for line in axis:
            out = _inv4([q[t] for t in line], _wrap64)
            for t, val in zip(line, out):
                q[t] = val
    # q 2^(e - 62) rounded once: exact rational, then the nearest double
    from fractions import Fraction
    return np.array([float(Fraction(v) * Fraction(2) ** (e - 62)) for v in q])
