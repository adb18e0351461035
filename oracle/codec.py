"""ctypes binding of the scalar C oracle ``zfp_oracle.c`` (test infrastructure).

ZFP fixed-rate coding of float32 data in 4^d blocks (paper Sec. II-C, the
fixed-rate mode of ZFP 1.0.1 in Sec. IV-B; the method itself is Lindstrom
2014).  Parity pinned by tests/test_oracle_codec.py and
tests/test_oracle_transform.py.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.zfpo_overflow_count.restype = ctypes.c_longlong
        L.zfpo_overflow_reset.restype = None
        L.zfpo_lift_forward_exact.argtypes = [ctypes.c_void_p]
        L.zfpo_lift_inverse_exact.argtypes = [ctypes.c_void_p]
        L.zfpo_lift_forward.argtypes = [ctypes.c_void_p]
        L.zfpo_lift_inverse.argtypes = [ctypes.c_void_p]
        L.zfpo_xform_forward.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.zfpo_xform_inverse.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.zfpo_sequency_order.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.zfpo_to_negabinary.argtypes = [ctypes.c_int32]
        L.zfpo_to_negabinary.restype = ctypes.c_uint32
        L.zfpo_from_negabinary.argtypes = [ctypes.c_uint32]
        L.zfpo_from_negabinary.restype = ctypes.c_int32
        L.zfpo_plane_bits.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]
        L.zfpo_plane_bits.restype = ctypes.c_int
        L.zfpo_encode_planes.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_void_p]
        L.zfpo_encode_planes.restype = ctypes.c_uint64
        L.zfpo_decode_planes.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64,
                                         ctypes.c_void_p]
        L.zfpo_decode_planes.restype = ctypes.c_uint64
        L.zfpo_encode_block.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.zfpo_decode_block.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.zfpo_block_count.argtypes = [ctypes.c_int, i64p]
        L.zfpo_block_count.restype = ctypes.c_int64
        L.zfpo_stream_bytes.argtypes = [ctypes.c_int, ctypes.c_int, i64p]
        L.zfpo_stream_bytes.restype = ctypes.c_int64
        L.zfpo_encode_array.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, i64p,
                                        i64p, ctypes.c_void_p, ctypes.c_int64]
        L.zfpo_decode_array.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, i64p,
                                        ctypes.c_void_p, i64p]
        L.zfpo_accuracy_kmin.argtypes = [ctypes.c_int, ctypes.c_int]
        L.zfpo_accuracy_minexp.argtypes = [ctypes.c_double]
        L.zfpo_accuracy_max_payload_bytes.argtypes = [i64p]
        L.zfpo_accuracy_max_payload_bytes.restype = ctypes.c_int64
        L.zfpo_encode_accuracy.argtypes = [ctypes.c_void_p, i64p, i64p, ctypes.c_double, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
        L.zfpo_decode_accuracy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, i64p, ctypes.c_void_p, i64p]
        L.zfpo_xform_forward_i64.argtypes = [ctypes.c_void_p]
        L.zfpo_xform_inverse_i64.argtypes = [ctypes.c_void_p]
        L.zfpo_stream_bytes_f64.argtypes = [ctypes.c_int, i64p]
        L.zfpo_stream_bytes_f64.restype = ctypes.c_int64
        L.zfpo_encode_block_f64.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.zfpo_decode_block_f64.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.zfpo_encode_array_f64.argtypes = [ctypes.c_int, ctypes.c_void_p, i64p, i64p, ctypes.c_void_p,
                                            ctypes.c_int64]
        L.zfpo_decode_array_f64.argtypes = [ctypes.c_int, ctypes.c_void_p, i64p, ctypes.c_void_p, i64p]
        L.zfpo_encode_precision.argtypes = [ctypes.c_void_p, i64p, i64p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
        _lib = L
    return _lib


def _i64x3(v):
    return (ctypes.c_int64 * 3)(*[int(x) for x in v])


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def overflow_reset():
    lib().zfpo_overflow_reset()


def overflow_count():
    return int(lib().zfpo_overflow_count())


# ---------------------------------------------------------------- transform
def lift_forward_exact(v):
    a = np.array(v, dtype=np.float64).copy()
    lib().zfpo_lift_forward_exact(_ptr(a))
    return a


def lift_inverse_exact(v):
    a = np.array(v, dtype=np.float64).copy()
    lib().zfpo_lift_inverse_exact(_ptr(a))
    return a


def lift_forward(v):
    a = np.array(v, dtype=np.int32).copy()
    lib().zfpo_lift_forward(_ptr(a))
    return a


def lift_inverse(v):
    a = np.array(v, dtype=np.int32).copy()
    lib().zfpo_lift_inverse(_ptr(a))
    return a


def xform_forward(dims, q):
    a = np.ascontiguousarray(q, dtype=np.int32).copy()
    lib().zfpo_xform_forward(dims, _ptr(a))
    return a


def xform_inverse(dims, q):
    a = np.ascontiguousarray(q, dtype=np.int32).copy()
    lib().zfpo_xform_inverse(dims, _ptr(a))
    return a


def sequency_order(dims):
    S = 4 ** dims
    a = np.zeros(S, dtype=np.int32)
    lib().zfpo_sequency_order(dims, _ptr(a))
    return a


def to_negabinary(q):
    return int(lib().zfpo_to_negabinary(int(q)))


def from_negabinary(u):
    return int(lib().zfpo_from_negabinary(int(u)))


# ---------------------------------------------------------------- coder
def plane_bits(S, plane, n):
    n_out = ctypes.c_int(0)
    bits = lib().zfpo_plane_bits(S, int(plane), int(n), ctypes.byref(n_out))
    return bits, n_out.value


def encode_planes(u, budget):
    u = np.ascontiguousarray(u, dtype=np.uint32)
    out = np.zeros((int(budget) + 7) // 8 + 8, dtype=np.uint8)
    used = lib().zfpo_encode_planes(len(u), _ptr(u), int(budget), _ptr(out))
    return out, int(used)


def decode_planes(S, stream, budget):
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    u = np.zeros(S, dtype=np.uint32)
    used = lib().zfpo_decode_planes(S, _ptr(stream), int(budget), _ptr(u))
    return u, int(used)


# ---------------------------------------------------------------- blocks / arrays
def block_bytes(dims, rate):
    return (4 ** dims) * rate // 8


def encode_block(dims, rate, v):
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1)
    assert v.size == 4 ** dims
    out = np.zeros(((4 ** dims) * rate + 7) // 8, dtype=np.uint8)
    rc = lib().zfpo_encode_block(dims, rate, _ptr(v), _ptr(out))
    if rc:
        raise ValueError("invalid dims/rate")
    return out


def decode_block(dims, rate, stream):
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    v = np.zeros(4 ** dims, dtype=np.float32)
    rc = lib().zfpo_decode_block(dims, rate, _ptr(stream), _ptr(v))
    if rc:
        raise ValueError("invalid dims/rate")
    return v


def block_count(dims, n):
    return int(lib().zfpo_block_count(dims, _i64x3(n)))


def stream_bytes(dims, rate, n):
    return int(lib().zfpo_stream_bytes(dims, rate, _i64x3(n)))


def _strides_elems(a):
    """Element strides of a float32 numpy array indexed [z][y][x] -> (sx, sy, sz)."""
    assert a.dtype == np.float32 and a.ndim == 3
    sz, sy, sx = (s // 4 for s in a.strides)
    return (sx, sy, sz)


def encode_array(dims, rate, a):
    """Encode a float32 array indexed [z][y][x] (any strides). Returns uint8 stream."""
    nz, ny, nx = a.shape
    n = (nx, ny, nz)
    nbytes = stream_bytes(dims, rate, n)
    out = np.zeros(max(nbytes, 1), dtype=np.uint8)
    rc = lib().zfpo_encode_array(dims, rate, a.ctypes.data_as(ctypes.c_void_p), _i64x3(n),
                                 _i64x3(_strides_elems(a)), _ptr(out), nbytes)
    if rc:
        raise ValueError("zfpo_encode_array failed: %d" % rc)
    return out[:nbytes]


def decode_array(dims, rate, stream, out):
    """Decode into the float32 array ``out`` indexed [z][y][x] (any strides, written in place)."""
    nz, ny, nx = out.shape
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    rc = lib().zfpo_decode_array(dims, rate, _ptr(stream), _i64x3((nx, ny, nz)),
                                 out.ctypes.data_as(ctypes.c_void_p),
                                 _i64x3(_strides_elems(out)))
    if rc:
        raise ValueError("zfpo_decode_array failed: %d" % rc)
    return out


# ---------------------------------------------------------------- accuracy mode
def accuracy_minexp(tol):
    return int(lib().zfpo_accuracy_minexp(float(tol)))


def accuracy_kmin(emax, minexp):
    return int(lib().zfpo_accuracy_kmin(int(emax), int(minexp)))


def encode_accuracy(a, tol):
    """Accuracy-mode coding of a float32 array indexed [z][y][x] (any strides) with
    3-D blocks.  Returns (lengths uint16 per block, payload bytes, total bits)."""
    return _encode_variable(a, float(tol), None)


def encode_precision(a, prec):
    """Precision-mode coding (the top `prec` bit planes of every block); the same
    output as encode_accuracy and decoded by decode_accuracy."""
    return _encode_variable(a, None, int(prec))


def _encode_variable(a, tol, prec):
    nz, ny, nx = a.shape
    n = (nx, ny, nz)
    nblk = block_count(3, n)
    cap = int(lib().zfpo_accuracy_max_payload_bytes(_i64x3(n)))
    lengths = np.zeros(max(nblk, 1), dtype=np.uint16)
    payload = np.zeros(max(cap, 1), dtype=np.uint8)
    bits = ctypes.c_uint64(0)
    args = (a.ctypes.data_as(ctypes.c_void_p), _i64x3(n), _i64x3(_strides_elems(a)))
    if prec is None:
        rc = lib().zfpo_encode_accuracy(*args, tol, _ptr(lengths), _ptr(payload), cap, ctypes.byref(bits))
    else:
        rc = lib().zfpo_encode_precision(*args, prec, _ptr(lengths), _ptr(payload), cap, ctypes.byref(bits))
    if rc:
        raise ValueError("variable-rate encode failed: %d" % rc)
    total = int(bits.value)
    return lengths[:nblk], payload[:(total + 7) // 8], total


def decode_accuracy(lengths, payload, out):
    """Decode into the float32 array ``out`` indexed [z][y][x] (written in place)."""
    nz, ny, nx = out.shape
    lengths = np.ascontiguousarray(lengths, dtype=np.uint16)
    payload = np.ascontiguousarray(np.concatenate([np.asarray(payload, np.uint8), np.zeros(8, np.uint8)]))
    rc = lib().zfpo_decode_accuracy(_ptr(lengths), _ptr(payload), _i64x3((nx, ny, nz)),
                                    out.ctypes.data_as(ctypes.c_void_p), _i64x3(_strides_elems(out)))
    if rc:
        raise ValueError("zfpo_decode_accuracy failed: %d" % rc)
    return out


# ---------------------------------------------------------------- float64 fields (3-D blocks)
def xform_forward_i64(q):
    a = np.ascontiguousarray(q, dtype=np.int64).copy()
    lib().zfpo_xform_forward_i64(_ptr(a))
    return a


def xform_inverse_i64(q):
    a = np.ascontiguousarray(q, dtype=np.int64).copy()
    lib().zfpo_xform_inverse_i64(_ptr(a))
    return a


def stream_bytes_f64(rate, n):
    return int(lib().zfpo_stream_bytes_f64(rate, _i64x3(n)))


def encode_block_f64(rate, v):
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    assert v.size == 64
    out = np.zeros(8 * rate, dtype=np.uint8)
    if lib().zfpo_encode_block_f64(rate, _ptr(v), _ptr(out)):
        raise ValueError("invalid rate")
    return out


def decode_block_f64(rate, stream):
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    v = np.zeros(64, dtype=np.float64)
    if lib().zfpo_decode_block_f64(rate, _ptr(stream), _ptr(v)):
        raise ValueError("invalid rate")
    return v


def _strides_f64(a):
    assert a.dtype == np.float64 and a.ndim == 3
    sz, sy, sx = (s // 8 for s in a.strides)
    return (sx, sy, sz)


def encode_array_f64(rate, a):
    """Encode a float64 array indexed [z][y][x] (any strides) with 3-D blocks."""
    nz, ny, nx = a.shape
    n = (nx, ny, nz)
    nbytes = stream_bytes_f64(rate, n)
    out = np.zeros(max(nbytes, 1), dtype=np.uint8)
    rc = lib().zfpo_encode_array_f64(rate, a.ctypes.data_as(ctypes.c_void_p), _i64x3(n), _i64x3(_strides_f64(a)),
                                     _ptr(out), nbytes)
    if rc:
        raise ValueError("zfpo_encode_array_f64 failed: %d" % rc)
    return out[:nbytes]


def decode_array_f64(rate, stream, out):
    nz, ny, nx = out.shape
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    rc = lib().zfpo_decode_array_f64(rate, _ptr(stream), _i64x3((nx, ny, nz)), out.ctypes.data_as(ctypes.c_void_p),
                                     _i64x3(_strides_f64(out)))
    if rc:
        raise ValueError("zfpo_decode_array_f64 failed: %d" % rc)
    return out
