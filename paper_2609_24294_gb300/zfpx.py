"""Python binding of libzfpx.so (include/zfpx.h): argument marshalling only.

Every compute call runs in the library's CUDA kernels; this module turns
torch tensors into device pointers and byte counts, passes the current CUDA
stream, and raises ``ZfpxError`` on a non-zero return code.  The functions
carry the C names.  If the library has not been built the first call raises.
"""
import ctypes
import os
import re

import torch

from . import build as _build

RATE_F32 = 0
RATE_F16 = -16
LAYOUT_SEND = 0
LAYOUT_RECV = 1
ROUND_NEAREST = 0
ROUND_ZERO = 1
SPLIT_BALANCED = 0
SPLIT_TABLE1 = 1

_lib = None


class ZfpxError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: zfpx error %d (%s)" % (what, code, _strerror(code)))


class View3(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64 * 3), ("stride", ctypes.c_int64 * 3)]


class Field(ctypes.Structure):
    _fields_ = [("d_src", ctypes.c_void_p), ("d_dst", ctypes.c_void_p), ("lev_stride", ctypes.c_int64),
                ("dst_lev_stride", ctypes.c_int64), ("nlev", ctypes.c_int32), ("dims", ctypes.c_int32),
                ("rate", ctypes.c_int32), ("row0", ctypes.c_int32), ("row1", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def library_path():
    return _build.LIB


def lib():
    """The loaded library; raises if libzfpx.so is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ZfpxError(-3, "libzfpx.so is not built (run paper_2609_24294_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    i64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "zfpx_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "zfpx_launch_count": ([], ctypes.c_uint64),
        "zfpx_plan_create": ([ctypes.POINTER(vp), ctypes.POINTER(View3), ctypes.POINTER(View3), ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_plan_destroy": ([vp], None),
        "zfpx_plan_prepare": ([vp, ctypes.c_int], ctypes.c_int),
        "zfpx_plan_num_messages": ([vp], ctypes.c_int),
        "zfpx_plan_message": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), i64p], ctypes.c_int),
        "zfpx_message_bytes": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], sz),
        "zfpx_message_offset": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], i64),
        "zfpx_buffer_bytes": ([vp, ctypes.c_int], sz),
        "zfpx_pack_compress": ([vp, ctypes.c_int, vp, vp, sz, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_decompress_unpack": ([vp, ctypes.c_int, vp, sz, vp, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_cast_fp16_pack": ([vp, ctypes.c_int, vp, vp, sz, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_fp16_unpack": ([vp, vp, sz, vp, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_pack": ([vp, vp, vp, sz, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_unpack": ([vp, vp, sz, vp, ctypes.c_int, vp], ctypes.c_int),
        "zfpx_permute": ([vp, ctypes.c_int, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_stream_bytes": ([ctypes.c_int, ctypes.c_int, i64p], sz),
        "zfpx_encode": ([ctypes.c_int, ctypes.c_int, vp, i64p, i64p, vp, sz, vp], ctypes.c_int),
        "zfpx_decode": ([ctypes.c_int, ctypes.c_int, vp, sz, i64p, i64p, vp, vp], ctypes.c_int),
        "zfpx_pair_graph_create": ([ctypes.POINTER(vp), vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, sz, ctypes.c_int],
                                   ctypes.c_int),
        "zfpx_graph_launch": ([vp, vp], ctypes.c_int),
        "zfpx_transpose_noalloc": ([vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "zfpx_pipeline_create": ([ctypes.POINTER(vp), vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_pipeline_pieces": ([vp], ctypes.c_int),
        "zfpx_pipeline_run": ([vp, vp, vp, vp, sz, vp, vp], ctypes.c_int),
        "zfpx_pipeline_destroy": ([vp], None),
        "zfpx_set_units_per_warp": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_get_units_per_warp": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_capture_begin": ([vp], ctypes.c_int),
        "zfpx_server_create": ([ctypes.POINTER(vp), i64p, ctypes.c_int, sz, ctypes.c_int, ctypes.c_int],
                               ctypes.c_int),
        "zfpx_server_destroy": ([vp], None),
        "zfpx_server_set_launch": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_server_set_unit_blocks": ([vp, ctypes.c_int], ctypes.c_int),
        "zfpx_server_set_claim_units": ([vp, ctypes.c_int], ctypes.c_int),
        "zfpx_server_set_batching": ([vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
        "zfpx_server_submit": ([vp, ctypes.POINTER(Field), i64p], ctypes.c_int),
        "zfpx_server_pump": ([vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "zfpx_server_poll": ([vp, i64p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "zfpx_server_result": ([vp, ctypes.c_int64, ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(vp),
                                ctypes.POINTER(sz)], ctypes.c_int),
        "zfpx_server_release": ([vp, ctypes.c_int64], ctypes.c_int),
        "zfpx_server_copy_result": ([vp, ctypes.c_int64, vp, sz, vp, sz], ctypes.c_int),
        "zfpx_server_stats": ([vp, i64p], ctypes.c_int),
        "zfpx_server_run": ([vp, ctypes.POINTER(Field), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "zfpx_capture_end": ([ctypes.POINTER(vp), vp], ctypes.c_int),
        "zfpx_batch_create": ([ctypes.POINTER(vp), i64p, ctypes.c_int, ctypes.POINTER(Field), ctypes.c_int],
                              ctypes.c_int),
        "zfpx_batch_destroy": ([vp], None),
        "zfpx_batch_bytes": ([vp], sz),
        "zfpx_batch_field_offset": ([vp, ctypes.c_int], i64),
        "zfpx_batch_field_bytes": ([vp, ctypes.c_int], sz),
        "zfpx_batch_set_launch": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_batch_set_unit_blocks": ([vp, ctypes.c_int], ctypes.c_int),
        "zfpx_batch_set_claim_units": ([vp, ctypes.c_int], ctypes.c_int),
        "zfpx_batch_encode": ([vp, vp, sz, vp], ctypes.c_int),
        "zfpx_batch_decode": ([vp, vp, sz, vp], ctypes.c_int),
        "zfpx_graph_num_kernels": ([vp], ctypes.c_int),
        "zfpx_accuracy_workspace_bytes": ([i64p], sz),
        "zfpx_accuracy_max_payload_bytes": ([i64p], sz),
        "zfpx_encode_accuracy": ([vp, i64p, i64p, ctypes.c_double, vp, vp, sz, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_decode_accuracy": ([vp, vp, sz, i64p, i64p, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_plan_accuracy_blocks": ([vp], sz),
        "zfpx_plan_accuracy_workspace_bytes": ([vp], sz),
        "zfpx_pack_compress_accuracy": ([vp, ctypes.c_double, vp, vp, vp, sz, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_pack_compress_precision": ([vp, ctypes.c_int, vp, vp, vp, sz, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_encode_precision": ([vp, i64p, i64p, ctypes.c_int, vp, vp, sz, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_exchange_accuracy": ([vp, vp, vp, vp, vp, vp, sz, vp, sz, vp], ctypes.c_int),
        "zfpx_decompress_unpack_accuracy": ([vp, vp, vp, vp, sz, vp, vp, sz, vp], ctypes.c_int),
        "zfpx_stream_bytes_f64": ([ctypes.c_int, i64p], sz),
        "zfpx_encode_f64": ([ctypes.c_int, vp, i64p, i64p, vp, sz, vp], ctypes.c_int),
        "zfpx_decode_f64": ([ctypes.c_int, vp, sz, i64p, i64p, vp, vp], ctypes.c_int),
        "zfpx_rfft_lon": ([vp, i64p, i64p, ctypes.c_int, vp, vp, i64p, vp], ctypes.c_int),
        "zfpx_count_nonfinite": ([vp, ctypes.c_int, i64p, i64p, vp, vp], ctypes.c_int),
        "zfpx_gauss_legendre": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                                ctypes.c_int),
        "zfpx_legendre_create": ([ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "zfpx_legendre_destroy": ([vp], None),
        "zfpx_legendre_status": ([vp], ctypes.c_int),
        "zfpx_decompress_rfft_workspace_bytes": ([vp], sz),
        "zfpx_decompress_rfft": ([vp, ctypes.c_int, vp, sz, ctypes.c_int, vp, vp, i64p, vp, sz, vp], ctypes.c_int),
        "zfpx_legendre_workspace_bytes": ([vp, ctypes.c_int64], sz),
        "zfpx_legendre_forward": ([vp, vp, vp, i64p, i64p, vp, vp, ctypes.c_int64, vp, sz, vp], ctypes.c_int),
        "zfpx_graph_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def declared_symbols():
    """Names of every entry point declared in include/zfpx.h."""
    hdr = os.path.join(os.path.dirname(_build.PKG), "include", "zfpx.h")
    return re.findall(r"ZFPX_API\s+[\w\s\*]*?\b(zfpx_\w+)\s*\(", open(hdr).read())


def _strerror(code):
    try:
        return lib().zfpx_strerror(int(code)).decode()
    except Exception:
        return "?"


def _check(rc, what):
    if rc != 0:
        raise ZfpxError(rc, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, what):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


def _nbytes(t):
    return t.numel() * t.element_size()


def _i64x3(v):
    return (ctypes.c_int64 * 3)(*[int(x) for x in v])


def field_view(t):
    """(n, strides) in (lon, lat, lev) order of a [lev][lat][lon] float32 tensor."""
    if t.dim() != 3:
        raise ValueError("field must be a 3-D [lev][lat][lon] tensor")
    return tuple(reversed(t.shape)), tuple(reversed(t.stride()))


def zfpx_launch_count():
    return int(lib().zfpx_launch_count())


class Plan:
    """A pencil-transposition plan (zfpx_plan_create / zfpx_plan_destroy)."""

    def __init__(self, n, pr, pc, transposition=0, dims=3, split=SPLIT_BALANCED,
                 src_strides=None, dst_strides=None):
        nlon, nlat, nlev = (int(x) for x in n)
        contiguous = (1, nlon, nlon * nlat)
        self.n = (nlon, nlat, nlev)
        self.src_strides = tuple(src_strides or contiguous)
        self.dst_strides = tuple(dst_strides or contiguous)
        self.pr, self.pc, self.transposition, self.dims = pr, pc, transposition, dims
        sv = View3(_i64x3(self.n), _i64x3(self.src_strides))
        dv = View3(_i64x3(self.n), _i64x3(self.dst_strides))
        h = ctypes.c_void_p()
        _check(lib().zfpx_plan_create(ctypes.byref(h), ctypes.byref(sv), ctypes.byref(dv), pr, pc,
                                      transposition, dims, split), "zfpx_plan_create")
        self._h = h

    @classmethod
    def for_fields(cls, src, pr, pc, transposition=0, dims=3, dst=None, split=SPLIT_BALANCED):
        n, ss = field_view(src)
        ds = field_view(dst)[1] if dst is not None else ss
        if dst is not None and field_view(dst)[0] != n:
            raise ValueError("src and dst fields differ in shape")
        return cls(n, pr, pc, transposition, dims, split, ss, ds)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.zfpx_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def prepare(self, rate):
        _check(lib().zfpx_plan_prepare(self.handle, rate), "zfpx_plan_prepare")

    def num_messages(self):
        return lib().zfpx_plan_num_messages(self.handle)

    def messages(self):
        out = []
        ranks = (ctypes.c_int32 * 4)()
        box = (ctypes.c_int64 * 6)()
        for i in range(self.num_messages()):
            _check(lib().zfpx_plan_message(self.handle, i, ranks, box), "zfpx_plan_message")
            out.append((tuple(ranks), tuple(box)))
        return out

    def message_bytes(self, rate, src, dst):
        return int(lib().zfpx_message_bytes(self.handle, rate, src, dst))

    def message_offset(self, rate, layout, src, dst):
        return int(lib().zfpx_message_offset(self.handle, rate, layout, src, dst))

    def buffer_bytes(self, rate):
        return int(lib().zfpx_buffer_bytes(self.handle, rate))

    def _check_field(self, t, strides, what):
        if t.dtype != torch.float32:
            raise ValueError("%s must be float32" % what)
        n, s = field_view(t)
        if tuple(n) != self.n or tuple(s) != tuple(strides):
            raise ValueError("%s shape/strides %s/%s do not match the plan %s/%s" % (what, n, s, self.n, strides))


def zfpx_pack_compress(plan, rate, src, out, layout=LAYOUT_SEND, stream=None):
    plan._check_field(src, plan.src_strides, "src")
    _check(lib().zfpx_pack_compress(plan.handle, rate, _dev(src, "src"), _dev(out, "out"), _nbytes(out), layout,
                                    _stream(stream)), "zfpx_pack_compress")


def zfpx_decompress_unpack(plan, rate, inp, dst, layout=LAYOUT_RECV, stream=None):
    plan._check_field(dst, plan.dst_strides, "dst")
    _check(lib().zfpx_decompress_unpack(plan.handle, rate, _dev(inp, "in"), _nbytes(inp), _dev(dst, "dst"), layout,
                                        _stream(stream)), "zfpx_decompress_unpack")


def zfpx_cast_fp16_pack(plan, round_mode, src, out, layout=LAYOUT_SEND, stream=None):
    plan._check_field(src, plan.src_strides, "src")
    _check(lib().zfpx_cast_fp16_pack(plan.handle, round_mode, _dev(src, "src"), _dev(out, "out"), _nbytes(out),
                                     layout, _stream(stream)), "zfpx_cast_fp16_pack")


def zfpx_fp16_unpack(plan, inp, dst, layout=LAYOUT_RECV, stream=None):
    plan._check_field(dst, plan.dst_strides, "dst")
    _check(lib().zfpx_fp16_unpack(plan.handle, _dev(inp, "in"), _nbytes(inp), _dev(dst, "dst"), layout,
                                  _stream(stream)), "zfpx_fp16_unpack")


def zfpx_pack(plan, src, out, layout=LAYOUT_SEND, stream=None):
    plan._check_field(src, plan.src_strides, "src")
    _check(lib().zfpx_pack(plan.handle, _dev(src, "src"), _dev(out, "out"), _nbytes(out), layout, _stream(stream)),
           "zfpx_pack")


def zfpx_unpack(plan, inp, dst, layout=LAYOUT_RECV, stream=None):
    plan._check_field(dst, plan.dst_strides, "dst")
    _check(lib().zfpx_unpack(plan.handle, _dev(inp, "in"), _nbytes(inp), _dev(dst, "dst"), layout, _stream(stream)),
           "zfpx_unpack")


def zfpx_permute(plan, rate, send, recv, stream=None):
    _check(lib().zfpx_permute(plan.handle, rate, _dev(send, "send"), _dev(recv, "recv"),
                              min(_nbytes(send), _nbytes(recv)), _stream(stream)), "zfpx_permute")


def zfpx_stream_bytes(dims, rate, n):
    return int(lib().zfpx_stream_bytes(dims, rate, _i64x3(n)))


def zfpx_encode(dims, rate, src, out, stream=None):
    if src.dtype != torch.float32:
        raise ValueError("src must be float32")
    n, s = field_view(src)
    _check(lib().zfpx_encode(dims, rate, _dev(src, "src"), _i64x3(n), _i64x3(s), _dev(out, "out"), _nbytes(out),
                             _stream(stream)), "zfpx_encode")


def zfpx_decode(dims, rate, inp, dst, stream=None):
    if dst.dtype != torch.float32:
        raise ValueError("dst must be float32")
    n, s = field_view(dst)
    _check(lib().zfpx_decode(dims, rate, _dev(inp, "in"), _nbytes(inp), _i64x3(n), _i64x3(s), _dev(dst, "dst"),
                             _stream(stream)), "zfpx_decode")


def zfpx_accuracy_workspace_bytes(n):
    return int(lib().zfpx_accuracy_workspace_bytes(_i64x3(n)))


def zfpx_accuracy_max_payload_bytes(n):
    return int(lib().zfpx_accuracy_max_payload_bytes(_i64x3(n)))


def zfpx_encode_accuracy(src, tolerance, lengths, payload, total_bits, work, stream=None):
    """Accuracy-mode encode of a [lev][lat][lon] float32 field (any strides) with 3-D
    blocks; lengths: uint16 tensor (one per block), payload: uint8 tensor of at least
    zfpx_accuracy_max_payload_bytes, total_bits: int64 tensor of one element, work:
    uint8 tensor of zfpx_accuracy_workspace_bytes (all on the device)."""
    if src.dtype != torch.float32:
        raise ValueError("src must be float32")
    n, s = field_view(src)
    _check(lib().zfpx_encode_accuracy(_dev(src, "src"), _i64x3(n), _i64x3(s), float(tolerance),
                                      _dev(lengths, "lengths"), _dev(payload, "payload"), _nbytes(payload),
                                      _dev(total_bits, "total_bits"), _dev(work, "work"), _nbytes(work),
                                      _stream(stream)), "zfpx_encode_accuracy")


def zfpx_encode_precision(src, precision, lengths, payload, total_bits, work, stream=None):
    """Precision-mode encode (every block keeps its top `precision` bit planes);
    the same buffers as zfpx_encode_accuracy, decoded by zfpx_decode_accuracy."""
    if src.dtype != torch.float32:
        raise ValueError("src must be float32")
    n, s = field_view(src)
    _check(lib().zfpx_encode_precision(_dev(src, "src"), _i64x3(n), _i64x3(s), int(precision),
                                       _dev(lengths, "lengths"), _dev(payload, "payload"), _nbytes(payload),
                                       _dev(total_bits, "total_bits"), _dev(work, "work"), _nbytes(work),
                                       _stream(stream)), "zfpx_encode_precision")


def zfpx_decode_accuracy(lengths, payload, dst, work, stream=None):
    """Accuracy-mode decode into the float32 field dst (any strides)."""
    n, s = field_view(dst)
    _check(lib().zfpx_decode_accuracy(_dev(lengths, "lengths"), _dev(payload, "payload"), _nbytes(payload),
                                      _i64x3(n), _i64x3(s), _dev(dst, "dst"), _dev(work, "work"), _nbytes(work),
                                      _stream(stream)), "zfpx_decode_accuracy")


def zfpx_stream_bytes_f64(rate, n):
    return int(lib().zfpx_stream_bytes_f64(int(rate), _i64x3(n)))


def zfpx_encode_f64(rate, src, out, stream=None):
    """Fixed-rate encode of a float64 [lev][lat][lon] tensor (any strides) into
    the uint8 tensor out (>= zfpx_stream_bytes_f64 bytes)."""
    if src.dtype != torch.float64:
        raise ValueError("src must be float64")
    n, s = field_view(src)
    _check(lib().zfpx_encode_f64(int(rate), _dev(src, "src"), _i64x3(n), _i64x3(s), _dev(out, "out"),
                                 _nbytes(out), _stream(stream)), "zfpx_encode_f64")


def zfpx_decode_f64(rate, stream_bytes, dst, stream=None):
    """Fixed-rate decode into the float64 tensor dst (any strides)."""
    if dst.dtype != torch.float64:
        raise ValueError("dst must be float64")
    n, s = field_view(dst)
    _check(lib().zfpx_decode_f64(int(rate), _dev(stream_bytes, "stream"), _nbytes(stream_bytes), _i64x3(n),
                                 _i64x3(s), _dev(dst, "dst"), _stream(stream)), "zfpx_decode_f64")


def zfpx_rfft_lon(src, re, im, stream=None):
    """Longitude transform of every row of the float32 [lev][lat][lon] tensor src:
    re / im (float32 [lev][lat][K], the same strides) get the real / imaginary
    parts of F_m = (1/N) sum_j x_j e^{-2 pi i j m / N}, m < K = re.shape[-1]."""
    for t, w in ((src, "src"), (re, "re"), (im, "im")):
        if t.dtype != torch.float32 or t.dim() != 3:
            raise ValueError("%s must be a 3-D float32 tensor" % w)
    if re.shape != im.shape or re.stride() != im.stride() or re.shape[:2] != src.shape[:2]:
        raise ValueError("re and im must have the same shape and strides, over src's rows")
    n, s = field_view(src)
    _, os_ = field_view(re)
    _check(lib().zfpx_rfft_lon(_dev(src, "src"), _i64x3(n), _i64x3(s), int(re.shape[-1]), _dev(re, "re"),
                               _dev(im, "im"), _i64x3(os_), _stream(stream)), "zfpx_rfft_lon")


def zfpx_count_nonfinite(src, count, stream=None):
    """Adds to count (a one-element int64 CUDA tensor) the number of infinities
    and NaNs in the float32 or float64 CUDA tensor src (1 to 3 dimensions, the
    last one fastest; any non-negative strides).  The codec codes a block
    holding one as a zero block; this is the debug report of such inputs."""
    if src.dtype not in (torch.float32, torch.float64) or not 1 <= src.dim() <= 3:
        raise ValueError("src must be a 1-D to 3-D float32 or float64 tensor")
    if count.dtype != torch.int64 or count.numel() != 1:
        raise ValueError("count must be a one-element int64 tensor")
    if src.numel() == 0:
        return
    n = tuple(reversed(src.shape)) + (1,) * (3 - src.dim())
    s = tuple(reversed(src.stride())) + (0,) * (3 - src.dim())
    _check(lib().zfpx_count_nonfinite(_dev(src, "src"), src.element_size(), _i64x3(n), _i64x3(s),
                                      _dev(count, "count"), _stream(stream)), "zfpx_count_nonfinite")


def zfpx_gauss_legendre(n):
    """(mu, w): the Gauss-Legendre latitudes (sin of latitude, north to south) and
    weights the Legendre plan uses, as two lists of n floats (host computation)."""
    mu = (ctypes.c_double * int(n))()
    w = (ctypes.c_double * int(n))()
    _check(lib().zfpx_gauss_legendre(int(n), mu, w), "zfpx_gauss_legendre")
    return list(mu), list(w)


class Legendre:
    """The Legendre transform on Gauss-Legendre latitudes (zfpx_legendre_create /
    zfpx_legendre_forward / zfpx_legendre_destroy); the workspace is a PyTorch
    allocation kept per level count."""

    def __init__(self, nlat, T):
        h = ctypes.c_void_p()
        _check(lib().zfpx_legendre_create(ctypes.byref(h), int(nlat), int(T)), "zfpx_legendre_create")
        self._h, self.nlat, self.T = h, int(nlat), int(T)
        self.ncoeffs = (self.T + 1) * (self.T + 2) // 2
        self._work = {}

    def close(self):
        if self._h:
            lib().zfpx_legendre_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, nlev):
        return int(lib().zfpx_legendre_workspace_bytes(self._h, int(nlev)))

    def status(self):
        """Synchronously checks that no earlier forward gave up on a bounded
        device-side wait (raises ZfpxError(ZFPX_ETIMEOUT) if one did)."""
        _check(lib().zfpx_legendre_status(self._h), "zfpx_legendre_status")

    def forward(self, re, im, are, aim, stream=None):
        """re, im: float32 [lev][nlat][K] wavenumber fields (same strides); are, aim:
        float32 [lev][>= ncoeffs] (same level stride), the coefficients a_l^m."""
        if not self._h:
            raise ValueError("plan destroyed")
        for t, w in ((re, "re"), (im, "im"), (are, "are"), (aim, "aim")):
            if t.dtype != torch.float32:
                raise ValueError("%s must be float32" % w)
        if re.shape != im.shape or re.stride() != im.stride() or re.dim() != 3:
            raise ValueError("re and im must be 3-D with the same shape and strides")
        if are.dim() != 2 or are.shape != aim.shape or are.stride() != aim.stride() or are.stride(1) != 1 \
                or are.shape[0] != re.shape[0] or are.shape[1] < self.ncoeffs:
            raise ValueError("are and aim must be [lev][>= (T+1)(T+2)/2] with unit inner stride")
        nlev = re.shape[0]
        work = self._work.get(nlev)
        if work is None:
            work = torch.empty(max(16, self.workspace_bytes(nlev)), dtype=torch.uint8, device=re.device)
            self._work[nlev] = work
        n, s = field_view(re)
        _check(lib().zfpx_legendre_forward(self._h, _dev(re, "re"), _dev(im, "im"), _i64x3(n), _i64x3(s),
                                           _dev(are, "are"), _dev(aim, "aim"), int(are.stride(0)), _dev(work, "work"),
                                           _nbytes(work), _stream(stream)), "zfpx_legendre_forward")


class AccuracyTransposition:
    """The accuracy (or precision) mode on a plan: pack+compress, the
    all-to-all-v and decompress+unpack with device buffers owned here (PyTorch
    allocations)."""

    def __init__(self, plan):
        self.plan = plan
        self.G = int(lib().zfpx_plan_accuracy_blocks(plan.handle))
        M = plan.num_messages()
        self.cap = max(8, 128 * self.G)
        dev = "cuda"
        self.len_send = torch.zeros(max(1, self.G), dtype=torch.int16, device=dev)
        self.len_recv = torch.zeros_like(self.len_send)
        self.pay_send = torch.zeros(self.cap, dtype=torch.uint8, device=dev)
        self.pay_recv = torch.zeros_like(self.pay_send)
        self.words = torch.zeros(max(1, M), dtype=torch.int64, device=dev)
        self.work = torch.zeros(int(lib().zfpx_plan_accuracy_workspace_bytes(plan.handle)), dtype=torch.uint8,
                                device=dev)

    def compress(self, src, tolerance, stream=None):
        self.plan._check_field(src, self.plan.src_strides, "src")
        _check(lib().zfpx_pack_compress_accuracy(self.plan.handle, float(tolerance), _dev(src, "src"),
                                                 _dev(self.len_send, "lengths"), _dev(self.pay_send, "payload"),
                                                 self.cap, _dev(self.words, "words"), _dev(self.work, "work"),
                                                 _nbytes(self.work), _stream(stream)), "zfpx_pack_compress_accuracy")

    def compress_precision(self, src, precision, stream=None):
        self.plan._check_field(src, self.plan.src_strides, "src")
        _check(lib().zfpx_pack_compress_precision(self.plan.handle, int(precision), _dev(src, "src"),
                                                  _dev(self.len_send, "lengths"), _dev(self.pay_send, "payload"),
                                                  self.cap, _dev(self.words, "words"), _dev(self.work, "work"),
                                                  _nbytes(self.work), _stream(stream)), "zfpx_pack_compress_precision")

    def exchange(self, stream=None):
        _check(lib().zfpx_exchange_accuracy(self.plan.handle, _dev(self.words, "words"),
                                            _dev(self.len_send, "len_send"), _dev(self.pay_send, "pay_send"),
                                            _dev(self.len_recv, "len_recv"), _dev(self.pay_recv, "pay_recv"),
                                            self.cap, _dev(self.work, "work"), _nbytes(self.work),
                                            _stream(stream)), "zfpx_exchange_accuracy")

    def decompress(self, dst, stream=None):
        self.plan._check_field(dst, self.plan.dst_strides, "dst")
        _check(lib().zfpx_decompress_unpack_accuracy(self.plan.handle, _dev(self.words, "words"),
                                                     _dev(self.len_recv, "len_recv"), _dev(self.pay_recv, "pay_recv"),
                                                     self.cap, _dev(dst, "dst"), _dev(self.work, "work"),
                                                     _nbytes(self.work), _stream(stream)),
               "zfpx_decompress_unpack_accuracy")


class PairGraph:
    """The transposition pair as one CUDA graph (zfpx_pair_graph_create):
    first plan src -> mid, second plan mid -> dst, with caller-owned send /
    receive scratch buffers.  The tensors must outlive the graph."""

    def __init__(self, first, second, rate, src, mid, dst, send, recv, fold_permute=False):
        first._check_field(src, first.src_strides, "src")
        first._check_field(mid, first.dst_strides, "mid")
        second._check_field(mid, second.src_strides, "mid")
        second._check_field(dst, second.dst_strides, "dst")
        h = ctypes.c_void_p()
        _check(lib().zfpx_pair_graph_create(ctypes.byref(h), first.handle, second.handle, rate, _dev(src, "src"),
                                            _dev(mid, "mid"), _dev(dst, "dst"), _dev(send, "send"),
                                            _dev(recv, "recv"), min(_nbytes(send), _nbytes(recv)),
                                            1 if fold_permute else 0), "zfpx_pair_graph_create")
        self._h = h
        self._keep = (first, second, src, mid, dst, send, recv)

    def launch(self, stream=None):
        _check(lib().zfpx_graph_launch(self._h, _stream(stream)), "zfpx_graph_launch")

    def num_kernels(self):
        return int(lib().zfpx_graph_num_kernels(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.zfpx_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A CUDA graph recorded from zfpx calls (zfpx_capture_begin / _end)."""

    def __init__(self, handle):
        self._h = handle

    def launch(self, stream=None):
        _check(lib().zfpx_graph_launch(self._h, _stream(stream)), "zfpx_graph_launch")

    def num_kernels(self):
        return int(lib().zfpx_graph_num_kernels(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.zfpx_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def capture(fn, stream):
    """Records every zfpx call fn() makes on `stream` (a torch.cuda.Stream,
    not the default stream) into a Graph."""
    _check(lib().zfpx_capture_begin(ctypes.c_void_p(stream.cuda_stream)), "zfpx_capture_begin")
    try:
        with torch.cuda.stream(stream):
            fn()
    finally:
        h = ctypes.c_void_p()
        rc = lib().zfpx_capture_end(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream))
    _check(rc, "zfpx_capture_end")
    return Graph(h)


class Batch:
    """Batched ragged-row fields (zfpx_batch_create): fields is a list of
    (src tensor or None, dst tensor or None, dims, rate) with tensors
    [nlev][points] float32 on the device."""

    def __init__(self, row_len, fields):
        self.row_len = [int(v) for v in row_len]
        arr = (ctypes.c_int64 * len(self.row_len))(*self.row_len)
        descs = (Field * len(fields))()
        self._keep = []
        for i, (src, dst, dims, rate) in enumerate(fields):
            t = src if src is not None else dst
            if t is None or t.dim() != 2 or t.dtype != torch.float32:
                raise ValueError("field %d: need a [nlev][points] float32 tensor" % i)
            for u in (src, dst):
                if u is not None and (u.shape != t.shape or u.stride() != t.stride() or not u.is_cuda):
                    raise ValueError("field %d: src and dst must match" % i)
            descs[i].d_src = src.data_ptr() if src is not None else None
            descs[i].d_dst = dst.data_ptr() if dst is not None else None
            descs[i].lev_stride = t.stride(0)
            descs[i].dst_lev_stride = 0
            descs[i].nlev = t.shape[0]
            descs[i].dims = dims
            descs[i].rate = rate
            descs[i].row0 = 0
            descs[i].row1 = 0
            descs[i].reserved = 0
            self._keep.append((src, dst))
        h = ctypes.c_void_p()
        _check(lib().zfpx_batch_create(ctypes.byref(h), arr, len(self.row_len), descs, len(fields)),
               "zfpx_batch_create")
        self._h = h
        self.nfields = len(fields)

    def nbytes(self):
        return int(lib().zfpx_batch_bytes(self._h))

    def field_offset(self, f):
        return int(lib().zfpx_batch_field_offset(self._h, f))

    def field_bytes(self, f):
        return int(lib().zfpx_batch_field_bytes(self._h, f))

    def set_launch(self, warps_per_cta, ctas_per_sm=0):
        _check(lib().zfpx_batch_set_launch(self._h, warps_per_cta, ctas_per_sm), "zfpx_batch_set_launch")

    def set_unit_blocks(self, blocks_per_lane_1d):
        _check(lib().zfpx_batch_set_unit_blocks(self._h, blocks_per_lane_1d), "zfpx_batch_set_unit_blocks")

    def set_claim_units(self, units_per_claim):
        _check(lib().zfpx_batch_set_claim_units(self._h, units_per_claim), "zfpx_batch_set_claim_units")

    def encode(self, out, stream=None):
        _check(lib().zfpx_batch_encode(self._h, _dev(out, "out"), _nbytes(out), _stream(stream)), "zfpx_batch_encode")

    def decode(self, inp, stream=None):
        _check(lib().zfpx_batch_decode(self._h, _dev(inp, "in"), _nbytes(inp), _stream(stream)), "zfpx_batch_decode")

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.zfpx_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 64 << 20


class Pipeline:
    """A transposition pipelined per piece (zfpx_pipeline_create): compression,
    the device-local all-to-all and decompression of successive pieces of the
    plan's messages overlap on three streams."""

    def __init__(self, plan, rate, pieces):
        h = ctypes.c_void_p()
        _check(lib().zfpx_pipeline_create(ctypes.byref(h), plan.handle, int(rate), int(pieces)),
               "zfpx_pipeline_create")
        self._h, self.plan, self.rate = h, plan, int(rate)
        self.pieces = int(lib().zfpx_pipeline_pieces(h))

    def run(self, src, send, recv, dst, stream=None):
        self.plan._check_field(src, self.plan.src_strides, "src")
        self.plan._check_field(dst, self.plan.dst_strides, "dst")
        nb = min(_nbytes(send), _nbytes(recv))
        _check(lib().zfpx_pipeline_run(self._h, _dev(src, "src"), _dev(send, "send"), _dev(recv, "recv"), nb,
                                       _dev(dst, "dst"), _stream(stream)), "zfpx_pipeline_run")

    def close(self):
        if self._h:
            lib().zfpx_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zfpx_decompress_rfft(plan, rate, recv, re, im, work=None, stream=None):
    """Decodes the received messages of a z -> lambda plan and transforms every
    longitude row into wavenumbers: re, im float32 [lev][lat][K] (unit inner
    stride).  `work`: scratch of zfpx_decompress_rfft_workspace_bytes bytes
    (allocated here if None).  Returns the work tensor for reuse."""
    if re.dtype != torch.float32 or im.dtype != torch.float32 or re.shape != im.shape or re.stride() != im.stride():
        raise ValueError("re and im must be float32 with the same shape and strides")
    if re.dim() != 3 or re.stride(2) != 1:
        raise ValueError("re and im must be [lev][lat][K] with unit inner stride")
    nbytes = int(lib().zfpx_decompress_rfft_workspace_bytes(plan.handle))
    if work is None or _nbytes(work) < nbytes:
        work = torch.empty(max(16, nbytes), dtype=torch.uint8, device=re.device)
    os_ = (1, re.stride(1), re.stride(0))
    _check(lib().zfpx_decompress_rfft(plan.handle, int(rate), _dev(recv, "recv"), _nbytes(recv), int(re.shape[2]),
                                      _dev(re, "re"), _dev(im, "im"), _i64x3(os_), _dev(work, "work"), _nbytes(work),
                                      _stream(stream)), "zfpx_decompress_rfft")
    return work


def zfpx_set_units_per_warp(encode, rate, upw):
    """Launch shape of the 3-D codec kernels: 32-block units per warp (0 = default)."""
    _check(lib().zfpx_set_units_per_warp(int(bool(encode)), rate, upw), "zfpx_set_units_per_warp")


def zfpx_get_units_per_warp(encode, rate):
    return int(lib().zfpx_get_units_per_warp(int(bool(encode)), rate))


def zfpx_transpose_noalloc(plan, rate, src, dst, stream=None):
    """Compress (receive layout) then decompress through the library's fixed
    device array; allocates nothing (see include/zfpx.h)."""
    plan._check_field(src, plan.src_strides, "src")
    plan._check_field(dst, plan.dst_strides, "dst")
    _check(lib().zfpx_transpose_noalloc(plan.handle, rate, _dev(src, "src"), _dev(dst, "dst"), _stream(stream)),
           "zfpx_transpose_noalloc")
