"""The C-ABI library without a GPU: it builds, loads, exports every declared
symbol, and its host-side plan agrees with the oracle's plan (Sec. II-B;
Table 1).  No call here launches a kernel."""
import ctypes
import math

import pytest

from oracle.plan import Plan as OPlan, message_bytes as omsg_bytes


@pytest.fixture(scope="module")
def zfpx():
    from paper_2609_24294_gb300 import build, zfpx as z
    build.build()
    z.lib()
    return z


def test_exports_every_declared_symbol(zfpx):
    names = zfpx.declared_symbols()
    assert len(names) >= 20
    L = ctypes.CDLL(zfpx.library_path())
    for n in names:
        assert hasattr(L, n), n


def test_strerror_and_counter(zfpx):
    L = zfpx.lib()
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert L.zfpx_strerror(code)
    assert zfpx.zfpx_launch_count() >= 0


@pytest.mark.parametrize("N", [4, 9, 16, 25, 36, 49, 64, 81, 100, 121])
def test_library_plan_reproduces_table1(zfpx, N):
    p = int(round(math.sqrt(N)))
    plan = zfpx.Plan((2560, 1280, 137), p, p, 0, 3, zfpx.SPLIT_TABLE1)
    op = OPlan(2560, 1280, 137, p, p, 0, 3, "table1")
    m = op.messages[0]
    for r in (0, -16, 8, 16):
        assert plan.message_bytes(r, m.src, m.dst) == omsg_bytes(m, r, 3)


@pytest.mark.parametrize("t", [0, 1])
@pytest.mark.parametrize("dims", [1, 2, 3])
@pytest.mark.parametrize("shape,pr,pc", [((37, 23, 17), 3, 2), ((64, 32, 8), 2, 2), ((5, 3, 1), 2, 3),
                                         ((1280, 640, 137), 8, 8)])
def test_library_plan_matches_oracle_plan(zfpx, t, dims, shape, pr, pc):
    plan = zfpx.Plan(shape, pr, pc, t, dims)
    op = OPlan(*shape, pr, pc, t, dims)
    msgs = plan.messages()
    assert len(msgs) == len(op.messages)
    for (ranks, box), m in zip(msgs, op.messages):
        assert ranks == (m.src, m.dst, m.src_peer, m.dst_peer)
        assert box == (m.x0, m.nx, m.y0, m.ny, m.z0, m.nz)
    for r in (0, -16, 8, 16):
        so, ro, total = op.layout(r)
        assert plan.buffer_bytes(r) == total
        for m in op.messages[:: max(1, len(op.messages) // 40)]:
            assert plan.message_bytes(r, m.src, m.dst) == omsg_bytes(m, r, dims)
            assert plan.message_offset(r, zfpx.LAYOUT_SEND, m.src, m.dst) == so[(m.src, m.dst)]
            assert plan.message_offset(r, zfpx.LAYOUT_RECV, m.src, m.dst) == ro[(m.src, m.dst)]


def test_plan_rejects_bad_arguments(zfpx):
    for args in [((0, 4, 4), 1, 1, 0, 3), ((4, 4, 4), 0, 1, 0, 3), ((4, 4, 4), 1, 1, 2, 3),
                 ((4, 4, 4), 1, 1, 0, 4), ((4, 4, 4), 1, 1, 0, 0)]:
        with pytest.raises(zfpx.ZfpxError) as e:
            zfpx.Plan(*args)
        assert e.value.code == -1


def test_calls_reject_bad_arguments_before_any_launch(zfpx):
    L = zfpx.lib()
    plan = zfpx.Plan((8, 8, 8), 1, 1)
    h = plan.handle
    # NULL pointers, bad rates, bad layouts: ZFPX_EINVAL, nothing launched
    before = zfpx.zfpx_launch_count()
    assert L.zfpx_pack_compress(h, 8, None, None, 0, 0, None) == -1
    assert L.zfpx_pack_compress(h, 12, ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 20, 0, None) == -1
    assert L.zfpx_pack_compress(h, 8, ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 20, 5, None) == -1
    assert L.zfpx_decompress_unpack(h, 4, ctypes.c_void_p(256), 1 << 20, ctypes.c_void_p(256), 0, None) == -1
    assert L.zfpx_cast_fp16_pack(h, 7, ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 20, 0, None) == -1
    assert L.zfpx_permute(h, 8, ctypes.c_void_p(256), ctypes.c_void_p(256), 1 << 20, None) == -1   # overlap
    # undersized buffers: ZFPX_ESIZE
    need = plan.buffer_bytes(8)
    assert L.zfpx_pack_compress(h, 8, ctypes.c_void_p(256), ctypes.c_void_p(4096), need - 1, 0, None) == -2
    assert L.zfpx_pack(h, ctypes.c_void_p(256), ctypes.c_void_p(4096), 16, 0, None) == -2
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    s = (ctypes.c_int64 * 3)(1, 8, 64)
    assert L.zfpx_encode(4, 8, ctypes.c_void_p(256), n, s, ctypes.c_void_p(4096), 1 << 20, None) == -1
    assert L.zfpx_encode(2, 8, ctypes.c_void_p(256), n, s, ctypes.c_void_p(4096), 10, None) == -2
    assert L.zfpx_encode(3, 8, ctypes.c_void_p(256), n, s, ctypes.c_void_p(4096), 10, None) == -2
    assert zfpx.zfpx_launch_count() == before
    assert zfpx.zfpx_stream_bytes(3, 8, (8, 8, 8)) == 8 * 64
    assert zfpx.zfpx_stream_bytes(1, 8, (9, 2, 3)) == 3 * 2 * 3 * 4
    assert zfpx.zfpx_stream_bytes(2, 8, (9, 6, 3)) == 3 * 2 * 3 * 16
