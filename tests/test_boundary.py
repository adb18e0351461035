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


def test_exports_nothing_undeclared(zfpx):
    """The library's dynamic symbol table holds exactly the calls the header
    declares: nothing outside the documented C ABI is reachable."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("no nm")
    out = subprocess.run([nm, "-D", "--defined-only", zfpx.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = {f[-1] for f in (ln.split() for ln in out.splitlines()) if len(f) >= 3 and f[1] in "TW"}
    exported = {n for n in exported if not n.startswith("_")}
    assert exported == set(zfpx.declared_symbols())


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


def test_float64_and_spectral_calls_reject_bad_arguments_before_any_launch(zfpx):
    """float64 codec, longitude FFT and Legendre transform: argument checks run
    on the host before any CUDA call (so here, without a GPU, they answer)."""
    L = zfpx.lib()
    before = zfpx.zfpx_launch_count()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    s = (ctypes.c_int64 * 3)(1, 8, 64)
    p, q = ctypes.c_void_p(256), ctypes.c_void_p(4096)
    # float64 codec (rates 1..32, 8-byte alignment, capacity)
    assert zfpx.zfpx_stream_bytes_f64(16, (9, 6, 5)) == 3 * 2 * 2 * 8 * 16
    assert zfpx.zfpx_stream_bytes_f64(0, (4, 4, 4)) == 0 and zfpx.zfpx_stream_bytes_f64(33, (4, 4, 4)) == 0
    for rate in (0, 33):
        assert L.zfpx_encode_f64(rate, p, n, s, q, 1 << 20, None) == -1
        assert L.zfpx_decode_f64(rate, q, 1 << 20, n, s, p, None) == -1
    assert L.zfpx_encode_f64(16, None, n, s, q, 1 << 20, None) == -1
    assert L.zfpx_encode_f64(16, p, n, s, ctypes.c_void_p(4097), 1 << 20, None) == -1
    assert L.zfpx_encode_f64(16, p, n, s, q, 8 * 16 * 8 - 1, None) == -2
    assert L.zfpx_decode_f64(16, q, 8 * 16 * 8 - 1, n, s, p, None) == -2
    # longitude FFT: N even with N/2 = 2^a 3^b 5^c, N <= 8192, 1 <= K <= N/2 + 1, rows contiguous
    for nx, K in [(7, 1), (14, 1), (16386, 1), (16, 0), (16, 10)]:
        nn = (ctypes.c_int64 * 3)(nx, 2, 2)
        ss = (ctypes.c_int64 * 3)(1, nx + nx % 2, 2 * (nx + nx % 2))
        os_ = (ctypes.c_int64 * 3)(1, 16, 32)
        assert L.zfpx_rfft_lon(p, nn, ss, K, q, q, os_, None) == -1, (nx, K)
    nn = (ctypes.c_int64 * 3)(16, 2, 2)
    assert L.zfpx_rfft_lon(p, nn, (ctypes.c_int64 * 3)(2, 32, 64), 8, q, q, (ctypes.c_int64 * 3)(1, 8, 16), None) == -1
    assert L.zfpx_rfft_lon(ctypes.c_void_p(260), nn, (ctypes.c_int64 * 3)(1, 16, 32), 8, q, q,
                           (ctypes.c_int64 * 3)(1, 8, 16), None) == -1                     # rows off 8 bytes
    assert L.zfpx_rfft_lon(p, nn, (ctypes.c_int64 * 3)(1, 17, 34), 8, q, q, (ctypes.c_int64 * 3)(1, 8, 16), None) == -1
    # Legendre plan: nlat even, at most 32768, 0 <= T <= nlat - 1
    h = ctypes.c_void_p()
    for nlat, T in [(3, 1), (0, 0), (8, 8), (8, -1), (1 << 16, 10)]:
        assert L.zfpx_legendre_create(ctypes.byref(h), nlat, T) == -1, (nlat, T)
    assert L.zfpx_legendre_workspace_bytes(None, 5) == 0
    assert L.zfpx_legendre_forward(None, p, p, n, s, q, q, 64, q, 1 << 20, None) == -1
    assert zfpx.zfpx_launch_count() == before


def test_plan_size_limits(zfpx):
    """The kernels index a message's 4-value groups along x, rows and blocks
    with 32-bit integers: a plan whose message holds 2^31 or more groups, or
    whose extent passes 2^31 - 8, is refused; the same field split over more
    ranks, or just inside the limits, is accepted.  A rank grid that would
    need more than 2^24 messages is refused before any table is built.
    Host-only: no launch."""
    L = zfpx.lib()
    before = zfpx.zfpx_launch_count()

    def create(n, pr, pc, dims):
        v = zfpx.View3((ctypes.c_int64 * 3)(*n), (ctypes.c_int64 * 3)(0, 0, 0))
        h = ctypes.c_void_p()
        rc = L.zfpx_plan_create(ctypes.byref(h), ctypes.byref(v), ctypes.byref(v), pr, pc, 0, dims, 0)
        if rc == 0:
            L.zfpx_plan_destroy(h)
        return rc

    big = (1 << 31) - 8
    # at most 2^24 messages: p_r p_c p_c (z -> lambda) or p_r p_c p_r (lambda -> theta)
    assert create((64, 64, 64), 1, 8192, 3) == -1
    assert create((64, 64, 64), 64, 64, 3) == 0                              # 2^18 messages
    assert create((big, 1, 1), 1, 1, 1) == 0
    assert create((big + 1, 1, 1), 1, 1, 1) == -1
    assert create((1, big, 1), 1, 1, 3) == 0
    assert create((1, 1, big + 1), 1, 1, 3) == -1
    for dims in (1, 2, 3):
        assert create((4, 1 << 16, (1 << 15) - 1), 1, 1, dims) == 0          # 2^31 - 2^16 groups
        assert create((4, 1 << 16, 1 << 15), 1, 1, dims) == -1               # 2^31 groups
        assert create((8, 1 << 20, 1 << 12), 1, 1, dims) == -1               # 2^33 groups in one message
        assert create((8, 1 << 20, 1 << 12), 4, 4, dims) == 0                # 2^28 in each of 64
    assert zfpx.zfpx_launch_count() == before


def test_count_nonfinite_rejects_bad_arguments_before_any_launch(zfpx):
    """The debug report of non-finite inputs checks its arguments on the host
    and launches nothing for an empty view."""
    L = zfpx.lib()
    before = zfpx.zfpx_launch_count()
    n = (ctypes.c_int64 * 3)(8, 8, 8)
    s = (ctypes.c_int64 * 3)(1, 8, 64)
    p, c = ctypes.c_void_p(256), ctypes.c_void_p(4096)
    assert L.zfpx_count_nonfinite(None, 4, n, s, c, None) == -1
    assert L.zfpx_count_nonfinite(p, 4, n, s, None, None) == -1
    for eb in (0, 2, 3, 16):
        assert L.zfpx_count_nonfinite(p, eb, n, s, c, None) == -1, eb
    assert L.zfpx_count_nonfinite(ctypes.c_void_p(258), 4, n, s, c, None) == -1      # src off 4 bytes
    assert L.zfpx_count_nonfinite(ctypes.c_void_p(260), 8, n, s, c, None) == -1      # src off 8 bytes
    assert L.zfpx_count_nonfinite(p, 4, n, s, ctypes.c_void_p(4100), None) == -1     # counter off 8 bytes
    assert L.zfpx_count_nonfinite(p, 4, (ctypes.c_int64 * 3)(8, -1, 8), s, c, None) == -1
    assert L.zfpx_count_nonfinite(p, 4, n, (ctypes.c_int64 * 3)(1, -8, 64), c, None) == -1
    for empty in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):
        assert L.zfpx_count_nonfinite(p, 8, (ctypes.c_int64 * 3)(*empty), s, c, None) == 0
    assert zfpx.zfpx_launch_count() == before


@pytest.mark.parametrize("n", [1, 2, 3, 32, 640, 1280, 2560])
def test_gauss_legendre_nodes_of_the_library(zfpx, n):
    """The nodes and weights behind the Legendre plan's table (host code, no GPU)
    against numpy's Gauss-Legendre routine, north to south."""
    import numpy as np
    mu, w = zfpx.zfpx_gauss_legendre(n)
    x, ww = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(mu, x[::-1], rtol=0, atol=4e-15)
    # numpy's weights near the poles carry relative errors up to ~1e-7 at n = 2560
    np.testing.assert_allclose(w, ww[::-1], rtol=5e-7, atol=0)
    assert abs(sum(w) - 2.0) < 1e-12
    with pytest.raises(zfpx.ZfpxError):
        zfpx.zfpx_gauss_legendre(0)
    # the outermost weights against a 40-digit Newton iteration on P_n
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def pn(t):
        p0, p1 = mp.mpf(1), t
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
        return p1, p0

    for i in range(min(n, 2)):
        t = mp.mpf(mu[i])
        for _ in range(4):
            p, pm = pn(t)
            t = t - p / (n * (t * p - pm) / (t * t - 1))
        p, pm = pn(t)
        d = n * (t * p - pm) / (t * t - 1)
        assert abs(mu[i] - t) < 1e-16
        assert abs((w[i] - 2 / ((1 - t * t) * d * d)) / w[i]) < 1e-9


def test_header_is_plain_c_and_links(zfpx, tmp_path):
    """A C99 program includes include/zfpx.h with every warning on, links the
    library and calls host-only entry points (no GPU)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "t.c"
    src.write_text(
        '#include "zfpx.h"\n#include <stdio.h>\n'
        "int main(void) {\n"
        "    double mu[4], w[4];\n"
        "    int64_t n[3] = {9, 6, 5};\n"
        "    zfpx_legendre p = 0;\n"
        "    if (zfpx_gauss_legendre(4, mu, w) != ZFPX_OK) return 1;\n"
        '    printf("%.17g %.17g %zu %d\\n", mu[0], w[0], zfpx_stream_bytes_f64(16, n),\n'
        "           zfpx_legendre_create(&p, 3, 1));\n"
        "    return 0;\n}\n")
    lib = zfpx.library_path()
    exe = tmp_path / "t"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                        str(src), "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert abs(float(out[0]) - 0.8611363115940526) < 1e-15          # the 4-point Gauss-Legendre node
    assert abs(float(out[1]) - 0.34785484513745385) < 1e-15         # and its weight
    assert int(out[2]) == 3 * 2 * 2 * 8 * 16 and int(out[3]) == -1
