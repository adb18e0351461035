"""zfpx_transpose_noalloc, the entry point for callers that cannot allocate
device memory where they call (inside another framework's allocator, in
loops that must not pay for an allocation, with a fixed memory map).  It
must give exactly what the allocating path gives -- zfpx_pack_compress into
a caller buffer in the receive layout, then zfpx_decompress_unpack -- call
after call, although every call reuses the same library-owned device array.
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _field(shape, seed, offset):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    x = np.linspace(0, 2 * np.pi, nx)[None, None, :]
    y = np.linspace(0, np.pi, ny)[None, :, None]
    zz = np.linspace(0, 1, nz)[:, None, None]
    f = offset + np.sin(3 * x + zz) * np.cos(2 * y) + 0.05 * rng.standard_normal(shape)
    return torch.from_numpy(f.astype(np.float32)).cuda()


def _allocating_path(z, plan, rate, src):
    buf = torch.zeros(plan.buffer_bytes(rate), dtype=torch.uint8, device="cuda")
    out = torch.full_like(src, float("nan"))
    z.zfpx_pack_compress(plan, rate, src, buf, z.LAYOUT_RECV)
    z.zfpx_decompress_unpack(plan, rate, buf, out, z.LAYOUT_RECV)
    return out


def test_noalloc_matches_allocating_path_calls_in_a_row(z):
    # five calls in a row, each on a different plan: 3-D, 2-D and 1-D blocks, both rates,
    # both transpositions, and a 2 x 8 x 8 field over 4 x 4 ranks whose longitude split
    # leaves some messages empty
    cases = [((20, 36, 52), 2, 3, 0, 16, 250.0, 1, 3), ((17, 26, 37), 3, 2, 1, 8, 0.0, 2, 3),
             ((9, 30, 44), 2, 2, 0, 8, 5.0, 3, 2), ((6, 10, 37), 2, 3, 0, 8, 1.0, 4, 1),
             ((8, 8, 2), 4, 4, 0, 16, 3.0, 5, 3)]
    for shape, pr, pc, t, rate, offset, seed, dims in cases:
        src = _field(shape, seed, offset)
        plan = z.Plan.for_fields(src, pr, pc, t, dims)
        ref = _allocating_path(z, plan, rate, src)
        got = torch.full_like(src, float("nan"))
        z.zfpx_transpose_noalloc(plan, rate, src, got)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), (shape, rate)


def test_noalloc_rejects_oversize(z):
    # 1280 x 640 x 137 at rate 16 needs ~262 MB of messages, beyond the 64 MiB array
    plan = z.Plan((1280, 640, 137), 8, 8, 0, 3)
    assert plan.buffer_bytes(16) > z.NOALLOC_SCRATCH_BYTES
    src = torch.empty((1, 1, 1), device="cuda")
    import ctypes
    rc = z.lib().zfpx_transpose_noalloc(plan.handle, 16, ctypes.c_void_p(src.data_ptr()),
                                        ctypes.c_void_p(src.data_ptr()), None)
    assert rc == -2                                      # ZFPX_ESIZE, nothing launched


def test_noalloc_refuses_stream_capture(z):
    # the message table comes from pageable host memory, which a capture cannot record
    import ctypes
    src = _field((8, 16, 16), 6, 0.0)
    dst = torch.empty_like(src)
    plan = z.Plan.for_fields(src, 2, 2, 0, 3)
    s = torch.cuda.Stream()
    h = ctypes.c_void_p(s.cuda_stream)
    assert z.lib().zfpx_capture_begin(h) == 0
    rc = z.lib().zfpx_transpose_noalloc(plan.handle, 8, ctypes.c_void_p(src.data_ptr()),
                                        ctypes.c_void_p(dst.data_ptr()), h)
    g = ctypes.c_void_p()
    assert z.lib().zfpx_capture_end(ctypes.byref(g), h) == 0
    z.lib().zfpx_graph_destroy(g)
    assert rc == -1                                      # ZFPX_EINVAL, nothing recorded
    # and the same call outside a capture still works
    ref = _allocating_path(z, plan, 8, src)
    got = torch.full_like(src, float("nan"))
    z.zfpx_transpose_noalloc(plan, 8, src, got)
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
