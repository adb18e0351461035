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


def test_noalloc_matches_allocating_path_two_calls(z):
    cases = [((20, 36, 52), 2, 3, 0, 16, 250.0, 1, 3), ((17, 26, 37), 3, 2, 1, 8, 0.0, 2, 3),
             ((9, 30, 44), 2, 2, 0, 8, 5.0, 3, 2)]
    for shape, pr, pc, t, rate, offset, seed, dims in cases:     # calls in a row, different plans and rates
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
