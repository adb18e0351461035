"""The debug report of non-finite inputs (zfpx_count_nonfinite): the paper
leaves infinities and NaNs unspecified, the codec codes a block holding one
as a zero block, and this call counts them.  The count must equal the number
of elements whose exponent field is all ones, on contiguous, strided and
sliced views of float32 and float64 tensors, and it accumulates."""
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


def _planted(dtype, shape, nbad, seed):
    r = np.random.default_rng(seed)
    x = r.standard_normal(shape).astype(dtype)
    flat = x.reshape(-1)
    idx = r.choice(flat.size, nbad, replace=False)
    bad = np.array([np.nan, np.inf, -np.inf], dtype=dtype)
    flat[idx] = bad[np.arange(nbad) % 3]
    # the largest finite values and subnormals are finite: never counted
    fi = np.finfo(dtype)
    good = np.setdiff1d(np.arange(flat.size), idx)[:4]
    flat[good] = [fi.max, -fi.max, fi.smallest_subnormal, -fi.tiny]
    return x


def _count(z, t):
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    z.zfpx_count_nonfinite(t, c)
    torch.cuda.synchronize()
    return int(c.item())


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,nbad", [((19, 53, 37), 0), ((19, 53, 37), 1), ((19, 53, 37), 250),
                                        ((137, 16, 160), 4097), ((1000,), 17), ((33, 70), 9)])
def test_counts_planted_values(z, dtype, shape, nbad):
    x = _planted(dtype, shape, nbad, seed=len(shape) * 1000 + nbad)
    assert _count(z, torch.from_numpy(x).cuda()) == nbad == np.count_nonzero(~np.isfinite(x))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_strided_views_and_accumulation(z, dtype):
    x = _planted(dtype, (12, 40, 90), 1500, seed=5)
    t = torch.from_numpy(x).cuda()
    for view, ref in ((t[:, ::2, 1::3], x[:, ::2, 1::3]), (t[3:9, 5:31, 7:88], x[3:9, 5:31, 7:88]),
                      (t.transpose(0, 2), x.transpose(2, 1, 0)), (t[:, 7, :], x[:, 7, :])):
        assert _count(z, view) == np.count_nonzero(~np.isfinite(ref))
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        z.zfpx_count_nonfinite(t, c)
    torch.cuda.synchronize()
    assert int(c.item()) == 3 * 1500
    e = torch.empty((0, 4, 4), dtype=t.dtype, device="cuda")
    assert _count(z, e) == 0


def test_rejects_other_dtypes(z):
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        z.zfpx_count_nonfinite(torch.zeros(8, dtype=torch.float16, device="cuda"), c)
    with pytest.raises(ValueError):
        z.zfpx_count_nonfinite(torch.zeros(8, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))
