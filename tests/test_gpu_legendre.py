"""GPU parity of the Legendre transform (the latitude transform after the
second transposition, Sec. II-A/B) through the C ABI against the float64
oracle.

Tolerance.  The GPU sums nlat/2 products per coefficient in float32 (fused
multiply-adds) after one rounding of the table entry w_j Pbar_l^m(mu_j) and
one of the fold S_j / A_j = F(mu_j) +- F(-mu_j).  The standard dot-product
bound then gives |error| <= (nlat/2 + 2) u sum_j |w_j Pbar_l^m(mu_j)|
|F_m(mu_j)| (u = 2^-24; the sum over all latitudes equals the folded one by
symmetry).  The oracle returns that sum; the test allows twice the bound."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from fieldgen import sht as gsht
from oracle import fourier as of
from oracle import legendre as ol

U = 2.0 ** -24


@pytest.fixture(scope="module")
def z():
    from paper_2609_24294_gb300 import build, zfpx
    build.build()
    zfpx.lib()
    return zfpx


def _gpu(z, plan, re, im, pad=0):
    nlev = re.shape[0]
    are = torch.full((nlev, plan.ncoeffs + pad), float("nan"), device="cuda")
    aim = torch.full((nlev, plan.ncoeffs + pad), float("nan"), device="cuda")
    plan.forward(re, im, are, aim)
    torch.cuda.synchronize()
    plan.status()                              # no bounded wait in the tensor-core kernel gave up
    a, b = are.cpu().numpy(), aim.cpu().numpy()
    if pad:
        assert np.isnan(a[:, plan.ncoeffs:]).all() and np.isnan(b[:, plan.ncoeffs:]).all()
    return a[:, :plan.ncoeffs].astype(np.float64), b[:, :plan.ncoeffs].astype(np.float64)


def _check(re_np, im_np, T, gre, gim, levels=None):
    if levels is not None:
        re_np, im_np, gre, gim = re_np[levels], im_np[levels], gre[levels], gim[levels]
    rre, rim, mag = ol.legendre_forward(re_np, im_np, T)
    nh = re_np.shape[1] // 2
    bound = 2 * (nh + 2) * U * mag + 1e-30
    for g, r in ((gre, rre), (gim, rim)):
        assert np.isfinite(g).all()
        ratio = np.abs(g - r) / bound
        assert ratio.max() <= 1.0, (float(ratio.max()), np.unravel_index(ratio.argmax(), ratio.shape))


@pytest.mark.parametrize("nlat,T,nlev,K", [(2, 0, 1, 1), (4, 3, 2, 4), (32, 21, 3, 33), (24, 23, 2, 24),
                                           (90, 70, 70, 80), (320, 159, 5, 160), (64, 40, 33, 64)])
def test_random_fields(z, nlat, T, nlev, K):
    rng = np.random.default_rng(nlat + T + nlev)
    re = (rng.standard_normal((nlev, nlat, K)) * 10.0 ** rng.uniform(-2, 2, (nlev, 1, 1))).astype(np.float32)
    im = (rng.standard_normal((nlev, nlat, K))).astype(np.float32)
    plan = z.Legendre(nlat, T)
    gre, gim = _gpu(z, plan, torch.from_numpy(re).cuda(), torch.from_numpy(im).cuda(), pad=3)
    _check(re, im, T, gre, gim)
    plan.close()


def test_generator_field_and_views(z):
    # F from the oracle's longitude transform of a synthesised field, held in
    # wider strided buffers
    nlon, nlat, T, nlev = 96, 48, 31, 4
    x = gsht.sht_field(nlon, nlat, nlev, T=T, slope=-1.5, seed=3)
    re, im = of.rfft_lon(x, T + 1)
    re, im = re.astype(np.float32), im.astype(np.float32)
    big_re = np.full((nlev + 1, nlat, T + 9), np.nan, np.float32)
    big_im = np.full((nlev + 1, nlat, T + 9), np.nan, np.float32)
    big_re[1:, :, 2:T + 3] = re
    big_im[1:, :, 2:T + 3] = im
    dre = torch.from_numpy(big_re).cuda()[1:, :, 2:T + 3]
    dim = torch.from_numpy(big_im).cuda()[1:, :, 2:T + 3]
    plan = z.Legendre(nlat, T)
    gre, gim = _gpu(z, plan, dre, dim)
    _check(re, im, T, gre, gim)
    # and the coefficients the generator drew, to float32 accuracy
    for lev in range(nlev):
        a = gsht._level_coeffs(T, 3, lev, -1.5)
        want = np.concatenate([a[m, m:T + 1] for m in range(T + 1)])
        np.testing.assert_allclose(gre[lev] + 1j * gim[lev], want, rtol=0, atol=2e-5 * np.abs(x[lev]).max())
    plan.close()


def test_t639_full_size_sampled_levels(z):
    # 137 levels x 640 Gaussian latitudes x 640 wavenumbers (T639); the oracle
    # checks a sample of levels
    x = gsht.sht_field(1280, 640, 6, T=639, slope=-1.5, seed=1)    # six levels of a T639 field
    re, im = of.rfft_lon(x, 640)                     # oracle input for the sampled levels
    rng = np.random.default_rng(11)
    F_re = rng.standard_normal((137, 640, 640)).astype(np.float32)
    F_im = rng.standard_normal((137, 640, 640)).astype(np.float32)
    F_re[:6], F_im[:6] = re, im
    plan = z.Legendre(640, 639)
    gre, gim = _gpu(z, plan, torch.from_numpy(F_re).cuda(), torch.from_numpy(F_im).cuda())
    levels = [0, 1, 2, 3, 4, 5, 70, 136]
    _check(F_re, F_im, 639, gre, gim, levels=levels)
    plan.close()


def test_errors(z):
    for nlat, T in [(3, 1), (8, 8), (0, 0), (8, -1)]:
        with pytest.raises(z.ZfpxError):
            z.Legendre(nlat, T)
    # tables larger than the device (T = 32767: about 70 TB) are refused before
    # any of them is built
    with pytest.raises(z.ZfpxError) as e:
        z.Legendre(1 << 15, (1 << 15) - 1)
    assert e.value.code == -6                                                    # ZFPX_ENOMEM
    plan = z.Legendre(8, 5)
    re = torch.zeros((2, 8, 6), device="cuda")
    a = torch.zeros((2, plan.ncoeffs), device="cuda")
    with pytest.raises(z.ZfpxError):
        plan.forward(torch.zeros((2, 8, 5), device="cuda"), torch.zeros((2, 8, 5), device="cuda"), a, a.clone())  # K < T + 1
    with pytest.raises(z.ZfpxError):
        plan.forward(torch.zeros((2, 6, 6), device="cuda"), torch.zeros((2, 6, 6), device="cuda"), a, a.clone())
    with pytest.raises(z.ZfpxError):
        t = torch.zeros((2, 6, 8), device="cuda").transpose(1, 2)                 # wavenumber stride != 1
        plan.forward(t, t.clone().transpose(1, 2).contiguous().transpose(1, 2), a, a.clone())
    plan.close()
