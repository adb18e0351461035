"""Pins of the oracle's longitude transform (the FFT that follows the first
transposition, Sec. II-A/B): the library FFT against the definition summed
directly, against closed forms for pure tones, against Parseval's identity and
the shift theorem; and the argument checks."""
import numpy as np
import pytest

from oracle import fourier


@pytest.mark.parametrize("N", [2, 4, 6, 10, 12, 30, 40, 64, 90, 160, 1280])
def test_matches_the_direct_sum(N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((3, N)).astype(np.float32)
    K = N // 2 + 1
    re, im = fourier.rfft_lon(x, K)
    dre, dim = fourier.dft_direct(x, K)
    np.testing.assert_allclose(re, dre, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))
    np.testing.assert_allclose(im, dim, rtol=0, atol=1e-12 * max(1.0, np.abs(x).max()))


def test_pure_tones():
    # x_j = a cos(m0 lambda_j + phi): F_m0 = (a/2) e^{i phi}, every other m < N/2 zero;
    # the zonal mean sits in F_0; at m0 = N/2 the tone is a cos(phi) (-1)^j
    N = 1280
    lam = 2.0 * np.pi * np.arange(N) / N
    for m0, a, phi in [(1, 2.0, 0.3), (7, -1.5, 2.0), (639, 0.25, -1.0), (100, 3.0, 0.0)]:
        x = 5.0 + a * np.cos(m0 * lam + phi)
        re, im = fourier.rfft_lon(x, N // 2)
        want = np.zeros(N // 2, complex)
        want[0] = 5.0
        want[m0] = 0.5 * a * np.exp(1j * phi)
        np.testing.assert_allclose(re + 1j * im, want, atol=1e-12)
    x = 0.5 * np.cos(np.pi * np.arange(N))
    re, im = fourier.rfft_lon(x, N // 2 + 1)
    assert abs(re[N // 2] - 0.5) < 1e-12 and np.abs(re[:N // 2]).max() < 1e-12


def test_parseval_and_shift():
    rng = np.random.default_rng(3)
    N = 640
    x = rng.standard_normal((5, N))
    re, im = fourier.rfft_lon(x, N // 2 + 1)
    p = re ** 2 + im ** 2
    # sum_j x_j^2 / N = |F_0|^2 + 2 sum_{0<m<N/2} |F_m|^2 + |F_{N/2}|^2
    np.testing.assert_allclose((x ** 2).sum(axis=1) / N, p[:, 0] + 2 * p[:, 1:-1].sum(axis=1) + p[:, -1], rtol=1e-12)
    s = 37                                                       # x_{j - s}: F_m e^{-i m 2 pi s / N}
    r2, i2 = fourier.rfft_lon(np.roll(x, s, axis=1), N // 2 + 1)
    m = np.arange(N // 2 + 1)
    np.testing.assert_allclose(r2 + 1j * i2, (re + 1j * im) * np.exp(-2j * np.pi * m * s / N), atol=1e-12)


def test_argument_checks():
    for N, K in [(5, 2), (8, 6), (8, 0), (1, 1)]:
        with pytest.raises(ValueError):
            fourier.rfft_lon(np.zeros(N), K)
