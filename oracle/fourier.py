"""The longitude transform of the spectral transform (test infrastructure;
oracle side: only the tests, the bench's CPU baseline and the smoke check use
it).

The transform that follows the first transposition (z -> lambda) runs along
the longitude of every lambda-pencil row (Sec. II-A: the SHT splits into an
FFT in longitude and a Legendre transform in latitude; Sec. II-B: the first
all-to-all exists so that the longitude FFT can run locally).  For a row of N
equally spaced longitudes lambda_j = 2 pi j / N the Fourier coefficient of
zonal wavenumber m is

    F_m = (1/N) sum_j x_j exp(-i m lambda_j),        m = 0 .. K - 1,

so that x_j = sum_m F_m exp(i m lambda_j) over m in (-N/2, N/2] with
F_-m = conj(F_m).  The paper does not print a normalisation; 1/N keeps the
coefficients on the field's scale (F_0 is the zonal mean).  K <= N/2 + 1
wavenumbers are kept (K = N/2 is the linear-grid truncation T = N/2 - 1).

The real and imaginary parts go to two float arrays [lev][lat][m]; the second
transposition (lambda -> theta) then moves these wavenumber fields, split over
m instead of longitude.

Here the DFT is numpy's FFT in float64 on the float32 input widened exactly, a
library routine used as the step the definition names; tests pin it to the
definition summed directly, to pure tones and to Parseval's identity.
"""
import numpy as np


def rfft_lon(x, K):
    """x: real array [..., N] (any float dtype); returns (re, im) float64 arrays
    [..., K] of F_m, m = 0 .. K - 1."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[-1]
    if N < 2 or N % 2 or not 1 <= K <= N // 2 + 1:
        raise ValueError("need an even N >= 2 and 1 <= K <= N/2 + 1")
    F = np.fft.rfft(x, axis=-1)[..., :K] / N
    return F.real.copy(), F.imag.copy()


def dft_direct(x, K):
    """The definition summed term by term (float64), for small cases."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[-1]
    j = np.arange(N)
    re = np.empty(x.shape[:-1] + (K,))
    im = np.empty(x.shape[:-1] + (K,))
    for m in range(K):
        ang = 2.0 * np.pi * ((m * j) % N) / N
        re[..., m] = (x * np.cos(ang)).sum(axis=-1) / N
        im[..., m] = -(x * np.sin(ang)).sum(axis=-1) / N
    return re, im
