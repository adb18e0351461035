"""Pins of the oracle's Legendre transform (the latitude transform after the
second transposition, Sec. II-A/B): the normalised associated Legendre
functions against closed forms and scipy's lpmv, their parity in mu,
orthonormality under Gauss-Legendre quadrature, and recovery of the known
spectral coefficients of fields synthesised by the input generator (longitude
transform, then this one)."""
import math

import numpy as np
import pytest

from fieldgen import sht as gsht
from oracle import fourier, legendre


def test_closed_forms():
    mu = np.linspace(-0.999, 0.999, 41)
    s = np.sqrt(1 - mu * mu)
    want = {
        (0, 0): np.full_like(mu, 1 / math.sqrt(2)),
        (1, 0): math.sqrt(1.5) * mu,
        (1, 1): -math.sqrt(3) / 2 * s,
        (2, 0): math.sqrt(2.5) * (3 * mu * mu - 1) / 2,
        (2, 1): -math.sqrt(15) / 2 * mu * s,
        (2, 2): math.sqrt(15) / 4 * s * s,
    }
    for (l, m), v in want.items():
        np.testing.assert_allclose(legendre.pbar_m(m, 2, mu)[l - m], v, rtol=0, atol=1e-14)


def test_against_scipy_lpmv():
    sp = pytest.importorskip("scipy.special")
    mu = np.linspace(-0.98, 0.98, 23)
    T = 30
    for m in (0, 1, 2, 5, 11, 20, 30):
        P = legendre.pbar_m(m, T, mu)
        for l in range(m, T + 1):
            norm = math.sqrt((2 * l + 1) / 2 * math.factorial(l - m) / math.factorial(l + m))
            np.testing.assert_allclose(P[l - m], norm * sp.lpmv(m, l, mu), rtol=1e-10, atol=1e-13)


def test_parity_and_orthonormality_under_quadrature():
    nlat, T = 32, 31
    mu, w = legendre.gauss_nodes(nlat)
    assert abs(w.sum() - 2) < 1e-13 and np.all(np.diff(mu) < 0)
    np.testing.assert_allclose(mu, -mu[::-1], atol=1e-15)
    for m in range(T + 1):
        P = legendre.pbar_m(m, T, mu)
        for i in range(T - m + 1):                     # Pbar_l^m(-mu) = (-1)^(l+m) Pbar_l^m(mu)
            np.testing.assert_allclose(P[i][::-1], (-1) ** (i + 2 * m) * P[i], atol=1e-13)
        G = (P * w) @ P.T
        np.testing.assert_allclose(G, np.eye(T - m + 1), atol=1e-12)


def test_layout():
    T = 5
    seen = [legendre.offset(m, T) + (l - m) for m in range(T + 1) for l in range(m, T + 1)]
    assert seen == list(range(legendre.ncoeffs(T)))


@pytest.mark.parametrize("nlon,nlat,T", [(64, 32, 21), (48, 24, 23), (96, 48, 31)])
def test_recovers_the_generator_coefficients(nlon, nlat, T):
    nlev, seed = 3, 7
    x = gsht.sht_field(nlon, nlat, nlev, T=T, slope=-1.5, seed=seed)       # float32
    re, im = fourier.rfft_lon(x, T + 1)
    a_re, a_im, mag = legendre.legendre_forward(re, im, T)
    for z in range(nlev):
        a = gsht._level_coeffs(T, seed, z, -1.5)                           # a[m, l]
        want = np.concatenate([a[m, m:T + 1] for m in range(T + 1)])
        got = a_re[z] + 1j * a_im[z]
        # the field is rounded to float32 once: a few ulps of its magnitude
        np.testing.assert_allclose(got, want, rtol=0, atol=3e-6 * np.abs(x[z]).max())
    assert np.all(mag >= np.abs(a_re) - 1e-12) and np.all(mag >= np.abs(a_im) - 1e-12)


def test_argument_checks():
    with pytest.raises(ValueError):
        legendre.legendre_forward(np.zeros((1, 8, 4)), np.zeros((1, 8, 4)), 4)    # T + 1 > K
    with pytest.raises(ValueError):
        legendre.legendre_forward(np.zeros((1, 4, 8)), np.zeros((1, 4, 8)), 4)    # T + 1 > nlat
