"""Inverse spherical-harmonic synthesis of seeded power-law spectra.

A field on N_lambda longitudes x N_theta Gauss-Legendre latitudes (Sec. II-A)
is built as f(lambda, mu) = sum_m sum_{l>=m} Re[a_lm Pbar_l^m(mu) e^{i m lambda}]
(m > 0 terms doubled), with a_lm = (g1 + i g2) (l+1)^slope, g ~ N(0,1),
a_l0 real, one independent draw per level.  Pbar are the orthonormal associated
Legendre functions (int_{-1}^{1} Pbar^2 dmu = 1) by the standard three-term
recurrence in l; values that underflow near the poles for large m are left at
zero, which only drops contributions below 1e-300.

The Legendre part runs per order m as a dense product (lat x l) @ (l x levels)
and the longitude part as an inverse real FFT; both in float64.  The result
is rounded once to float32.
"""
import numpy as np


def gaussian_latitudes(nlat):
    """mu = sin(latitude) at the Gauss-Legendre nodes, north to south."""
    x, _ = np.polynomial.legendre.leggauss(nlat)
    return x[::-1].copy()


def _level_coeffs(T, seed, level, slope):
    rng = np.random.default_rng([int(seed), int(level)])
    re = rng.standard_normal((T + 1, T + 1))
    im = rng.standard_normal((T + 1, T + 1))
    l = np.arange(T + 1, dtype=np.float64)
    amp = (l + 1.0) ** slope                       # indexed by l
    a = (re + 1j * im) * amp[None, :]              # a[m, l]
    a[0, :] = re[0, :] * amp                       # m = 0 real
    # keep l >= m only
    mask = l[None, :] >= np.arange(T + 1)[:, None]
    return a * mask


def sht_field(nlon, nlat, nlev, T, slope=-1.5, seed=0, level_chunk=160):
    """float32 array [nlev][nlat][nlon]."""
    if 2 * T + 1 > nlon:
        raise ValueError("truncation T too large for nlon")
    mu = gaussian_latitudes(nlat)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    out = np.empty((nlev, nlat, nlon), dtype=np.float32)
    for z0 in range(0, nlev, level_chunk):
        z1 = min(nlev, z0 + level_chunk)
        coeffs = [_level_coeffs(T, seed, z, slope) for z in range(z0, z1)]
        F = np.zeros((nlat, nlon // 2 + 1, z1 - z0), dtype=np.complex128)
        pmm = np.full(nlat, np.sqrt(0.5))          # Pbar_0^0
        for m in range(T + 1):
            if m > 0:
                pmm = -np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
            L = T - m + 1
            P = np.empty((L, nlat))
            P[0] = pmm
            if L > 1:
                P[1] = np.sqrt(2.0 * m + 3.0) * mu * pmm
            for i in range(2, L):
                l = m + i
                a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                P[i] = a * (mu * P[i - 1] - b * P[i - 2])
            C = np.stack([c[m, m:T + 1] for c in coeffs], axis=1)   # L x nz
            Cr = np.concatenate([C.real, C.imag], axis=1)           # L x 2nz
            R = P.T @ Cr                                            # nlat x 2nz
            nz = z1 - z0
            F[:, m, :] = R[:, :nz] + 1j * R[:, nz:]
        g = np.fft.irfft(F, n=nlon, axis=1) * nlon                  # nlat x nlon x nz
        out[z0:z1] = np.transpose(g, (2, 0, 1)).astype(np.float32)
    return out
