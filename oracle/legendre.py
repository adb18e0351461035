"""The Legendre transform of the spectral transform (test infrastructure;
oracle side: only the tests, the bench's CPU baseline and the smoke check use
it).

After the second transposition (lambda -> theta, Sec. II-B) every rank holds
whole latitude columns of the wavenumber fields F_m(mu_j) (the longitude
transform's output, F_m = (1/N) sum_k x_k e^{-i m lambda_k}).  The latitude
transform (Sec. II-A: associated Legendre functions, Gauss-Legendre
quadrature) gives the spectral coefficients

    a_l^m = sum_j w_j Pbar_l^m(mu_j) F_m(mu_j),     0 <= m <= l <= T,

with mu_j the Gauss-Legendre nodes (north to south), w_j their weights
(sum 2), and Pbar_l^m the associated Legendre functions normalised so that
int_{-1}^{1} Pbar_l^m Pbar_l'^m dmu = delta_ll' (with the Condon-Shortley
phase (-1)^m).  Quadrature on nlat >= T + 1 nodes is exact for these
products, so a field synthesised as sum_l a_l^m Pbar_l^m e^{i m lambda}
(conjugate terms for -m) comes back exactly.

Pbar by the standard recurrences (Sec. II-A names the functions only):
  Pbar_0^0 = 1/sqrt(2),
  Pbar_m^m = -sqrt((2m+1)/(2m)) sqrt(1 - mu^2) Pbar_{m-1}^{m-1},
  Pbar_{m+1}^m = sqrt(2m+3) mu Pbar_m^m,
  Pbar_l^m = a_lm (mu Pbar_{l-1}^m - b_lm Pbar_{l-2}^m),
  a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
Values that underflow float64 near the poles for large m stay 0.

Output layout: for every level, the coefficients in order m = 0 .. T and, for
each m, l = m .. T (offset(m) = m (T+1) - m (m-1) / 2), real and imaginary
parts in two arrays [lev][(T+1)(T+2)/2].  The nodes come from numpy's
Gauss-Legendre routine, a library step; everything else is the definition,
summed in float64.
"""
import numpy as np


def gauss_nodes(nlat):
    """(mu, w): Gauss-Legendre nodes north to south (mu decreasing) and weights."""
    x, w = np.polynomial.legendre.leggauss(nlat)
    return x[::-1].copy(), w[::-1].copy()


def offset(m, T):
    return m * (T + 1) - m * (m - 1) // 2


def ncoeffs(T):
    return (T + 1) * (T + 2) // 2


def pbar_m(m, T, mu):
    """Pbar_l^m(mu) for l = m .. T: array [T - m + 1][len(mu)] (float64)."""
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    p = np.full(mu.shape, np.sqrt(0.5))
    for k in range(1, m + 1):
        p = -np.sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * p
    out = np.empty((T - m + 1,) + mu.shape)
    out[0] = p
    if T > m:
        out[1] = np.sqrt(2.0 * m + 3.0) * mu * p
    for i in range(2, T - m + 1):
        l = m + i
        a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        out[i] = a * (mu * out[i - 1] - b * out[i - 2])
    return out


def legendre_forward(re, im, T):
    """re, im: wavenumber fields [lev][nlat][K] (K >= T + 1), latitudes at the
    Gauss-Legendre nodes north to south.  Returns (a_re, a_im) float64
    [lev][(T+1)(T+2)/2] and, for error bounds, mag = sum_j |w_j Pbar_l^m(mu_j)|
    |F_m(mu_j)| in the same layout."""
    re = np.asarray(re, dtype=np.float64)
    im = np.asarray(im, dtype=np.float64)
    nlev, nlat, K = re.shape
    if T < 0 or T + 1 > K or T + 1 > nlat:
        raise ValueError("need T + 1 <= K and T + 1 <= nlat")
    mu, w = gauss_nodes(nlat)
    a_re = np.empty((nlev, ncoeffs(T)))
    a_im = np.empty((nlev, ncoeffs(T)))
    mag = np.empty((nlev, ncoeffs(T)))
    for m in range(T + 1):
        P = pbar_m(m, T, mu) * w[None, :]                   # [l][j]
        o = offset(m, T)
        L = T - m + 1
        a_re[:, o:o + L] = re[:, :, m] @ P.T                  # [lev][j] x [j][l]
        a_im[:, o:o + L] = im[:, :, m] @ P.T
        mag[:, o:o + L] = np.hypot(re[:, :, m], im[:, :, m]) @ np.abs(P).T
    return a_re, a_im, mag
