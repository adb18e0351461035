"""Inverse spherical-harmonic synthesis on a device (torch), for large grids.

Same construction as ``sht.sht_field`` -- orthonormal associated Legendre
functions on Gauss-Legendre latitudes, a_lm = (g1 + i g2)(l+1)^slope with a
real m = 0 column, one independent draw per level, inverse real FFT in
longitude -- but the Legendre recurrence runs over l for all orders m at
once and the sums are accumulated on the device in float32, so a
2560 x 1280 x 137 field at T1279 takes seconds on a GPU instead of tens of
minutes on a CPU.  The random numbers come from torch's generator, so the
field differs from ``sht.sht_field``'s for the same seed; each consumer
uses the one array it is given.
"""
import numpy as np
import torch

from .sht import gaussian_latitudes


def sht_field_torch(nlon, nlat, nlev, T, slope=-1.5, seed=0, device="cuda", level_chunk=160):
    if 2 * T + 1 > nlon:
        raise ValueError("truncation T too large for nlon")
    mu = torch.from_numpy(gaussian_latitudes(nlat)).to(device=device, dtype=torch.float64)
    s = torch.sqrt(torch.clamp(1.0 - mu * mu, min=0.0))
    M = T + 1
    m = torch.arange(M, dtype=torch.float64, device=device)
    # Pbar_m^m for all m (log form against underflow), shape [nlat, M]
    logs = torch.log(torch.clamp(s, min=1e-300))
    fac = torch.zeros(M, dtype=torch.float64, device=device)
    if M > 1:
        fac[1:] = torch.cumsum(0.5 * torch.log((2.0 * m[1:] + 1.0) / (2.0 * m[1:])), 0)
    pmm = torch.exp(np.log(np.sqrt(0.5)) + fac[None, :] + m[None, :] * logs[:, None])
    sign = torch.where((m.long() % 2) == 1, -1.0, 1.0).to(torch.float64)
    pmm = pmm * sign[None, :]
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 7919 + 3)
    out = torch.empty((nlev, nlat, nlon), dtype=torch.float32, device=device)
    amp_l = (torch.arange(M, dtype=torch.float64, device=device) + 1.0) ** slope
    for z0 in range(0, nlev, level_chunk):
        nz = min(level_chunk, nlev - z0)
        a = torch.randn((nz, M, M, 2), dtype=torch.float32, device=device, generator=gen)   # [lev][m][l]
        coef = torch.complex(a[..., 0], a[..., 1])
        coef[:, 0, :] = torch.complex(a[:, 0, :, 0], torch.zeros_like(a[:, 0, :, 0]))
        coef = coef * amp_l.to(torch.float32)[None, None, :]
        F = torch.zeros((nz, nlat, M), dtype=torch.complex64, device=device)
        p_prev2 = None
        p_prev = pmm                                                     # Pbar_l^m at l = m (diagonal)
        # run l from 0..T; for order m the recurrence starts at l = m
        P_l = torch.zeros((nlat, M), dtype=torch.float64, device=device)
        P_lm1 = torch.zeros((nlat, M), dtype=torch.float64, device=device)
        for l in range(M):
            # Pbar_l^m for all m <= l
            Pn = torch.zeros((nlat, M), dtype=torch.float64, device=device)
            if l >= 1:
                mm = m[:l]                                                  # orders below l
                a_l = torch.sqrt((4.0 * l * l - 1.0) / (l * l - mm * mm))
                b_l = torch.sqrt(torch.clamp(((l - 1.0) ** 2 - mm * mm) / (4.0 * (l - 1.0) ** 2 - 1.0), min=0.0))
                Pn[:, :l] = a_l[None, :] * (mu[:, None] * P_l[:, :l] - b_l[None, :] * P_lm1[:, :l])
            Pn[:, l] = pmm[:, l]
            P_lm1, P_l = P_l, Pn
            # F[z, lat, m] += Pbar_l^m(lat) a_lm[z]
            F += Pn.to(torch.float32)[None, :, :] * coef[:, :, l][:, None, :]
        del p_prev, p_prev2
        full = torch.zeros((nz, nlat, nlon // 2 + 1), dtype=torch.complex64, device=device)
        full[:, :, :M] = F
        out[z0:z0 + nz] = torch.fft.irfft(full, n=nlon, dim=2) * float(nlon)
    return out
