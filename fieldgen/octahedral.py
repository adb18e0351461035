"""Seeded fields on an octahedral reduced Gaussian grid (ragged rows).

Grid O<N>: 2N latitude rows; row i of the northern half (i = 0..N-1) has
20 + 4i points, mirrored in the southern half, so O1280 has 2560 rows,
6,599,680 points per level and a longest row of 5136 points.  A field is a
float32 array [level][point] with the rows stored back to back.

A full inverse spherical-harmonic transform on O1280 for hundreds of levels
is too slow to be an input generator, so the stand-in is a 1-D spectral
synthesis along rows: every row is the first L_r samples of a periodic
signal of length L_max with Fourier amplitudes (k+1)^-1.5 and Gaussian
coefficients that are AR(1)-correlated (rho = 0.95) from row to row and from
level to level; g = that synthesis scaled to unit variance.  Flavours
follow the paper's variable classes (Sec. IV-A): "power" (wind like, g),
"temperature" (250 + 20 g: the mean offset of the paper's T) and
"humidity" (lognormal, exp(-8 + 2 g)).  Seeded, float64 with one rounding to float32, computed with torch
on the given device so the 22.9 GB ten-field workload takes seconds on a GPU.
"""
import numpy as np
import torch


def row_lengths(N):
    north = 20 + 4 * np.arange(N, dtype=np.int64)
    return np.concatenate([north, north[::-1]])


def row_offsets(lengths):
    return np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int64)


def _ar1_rows(w, rho):
    """c[r] = rho c[r-1] + sqrt(1-rho^2) w[r], c[0] = w[0], along dim 0 (float64)."""
    n = w.shape[0]
    r = torch.arange(n, dtype=torch.float64, device=w.device).view(-1, *([1] * (w.dim() - 1)))
    s = float(np.sqrt(1.0 - rho * rho))
    scaled = w * (rho ** (-r))
    scaled[1:] *= s
    return torch.cumsum(scaled, dim=0) * (rho ** r)


def octahedral_field(N, nlev, seed, kind="power", device="cpu", rho=0.95, slope=-1.5):
    """float32 tensor [nlev][points] on `device`."""
    lens = row_lengths(N)
    offs = row_offsets(lens)
    Lmax = int(lens.max())
    kmax = Lmax // 2 + 1
    nrows = len(lens)
    npts = int(lens.sum())
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed) * 1000003 + 17)
    # flat index of every grid point in the [row][Lmax] synthesis array
    idx = np.concatenate([r * Lmax + np.arange(L) for r, L in enumerate(lens)])
    idx = torch.from_numpy(idx).to(device)
    amp = (torch.arange(kmax, dtype=torch.float64, device=device) + 1.0) ** slope
    s = float(np.sqrt(1.0 - rho * rho))
    out = torch.empty((nlev, npts), dtype=torch.float32, device=device)
    prev = None
    for z in range(nlev):
        w = torch.randn((nrows, kmax, 2), dtype=torch.float64, device=device, generator=gen)
        c = _ar1_rows(w, rho)
        if prev is not None:
            c = rho * prev + s * c
        prev = c
        coef = torch.complex(c[..., 0], c[..., 1]) * amp
        coef[:, 0] = torch.complex(coef[:, 0].real, torch.zeros_like(coef[:, 0].real))
        vals = torch.fft.irfft(coef, n=Lmax, dim=1) * float(np.sqrt(Lmax))
        out[z] = vals.reshape(-1)[idx].to(torch.float32)
    g = out.double()
    g = (g - g.mean()) / g.std()
    if kind == "power":
        out = g.to(torch.float32)
    elif kind == "temperature":
        out = (250.0 + 20.0 * g).to(torch.float32)
    elif kind == "humidity":
        out = torch.exp(-8.0 + 2.0 * g).to(torch.float32)
    else:
        raise ValueError(kind)
    return out


# The ten fields of the batched workload: (levels, flavour, block dims, rate).
O1280_TEN_FIELDS = [
    (137, "temperature", 3, 8), (137, "power", 3, 16), (137, "humidity", 3, 8), (137, "power", 3, 16),
    (1, "temperature", 1, 8), (137, "humidity", 3, 16), (91, "power", 3, 8), (60, "humidity", 3, 16),
    (30, "temperature", 3, 8), (1, "humidity", 1, 16),
]


def serving_requests(n, fields_nlev, fields_dims, seed, lens, min_bytes=16 << 10, max_bytes=64 << 20,
                     median_bytes=1 << 20, sigma=1.34):
    """Request mix for the serving workload: sizes lognormal (median 1 MiB,
    sigma 1.34, clipped to [16 KiB, 64 MiB]), each a slab of rows x levels of
    a random field: 3-D fields take whole row-quads and up to 16 levels, 1-D
    (single-level) fields take rows; rate 8 or 16 uniformly.  Returns dicts
    (field, z0, nz, row0, row1, rate, dims, bytes)."""
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.exp(np.log(median_bytes) + sigma * rng.standard_normal(n)), min_bytes, max_bytes)
    offs = np.concatenate([[0], np.cumsum(lens)])
    nrows = len(lens)
    out = []
    for s in sizes:
        f = int(rng.integers(len(fields_nlev)))
        nlev, dims = fields_nlev[f], fields_dims[f]
        nz = 1 if dims == 1 else int(rng.integers(1, min(16, nlev) + 1))
        z0 = int(rng.integers(0, nlev - nz + 1))
        target_pts = max(1, int(s) // (4 * nz))
        step = 4 if dims == 3 else 1
        r0 = int(rng.integers(0, nrows // step)) * step
        r1 = r0
        while r1 < nrows and offs[r1] - offs[r0] < target_pts:
            r1 = min(nrows, r1 + step)
        while r0 > 0 and offs[r1] - offs[r0] < target_pts:      # ran into the last row: grow downwards
            r0 -= step
        out.append(dict(field=f, z0=z0, nz=nz, row0=r0, row1=r1, rate=int(rng.choice([8, 16])), dims=dims,
                        bytes=int(4 * nz * (offs[r1] - offs[r0]))))
    return out
