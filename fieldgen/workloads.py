"""The seeded workloads (stand-ins for the paper's DYAMOND fields, Sec. IV-A).

* ``t21_field``: 64 lon x 32 Gaussian lat x 8 levels, T21 spectrum with
  complex N(0,1) (l+1)^-1.5 amplitudes, one draw per level, seed 0.
* ``t639_field``: 1280 x 640 x 137, T639 (l+1)^-1.5 spectrum, one draw per
  level, each level scaled to unit RMS, plus N(0, 0.01^2) white noise, seed 1.
* ``temperature_like``: 250 + 20 * field -- the paper's temperature has a
  large mean offset, which is what makes its relative error small.
* ``graded_blocks``: blocks with geometrically graded cosine spectra, a test
  input that makes the bit-plane coder meet new ones on many planes.
"""
import numpy as np

from .sht import sht_field


def t21_field():
    return sht_field(64, 32, 8, T=21, slope=-1.5, seed=0)


def unit_rms_plus_noise(f, noise, seed):
    f = f.astype(np.float64)
    rms = np.sqrt(np.mean(f * f, axis=(1, 2), keepdims=True))
    f = f / np.where(rms > 0, rms, 1.0)
    rng = np.random.default_rng([int(seed), 0x5eed])
    f = f + noise * rng.standard_normal(f.shape)
    return f.astype(np.float32)


def t639_field(nlon=1280, nlat=640, nlev=137, T=639, seed=1, noise=0.01):
    f = sht_field(nlon, nlat, nlev, T=T, slope=-1.5, seed=seed)
    return unit_rms_plus_noise(f, noise, seed)


def temperature_like(f):
    return (250.0 + 20.0 * f.astype(np.float64)).astype(np.float32)


def graded_blocks(nblocks, seed):
    """float32 [4][4][4 nblocks]: nblocks 4x4x4 blocks side by side, each a sum
    of separable cosines whose amplitudes fall off geometrically with the
    total frequency (random rate, sign and overall scale per block).  Blocks
    like these gain newly significant coefficients a few at a time over many
    bit planes, so the coder visits many planes with new ones."""
    r = np.random.default_rng(seed)
    t = np.arange(4)
    C = np.cos(np.pi * (2 * t[None, :] + 1) * t[:, None] / 8.0)     # [frequency][position]
    fsum = t[:, None, None] + t[None, :, None] + t[None, None, :]
    out = np.empty((4, 4, 4 * nblocks))
    for b in range(nblocks):
        step = r.uniform(0.4, 2.5)
        amp = r.choice([-1.0, 1.0], (4, 4, 4)) * 2.0 ** (-step * fsum * r.uniform(0.8, 1.2, (4, 4, 4))
                                                          - r.uniform(0, 1, (4, 4, 4)))
        blk = np.einsum("abc,az,by,cx->zyx", amp, C, C, C)
        out[:, :, 4 * b:4 * b + 4] = blk * 10.0 ** r.uniform(-5, 5)
    return out.astype(np.float32)
