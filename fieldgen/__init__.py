"""Seeded synthetic input fields (shared by tests, bench and smoke).

This package holds only input generation -- none of the compression method's
arithmetic -- so both the CUDA path and the oracle can be fed from it.

The paper's fields are DYAMOND float32 temperature and ozone on a Gaussian
grid (Sec. IV-A), which are not available here; the stand-ins are inverse
spherical-harmonic transforms of seeded power-law spectra on Gauss-Legendre
latitudes (Sec. II-A describes the grid and the transform).
"""
from .sht import gaussian_latitudes, sht_field  # noqa: F401
from .workloads import t21_field, t639_field, graded_blocks, temperature_like  # noqa: F401
