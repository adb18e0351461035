"""float32 -> float16 casts for the comparator (test infrastructure; oracle side).

The paper's comparator casts the exchanged buffer to half precision and back
(Sec. I; Sec. IV-D treats the cast as costing nothing; Sec. IV-F measures
its error by a round trip float32 -> float16 -> float32).

* ``to_f16_rn``: IEEE 754 round-to-nearest-even, overflow to +-inf, subnormal
  halves kept -- this is numpy's float32 -> float16 conversion, used as is
  (a library routine; pinned against the definition in
  tests/test_oracle_packs.py, test_fp16_rn_definition).
* ``to_f16_rz``: round toward zero (the paper calls the cast a truncation): the
  float16 of largest magnitude not above |x|, same sign; finite values beyond
  the float16 range give +-65504 (IEEE round-toward-zero overflow), inf stays
  inf, NaN stays NaN.  Pinned by brute force over neighbouring float16 values.

Results are returned as uint16 bit patterns.
"""
import numpy as np


def to_f16_rn(x):
    x = np.asarray(x, dtype=np.float32)
    return x.astype(np.float16).view(np.uint16)


def to_f16_rz(x):
    x = np.asarray(x, dtype=np.float32)
    h = x.astype(np.float16)                 # nearest
    hx = h.astype(np.float32)
    ax = np.abs(x)
    ah = np.abs(hx)
    # where rounding went away from zero, step one float16 toward zero
    away = np.isfinite(x) & (ah > ax)
    hb = h.view(np.uint16).copy()
    hb[away] = hb[away] - 1                  # magnitude bits minus one ulp (sign kept)
    # finite values that overflowed to inf under nearest rounding
    ovf = np.isfinite(x) & np.isinf(hx)
    hb[ovf] = np.where(x[ovf] > 0, np.uint16(0x7BFF), np.uint16(0xFBFF))
    return hb


def from_f16(bits):
    return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float32)
