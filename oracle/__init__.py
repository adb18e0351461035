"""CPU oracle for the fused pencil-transposition pack + ZFP fixed-rate path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_2609_24294_gb300``) and never
imports it; the CUDA path never imports this package.

Contents (each module cites the passage of the paper it restates):

* ``codec``   -- ctypes binding of ``zfp_oracle.c`` (ZFP fixed-rate blocks and
                 arrays, Sec. II-C; Lindstrom 2014).
* ``plan``    -- pencil decomposition and message layout of the two
                 transpositions (Sec. II-B; Table 1).
* ``packs``   -- plain float32 pack, float16-cast pack, the all-to-all as a
                 buffer permutation, and pack+compress / decompress+unpack over
                 a whole plan (Sec. I; Sec. IV-C/D).
* ``fp16``    -- float32 -> float16 casts, round-to-nearest-even and
                 round-toward-zero (Sec. I: the exchanged buffer cast to
                 half precision).

Parity status: see the header of each module.
"""
from . import codec, plan, packs, fp16  # noqa: F401
