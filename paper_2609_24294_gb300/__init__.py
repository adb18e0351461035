"""zfpx: GB300 (sm_103a) fused pencil-transposition pack + ZFP fixed-rate codec.

The compute path is ``libzfpx.so`` (hand-written CUDA in ``csrc/``, C ABI in
``include/zfpx.h``); ``zfpx`` is its ctypes binding.  PyTorch provides device
memory and streams only.
"""
from . import zfpx  # noqa: F401
from .zfpx import (  # noqa: F401
    Plan, ZfpxError, RATE_F32, RATE_F16, LAYOUT_SEND, LAYOUT_RECV, ROUND_NEAREST, ROUND_ZERO,
    SPLIT_BALANCED, SPLIT_TABLE1,
)
