"""GB300 (sm_103a) mixed-precision lattice Boltzmann stream-collide library.

Implements the hot path of Lehmann et al., arXiv 2112.08926: the fused
stream-collide step with shifted populations stored in FP64, FP32 or the
paper's 16-bit formats (FP16, FP16S, FP16C, P16_0S, P16_1S, P16_2C and the
unscaled posits), collision arithmetic in FP32 (or FP64) registers.  The C ABI
is declared in include/lbm.h; this package is its thin ctypes binding.
"""
from .lbm import (  # noqa: F401
    ARITHS, COLLISIONS, EQ, EXPORTS, FREESLIP, MOVING, OUTFLOW, Q, SCHEMES, STORAGES, VELSETS, WALL,
    Ensemble, LBMError, Lattice, codec_decode, codec_encode, codec_encode_bits, load, lbm_create,
    lbm_status_string,
)
