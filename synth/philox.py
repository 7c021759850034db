"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from its
published definition so that the NumPy generator here and the CUDA generator
in ``synth/csrc/synth.cu`` draw the same numbers for the same (key, counter).

Each call maps a 128-bit counter and a 64-bit key to four uint32 words.
One round multiplies words 0 and 2 by fixed odd constants, keeps both halves
of the 64-bit products and mixes them with words 1 and 3 and the key; the key
is bumped by two Weyl constants between rounds; ten rounds are applied.

This module holds random-number plumbing only; it contains none of the
TACAW arithmetic.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

TWO_M32 = 2.0 ** -32


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10. All arguments broadcast; returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (x.copy() for x in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            p0 = PHILOX_M0 * c0.astype(np.uint64)
            p1 = PHILOX_M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if r != 9:
                k0 = np.uint32(k0 + PHILOX_W0)
                k1 = np.uint32(k1 + PHILOX_W1)
    return c0, c1, c2, c3


def u01(x):
    """uint32 -> float64 uniform in the open interval (0, 1): (x + 1/2) / 2^32 (exact in FP64)."""
    return (np.asarray(x, dtype=np.float64) + 0.5) * TWO_M32
