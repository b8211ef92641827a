"""E4M3 8-bit floating point (OCP 8-bit Floating Point Specification, the
"E4M3" format): 1 sign bit, 4 exponent bits with bias 7, 3 significand
bits; no infinities; largest finite magnitude 448 (exponent field 15,
significand 110); subnormals down to 2^-9.

TEST INFRASTRUCTURE ONLY (part of the oracle): models the rounding the
FP8 tensor-core path applies, so tests can compare that path against a
float64 computation with the same roundings.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def round_e4m3(x, saturate: bool = True) -> np.ndarray:
    """Nearest E4M3 value (ties to even), as float64.

    Normal numbers 2^e (1 + m/8) with e in [-6, 8]; below 2^-6 the spacing
    is fixed at 2^-9 (subnormals).  Magnitudes above 448 saturate to 448.
    """
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    # exponent of the binade, clamped to the subnormal floor
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)
    ulp = np.exp2(e - 3.0)                     # 3 significand bits
    q = np.round(a / ulp) * ulp                # np.round: ties to even
    if saturate:
        q = np.minimum(q, E4M3_MAX)
    return np.where(np.isnan(x), np.nan, np.sign(x) * np.where(a > 0, q, 0.0))


def e4m3_scale(amax: float) -> float:
    """Per-tensor scale that maps the largest magnitude onto E4M3's 448."""
    return E4M3_MAX / amax if amax > 0 else 1.0
