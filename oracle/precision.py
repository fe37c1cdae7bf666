"""Rounding to the leaf formats, written from the IEEE-754 / OCP definitions.

Oracle module (test infrastructure only; see the package docstring).

A binary floating-point format with p significand bits (hidden bit included)
and minimum normal exponent emin represents x = m * 2^E with 1 <= |m| < 2;
the spacing of representable numbers near x is 2^(max(E, emin) - p + 1).
Round-to-nearest-even picks the nearest multiple of that spacing, ties to
the even multiple.  Everything here is float64 arithmetic on exact
power-of-two scalings, so the only rounding is the one being modelled.
"""
from __future__ import annotations

import numpy as np

# name: (p, emin, max_finite)
FORMATS = {
    "fp32": (24, -126, float.fromhex("0x1.fffffep127")),
    "bf16": (8, -126, float.fromhex("0x1.fep127")),
    "fp16": (11, -14, 65504.0),
    "e4m3": (4, -6, 448.0),   # OCP FP8 E4M3 (no infinities), saturating
}

# unit roundoff u = 2^-p of each format (the eps of Sec. 4.2, reading)
UNIT_ROUNDOFF = {k: 2.0 ** -v[0] for k, v in FORMATS.items()}


def round_to(x, fmt: str, saturate: bool = False) -> np.ndarray:
    """Round float64 values to the nearest ``fmt`` value, ties to even.
    Overflow gives +-inf (or +-max_finite if ``saturate``; e4m3 always
    saturates)."""
    p, emin, big = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = (x != 0) & np.isfinite(x)
    _, e = np.frexp(x[nz])           # x = f 2^e, 0.5 <= |f| < 1  ->  E = e - 1
    E = np.maximum(e - 1, emin)
    quantum = np.ldexp(1.0, E - (p - 1))
    r = np.rint(x[nz] / quantum) * quantum   # rint = round half to even
    over = np.abs(r) > big
    if saturate or fmt == "e4m3":
        r[over] = np.sign(r[over]) * big
    else:
        r[over] = np.sign(r[over]) * np.inf
    out[nz] = r
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    return out


def split_bf16(x):
    """hi = rn_bf16(x), lo = rn_bf16(x - hi): the two-term bf16 split used by
    the three-product (bf16x3) leaf mode.  x - hi is exact in float64."""
    hi = round_to(x, "bf16")
    lo = round_to(np.asarray(x, np.float64) - hi, "bf16")
    return hi, lo


def to_fp32(x):
    """Round to IEEE binary32 (nearest even)."""
    return round_to(x, "fp32")
