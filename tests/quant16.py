"""Rounding of FP64 values to a binary floating-point format with `mant`
stored fraction bits and minimum normal exponent `emin` (FP16: 10, -14;
BF16: 7, -126), to nearest with ties to even, done exactly in FP64.

Test helper for the 16-bit storage of the geometric factors: it defines the
stored values independently of the CUDA conversion intrinsics.  Values are
assumed well inside the format's range (no overflow handling).
"""

import numpy as np


def round_to_format(v, mant, emin):
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, x = np.frexp(a)                     # a = m 2^x, m in [0.5, 1)
    e = np.maximum(x - 1, emin)            # exponent of the leading bit (or emin)
    ulp = np.ldexp(1.0, e - mant)          # spacing of the format near a
    q = np.round(a / ulp) * ulp            # a / ulp is exact; np.round ties to even
    return np.where(a == 0, v, np.copysign(q, v))


def fp16(v):
    return round_to_format(v, 10, -14)


def bf16(v):
    return round_to_format(v, 7, -126)


def quantise_factors(G, E, Np3, kind):
    """Stored 16-bit factors as the operator uses them: per element e,
    scale = float32(max |G| over its six factors and points) (1 if zero),
    q = round16(G / scale); the operator computes with q and multiplies its
    result by the scale, i.e. it applies the factors q * scale exactly.
    Returns those factors (float64, exact) and the scales."""
    G = np.asarray(G, dtype=np.float64).reshape(E, 6 * Np3)
    m = np.abs(G).max(axis=1)
    sc = np.where(m > 0, m.astype(np.float32), np.float32(1.0))
    v = G / sc[:, None].astype(np.float64)
    q = fp16(v) if kind == "f16" else bf16(v)
    Gq = q * sc[:, None].astype(np.float64)  # 11- or 8-bit times 24-bit: exact in FP64
    return Gq.reshape(-1), sc
