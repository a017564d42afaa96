"""The stored cell-relative coordinates (Eq. 6) evaluated on the CPU from
their FP64 definition, for tests that check the GPU's bits or emulate its
reduced-precision arithmetic.

s = 2 (x - lo) / h_c rounded to FP64 (one fused multiply-add s = RN(x t + b)
with t = RN(2 / h_c), b = RN(-lo t) when every coordinate lies within 2^17 u
of the origin, else RN(RN(x - lo) t)), c = clamp(floor(s / 2), 0, n_k - 1),
FP32 = RN32(s - (2c + 1)), FP16 = RN16(FP32); the FP16 record's fourth entry
is the cell x modulo 2^16.  The fused multiply-add is evaluated exactly with
rationals and rounded once (Python's float(Fraction) rounds to nearest).
"""
from fractions import Fraction
import math

import numpy as np


def reference(xyz, kh, cells=False):
    """FP32 and FP16 relative coordinates of every input particle (and, with
    cells=True, the integer cell coordinates and the cells per axis)."""
    n, dim = xyz.shape
    hc = kh * (1.0 + 2.0 ** -30)
    t = 2.0 / hc
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    nk = [max(1, int(math.ceil((hi[k] - lo[k]) / hc))) for k in range(dim)]
    fma = all(max(abs(lo[k]), abs(lo[k] + nk[k] * hc)) * t <= 131072.0 for k in range(dim))
    f32 = np.zeros((n, 4), dtype=np.float32)
    cc = np.zeros((n, dim), dtype=np.int64)
    for k in range(dim):
        b = -lo[k] * t
        if fma:
            ft, fb = Fraction(t), Fraction(b)
            s = np.array([float(Fraction(float(x)) * ft + fb) for x in xyz[:, k]])
        else:
            s = (xyz[:, k] - lo[k]) * t
        c = np.minimum(np.floor(s).astype(np.int64) >> 1, nk[k] - 1)
        c = np.maximum(c, 0)
        cc[:, k] = c
        a = s - (2 * c + 1).astype(np.float64)
        f32[:, k] = a.astype(np.float32)
    f16 = f32.astype(np.float16).view(np.uint16).copy()
    f16[:, 3] = (cc[:, 0] & 0xFFFF).astype(np.uint16)
    if cells:
        return f32, f16, fma, cc, nk, hc
    return f32, f16, fma
