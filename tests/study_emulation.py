"""CPU emulation of the precision study's reduced-precision decisions
(Tables 1-2 and approach II of Table 4 of arXiv 2401.08586), operation by
operation with one IEEE rounding (to nearest, ties to even) per step, so the
GPU's wrong-decision counts can be compared as exact integers.

Each fused multiply-add is evaluated exactly (the product of two FP16 or FP32
values is exact in FP64; the sum is split exactly into s + e by TwoSum and
rounded to odd, which has more than two bits to spare over FP32 and FP16), then
rounded once to the target format.  numpy's FP64 -> FP16 and FP64 -> FP32
conversions round to nearest even.  The exact decision comes from the oracle's
neighbour list; the candidate pairs are every ordered pair (i, j != i) in the
3^d cells around i's cell, with the cells of the stored relative coordinates
(tests/relref.py).
"""
import numpy as np

import oracle
from relref import reference


def _round_odd(s, e):
    """s + e (s = RN(s + e)) rounded to odd in FP64."""
    fix = (e != 0) & ((s.view(np.int64) & 1) == 0)
    if np.any(fix):
        s = s.copy()
        s[fix] = np.nextafter(s[fix], np.where(e[fix] > 0, np.inf, -np.inf))
    return s


def fma(a, b, c, dtype):
    """RN_dtype(a * b + c) for FP16/FP32 values a, b, c given as FP64 arrays."""
    p = a * b                      # exact
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)  # TwoSum: s + e == p + c exactly
    return _round_odd(s, e).astype(dtype).astype(np.float64)


def rnd(x, dtype):
    return np.asarray(x, dtype=np.float64).astype(dtype).astype(np.float64)


def candidate_pairs(cc, nk, dim, rows):
    """(i, j, offset) of every ordered pair j != i in the 3^d cells around
    i's cell, for i in rows."""
    nx = nk[0]
    ny = nk[1]
    nz = nk[2] if dim == 3 else 1
    cz = cc[:, 2] if dim == 3 else np.zeros(len(cc), dtype=np.int64)
    lin = (cz * ny + cc[:, 1]) * nx + cc[:, 0]
    order = np.argsort(lin, kind="stable")
    start = np.zeros(nx * ny * nz + 1, dtype=np.int64)
    np.cumsum(np.bincount(lin, minlength=nx * ny * nz), out=start[1:])
    out = []
    offs = [(dx, dy, dz) for dz in ((-1, 0, 1) if dim == 3 else (0,)) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    for dx, dy, dz in offs:
        x, y, z = cc[rows, 0] + dx, cc[rows, 1] + dy, cz[rows] + dz
        ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
        i = rows[ok]
        c = (z[ok] * ny + y[ok]) * nx + x[ok]
        cnt = start[c + 1] - start[c]
        ii = np.repeat(i, cnt)
        base = np.repeat(start[c] - np.concatenate([[0], np.cumsum(cnt)[:-1]]), cnt)
        jj = order[base + np.arange(cnt.sum())]
        keep = jj != ii
        out.append((ii[keep], jj[keep], (dx, dy, dz)))
    return out


def counts(xyz, kh, row_begin=0, row_end=None):
    """candidates, neighbours and the wrong decisions of FP16 absolute, FP32
    absolute and FP16 cell-relative coordinates, as the study reports them."""
    n, dim = xyz.shape
    row_end = n if row_end is None else row_end
    rows = np.arange(row_begin, row_end, dtype=np.int64)
    f32, f16, _fma, cc, nk, hc = reference(xyz, kh, cells=True)
    q16 = f16[:, :3].copy().view(np.float16).astype(np.float64)  # x, y, z of the FP16 record
    rp, col = oracle.cll(xyz, kh)
    keys = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp)) * n + col.astype(np.int64)
    kh2_16 = rnd(kh * kh, np.float16)
    kh2_32 = rnd(kh * kh, np.float32)
    u = hc * 0.5
    t16 = rnd(kh * kh / (u * u), np.float16)
    a16 = rnd(xyz, np.float16)
    a32 = rnd(xyz, np.float32)
    c = dict(candidates=0, neighbours=0, wrong_fp16_abs=0, wrong_fp32_abs=0, wrong_fp16_rcll=0)
    for i, j, (dx, dy, dz) in candidate_pairs(cc, nk, dim, rows):
        if i.size == 0:
            continue
        ex = np.isin(i * n + j, keys)
        r16 = np.zeros(i.size)
        r32 = np.zeros(i.size)
        for k in range(dim):
            d = rnd(a16[i, k] - a16[j, k], np.float16)
            r16 = fma(d, d, r16, np.float16)
            d = rnd(a32[i, k] - a32[j, k], np.float32)
            r32 = fma(d, d, r32, np.float32)
        # FP16 RCLL: d = (q_j - q_i) + 2 dc per axis, r^2 = d_x^2, then FMAs
        shift = (dx, dy, dz)
        r = None
        for k in range(dim):
            d = rnd(rnd(q16[j, k] - q16[i, k], np.float16) + 2.0 * shift[k], np.float16)
            r = rnd(d * d, np.float16) if r is None else fma(d, d, r, np.float16)
        c["candidates"] += int(i.size)
        c["neighbours"] += int(ex.sum())
        c["wrong_fp16_abs"] += int(((r16 < kh2_16) != ex).sum())
        c["wrong_fp32_abs"] += int(((r32 < kh2_32) != ex).sum())
        c["wrong_fp16_rcll"] += int(((r < t16) != ex).sum())
    return c
