"""Soundness of the FP16 test band and the FP32 re-decision band (no GPU).

The search keeps a candidate pair when its FP16 value e = r2 - T is below
tau16, re-decides kept pairs in FP32 with the band tau32 and falls back to the
FP64 definition inside that band.  Bit-exact neighbour lists need: (1) every
true neighbour passes the FP16 test, (2) an FP32 decision outside the band
equals the exact decision.  This file emulates, in numpy, the exact sequence of
IEEE operations the kernel performs (round-to-nearest-even at each step; an
FMA is evaluated exactly in float64 and rounded once, which is exact here
because the operands are FP16/FP32 values of bounded range) on millions of
random and adversarial pairs, and checks both properties and the analytic
worst-case bounds (0.0199 u^2 and 4.7e-6 u^2) against the library's bands.
The stored FP16 coordinate is the FP16 rounding of the FP32 one (at most
2^-25 u further from the FP64 value than a direct rounding).
"""
import numpy as np
import pytest

from paper_2401_08586_gb300 import sph

RNG = np.random.default_rng(1234)


def t16_up(T):
    """Smallest FP16 value >= T (the library rounds the threshold upward)."""
    t = np.float16(T)
    while float(t) < T:
        t = np.nextafter(t, np.float16(np.inf))
    return t


def f16_of_f32(x):
    """The stored FP16 coordinate: the FP32 rounding of the FP64 value, rounded
    again to FP16 (as the library stores rel16)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float16).astype(np.float64)


def fp16_e(ai, aj, sh, T):
    """e = ((dx^2 - T16) + dy^2) + dz^2 with the kernel's FP16 roundings."""
    f16 = lambda x: np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)
    qi, qj = f16_of_f32(ai), f16_of_f32(aj)
    p = f16(qj + 2.0 * sh)          # pre-shifted candidate (__hadd2)
    d = f16(p - qi)                  # __hsub2
    e = f16(d[:, 0] * d[:, 0] - float(t16_up(T)))   # __hfma2
    for k in range(1, ai.shape[1]):
        e = f16(d[:, k] * d[:, k] + e)
    return e


def fp32_r2(ai, aj, sh):
    f32 = lambda x: np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    ri, rj = f32(ai), f32(aj)
    d = f32(f32(rj + 2.0 * sh) - ri)
    r2 = f32(d[:, 0] * d[:, 0])
    for k in range(1, ai.shape[1]):
        r2 = f32(d[:, k] * d[:, k] + r2)
    return r2


def pairs_near_threshold(m, dim, T, width=0.08):
    """Home particle anywhere in its cell, partner at |D| within +-width of sqrt(T),
    expressed relative to the partner's own cell (|dc| <= 1 per axis)."""
    xi = RNG.uniform(-1, 1, size=(m, dim))
    v = RNG.normal(size=(m, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = np.sqrt(T) + RNG.uniform(-width, width, size=m)
    xj = xi + v * r[:, None]
    c = np.floor((xj + 1.0) / 2.0)
    ok = np.all(np.abs(c) <= 1, axis=1)
    aj = xj - 2.0 * c
    return xi[ok], np.clip(aj[ok], -1, 1), c[ok]


def adversarial_pairs(dim, T):
    """Coordinates on and beside cell faces and centres, all cell offsets."""
    vals = np.array([-1.0, -1 + 2 ** -11, -1 + 2 ** -12, -0.5, -2 ** -12, 0.0, 2 ** -12, 0.5,
                     1 - 2 ** -12, 1 - 2 ** -11, 1.0])
    m = 400000
    ai = RNG.choice(vals, size=(m, dim)) + RNG.uniform(-2e-4, 2e-4, size=(m, dim)) * RNG.integers(0, 2, (m, dim))
    aj = RNG.choice(vals, size=(m, dim)) + RNG.uniform(-2e-4, 2e-4, size=(m, dim)) * RNG.integers(0, 2, (m, dim))
    ai, aj = np.clip(ai, -1, 1), np.clip(aj, -1, 1)
    sh = RNG.integers(-1, 2, size=(m, dim)).astype(np.float64)
    return ai, aj, sh


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("T", [4.0 * (1 - 2.0 ** -29), 4.0 / 1.5 ** 2, 4.0 / 1.01 ** 2])
def test_fp16_band_sound(dim, T):
    tau16, _ = sph.sph_precision_bands()
    worst = -np.inf
    for gen in (lambda: pairs_near_threshold(1_500_000, dim, T),
                lambda: adversarial_pairs(dim, T)):
        ai, aj, sh = gen()
        D2 = np.sum((aj + 2.0 * sh - ai) ** 2, axis=1)
        e = fp16_e(ai, aj, sh, T)
        true_nb = D2 < T
        assert true_nb.sum() > 1000
        # every true neighbour survives the FP16 test
        assert np.all(e[true_nb] < tau16)
        err = e - (D2 - T)
        close = np.abs(D2 - T) < 0.5
        worst = max(worst, float(err[close].max()))
    # the analytic worst case of the op sequence, and the library band above it
    assert worst <= 0.0199
    assert 0.0199 < tau16


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("T", [4.0 * (1 - 2.0 ** -29), 4.0 / 1.5 ** 2])
def test_fp32_band_sound(dim, T):
    _, tau32 = sph.sph_precision_bands()
    ai, aj, sh = pairs_near_threshold(1_500_000, dim, T, width=1e-5)
    D2 = np.sum((aj + 2.0 * sh - ai) ** 2, axis=1)
    r2 = fp32_r2(ai, aj, sh)
    err = np.abs(r2 - D2)
    assert err.max() <= 4.7e-6
    t_in = np.float32(T - tau32)
    t_out = np.float32(T + tau32)
    t_in = t_in if float(t_in) <= T - tau32 else np.nextafter(t_in, np.float32(-np.inf))
    t_out = t_out if float(t_out) >= T + tau32 else np.nextafter(t_out, np.float32(np.inf))
    said_in = r2 < float(t_in)
    said_out = r2 > float(t_out)
    assert np.all(D2[said_in] < T)
    assert np.all(D2[said_out] >= T)
    # the band is narrow: only pairs within ~tau32 of the threshold reach FP64
    undecided = ~(said_in | said_out)
    assert np.all(np.abs(D2[undecided] - T) < 2 * tau32 + 5e-6)


def fp16_e_frame(ai, aj, oi, oj, T):
    """Row-tile arithmetic: both coordinates re-expressed in a frame cell,
    X = fl16(q + 2 o) with integer cell offsets o, then the same e chain."""
    f16 = lambda x: np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)
    Xi = f16(f16_of_f32(ai) + 2.0 * oi)
    Xj = f16(f16_of_f32(aj) + 2.0 * oj)
    d = f16(Xj - Xi)
    e = f16(d[:, 0] * d[:, 0] - float(t16_up(T)))
    for k in range(1, ai.shape[1]):
        e = f16(d[:, k] * d[:, k] + e)
    return e


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("maxoff,tau", [(1, 0.03), (3, 0.06)])
def test_fp16_band_sound_in_tile_frame(dim, maxoff, tau):
    """Frame coordinates with x cell offsets up to +-maxoff (|X| < 4 for 1,
    |X| < 8 for 3): every true neighbour keeps e below the band the tile
    search uses for that magnitude."""
    T = 4.0 * (1 - 2.0 ** -29)
    ai, aj, sh = pairs_near_threshold(1_500_000, dim, T, width=0.1)
    oi = np.zeros_like(ai)
    oi[:, 0] = RNG.integers(-maxoff + 1, maxoff, size=ai.shape[0]) if maxoff > 1 else 0
    oj = oi + sh
    ok = np.abs(oj[:, 0]) <= maxoff
    if dim == 3:
        ok &= np.all(np.abs(oj[:, 1:]) <= 1, axis=1)
    ai, aj, oi, oj, sh = ai[ok], aj[ok], oi[ok], oj[ok], sh[ok]
    D2 = np.sum((aj + 2.0 * sh - ai) ** 2, axis=1)
    e = fp16_e_frame(ai, aj, oi, oj, T)
    nb = D2 < T
    assert nb.sum() > 1000
    assert np.all(e[nb] < tau)
    assert float((e - (D2 - T))[np.abs(D2 - T) < 0.5].max()) <= (0.0199 if maxoff == 1 else 0.044)


def fp16_e_shift(ai, aj, si, sj, T):
    """Row-tile arithmetic with any integer frame shifts s (X = fl16(q + s)):
    odd shifts are the frames centred on the face between a two-cell group's
    cells."""
    f16 = lambda x: np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)
    Xi = f16(f16_of_f32(ai) + si)
    Xj = f16(f16_of_f32(aj) + sj)
    d = f16(Xj - Xi)
    e = f16(d[:, 0] * d[:, 0] - float(t16_up(T)))
    for k in range(1, ai.shape[1]):
        e = f16(d[:, k] * d[:, k] + e)
    return e


@pytest.mark.parametrize("dim", [2, 3])
def test_fp16_band_sound_in_face_centred_frame(dim):
    """Two-cell home groups with the FP16 frame centre on the face between
    their cells: x shifts 2 o - 1 for cell offsets o in -1..2, so |X| <= 4;
    every true neighbour keeps e below the narrow band, and the rounding
    stays under the |X| <= 4 bound."""
    T = 4.0 * (1 - 2.0 ** -29)
    ai, aj, sh = pairs_near_threshold(1_500_000, dim, T, width=0.1)
    oi = np.zeros_like(ai)
    oi[:, 0] = RNG.integers(0, 2, size=ai.shape[0])  # the home in either cell
    oj = oi + sh
    ok = (oj[:, 0] >= -1) & (oj[:, 0] <= 2)
    if dim == 3:
        ok &= np.all(np.abs(oj[:, 1:]) <= 1, axis=1)
    ai, aj, oi, oj, sh = ai[ok], aj[ok], oi[ok], oj[ok], sh[ok]
    si = 2.0 * oi
    sj = 2.0 * oj
    si[:, 0] -= 1.0
    sj[:, 0] -= 1.0
    assert np.abs(ai[:, 0] + si[:, 0]).max() <= 4 and np.abs(aj[:, 0] + sj[:, 0]).max() <= 4
    D2 = np.sum((aj + 2.0 * sh - ai) ** 2, axis=1)
    e = fp16_e_shift(ai, aj, si, sj, T)
    nb = D2 < T
    assert nb.sum() > 1000
    assert np.all(e[nb] < 0.03)
    assert float((e - (D2 - T))[np.abs(D2 - T) < 0.5].max()) <= 0.0199


def test_fp16_band_is_needed():
    """Without the band the FP16 test would lose true neighbours (so the test
    above is not vacuous)."""
    T = 4.0 * (1 - 2.0 ** -29)
    ai, aj, sh = pairs_near_threshold(400_000, 3, T, width=0.02)
    D2 = np.sum((aj + 2.0 * sh - ai) ** 2, axis=1)
    e = fp16_e(ai, aj, sh, T)
    assert np.any((D2 < T) & (e >= 0))
