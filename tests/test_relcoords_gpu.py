"""Stored cell-relative coordinates (Eq. 6) bit for bit against their FP64
definition, evaluated here on the CPU: s = 2 (x - lo) / h_c rounded to FP64
(one fused multiply-add s = RN(x t + b) with t = RN(2 / h_c), b = RN(-lo t)
when every coordinate lies within 2^17 u of the origin, else RN(RN(x - lo) t)),
c = min(floor(s / 2), n_k - 1), FP32 = RN32(s - (2c + 1)), FP16 = RN16(FP32);
the FP16 record's fourth entry is the cell x modulo 2^16.
The fused multiply-add is evaluated exactly with rationals and rounded once
(Python's float(Fraction) rounds to nearest).  Covers the particle at the
lower bound (s = 0), the half cell next to it (s < 1), the upper clamp, and a
grid far from the origin (the subtraction route).  GPU required."""
import numpy as np
import pytest

from paper_2401_08586_gb300 import workloads as W
from relref import reference

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


def check(sph, xyz, h, expect_fma):
    kh = 2.0 * h
    x = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
    g = sph.Grid(x, h, kh)
    r16, r32 = g.relative_coordinates()
    orig = g.orig_id().cpu().numpy()
    f32, f16, fma = reference(xyz, kh)
    assert fma == expect_fma
    got32 = r32.cpu().numpy().view(np.uint32)
    got16 = r16.cpu().numpy().view(np.uint16)
    want32 = f32[orig].view(np.uint32)
    want16 = f16[orig]
    bad = np.nonzero((got32 != want32).any(axis=1))[0]
    assert bad.size == 0, (bad[:5], got32[bad[:5]], want32[bad[:5]])
    assert np.array_equal(got16, want16)


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_near_origin(sph, dim):
    side = 30 if dim == 3 else 150
    xyz = W.lattice((side,) * dim, 0.01, 0.1, 5)
    check(sph, xyz, 0.013, True)


def test_random_offset_box(sph):
    rng = np.random.default_rng(8)
    xyz = 1000.0 + rng.uniform(0.0, 1.0, size=(20000, 3))
    check(sph, xyz, 0.03, True)


def test_points_on_cell_faces(sph):
    """Coordinates at lo + j h_c / 2 (cell faces and centres, s near integers)
    and the upper bound exactly n_k cells away (the clamp)."""
    h = 0.02
    hc = 2 * h * (1.0 + 2.0 ** -30)
    j = np.arange(0, 41)
    base = j * (hc / 2.0)
    rng = np.random.default_rng(3)
    xyz = np.stack([rng.permutation(base) for _ in range(3)], axis=1)
    xyz = np.vstack([xyz, xyz + np.nextafter(0.0, 1.0), xyz[:5] * (1 + 2e-16)])
    check(sph, xyz, h, True)


def test_far_from_origin(sph):
    """|x| 2 / h_c beyond 2^17: the subtraction route."""
    rng = np.random.default_rng(9)
    xyz = 1.0e6 + rng.uniform(0.0, 1.0, size=(5000, 3))
    check(sph, xyz, 0.05, False)
