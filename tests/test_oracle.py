"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed forms
of Eq. 3, the normalisation integral of the kernel (scipy quadrature), a
library neighbour search (scipy cKDTree), exact lattice counts from integer
enumeration, pair symmetry, brute force against the cell link-list, and exact
identities of the Appendix A5 gradient on linear fields.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

import oracle
from paper_2401_08586_gb300 import workloads as W
from conftest import read_golden


def pairs_of(row_ptr, col):
    rows = np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))
    return set(zip(rows.tolist(), col.tolist()))


# ---------------------------------------------------------------- kernel, Eq. 3

def test_kernel_golden_values():
    for dim, R, _frac, w in read_golden("kernel_values.txt"):
        got = oracle.kernel_w(int(dim), float(R), 1.0)[0]
        assert got == pytest.approx(float(w), rel=1e-15, abs=1e-300), (dim, R)


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("h", [1.0, 0.013, 3.7])
def test_kernel_closed_forms(dim, h):
    a = oracle.kernel_alpha(dim, h)
    assert a == pytest.approx({1: 1 / h, 2: 15 / (7 * math.pi * h * h),
                               3: 3 / (2 * math.pi * h ** 3)}[dim], rel=1e-15)
    w = lambda R: oracle.kernel_w(dim, R, h)[0]
    assert w(0.0) == pytest.approx(2 * a / 3, rel=1e-15)
    # both branches give alpha/6 at R = 1 (continuity)
    assert w(1.0) == pytest.approx(a / 6, rel=1e-15)
    assert w(1.0 - 1e-12) == pytest.approx(a / 6, rel=1e-9)
    assert w(2.0) == 0.0 and w(2.5) == 0.0 and w(1e6) == 0.0
    assert w(2.0 - 1e-4) == pytest.approx(a * 1e-12 / 6, rel=1e-6)
    # monotone decreasing on [0, 2]
    R = np.linspace(0, 2, 4001)
    vals = oracle.kernel_w(dim, R, h)
    assert np.all(np.diff(vals) <= 0)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_normalisation(dim):
    """The kernel integrates to one over its support: this pins alpha_d and
    both polynomial branches of Eq. 3 (a dropped term or wrong sign fails)."""
    h = 0.7
    w = lambda r: oracle.kernel_w(dim, r / h, h)[0]
    shell = {1: lambda r: 2.0, 2: lambda r: 2 * math.pi * r, 3: lambda r: 4 * math.pi * r * r}[dim]
    total = sum(integrate.quad(lambda r: w(r) * shell(r), a, b, epsabs=1e-14, epsrel=1e-13)[0]
                for a, b in ((0, h), (h, 2 * h)))
    assert total == pytest.approx(1.0, abs=1e-10)


# ------------------------------------------------------------ neighbour search

@pytest.mark.parametrize("dim,n,seed", [(2, 600, 0), (3, 700, 1), (2, 1500, 2), (3, 2000, 3)])
def test_allpairs_matches_kdtree(dim, n, seed):
    xyz = W.random_uniform(n, dim, seed)
    kh = 0.08 if dim == 2 else 0.15
    rp, col = oracle.allpairs(xyz, kh)
    got = pairs_of(rp, col)
    tree = cKDTree(xyz)
    ref = set()
    for i, j in tree.query_pairs(kh, output_type="ndarray").tolist():
        ref.add((i, j))
        ref.add((j, i))
    assert got == ref
    # columns ascending within each row
    for i in range(n):
        seg = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_allpairs_hand_cases():
    kh = 0.25
    # two particles just inside / just outside / exactly at kh (strict test)
    for d, expect in ((kh * (1 - 1e-12), 1), (kh * (1 + 1e-12), 0)):
        rp, col = oracle.allpairs(np.array([[0.0, 0.0], [d, 0.0]]), kh)
        assert rp.tolist() == [0, expect, 2 * expect]
    rp, _ = oracle.allpairs(np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.25]]), kh)  # exact tie
    assert rp.tolist() == [0, 0, 0]
    # coincident particles are neighbours of each other but not of themselves
    rp, col = oracle.allpairs(np.zeros((3, 3)), kh)
    assert rp.tolist() == [0, 2, 4, 6] and col.tolist() == [1, 2, 0, 2, 0, 1]
    # empty and single inputs
    rp, col = oracle.allpairs(np.zeros((0, 3)), kh)
    assert rp.tolist() == [0] and col.size == 0
    rp, col = oracle.allpairs(np.zeros((1, 2)), kh)
    assert rp.tolist() == [0, 0] and col.size == 0


def _cases():
    yield "lattice2d", W.c1_2d_10k(side=40).xyz, 2.4 * 0.025
    yield "lattice3d", W.c2_3d_1m(side=14).xyz, 0.026
    yield "random2d", W.random_uniform(3000, 2, 5), 0.03
    yield "random3d", W.random_uniform(3000, 3, 6), 0.09
    yield "faces3d", W.face_set(0.1, 3, 7), 0.1
    yield "faces2d", W.face_set(0.1, 2, 8), 0.1
    yield "circle2d", W.circle_pairs(0.05, 1e-9, 400, 2, 9), 0.05
    yield "circle3d", W.circle_pairs(0.05, 1e-12, 400, 3, 10), 0.05
    yield "one_cell", W.random_uniform(200, 3, 11, extent=0.05), 0.2
    yield "coincident", np.full((50, 3), 0.3), 0.1
    yield "line", np.stack([np.linspace(0, 1, 500), np.zeros(500), np.zeros(500)], 1), 0.0101
    yield "two", np.array([[0.0, 0.0], [0.01, 0.0]]), 0.02
    yield "one", np.array([[0.5, 0.5, 0.5]]), 0.1
    yield "empty", np.zeros((0, 3)), 0.1
    ps = W.c3_3d_dambreak(side=16)
    yield "dambreak_small", ps.xyz, ps.kh


@pytest.mark.parametrize("name,xyz,kh", list(_cases()), ids=[c[0] for c in _cases()])
def test_cll_equals_allpairs(name, xyz, kh):
    rp_a, col_a = oracle.allpairs(xyz, kh)
    rp_c, col_c = oracle.cll(xyz, kh)
    assert np.array_equal(rp_a, rp_c)
    assert np.array_equal(col_a, col_c)


@pytest.mark.parametrize("name,xyz,kh", [c for c in _cases() if c[1].shape[0] >= 2],
                         ids=[c[0] for c in _cases() if c[1].shape[0] >= 2])
def test_cll_rows_equal_allpairs_rows(name, xyz, kh):
    """Sampled rows (shuffled, repeated) are the brute-force rows."""
    rp_a, col_a = oracle.allpairs(xyz, kh)
    rng = np.random.default_rng(3)
    rows = rng.integers(0, xyz.shape[0], size=min(300, 3 * xyz.shape[0]))
    rp, col = oracle.cll_rows(xyz, kh, rows, threads=2)
    for r, i in enumerate(rows):
        assert np.array_equal(col[rp[r]:rp[r + 1]], col_a[rp_a[i]:rp_a[i + 1]])
    rho = oracle.density_rows(xyz, 0.5 * kh, rows, rp, col)
    rho_all = oracle.density(xyz, 0.5 * kh, rp_a, col_a)
    assert np.array_equal(rho, rho_all[rows])


def test_cll_threads_identical():
    ps = W.c2_3d_1m(side=20)
    a = oracle.cll(ps.xyz, ps.kh, threads=1)
    b = oracle.cll(ps.xyz, ps.kh, threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _lattice_interior_counts(dim, side, dx, kh):
    xyz = W.exact_lattice(side, dim, dx)
    rp, col = oracle.cll(xyz, kh)
    idx = np.arange(side ** dim)
    coords = np.stack(np.unravel_index(idx, (side,) * dim)[::-1], axis=1)
    m = int(math.ceil(kh / dx)) + 1
    interior = np.all((coords >= m) & (coords < side - m), axis=1)
    return np.diff(rp)[interior], rp, col


@pytest.mark.parametrize("dim,khr,count,ties", [tuple(map(float, r)) for r in
                                               read_golden("lattice_counts.txt")])
def test_lattice_invariant(dim, khr, count, ties):
    """Interior counts on an unjittered lattice equal the integer-vector count
    |v|^2 < (kh/dx)^2.  dx = 1/256 makes every coordinate and squared distance
    exact, so kh/dx = 3 and 2 produce exact ties that the strict test drops."""
    dim = int(dim)
    dx = 1.0 / 256
    kh = khr * dx
    side = 12 if dim == 3 else 20
    counts, _, _ = _lattice_interior_counts(dim, side, dx, kh)
    assert counts.size > 0
    assert np.all(counts == int(count))
    # cross-check the table itself by enumerating integer vectors
    r = int(math.ceil(khr))
    vs = [v for v in itertools.product(range(-r, r + 1), repeat=dim) if any(v)]
    n2 = [sum(c * c for c in v) for v in vs]
    k2 = round(khr * khr * 100)
    assert sum(1 for s in n2 if s * 100 < k2) == int(count)
    assert sum(1 for s in n2 if s * 100 == k2) == int(ties)


def test_lattice_invariant_decimal_spacing():
    """The shapes used by the workloads (dx = 0.01, h = 1.2 dx in 2D and 1.3 dx in
    3D) sit between lattice shells, so rounding cannot move a count."""
    for dim, khr, count in ((2, 2.4, 20), (3, 2.6, 80)):
        counts, _, _ = _lattice_interior_counts(dim, 14, 0.01, khr * 0.01)
        assert np.all(counts == count)


@pytest.mark.parametrize("maker", [lambda: W.c1_2d_10k(side=50), lambda: W.c2_3d_1m(side=16),
                                   lambda: W.c3_3d_dambreak(side=14)])
def test_symmetry(maker):
    ps = maker()
    rp, col = oracle.cll(ps.xyz, ps.kh)
    p = pairs_of(rp, col)
    assert p == {(j, i) for (i, j) in p}
    assert all(i != j for i, j in p)


# ----------------------------------------------------------------- density

def test_density_single_and_pair():
    h = 0.01
    rp, col = oracle.cll(np.array([[0.3, 0.3, 0.3]]), 2 * h)
    rho = oracle.density(np.array([[0.3, 0.3, 0.3]]), h, rp, col, mass=2.5)
    assert rho[0] == pytest.approx(2.5 * 2 / 3 * 3 / (2 * math.pi * h ** 3), rel=1e-14)
    # pair at r = h: each sees W(0) + W(1) = alpha (2/3 + 1/6)
    xy = np.array([[0.0, 0.0], [h, 0.0]])
    rp, col = oracle.cll(xy, 2 * h)
    rho = oracle.density(xy, h, rp, col)
    a = 15 / (7 * math.pi * h * h)
    assert rho == pytest.approx([a * 5 / 6, a * 5 / 6], rel=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 800), (3, 900)])
def test_density_equals_full_kernel_sum(dim, n):
    """Because W vanishes at R >= 2, summing W over *every* particle (self
    included) must equal the neighbour-list sum: pins the self term, the use of
    h (not kh) in R, and the row/column bookkeeping."""
    xyz = W.random_uniform(n, dim, 12 + dim)
    h = 0.03 if dim == 2 else 0.07
    rp, col = oracle.cll(xyz, 2 * h)
    rho = oracle.density(xyz, h, rp, col, mass=0.5)
    d = np.sqrt(((xyz[:, None, :] - xyz[None, :, :]) ** 2).sum(-1))
    full = 0.5 * oracle.kernel_w(dim, (d / h).reshape(-1), h).reshape(n, n).sum(1)
    assert rho == pytest.approx(full, rel=1e-12)


@pytest.mark.parametrize("dim,hr,target", [(2, 1.2, 0.99976), (3, 1.3, 0.99726), (3, 1.5, 1.00179)])
def test_partition_of_unity(dim, hr, target):
    """Interior lattice density times dx^d is the lattice sum of W dx^d, close to
    the kernel integral 1 (a sanity check on alpha_d, not a tolerance)."""
    dx = 0.01
    side = 16 if dim == 3 else 30
    xyz = W.exact_lattice(side, dim, dx)
    rp, col = oracle.cll(xyz, 2 * hr * dx)
    rho = oracle.density(xyz, hr * dx, rp, col)
    counts, _, _ = _lattice_interior_counts(dim, side, dx, 2 * hr * dx)
    full = np.diff(rp) == counts.max()
    val = rho[full] * dx ** dim
    assert np.allclose(val, target, atol=2e-5)
    assert abs(val.mean() - 1.0) < 3e-3


# ------------------------------------------------------------- gradient, A5

@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_a5_linear_exact(dim):
    """A5 reproduces the slope of a field that varies along one axis only:
    (f_j - f_i) = a (x_j - x_i) on that axis, so numerator = a * denominator."""
    ps = W.c2_3d_1m(side=10) if dim == 3 else W.c1_2d_10k(side=30)
    rp, col = oracle.cll(ps.xyz, ps.kh)
    for ax in range(dim):
        f = 3.5 * ps.xyz[:, ax] - 1.25
        g = oracle.gradient_a5(ps.xyz, ps.h, f, rp, col)
        assert np.allclose(g[:, ax], 3.5, rtol=1e-10)


def test_gradient_a5_first_order():
    """For f = x^3 on a 2D lattice the interior error falls linearly with dx
    (the first-order accuracy the paper reports in Table 3)."""
    errs = []
    for side in (25, 50):
        dx = 1.0 / side
        xyz = W.lattice((side, side), dx, 0.1, seed=3)
        h = 1.2 * dx
        rp, col = oracle.cll(xyz, 2 * h)
        g = oracle.gradient_a5(xyz, h, xyz[:, 0] ** 3, rp, col)
        inner = np.all((xyz > 0.2) & (xyz < 0.8), axis=1)
        errs.append(np.sqrt(np.mean((g[inner, 0] - 3 * xyz[inner, 0] ** 2) ** 2)))
    assert errs[1] < errs[0] * 0.75


# ------------------------------------------- kernel derivative (Eq. 3, A5)

def _golden_derivative():
    from fractions import Fraction
    table, a5 = [], []
    for row in read_golden("kernel_derivative.txt"):
        if row[0] == "A5":
            a5.append(row[1:])
        else:
            table.append((Fraction(row[0]), Fraction(row[1])))
    return table, a5


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("h", [1.0, 0.013])
def test_kernel_derivative_hand_values(dim, h):
    """dW/dR against Eq. 3 differentiated by hand (tests/golden/kernel_derivative.txt):
    both branches, their junction at R = 1 and the ends of the support."""
    a = oracle.kernel_alpha(dim, h)
    table, _ = _golden_derivative()
    for R, dP in table:
        got = oracle.kernel_dwdr(dim, float(R), h)[0]
        assert got == pytest.approx(a * float(dP), rel=1e-15, abs=1e-300), (dim, R)
    # just below the support's end the derivative is -(2 - R)^2 / 2 -> 0
    assert oracle.kernel_dwdr(dim, 2.0 - 1e-6, h)[0] == pytest.approx(-a * 0.5e-12, rel=1e-6)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kernel_derivative_central_differences(dim):
    """dW/dR against central differences of W (pinned above by closed forms and
    its normalisation integral) at points inside both branches."""
    h = 0.37
    eps = 1e-6
    for R in np.concatenate([np.linspace(0.01, 0.99, 23), np.linspace(1.01, 1.99, 23)]):
        w_hi = oracle.kernel_w(dim, R + eps, h)[0]
        w_lo = oracle.kernel_w(dim, R - eps, h)[0]
        fd = (w_hi - w_lo) / (2 * eps)
        got = oracle.kernel_dwdr(dim, R, h)[0]
        assert got == pytest.approx(fd, rel=1e-6, abs=1e-9 * oracle.kernel_alpha(dim, h)), R


def test_gradient_a5_hand_worked():
    """Appendix A5 on the three-particle line of tests/golden/kernel_derivative.txt
    (f = x^2, one neighbour in each branch of the kernel): -1/4 along x, 0 along y."""
    from fractions import Fraction
    _, a5 = _golden_derivative()
    for dim, h, xi, yi, x1, y1, x2, y2, field, ex, ey in a5:
        assert field == "x^2"
        xyz = np.array([[float(Fraction(xi)), float(Fraction(yi))],
                        [float(Fraction(x1)), float(Fraction(y1))],
                        [float(Fraction(x2)), float(Fraction(y2))]])
        f = xyz[:, 0] ** 2
        rp, col = oracle.allpairs(xyz, 2 * float(h))
        assert col[rp[0]:rp[1]].tolist() == [1, 2]
        g = oracle.gradient_a5(xyz, float(h), f, rp, col)
        assert g[0, 0] == pytest.approx(float(Fraction(ex)), rel=1e-14)
        assert g[0, 1] == float(Fraction(ey))


def test_gradient_a5_off_axis_against_finite_difference_weights():
    """A5 for four particles off the axes (f = x^2 + 3 y^2), the expected value
    built from the A5 sums with weights W' taken by central differences of the
    pinned W (not the oracle's derivative): a wrong branch, coefficient or a
    W in place of W' moves the ratio."""
    h = 1.0
    xyz = np.array([[0.0, 0.0], [0.4, 0.3], [-1.1, 0.5], [0.2, -1.3], [-0.7, -0.9]])
    f = xyz[:, 0] ** 2 + 3 * xyz[:, 1] ** 2
    rp, col = oracle.allpairs(xyz, 2 * h)
    g = oracle.gradient_a5(xyz, h, f, rp, col)
    eps = 1e-6
    num, den = np.zeros(2), np.zeros(2)
    for j in col[rp[0]:rp[1]]:
        d = xyz[0] - xyz[j]
        r = math.hypot(d[0], d[1])
        wp = (oracle.kernel_w(2, r / h + eps, h)[0] - oracle.kernel_w(2, r / h - eps, h)[0]) / (2 * eps) / h
        dwdx = wp * d / r
        num += (f[j] - f[0]) * dwdx
        den += (xyz[j] - xyz[0]) * dwdx
    assert len(col[rp[0]:rp[1]]) == 4
    assert np.allclose(g[0], num / den, rtol=1e-7)
