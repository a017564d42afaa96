"""Parity of the CUDA path with the FP64 oracle (GPU required).

Neighbour lists must be identical (bit-exact integer CSR); densities within
1e-5 relative of the FP64 oracle (the FP32-accumulation tolerance of the
path).  Every call goes through the C ABI (paper_2401_08586_gb300.sph).
"""
import numpy as np
import pytest

import oracle
from paper_2401_08586_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO_RTOL = 1e-5


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


def run(sph, xyz, h, kh, order, precision=0, density=True, mass=1.0, box=None, cell_size=0.0, fused=True):
    x = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float64)).cuda()
    g = sph.Grid(x, h, kh, order=order, precision=precision, mass=mass, box=box, cell_size=cell_size)
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_FUSED, int(fused))
    rp, col, rho = g.query(density=density)
    torch.cuda.synchronize()
    out = dict(rp=rp.cpu().numpy(), col=col.cpu().numpy(), rho=None if rho is None else rho.cpu().numpy(),
               orig=g.orig_id().cpu().numpy(), rank=g.rank().cpu().numpy(), info=g.info(), grid=g, x=x)
    return out


def to_canonical(rp, col, orig):
    """CELL-order CSR (rows/cols are sorted positions) -> input-order CSR."""
    n = rp.size - 1
    lens = np.diff(rp)
    rows_in = orig  # row r is input particle orig[r]
    new_len = np.empty(n, dtype=np.int64)
    new_len[rows_in] = lens
    new_rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(new_len, out=new_rp[1:])
    new_col = np.empty_like(col)
    for r in range(n):
        seg = np.sort(orig[col[rp[r]:rp[r + 1]]])
        i = rows_in[r]
        new_col[new_rp[i]:new_rp[i + 1]] = seg
    return new_rp, new_col


def check_against_oracle(out, xyz, h, kh, order, mass=1.0, density=True):
    rp_ref, col_ref = oracle.cll(xyz, kh)
    rp, col = out["rp"], out["col"]
    if order == 0:
        # columns ascending within each row in cell order
        for r in range(min(rp.size - 1, 2000)):
            assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)
        rp, col = to_canonical(rp, col, out["orig"])
    assert np.array_equal(rp, rp_ref), "row_ptr differs"
    assert np.array_equal(col, col_ref), "col differs"
    if density:
        rho_ref = oracle.density(xyz, h, rp_ref, col_ref, mass=mass)
        rho = out["rho"].astype(np.float64)
        if order == 0:
            r2 = np.empty_like(rho)
            r2[out["orig"]] = rho
            rho = r2
        rel = np.abs(rho - rho_ref) / np.abs(rho_ref)
        assert rel.max() <= RHO_RTOL, rel.max()
        return rel.max()
    return None


CASES = {
    "c1_2d_10k": lambda: (W.c1_2d_10k().xyz, W.c1_2d_10k().h),
    "lattice3d_27k": lambda: (W.c2_3d_1m(side=30).xyz, 0.013),
    "random2d": lambda: (W.random_uniform(5000, 2, 3), 0.006),
    "random3d": lambda: (W.random_uniform(6000, 3, 4), 0.03),
    "faces3d": lambda: (W.face_set(0.1, 3, 7), 0.05),
    "faces2d": lambda: (W.face_set(0.1, 2, 8), 0.05),
    "circle2d_1e-8": lambda: (W.circle_pairs(0.05, 1e-8, 2000, 2, 9), 0.025),
    "circle3d_1e-12": lambda: (W.circle_pairs(0.05, 1e-12, 2000, 3, 10), 0.025),
    "circle3d_1e-3": lambda: (W.circle_pairs(0.05, 1e-3, 2000, 3, 11), 0.025),
    "dambreak_small": lambda: (W.c3_3d_dambreak(side=24).xyz, W.c3_3d_dambreak(side=24).h),
    "one": lambda: (np.array([[0.3, 0.3, 0.3]]), 0.01),
    "two": lambda: (np.array([[0.0, 0.0], [0.01, 0.0]]), 0.01),
    "line": lambda: (np.stack([np.linspace(0, 1, 3000), np.zeros(3000), np.zeros(3000)], 1), 0.0005),
}


VARIANTS = [(0, 1), (0, 2), (0, 0), (1, 1), (1, 0)]
VARIANT_IDS = ["cell-tile", "cell-cta", "cell-twopass", "canonical-tile", "canonical-twopass"]


@pytest.mark.parametrize("order,fused", VARIANTS, ids=VARIANT_IDS)
@pytest.mark.parametrize("case", sorted(CASES))
def test_parity_fp16_rcll(sph, case, order, fused):
    xyz, h = CASES[case]()
    out = run(sph, xyz, h, 2 * h, order, fused=fused)
    check_against_oracle(out, xyz, h, 2 * h, order)
    assert sph.sph_grid_check(out["grid"].handle) == 0


FP64_VARIANTS = [(0, 1), (1, 1), (1, 0)]
FP64_VARIANT_IDS = ["cell-tile", "canonical-tile", "canonical-twopass"]


@pytest.mark.parametrize("order,fused", FP64_VARIANTS, ids=FP64_VARIANT_IDS)
@pytest.mark.parametrize("case", ["c1_2d_10k", "lattice3d_27k", "faces3d", "circle3d_1e-12", "dambreak_small",
                                  "random2d", "line", "one", "two"])
def test_parity_fp64_cll(sph, case, order, fused):
    """The FP64 cell link-list (the FP64 tile search by default, the two-pass
    search with SPH_OPT_FUSED 0): the oracle's CSR bit for bit, density within
    the FP32 output's tolerance."""
    xyz, h = CASES[case]()
    out = run(sph, xyz, h, 2 * h, order, precision=sph.SPH_PREC_FP64_CLL, fused=fused)
    check_against_oracle(out, xyz, h, 2 * h, order)
    assert sph.sph_grid_check(out["grid"].handle) == 0


def test_fp64_tile_ties_and_count_only(sph):
    """Exact ties at kh (power-of-two lattice) are excluded by the FP64 tile
    search's strict test; its count-only query gives the same row pointers."""
    dx = 1.0 / 256
    xyz = W.exact_lattice(14, 3, dx)
    out = run(sph, xyz, 1.5 * dx, 3 * dx, 0, precision=sph.SPH_PREC_FP64_CLL)
    check_against_oracle(out, xyz, 1.5 * dx, 3 * dx, 0)
    rp = torch.empty(xyz.shape[0] + 1, dtype=torch.int64, device="cuda")
    nnz = sph.sph_nnps_query(out["grid"].handle, rp, None, 0, True, None)
    assert nnz == out["rp"][-1] and np.array_equal(rp.cpu().numpy(), out["rp"])


def test_exact_ties_power_of_two_lattice(sph):
    """dx = 1/256 and kh = 3 dx: 30 exact ties per interior particle, all
    excluded by the strict test; they reach the FP64 tier."""
    dx = 1.0 / 256
    xyz = W.exact_lattice(14, 3, dx)
    out = run(sph, xyz, 1.5 * dx, 3 * dx, 1)
    check_against_oracle(out, xyz, 1.5 * dx, 3 * dx, 1)
    assert out["grid"].info().stat_fp64_pairs > 0


@pytest.mark.parametrize("order,fused", VARIANTS, ids=VARIANT_IDS)
def test_coincident_and_crowded_cells(sph, order, fused):
    """Cells with more than 32 particles (several home batches) and more than
    1024 candidates (several candidate windows); in the single-pass search
    these take the general path around the look-back."""
    rng = np.random.default_rng(5)
    xyz = np.vstack([np.full((70, 3), 0.5), rng.uniform(0.45, 0.55, size=(1500, 3)),
                     rng.uniform(0, 1, size=(500, 3))])
    out = run(sph, xyz, 0.02, 0.04, order, fused=fused)
    check_against_oracle(out, xyz, 0.02, 0.04, order)


@pytest.mark.parametrize("variant", [1, 2])
def test_fused_matches_twopass(sph, variant):
    """The single-pass searches give the same CSR as the two-pass search and
    the same density up to FP32 summation order."""
    ps = W.c2_3d_1m(side=30)
    a = run(sph, ps.xyz, ps.h, ps.kh, 0, fused=variant)
    b = run(sph, ps.xyz, ps.h, ps.kh, 0, fused=0)
    assert np.array_equal(a["rp"], b["rp"]) and np.array_equal(a["col"], b["col"])
    rel = np.abs(a["rho"].astype(np.float64) - b["rho"]) / b["rho"]
    assert rel.max() <= 2e-6


def test_sparse_rows_several_groups(sph):
    """Row tiles whose 32 particles span more than four cells (sparse spray)
    are split into home groups and take the two-step path."""
    rng = np.random.default_rng(17)
    xyz = np.vstack([rng.uniform(0, 1, size=(3000, 3)) * [1.0, 0.05, 0.05], rng.uniform(0, 1, size=(2000, 3))])
    out = run(sph, xyz, 0.004, 0.008, 0, fused=1)
    check_against_oracle(out, xyz, 0.004, 0.008, 0)


def test_empty_input(sph):
    x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    g = sph.Grid(x, 0.01)
    rp, col, rho = g.query()
    assert rp.cpu().tolist() == [0] and col.numel() == 0


def test_mass_and_cell_size(sph):
    ps = W.c1_2d_10k(side=50)
    out = run(sph, ps.xyz, ps.h, ps.kh, 1, mass=2.5, cell_size=ps.kh * 1.7)
    check_against_oracle(out, ps.xyz, ps.h, ps.kh, 1, mass=2.5)


def test_user_box(sph):
    ps = W.c2_3d_1m(side=16)
    out = run(sph, ps.xyz, ps.h, ps.kh, 1, box=((-0.01, -0.01, -0.01), (0.2, 0.2, 0.2)))
    check_against_oracle(out, ps.xyz, ps.h, ps.kh, 1)
    # a particle outside the box is reported
    bad = ps.xyz.copy()
    bad[0, 0] = 0.5
    x = torch.from_numpy(bad).cuda()
    with pytest.raises(sph.SphError) as ei:
        g = sph.Grid(x, ps.h, ps.kh, box=((-0.01,) * 3, (0.2,) * 3))
        g.query()
    assert ei.value.code == sph.SPH_ERR_INVALID


def test_nonfinite_rejected(sph):
    xyz = W.random_uniform(100, 3, 1)
    xyz[7, 1] = np.nan
    with pytest.raises(sph.SphError) as ei:
        sph.Grid(torch.from_numpy(xyz).cuda(), 0.05)
    assert ei.value.code == sph.SPH_ERR_INVALID


def test_capacity_error_writes_nothing(sph):
    ps = W.c1_2d_10k(side=30)
    x = torch.from_numpy(ps.xyz).cuda()
    g = sph.Grid(x, ps.h, ps.kh)
    rp = torch.empty(ps.n + 1, dtype=torch.int64, device="cuda")
    nnz = sph.sph_nnps_query(g.handle, rp, None, 0)
    cap = nnz - 10
    buf = torch.full((nnz + 100,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SphError) as ei:
        sph.sph_nnps_query(g.handle, rp, buf, cap)
    assert ei.value.code == sph.SPH_ERR_CAPACITY
    assert torch.all(buf[cap:] == -7)  # nothing at or past the capacity
    # the same grid, queried again with room: succeeds (the flag was per query)
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    assert sph.sph_nnps_query(g.handle, rp, col, nnz) == nnz
    rp_ref, col_ref = oracle.cll(ps.xyz, ps.kh)
    # cell order -> input order
    orig = g.orig_id().cpu().numpy()
    crp, ccol = to_canonical(rp.cpu().numpy(), col.cpu().numpy(), orig)
    assert np.array_equal(crp, rp_ref) and np.array_equal(ccol, col_ref)


def test_unfused_density_matches(sph):
    for order in (0, 1):
        ps = W.c2_3d_1m(side=20)
        out = run(sph, ps.xyz, ps.h, ps.kh, order)
        g = out["grid"]
        rp = torch.from_numpy(out["rp"]).cuda()
        col = torch.from_numpy(out["col"]).cuda()
        rho2 = g.density(rp, col).cpu().numpy()
        rel = np.abs(rho2.astype(np.float64) - out["rho"]) / out["rho"]
        assert rel.max() <= 2e-6


def test_rebin_in_place(sph):
    a = W.c2_3d_1m(side=12)
    b = W.c2_3d_1m(side=18, seed=9)
    x = torch.from_numpy(a.xyz).cuda()
    g = sph.Grid(x, a.h, a.kh, order=1)
    g.query()
    g.rebin(torch.from_numpy(b.xyz).cuda())
    rp, col, rho = g.query()
    rp_ref, col_ref = oracle.cll(b.xyz, b.kh)
    assert np.array_equal(rp.cpu().numpy(), rp_ref) and np.array_equal(col.cpu().numpy(), col_ref)


def test_deterministic(sph):
    ps = W.c2_3d_1m(side=24)
    a = run(sph, ps.xyz, ps.h, ps.kh, 0)
    b = run(sph, ps.xyz, ps.h, ps.kh, 0)
    assert np.array_equal(a["rp"], b["rp"]) and np.array_equal(a["col"], b["col"])
    assert np.array_equal(a["rho"], b["rho"])
    assert np.array_equal(a["orig"], b["orig"])


@pytest.mark.parametrize("dim", [2, 3])
def test_unaligned_coordinates(sph, dim):
    """Coordinates at an address that is 8- but not 16-byte aligned (the
    bounds pass then reads value by value) give the same CSR."""
    ps = W.c1_2d_10k(side=37) if dim == 2 else W.c2_3d_1m(side=17)
    flat = torch.zeros(ps.n * dim + 1, dtype=torch.float64, device="cuda")
    flat[1:] = torch.from_numpy(ps.xyz.reshape(-1))
    x = flat[1:].view(ps.n, dim)
    assert x.data_ptr() % 16 == 8
    g = sph.Grid(x, ps.h, ps.kh, order=1)
    rp, col, rho = g.query()
    rp_ref, col_ref = oracle.cll(ps.xyz, ps.kh)
    assert np.array_equal(rp.cpu().numpy(), rp_ref) and np.array_equal(col.cpu().numpy(), col_ref)


@pytest.mark.parametrize("where", ["first", "last"])
def test_nonfinite_in_tail_rejected(sph, where):
    """A non-finite value in the last (scalar tail) or first coordinate."""
    xyz = W.random_uniform(101, 3, 2)  # 303 values: 50 six-value steps + a tail of 3
    if where == "last":
        xyz[100, 2] = np.inf
    else:
        xyz[0, 0] = -np.inf
    with pytest.raises(sph.SphError) as ei:
        sph.Grid(torch.from_numpy(xyz).cuda(), 0.05)
    assert ei.value.code == sph.SPH_ERR_INVALID


@pytest.mark.parametrize("shape,staging", [(0, 0), (1, 0), (0, 4096), (1, 2048)])
@pytest.mark.parametrize("case", ["c1_2d_10k", "lattice3d_27k", "dambreak_small", "random3d_dense", "lattice3d_wide"])
def test_tile_shapes_and_staging(sph, case, shape, staging):
    """Both shared-memory shapes of the tile search, with and without extra
    staging, give the oracle's lists and densities.  lattice3d_wide (kh =
    3.2 dx, ~130 neighbours per particle) gives tiles whose output is larger
    than the staging area, so it is staged and copied in several chunks."""
    if case == "random3d_dense":
        xyz, h = W.random_uniform(20000, 3, 21), 0.05  # ~110 neighbours per particle
    elif case == "lattice3d_wide":
        xyz, h = W.c2_3d_1m(side=24).xyz, 0.016
    else:
        xyz, h = CASES[case]()
    x = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
    g = sph.Grid(x, h, 2 * h, order=0)
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_TILE_SHAPE, shape)
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_STAGING, staging)
    rp, col, rho = g.query()
    out = dict(rp=rp.cpu().numpy(), col=col.cpu().numpy(), rho=rho.cpu().numpy(), orig=g.orig_id().cpu().numpy())
    check_against_oracle(out, xyz, h, 2 * h, 0)


@pytest.mark.parametrize("case", ["c1_2d_10k", "lattice3d_27k", "random3d_dense", "lattice3d_wide"])
def test_density_bits_independent_of_tile_shape(sph, case):
    """The two shared-memory shapes cut the kept candidates into windows of
    192 and 256 (and passes of 672 and 832) and batch the walk's bits
    differently; each row's Eq. 3 sum still adds its pairs in candidate order,
    one weight per pair computed the same way in every batch slot, so the
    densities agree bit for bit, and the lists are the same."""
    if case == "random3d_dense":
        xyz, h = W.random_uniform(20000, 3, 21), 0.05
    elif case == "lattice3d_wide":
        xyz, h = W.c2_3d_1m(side=24).xyz, 0.016
    else:
        xyz, h = CASES[case]()
    x = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
    res = []
    for shape in (0, 1):
        g = sph.Grid(x, h, 2 * h, order=0)
        sph.sph_grid_set_option(g.handle, sph.SPH_OPT_TILE_SHAPE, shape)
        rp, col, rho = g.query()
        res.append((rp.cpu().numpy(), col.cpu().numpy(), rho.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2])
    with pytest.raises(sph.SphError):
        sph.sph_grid_set_option(g.handle, sph.SPH_OPT_TILE_SHAPE, 2)


@pytest.mark.parametrize("dim,n,h", [(3, 200000, 0.0025), (2, 300000, 0.0001)])
def test_large_sparse_grid(sph, dim, n, h):
    """A sparse set over a fine grid (8M cells in 3D, 25M in 2D): the
    one-launch cell scan has more tiles of 4096 cells, and the one-launch
    tile-list builder more chunks of rows, than blocks, so blocks take several
    of them in ticket order."""
    xyz = W.random_uniform(n, dim, 31 + dim)
    out = run(sph, xyz, h, 2 * h, 0)
    info = out["info"]
    assert info.ncell > 152 * 4 * 4096
    check_against_oracle(out, xyz, h, 2 * h, 0)


@pytest.mark.parametrize("case", ["c1_2d_10k", "lattice3d_27k", "random3d", "faces3d", "dambreak_small"])
def test_density_half_stencil(sph, case):
    """The summation density over the half stencil (each pair tested once,
    no neighbour list) against the oracle's density and the search's."""
    xyz, h = CASES[case]()
    out = run(sph, xyz, h, 2 * h, 0)
    half = out["grid"].density_half().cpu().numpy().astype(np.float64)
    rp_ref, col_ref = oracle.cll(xyz, 2 * h)
    rho_ref = oracle.density(xyz, h, rp_ref, col_ref)
    r = np.empty_like(rho_ref)
    r[out["orig"]] = half
    assert (np.abs(r - rho_ref) / rho_ref).max() <= RHO_RTOL
    assert (np.abs(half - out["rho"]) / out["rho"]).max() <= 2e-6


@pytest.mark.parametrize("dim,khr", [(2, 2.4), (2, 4.0), (3, 2.6), (3, 3.6), (3, 4.6)])
def test_canonical_row_lengths(sph, dim, khr):
    """Canonical order sorts each row's input-order columns: rows of about
    20, 50, 80, 190 and 400 neighbours exercise the one-register, 64-, 128-
    and 256-key register networks and the shared-memory network."""
    side = 60 if dim == 2 else 16
    dx = 1.0 / side
    xyz = W.lattice((side,) * dim, dx, 0.1, seed=31 + int(10 * khr))
    h = 0.5 * khr * dx
    out = run(sph, xyz, h, 2 * h, 1)
    check_against_oracle(out, xyz, h, 2 * h, 1)
    lens = np.diff(out["rp"])
    assert lens.max() > {2.4: 16, 4.0: 40, 2.6: 64, 3.6: 128, 4.6: 256}[khr]


@pytest.mark.parametrize("case", ["c1_2d_10k", "lattice3d_27k", "random3d", "faces3d", "dambreak_small", "two"])
def test_half_stencil_csr(sph, case):
    """sph_nnps_query_half (each pair decided once, written into both rows,
    rows sorted) gives the tile search's CSR exactly and the oracle's density
    within the tolerance; its count-only call gives the same row pointers;
    a short capacity is refused with nothing written."""
    xyz, h = CASES[case]()
    out = run(sph, xyz, h, 2 * h, 0)
    g = out["grid"]
    n = xyz.shape[0]
    nnz = int(out["rp"][-1])
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    assert sph.sph_nnps_query_half(g.handle, rp) == nnz
    assert np.array_equal(rp.cpu().numpy(), out["rp"])
    col = torch.full((nnz + 64,), -7, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    assert sph.sph_nnps_query_half(g.handle, rp, col, col.numel(), rho) == nnz
    assert np.array_equal(rp.cpu().numpy(), out["rp"])
    assert np.array_equal(col[:nnz].cpu().numpy(), out["col"])
    half = dict(out, rho=rho.cpu().numpy())
    check_against_oracle(half, xyz, h, 2 * h, 0)
    if nnz > 0:
        col2 = torch.full((nnz,), -7, dtype=torch.int32, device="cuda")
        with pytest.raises(sph.SphError) as ei:
            sph.sph_nnps_query_half(g.handle, rp, col2, nnz - 1)
        assert ei.value.code == sph.SPH_ERR_CAPACITY
        assert np.all(col2.cpu().numpy() == -7)


@pytest.mark.parametrize("share", [100, 40, 1])
def test_sm_share_same_result(sph, share):
    """SPH_OPT_SM_SHARE only sizes the persistent grid: the CSR and the
    density bits are those of the full grid, down to one CTA."""
    xyz, h = CASES["lattice3d_27k"]()
    full = run(sph, xyz, h, 2 * h, 0)
    x = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
    g = sph.Grid(x, h, 2 * h)
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_SM_SHARE, share)
    rp, col, rho = g.query(density=True)
    assert np.array_equal(rp.cpu().numpy(), full["rp"])
    assert np.array_equal(col.cpu().numpy(), full["col"])
    assert np.array_equal(rho.cpu().numpy(), full["rho"])
    with pytest.raises(sph.SphError):
        sph.sph_grid_set_option(g.handle, sph.SPH_OPT_SM_SHARE, 0)


def test_search_host_async_matches_sync(sph):
    """sph_search_host_async / _finish on two grids and two streams give the
    synchronous call's density, nnz and CSR; a set whose neighbours outgrow
    the grid's column buffer is reported by _finish as SPH_ERR_CAPACITY and
    the synchronous call then grows the buffer."""
    xyz, h = CASES["lattice3d_27k"]()
    n = xyz.shape[0]
    params = sph.make_params(3, h, 2 * h, order=sph.SPH_ORDER_CELL)
    xh = torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory()
    rho_ref = torch.empty(n, dtype=torch.float32).pin_memory()
    g_ref, nnz_ref = sph.sph_search_host(params, xh, n, rho_ref, None, None)
    rp_ref = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    col_ref = torch.empty(nnz_ref, dtype=torch.int32).pin_memory()
    sph.sph_grid_csr_copy(g_ref, rp_ref, col_ref)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    rhos = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    gs = [None, None]
    for rnd in range(3):
        for b in range(2):
            gs[b] = sph.sph_search_host_async(params, xh, n, rhos[b], streams[b].cuda_stream, gs[b])
        for b in range(2):
            assert sph.sph_search_host_finish(gs[b]) == nnz_ref
            assert torch.equal(rhos[b], rho_ref)
            rp = torch.empty(n + 1, dtype=torch.int64).pin_memory()
            col = torch.empty(nnz_ref, dtype=torch.int32).pin_memory()
            sph.sph_grid_csr_copy(gs[b], rp, col)
            assert torch.equal(rp, rp_ref) and torch.equal(col, col_ref)
    # a denser set of the same size: the grid's column buffer is too small
    dense = sph.make_params(3, 1.6 * h, 3.2 * h, order=sph.SPH_ORDER_CELL)
    sph.sph_search_host_async(dense, xh, n, rhos[0], streams[0].cuda_stream, gs[0])
    with pytest.raises(sph.SphError) as ei:
        sph.sph_search_host_finish(gs[0])
    assert ei.value.code == sph.SPH_ERR_CAPACITY
    _, nnz_dense = sph.sph_search_host(dense, xh, n, rhos[0], None, gs[0])
    rp_o, col_o = oracle.cll(xyz, 3.2 * h)
    assert nnz_dense == col_o.size
    for g in gs + [g_ref]:
        sph.sph_grid_free(g)
