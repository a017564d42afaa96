"""sph_nnps_query_static: the neighbour search for callers that cannot allocate
device memory when they call it (for example a process whose device memory is
all reserved up front by its own allocator or budget, or a latency-critical
loop that cannot pay for an allocation).  The entry point keeps its working
memory in a fixed array inside the library instead of allocating.

Checked here through the C ABI: on two calls in a row, and after a call on
another grid (the shared array keeps the previous call's contents), it gives
the same CSR and density as sph_nnps_query on the same grid; sizes above its
limit are refused with a clear error.  At its limits: a set of about 2^20
particles with more than 16,384 rows of cells (the multi-block row scan inside
the fixed array), a col_capacity below nnz (SPH_ERR_CAPACITY from the next
sph_grid_check, nothing written past the capacity), and a grid of more than
65,536 rows (refused).  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

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


def regular(sph, g):
    """Reference result from the allocating entry point sph_nnps_query."""
    rp, col, rho = g.query(density=True)
    torch.cuda.synchronize()
    return rp.cpu().numpy(), col.cpu().numpy(), rho.cpu().numpy()


def static_call(sph, g, cap):
    n = g.n
    rp = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    col = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    rho = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    sph.sph_nnps_query_static(g.handle, rp, col, cap, rho)
    torch.cuda.synchronize()
    assert sph.sph_grid_check(g.handle) == 0
    rp = rp.cpu().numpy()
    return rp, col.cpu().numpy()[:rp[-1]], rho.cpu().numpy()


def same(a, b):
    assert np.array_equal(a[0], b[0]), "row_ptr differs"
    assert np.array_equal(a[1], b[1]), "col differs"
    rel = np.abs(a[2].astype(np.float64) - b[2]) / np.abs(b[2])
    assert rel.max() <= RHO_RTOL, rel.max()


def test_static_query_matches_regular_query(sph):
    a = W.c2_3d_1m(side=40)                  # 64,000 particles, 3D
    b = W.c1_2d_10k()                        # 10,000 particles, 2D
    ga = sph.Grid(torch.from_numpy(a.xyz).cuda(), a.h, a.kh)
    gb = sph.Grid(torch.from_numpy(b.xyz).cuda(), b.h, b.kh)
    ref_a, ref_b = regular(sph, ga), regular(sph, gb)
    cap_a, cap_b = int(ref_a[0][-1]) + 64, int(ref_b[0][-1]) + 64
    # two calls in a row on the same grid
    same(static_call(sph, ga, cap_a), ref_a)
    same(static_call(sph, ga, cap_a), ref_a)
    # another grid in between: the array's leftover contents must not matter
    same(static_call(sph, gb, cap_b), ref_b)
    same(static_call(sph, ga, cap_a), ref_a)
    ga.close()
    gb.close()


def test_static_query_refuses_oversized_grids(sph):
    ps = W.c2_3d_1m(side=102)                # 1,061,208 particles > 2^20
    g = sph.Grid(torch.from_numpy(ps.xyz).cuda(), ps.h, ps.kh)
    rp = torch.empty(ps.n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SphError) as ei:
        sph.sph_nnps_query_static(g.handle, rp, col, 16)
    assert ei.value.code == sph.SPH_ERR_INVALID
    assert "1048576" in str(ei.value)
    g.close()
    # a canonical-order grid is refused too
    small = W.c2_3d_1m(side=10)
    g = sph.Grid(torch.from_numpy(small.xyz).cuda(), small.h, small.kh, order=sph.SPH_ORDER_CANONICAL)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_nnps_query_static(g.handle, rp, col, 16)
    assert ei.value.code == sph.SPH_ERR_INVALID
    g.close()


def test_static_query_dense_set(sph):
    """A lattice with ~140 neighbours per particle: the grid's tile choice is
    the dense shape, which the no-allocation call takes over."""
    xyz = W.lattice((36, 36, 36), 1.0 / 36, 0.1, seed=17)
    h = 1.6 / 36
    g = sph.Grid(torch.from_numpy(xyz).cuda(), h, 2 * h)
    ref = regular(sph, g)
    assert ref[0][-1] / g.n > 110
    cap = int(ref[0][-1])
    same(static_call(sph, g, cap), ref)
    same(static_call(sph, g, cap), ref)
    g.close()


def thin_slab(n, seed):
    """Uniform random particles in a 0.05 x 1.5 x 1.5 slab: with kh = 0.01 the
    grid has 5 x 150 x 150 cells, i.e. 22,500 rows of cells."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n, 3)) * np.array([0.05, 1.5, 1.5])


def test_static_query_near_its_limits(sph):
    n = (1 << 20) - 7
    xyz = thin_slab(n, 21)
    g = sph.Grid(torch.from_numpy(xyz).cuda(), 0.005, 0.01)
    info = g.info()
    assert int(info.nk[1]) * int(info.nk[2]) > 16384
    ref = regular(sph, g)
    cap = int(ref[0][-1])
    same(static_call(sph, g, cap), ref)
    same(static_call(sph, g, cap), ref)
    g.close()


def test_static_query_capacity_below_nnz(sph):
    ps = W.c2_3d_1m(side=30)
    g = sph.Grid(torch.from_numpy(ps.xyz).cuda(), ps.h, ps.kh)
    ref = regular(sph, g)
    nnz = int(ref[0][-1])
    cap = nnz // 2
    rp = torch.empty(g.n + 1, dtype=torch.int64, device="cuda")
    col = torch.full((nnz + 1024,), -7, dtype=torch.int32, device="cuda")
    sph.sph_nnps_query_static(g.handle, rp, col, cap)
    torch.cuda.synchronize()
    with pytest.raises(sph.SphError) as ei:
        sph.sph_grid_check(g.handle)
    assert ei.value.code == sph.SPH_ERR_CAPACITY
    assert np.all(col[cap:].cpu().numpy() == -7)
    # row pointers are complete even when the columns do not fit
    assert np.array_equal(rp.cpu().numpy(), ref[0])
    # and a call with enough room afterwards is exact
    same(static_call(sph, g, nnz), ref)
    g.close()


def test_static_query_refuses_too_many_rows(sph):
    rng = np.random.default_rng(5)
    xyz = rng.uniform(0.0, 1.0, size=(20000, 3)) * np.array([0.05, 2.6, 2.6])  # 260 x 260 rows of cells
    g = sph.Grid(torch.from_numpy(xyz).cuda(), 0.005, 0.01)
    info = g.info()
    assert int(info.nk[1]) * int(info.nk[2]) > 65536
    rp = torch.empty(g.n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(sph.SphError) as ei:
        sph.sph_nnps_query_static(g.handle, rp, col, 16)
    assert ei.value.code == sph.SPH_ERR_INVALID
    assert "65536" in str(ei.value)
    g.close()
