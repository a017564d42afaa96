"""Parity at the full workload sizes, in the configuration the benchmark
times (cell order, single-pass tile search with fused density).

3D 1M jittered lattice: the whole CSR and every density against the oracle.
3D 8M dam-break (block + 5% spray): every row length against the oracle's
row pointer, the full rows and densities of a seeded sample of particles,
and the symmetry of the whole neighbour relation (i in N(j) iff j in N(i)).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2401_08586_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO_RTOL = 1e-5
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


def bench_query(sph, ps):
    """Bin and query exactly as the benchmark step does (capacity from a
    count-only query first)."""
    x = torch.from_numpy(ps.xyz).cuda()
    params = sph.make_params(ps.dim, ps.h, ps.kh, order=sph.SPH_ORDER_CELL)
    g = sph.sph_bin_cells(params, x, ps.n, None, None)
    rp = torch.empty(ps.n + 1, dtype=torch.int64, device="cuda")
    nnz = sph.sph_nnps_query(g, rp, None, 0, True, None, None)
    col = torch.empty(nnz + 1024, dtype=torch.int32, device="cuda")
    rho = torch.empty(ps.n, dtype=torch.float32, device="cuda")
    nnz2 = sph.sph_nnps_query(g, rp, col, col.numel(), True, rho, None)
    assert nnz2 == nnz
    orig = torch.empty(ps.n, dtype=torch.int32, device="cuda")
    rank = torch.empty(ps.n, dtype=torch.int32, device="cuda")
    sph.sph_grid_export(g, orig, rank, None, None)
    torch.cuda.synchronize()
    return g, x, rp, col[:nnz], rho, orig.long(), rank.long()


def input_order_counts(rp, orig, n):
    cnt = torch.empty(n, dtype=torch.int64, device=rp.device)
    cnt[orig] = rp[1:] - rp[:-1]
    return cnt


def rows_in_input_ids(rp, col, orig, rank, rows):
    """Neighbour lists of input particles `rows`, as sorted input indices."""
    out = []
    for i in rows:
        r = int(rank[i])
        seg = orig[col[int(rp[r]):int(rp[r + 1])].long()]
        out.append(np.sort(seg.cpu().numpy()))
    return out


def symmetric(rp, col, n):
    """i in N(j) iff j in N(i), checked as equal multisets of (row, col)
    pairs and their transposes under a random 64-bit mixing hash."""
    rows = torch.repeat_interleave(torch.arange(n, device=rp.device), rp[1:] - rp[:-1])
    c = col.long()

    def mix(a, b):  # int64 arithmetic wraps; the constants are 64-bit odd multipliers
        v = a * (-7046029254386353131) + b * (-4417276706812531889)
        v = v ^ (v >> 29)
        return v * (1609587929392839161)

    return bool(torch.equal(torch.sort(mix(rows, c)).values, torch.sort(mix(c, rows)).values))


def test_full_csr_and_density_3d_1m(sph):
    ps = W.c2_3d_1m()
    g, x, rp, col, rho, orig, rank = bench_query(sph, ps)
    rp_ref, col_ref = oracle.cll(ps.xyz, ps.kh, threads=THREADS)
    # rows to input order
    cnt = input_order_counts(rp, orig, ps.n).cpu().numpy()
    assert np.array_equal(np.diff(rp_ref), cnt)
    # columns: map to input ids, sort within rows (rows in input order)
    n = ps.n
    rows_sorted = torch.repeat_interleave(torch.arange(n, device="cuda"), rp[1:] - rp[:-1])
    key = orig[rows_sorted] * n + orig[col.long()]
    key = torch.sort(key).values
    assert np.array_equal((key % n).to(torch.int32).cpu().numpy(), col_ref)
    rho_ref = oracle.density(ps.xyz, ps.h, rp_ref, col_ref, threads=THREADS)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    r[orig] = rho.double()
    rel = np.abs(r.cpu().numpy() - rho_ref) / rho_ref
    assert rel.max() <= RHO_RTOL
    sph.sph_grid_free(g)


def test_sampled_rows_counts_symmetry_3d_8m(sph):
    ps = W.c3_3d_dambreak()
    g, x, rp, col, rho, orig, rank = bench_query(sph, ps)
    n = ps.n
    rp_ref = oracle.cll_counts(ps.xyz, ps.kh, threads=THREADS)
    cnt = input_order_counts(rp, orig, n).cpu().numpy()
    assert np.array_equal(np.diff(rp_ref), cnt)
    # a seeded sample: uniform over all particles plus the spray (z > 1)
    rng = np.random.default_rng(88)
    spray = np.nonzero(ps.xyz[:, 2] > 1.0)[0]
    rows = np.concatenate([rng.choice(n, 3000, replace=False), rng.choice(spray, 1000, replace=False)])
    srp, scol = oracle.cll_rows(ps.xyz, ps.kh, rows, threads=THREADS)
    got = rows_in_input_ids(rp, col, orig, rank, rows)
    for k in range(rows.size):
        assert np.array_equal(got[k], scol[srp[k]:srp[k + 1]]), "row of particle %d differs" % rows[k]
    srho = oracle.density_rows(ps.xyz, ps.h, rows, srp, scol)
    grho = rho[rank[torch.from_numpy(rows).cuda()]].double().cpu().numpy()
    assert (np.abs(grho - srho) / srho).max() <= RHO_RTOL
    assert symmetric(rp, col, n)
    sph.sph_grid_free(g)
