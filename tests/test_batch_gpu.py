"""Batched runs (sph_batch_run): every system of a batch against the oracle,
against a single-system run of the same system, and the workspace's CUDA
graph replay and staging tuning (GPU required)."""
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


def mixed_systems(sph, dim=3, seed=0):
    """Uneven sizes (including empty and one-particle systems), different
    h / kh / mass, one with a caller box."""
    rng = np.random.default_rng(seed)
    out = []
    sizes = [0, 1, 2, 37, 500, 2100, 4000, 6859 if dim == 3 else 4900, 900, 3]
    for k, n in enumerate(sizes):
        dx = rng.uniform(0.005, 0.02)
        hr = rng.uniform(1.2, 1.5)
        if k % 3 == 0 and n > 10:
            xyz = W.random_uniform(n, dim, seed + k, extent=dx * n ** (1.0 / dim))
        else:
            side = int(np.ceil(n ** (1.0 / dim))) if n > 0 else 1
            xyz = W.lattice((side,) * dim, dx, 0.0, count=n) if n > 0 else np.zeros((0, dim))
            xyz = xyz + rng.uniform(-0.1 * dx, 0.1 * dx, size=xyz.shape)
        box = None
        if k == 4:
            box = (tuple(xyz.min(0) - 0.5 * dx), tuple(xyz.max(0) + 0.7 * dx))
        p = sph.make_params(dim, hr * dx, 2 * hr * dx, order=sph.SPH_ORDER_CELL, mass=1.0 + 0.25 * k, box=box)
        out.append((np.ascontiguousarray(xyz, dtype=np.float64), p))
    return out


def per_system(rp, col, rho, orig, first, s):
    """System s's CSR in its own input order, and its densities."""
    a, b = first[s], first[s + 1]
    n = b - a
    rp = rp.cpu().numpy()
    col = col.cpu().numpy()
    orig = orig.cpu().numpy()
    lens = np.diff(rp[a:b + 1])
    rows_in = orig[a:b]
    new_len = np.empty(n, dtype=np.int64)
    new_len[rows_in] = lens
    new_rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(new_len, out=new_rp[1:])
    new_col = np.empty(int(new_rp[-1]), dtype=np.int32)
    for r in range(n):
        seg = col[rp[a + r]:rp[a + r + 1]]
        assert np.all((seg >= a) & (seg < b)), "column outside the system"
        assert np.all(np.diff(seg) > 0)
        i = rows_in[r]
        new_col[new_rp[i]:new_rp[i + 1]] = np.sort(orig[seg])
    r2 = None
    if rho is not None:
        r2 = np.empty(n)
        r2[rows_in] = rho.cpu().numpy()[a:b]
    return new_rp, new_col, r2


def check_batch(sph, systems, res):
    rp, col, rho, orig, first = res
    for s, (xyz, p) in enumerate(systems):
        grp, gcol, grho = per_system(rp, col, rho, orig, first, s)
        rp_ref, col_ref = oracle.cll(xyz, p.kh)
        assert np.array_equal(grp, rp_ref), "system %d row_ptr" % s
        assert np.array_equal(gcol, col_ref), "system %d col" % s
        if xyz.shape[0]:
            rho_ref = oracle.density(xyz, p.h, rp_ref, col_ref, mass=p.mass)
            assert (np.abs(grho - rho_ref) / rho_ref).max() <= RHO_RTOL, "system %d rho" % s


def run(sph, systems, batch=None, **kw):
    b = batch or sph.Batch()
    res = b.run([(torch.from_numpy(x).cuda(), p) for x, p in systems], **kw)
    torch.cuda.synchronize()
    return b, res


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_matches_oracle(sph, dim):
    systems = mixed_systems(sph, dim, seed=dim)
    b, res = run(sph, systems)
    check_batch(sph, systems, res)
    b.close()


def test_batch_equals_single_system_runs(sph):
    """Each system's rows, columns (shifted by its first position) and
    densities are bit-identical to a single-system cell-order query."""
    systems = mixed_systems(sph, 3, seed=7)
    b, (rp, col, rho, orig, first) = run(sph, systems)
    for s, (xyz, p) in enumerate(systems):
        if xyz.shape[0] == 0:
            continue
        g = sph.Grid(torch.from_numpy(xyz).cuda(), p.h, p.kh, order=0, mass=p.mass,
                     box=(tuple(p.box_lo[:3]), tuple(p.box_hi[:3])) if p.have_box else None)
        grp, gcol, grho = g.query()
        a, e = first[s], first[s + 1]
        assert torch.equal(rp[a:e + 1] - rp[a], grp)
        assert torch.equal(col[rp[a]:rp[e]] - a, gcol)
        assert torch.equal(rho[a:e], grho)
        assert torch.equal(orig[a:e], g.orig_id())
        g.close()
    b.close()


def test_graph_replay_and_tuning(sph):
    systems = mixed_systems(sph, 3, seed=11)
    b = sph.Batch()
    _, r1 = run(sph, systems, b)  # count-only run, then the tuned run
    r1 = [t.clone() if isinstance(t, torch.Tensor) else t for t in r1]
    st = b.stats()
    assert st.tuned_candidates == 5 and st.tuned_staging in (0, 2048, 4096) and st.tuned_shape in (0, 1)
    captures = st.graph_captures
    assert captures == 2  # one per distinct launch sequence (count-only, full)
    launches = sph.sph_launch_count()
    _, r2 = run(sph, systems, b)
    _, r3 = run(sph, systems, b)
    st = b.stats()
    assert st.graph_replays == 2 and st.graph_captures == captures
    assert sph.sph_launch_count() > launches  # replayed kernels are counted
    # a replayed run is one graph launch (binning, tile list, counter reset and
    # the persistent search) plus five small kernels outside it: the status
    # reset and the bounds before it, the bounds' and the result's read-backs
    assert st.graph_launched == 1 and st.direct_launches <= 5
    for a, c in zip(r1[:4], r3[:4]):
        assert torch.equal(a, c)
    check_batch(sph, systems, r3)
    b.close()


@pytest.mark.parametrize("staging", [0, 4096, 16384])
def test_fixed_staging_same_result(sph, staging):
    systems = mixed_systems(sph, 3, seed=5)
    b0, r0 = run(sph, systems)
    b = sph.Batch()
    b.set_option(sph.SPH_BATCH_OPT_STAGING, staging)
    b.set_option(sph.SPH_BATCH_OPT_GRAPH, 0)
    _, r = run(sph, systems, b)
    for x, y in zip(r0[:4], r[:4]):
        assert torch.equal(x, y)
    assert b.stats().graph_captures == 0
    b.close()
    b0.close()


def test_batched_uneven_workload_sample(sph):
    """Systems drawn like the batched workload (log-uniform sizes, random
    spacing and h/dx), fewer and smaller so the oracle stays quick."""
    systems = [(ps.xyz, sph.make_params(3, ps.h, ps.kh, order=sph.SPH_ORDER_CELL))
               for ps in W.c4_batched(seed=4, nsys=24, nmin=200, nmax=20000)]
    b, res = run(sph, systems)
    check_batch(sph, systems, res)
    b.close()


def test_capacity_and_invalid(sph):
    systems = mixed_systems(sph, 3, seed=3)
    b, (rp, col, rho, orig, first) = run(sph, systems)
    nnz = int(rp[-1])
    xs = [torch.from_numpy(x).cuda() for x, _ in systems]
    ps = [p for _, p in systems]
    buf = torch.full((nnz + 64,), -7, dtype=torch.int32, device="cuda")
    rp2 = torch.empty_like(rp)
    cap = nnz - 5
    out = sph.sph_batch_out(rp2.data_ptr(), buf.data_ptr(), cap, None, None, None, 0)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_batch_run(b.handle, ps, xs, out)
    assert ei.value.code == sph.SPH_ERR_CAPACITY and out.nnz == nnz
    assert torch.all(buf[cap:] == -7)
    # mixed dimensions
    p2 = sph.make_params(2, 0.01, 0.02, order=sph.SPH_ORDER_CELL)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_batch_run(b.handle, ps[:2] + [p2], xs[:2] + [torch.zeros(5, 2, dtype=torch.float64, device="cuda")],
                          out)
    assert ei.value.code == sph.SPH_ERR_INVALID
    # non-finite coordinate
    bad = xs[5].clone()
    bad[3, 1] = float("nan")
    with pytest.raises(sph.SphError) as ei:
        sph.sph_batch_run(b.handle, ps, xs[:5] + [bad] + xs[6:], out)
    assert ei.value.code == sph.SPH_ERR_INVALID
    # the workspace still works afterwards
    _, res = run(sph, systems, b)
    check_batch(sph, systems, res)
    b.close()
