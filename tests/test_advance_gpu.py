"""Time step of Eq. 8-9 (sph_advance): after each step the neighbour lists
and densities are those of the FP64 oracle on the updated positions (GPU
required)."""
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


def canonical(rp, col, orig):
    rp, col, orig = rp.cpu().numpy(), col.cpu().numpy(), orig.cpu().numpy()
    n = rp.size - 1
    lens = np.diff(rp)
    new_len = np.empty(n, dtype=np.int64)
    new_len[orig] = lens
    new_rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(new_len, out=new_rp[1:])
    new_col = np.empty(int(new_rp[-1]), dtype=np.int32)
    for r in range(n):
        i = orig[r]
        new_col[new_rp[i]:new_rp[i + 1]] = np.sort(orig[col[rp[r]:rp[r + 1]]])
    return new_rp, new_col


def check(g, x, h):
    rp, col, rho = g.query()
    orig = g.orig_id()
    crp, ccol = canonical(rp, col, orig)
    rp_ref, col_ref = oracle.cll(x, 2 * h)
    assert np.array_equal(crp, rp_ref) and np.array_equal(ccol, col_ref)
    r = np.empty(x.shape[0])
    r[orig.cpu().numpy()] = rho.cpu().numpy()
    rho_ref = oracle.density(x, h, rp_ref, col_ref)
    assert (np.abs(r - rho_ref) / rho_ref).max() <= RHO_RTOL


def swirl(x, speed, rng):
    """A smooth rotating field plus noise (particles cross cell faces in
    every direction)."""
    c = x.mean(0)
    v = np.zeros_like(x)
    v[:, 0] = -(x[:, 1] - c[1])
    v[:, 1] = x[:, 0] - c[0]
    v = speed * v / (np.abs(v).max() + 1e-30)
    return v + rng.uniform(-0.5 * speed, 0.5 * speed, size=x.shape)


@pytest.mark.parametrize("dim", [2, 3])
def test_steps_match_oracle(sph, dim):
    ps = W.c2_3d_1m(side=28) if dim == 3 else W.c1_2d_10k(side=90)
    rng = np.random.default_rng(dim)
    x = ps.xyz.copy()
    g = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=0)
    dt = 1.0
    for step in range(12):
        v = swirl(x, 0.3 * ps.dx, rng)
        x_new = x + v * dt
        g.advance(torch.from_numpy(x_new).cuda(), torch.from_numpy(v).cuda(), dt)
        x = x_new
        if step % 3 == 2:
            check(g, x, ps.h)
    check(g, x, ps.h)
    g.close()


def test_fast_motion_and_leaving_the_box(sph):
    """Displacements of several cells per step, and particles that leave
    the grid's box (the grid is then binned again)."""
    ps = W.c2_3d_1m(side=20)
    rng = np.random.default_rng(7)
    x = ps.xyz.copy()
    g = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=0)
    for step in range(4):
        v = rng.uniform(-2.5 * ps.kh, 2.5 * ps.kh, size=x.shape)
        x_new = x + v
        g.advance(torch.from_numpy(x_new).cuda(), torch.from_numpy(v).cuda(), 1.0)
        x = x_new
        check(g, x, ps.h)
    g.close()


def test_same_lists_as_fresh_binning(sph):
    ps = W.c2_3d_1m(side=24)
    rng = np.random.default_rng(3)
    x = ps.xyz.copy()
    g = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=1)
    for step in range(30):
        v = swirl(x, 0.2 * ps.dx, rng)
        x = x + v
        g.advance(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), 1.0)
    rp, col, rho = g.query()
    f = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=1)
    rp2, col2, rho2 = f.query()
    assert torch.equal(rp, rp2) and torch.equal(col, col2)
    assert ((rho - rho2).abs() / rho2).max().item() <= 2e-6
    g.close()
    f.close()


def test_box_and_nonfinite(sph):
    ps = W.c2_3d_1m(side=12)
    x = ps.xyz
    box = (tuple(x.min(0) - 0.01), tuple(x.max(0) + 0.01))
    g = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=0, box=box)
    v = np.zeros_like(x)
    v[0, 0] = -1.0  # far outside the caller's box
    with pytest.raises(sph.SphError) as ei:
        g.advance(torch.from_numpy(x + v).cuda(), torch.from_numpy(v).cuda(), 1.0)
    assert ei.value.code == sph.SPH_ERR_INVALID
    g2 = sph.Grid(torch.from_numpy(x).cuda(), ps.h, ps.kh, order=0)
    v = np.zeros_like(x)
    v[3, 1] = np.nan
    with pytest.raises(sph.SphError) as ei:
        g2.advance(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), 1.0)
    assert ei.value.code == sph.SPH_ERR_INVALID
    g.close()
    g2.close()
