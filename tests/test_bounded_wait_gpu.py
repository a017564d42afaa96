"""The look-back wait of the single-pass search is bounded: a wait that runs
out records a timeout status and returns instead of hanging.  The test makes
the wait run out on purpose, through the test-only grid option
SPH_OPT_TEST_LOOKBACK: the search leaves its first tile out, so every later
tile waits on a predecessor that never publishes, for 1,024 polls.  Checked:
the query reports SPH_ERR_TIMEOUT (and sph_grid_check does), it ends in well
under a second, nothing is written at or past col_capacity, and the next
normal query on the same grid is exact again.  GPU required."""
import time

import numpy as np
import pytest

import oracle
from paper_2401_08586_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 4096
SENTINEL = -7


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


@pytest.mark.parametrize("dim", [2, 3])
def test_lookback_wait_times_out_and_recovers(sph, dim):
    ps = W.c2_3d_1m(side=30) if dim == 3 else W.c1_2d_10k()
    g = sph.Grid(torch.from_numpy(ps.xyz).cuda(), ps.h, ps.kh)
    rp_ref, col_ref, rho_ref = g.query(density=True)
    nnz = int(rp_ref[-1].item())
    n = g.n

    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.full((nnz + GUARD,), SENTINEL, dtype=torch.int32, device="cuda")
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_TEST_LOOKBACK, 1024)
    t0 = time.perf_counter()
    with pytest.raises(sph.SphError) as ei:
        sph.sph_nnps_query(g.handle, rp, col, nnz, True, rho)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    assert ei.value.code == sph.SPH_ERR_TIMEOUT, str(ei.value)
    with pytest.raises(sph.SphError) as ei:
        sph.sph_grid_check(g.handle)
    assert ei.value.code == sph.SPH_ERR_TIMEOUT
    assert elapsed < 1.0, elapsed
    # nothing at or past the capacity
    tail = col[nnz:].cpu().numpy()
    assert np.all(tail == SENTINEL)

    # back to normal: the same grid gives the exact result again
    sph.sph_grid_set_option(g.handle, sph.SPH_OPT_TEST_LOOKBACK, 0)
    rp2, col2, rho2 = g.query(density=True)
    assert sph.sph_grid_check(g.handle) == 0
    assert torch.equal(rp2, rp_ref) and torch.equal(col2, col_ref) and torch.equal(rho2, rho_ref)
    # and it is the oracle's neighbour set (cell order -> input order)
    orig = g.orig_id().cpu().numpy()
    rp_o, col_o = oracle.cll(ps.xyz, ps.kh)
    r = np.diff(rp2.cpu().numpy())
    assert np.array_equal(r, np.diff(rp_o)[orig])
    g.close()
