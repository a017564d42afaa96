"""Request server (sph_server_*): results against the oracle, continuous
batching, failure isolation, the memory budget and small-behind-large
latency (GPU required)."""
import time

import numpy as np
import pytest

import oracle
from paper_2401_08586_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO_RTOL = 1e-5
GB = 1 << 30


@pytest.fixture(scope="module")
def sph():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_08586_gb300 import sph as _sph
    _sph.load()
    return _sph


def lattice_system(n, dim, seed, hr=1.3):
    side = int(np.ceil(n ** (1.0 / dim)))
    dx = 1.0 / side
    rng = np.random.default_rng(seed)
    xyz = W.lattice((side,) * dim, dx, 0.0, count=n)
    xyz = xyz + rng.uniform(-0.1 * dx, 0.1 * dx, size=xyz.shape)
    return np.ascontiguousarray(xyz), hr * dx


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


def check(server, t, xyz, h, order):
    rp, col, rho, orig = server.fetch(t)
    rp_ref, col_ref = oracle.cll(xyz, 2 * h)
    if order == 0:
        crp, ccol = canonical(rp, col, orig)
        r = np.empty(xyz.shape[0])
        r[orig.cpu().numpy()] = rho.cpu().numpy()
    else:
        crp, ccol = rp.cpu().numpy(), col.cpu().numpy()
        r = rho.cpu().numpy()
    assert np.array_equal(crp, rp_ref) and np.array_equal(ccol, col_ref)
    rho_ref = oracle.density(xyz, h, rp_ref, col_ref)
    assert (np.abs(r - rho_ref) / rho_ref).max() <= RHO_RTOL


def test_mixed_requests_match_oracle(sph):
    srv = sph.Server(8 * GB, streams=2)
    cases = []
    for k, (n, dim, order, dev) in enumerate([(20000, 3, 0, False), (3000, 2, 0, True), (50000, 3, 1, False),
                                              (700, 3, 0, False), (12000, 2, 1, True), (1, 3, 0, False)]):
        xyz, h = lattice_system(n, dim, k)
        p = sph.make_params(dim, h, 2 * h, order=order)
        t = srv.submit(torch.from_numpy(xyz).cuda() if dev else xyz, p)
        cases.append((t, xyz, h, order))
    for t, xyz, h, order in cases:
        res = srv.wait(t)
        assert res.status == sph.SPH_OK
        assert res.t_submit_ns <= res.t_admit_ns <= res.t_done_ns
        check(srv, t, xyz, h, order)
        srv.release(t)
    st = srv.stats()
    assert st.completed == len(cases) and st.failed == 0 and st.held_bytes == 0
    srv.close()


def test_continuous_batching_and_isolation(sph):
    """Many small requests submitted at once run in batches; a request with a
    non-finite coordinate fails alone."""
    srv = sph.Server(8 * GB, streams=1, small_n=5000)
    big, hb = lattice_system(1_000_000, 3, 99)
    smalls = []
    for k in range(24):
        xyz, h = lattice_system(int(200 + 150 * k), 3 if k % 4 else 2, 100 + k)
        if k == 9:
            xyz = xyz.copy()
            xyz[5, 0] = np.nan
        smalls.append((xyz, h, k == 9))
    # occupy the worker so that the small requests queue up behind it
    tb = srv.submit(big, sph.make_params(3, hb, 2 * hb, order=0))
    items = [(srv.submit(x, sph.make_params(x.shape[1], h, 2 * h, order=0)), x, h, bad) for x, h, bad in smalls]
    assert srv.wait(tb).status == sph.SPH_OK
    for t, xyz, h, bad in items:
        res = srv.wait(t)
        if bad:
            assert res.status == sph.SPH_ERR_INVALID
            with pytest.raises(sph.SphError):
                srv.fetch(t)
        else:
            assert res.status == sph.SPH_OK
            check(srv, t, xyz, h, 0)
        srv.release(t)
    st = srv.stats()
    assert st.batches >= 1 and st.batched_requests >= 2
    assert st.failed == 1
    srv.release(tb)
    srv.close()


def test_budget(sph):
    srv = sph.Server(200 << 20, streams=2)
    xyz, h = lattice_system(2_000_000, 3, 1)
    with pytest.raises(sph.SphError) as ei:
        srv.submit(xyz, sph.make_params(3, h, 2 * h))
    assert ei.value.code == sph.SPH_ERR_BUDGET
    # requests that fit one or two at a time: the reserved bytes stay within
    # the budget while results are held and released
    items = []
    for k in range(8):
        x, hh = lattice_system(120000, 3, 10 + k)
        items.append((srv.submit(x, sph.make_params(3, hh, 2 * hh, order=0)), x, hh))
    for t, x, hh in items:
        assert srv.wait(t).status == sph.SPH_OK
        check(srv, t, x, hh, 0)
        srv.release(t)
    st = srv.stats()
    assert st.peak_held_bytes <= 200 << 20
    assert st.held_bytes == 0
    srv.close()


def test_small_request_not_stuck_behind_large(sph):
    """With two workers, a small request submitted just after a large one
    finishes first."""
    srv = sph.Server(16 * GB, streams=2)
    big, hb = lattice_system(2_000_000, 3, 3)
    small, hs = lattice_system(2000, 3, 4)
    for _ in range(2):  # warm both workers
        t = srv.submit(small, sph.make_params(3, hs, 2 * hs))
        srv.wait(t)
        srv.release(t)
    tb = srv.submit(big, sph.make_params(3, hb, 2 * hb))
    ts = srv.submit(small, sph.make_params(3, hs, 2 * hs))
    rs, rb = srv.wait(ts), srv.wait(tb)
    assert rs.status == sph.SPH_OK and rb.status == sph.SPH_OK
    assert rs.t_done_ns < rb.t_done_ns
    srv.release(ts)
    srv.release(tb)
    srv.close()


def test_tickets_and_shutdown(sph):
    srv = sph.Server(4 * GB)
    with pytest.raises(sph.SphError) as ei:
        srv.poll(12345)
    assert ei.value.code == sph.SPH_ERR_NOT_FOUND
    xyz, h = lattice_system(5000, 3, 7)
    t = srv.submit(xyz, sph.make_params(3, h, 2 * h))
    assert srv.wait(t).status == sph.SPH_OK
    srv.release(t)
    with pytest.raises(sph.SphError) as ei:
        srv.release(t)
    assert ei.value.code == sph.SPH_ERR_NOT_FOUND
    # bad parameters are refused at submission
    with pytest.raises(sph.SphError) as ei:
        srv.submit(xyz, sph.make_params(3, h, -1.0))
    assert ei.value.code == sph.SPH_ERR_INVALID
    # destroy with requests queued and running: returns, frees everything
    for k in range(6):
        x, hh = lattice_system(300000, 3, 20 + k)
        srv.submit(x, sph.make_params(3, hh, 2 * hh))
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 60


def _fetch_host(srv, t):
    rp, col, rho, orig = srv.fetch(t)
    return (rp.cpu().numpy(), col.cpu().numpy(), rho.cpu().numpy(),
            None if orig is None else orig.cpu().numpy())


def test_same_result_alone_and_in_the_mix(sph):
    """Each request's result is the same when it is served alone and when it
    is served inside a mixed load: small requests of both dimensions batched
    together (continuous batching, results split by the rebase kernels), a
    large request on its low-priority stream with a share of the GPU, and
    canonical-order requests, all submitted at once to four workers.  CSR
    identical; density within 1e-5 relative (the batched search may pick
    another tile shape, whose summation order differs in the last bits); the
    cell-order permutation identical."""
    specs = [(300000, 3, 0), (4000, 3, 0), (2500, 3, 0), (9000, 3, 0), (1500, 2, 0), (6000, 2, 0),
             (20000, 3, 1), (3000, 2, 1), (700, 3, 0), (12000, 3, 0), (60000, 2, 0), (5000, 3, 0)]
    systems = []
    for k, (n, dim, order) in enumerate(specs):
        xyz, h = lattice_system(n, dim, 100 + k, hr=1.2 + 0.025 * k)
        systems.append((torch.from_numpy(xyz).cuda(), sph.make_params(dim, h, 2 * h, order=order)))

    # alone: one worker, one request at a time, no batching partner
    srv = sph.Server(16 * GB, streams=1)
    alone = []
    for x, p in systems:
        t = srv.submit(x, p)
        assert srv.wait(t).status == sph.SPH_OK
        alone.append(_fetch_host(srv, t))
        srv.release(t)
    assert srv.stats().batches == 0
    srv.close()

    # in the mix: everything at once
    srv = sph.Server(16 * GB, streams=4, large_n=100000, large_sm_percent=60)
    ts = [srv.submit(x, p) for x, p in systems]
    mixed = []
    for t in ts:
        assert srv.wait(t).status == sph.SPH_OK
        mixed.append(_fetch_host(srv, t))
    st = srv.stats()
    srv.close()
    assert st.batches >= 1 and st.batched_requests >= 2

    for k, (a, b) in enumerate(zip(alone, mixed)):
        assert np.array_equal(a[0], b[0]), ("row_ptr", k)
        assert np.array_equal(a[1], b[1]), ("col", k)
        if a[3] is not None or b[3] is not None:
            assert np.array_equal(a[3], b[3]), ("orig_id", k)
        rel = np.abs(a[2].astype(np.float64) - b[2]) / np.abs(a[2].astype(np.float64))
        assert rel.max() <= RHO_RTOL, (k, rel.max())
