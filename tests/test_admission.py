"""Admission policy of the request server (host logic, no GPU): the policy
header is compiled alone with the host compiler and driven through a small
C shim."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SHIM = os.path.join(HERE, "native", "admission_shim.cpp")


@pytest.fixture(scope="module")
def adm(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("adm") / "libadm.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", SHIM, "-o", out])
    lib = ctypes.CDLL(out)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.adm_pick.restype = ctypes.c_int
    lib.adm_pick.argtypes = [i64p, i32p, i64p, i64p, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                             ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, i32p]
    lib.adm_request_bytes.restype = ctypes.c_int64
    lib.adm_request_bytes.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]
    return lib


CFG = dict(budget=1000, small_n=10, batch_max_n=40, max_batch=3, max_wait=100)


def pick(adm, q, held, now, **kw):
    c = dict(CFG)
    c.update(kw)
    n = np.array([r[0] for r in q], dtype=np.int64)
    dim = np.array([r[1] for r in q], dtype=np.int32)
    est = np.array([r[2] for r in q], dtype=np.int64)
    ts = np.array([r[3] for r in q], dtype=np.int64)
    out = np.zeros(max(len(q), 1), dtype=np.int32)
    P = lambda a, t: a.ctypes.data_as(ctypes.POINTER(t))
    k = adm.adm_pick(P(n, ctypes.c_int64), P(dim, ctypes.c_int32), P(est, ctypes.c_int64), P(ts, ctypes.c_int64),
                     len(q), held, c["budget"], c["small_n"], c["batch_max_n"], c["max_batch"], c["max_wait"], now,
                     P(out, ctypes.c_int32))
    return out[:k].tolist()


def test_empty_and_fifo(adm):
    assert pick(adm, [], 0, 0) == []
    # (n, dim, est_bytes, t_submit)
    q = [(100, 3, 600, 0), (200, 3, 300, 1)]
    assert pick(adm, q, 0, 5) == [0]          # head fits: it starts (large: alone)
    assert pick(adm, q, 500, 5) == [1]        # head does not fit, young: the next one passes


def test_old_blocked_head_is_not_passed(adm):
    q = [(100, 3, 600, 0), (200, 3, 300, 1)]
    assert pick(adm, q, 500, 100) == []       # head waited max_wait: nobody passes it
    assert pick(adm, q, 500, 99) == [1]
    # an old request further back blocks only those behind it
    q = [(100, 3, 300, 50), (200, 3, 900, 0), (5, 3, 10, 60)]
    assert pick(adm, q, 750, 120) == []       # q[0] does not fit (young), q[1] old and blocked
    assert pick(adm, q, 100, 120) == [0]


def test_continuous_batching(adm):
    q = [(5, 3, 100, 0), (50, 3, 100, 1), (6, 2, 100, 2), (7, 3, 100, 3), (8, 3, 100, 4), (9, 3, 100, 5)]
    # small head takes later small ones of its dimension, up to max_batch
    assert pick(adm, q, 0, 10) == [0, 3, 4]
    # particle limit: 5 + 7 = 12 <= 15, + 8 > 15
    assert pick(adm, q, 0, 10, batch_max_n=15) == [0, 3]
    # budget limit
    assert pick(adm, q, 750, 10) == [0, 3]
    # a large head is never batched
    assert pick(adm, [(50, 3, 10, 0), (5, 3, 10, 1)], 0, 1) == [0]


def test_request_bytes(adm):
    a = adm.adm_request_bytes(1000, 3, 128)
    assert a == 1000 * (72 + 24 + 16 + 512) + 8 + 4096
    assert adm.adm_request_bytes(2000, 3, 128) > a > adm.adm_request_bytes(1000, 2, 40)


def test_simulation_budget_liveness_aging(adm):
    """Random arrivals and completions: the reserved bytes never exceed the
    budget, every request is eventually admitted, and a request that has
    waited max_wait is never passed."""
    rng = np.random.default_rng(5)
    budget, max_wait = 10_000, 30
    arrivals = sorted(rng.integers(0, 400, size=300).tolist())
    reqs = []
    for k, t in enumerate(arrivals):
        n = int(rng.integers(1, 40))
        reqs.append(dict(id=k, n=n, dim=int(rng.choice([2, 3])), est=int(rng.integers(50, 4000)), t=t))
    queue, running, held = [], [], 0
    admitted_at = {}
    nxt = 0
    for now in range(0, 5000):
        while nxt < len(reqs) and reqs[nxt]["t"] <= now:
            queue.append(reqs[nxt])
            nxt += 1
        for r in [r for r in running if r["done"] <= now]:
            running.remove(r)
            held -= r["est"]
        while queue:
            idx = pick(adm, [(r["n"], r["dim"], r["est"], r["t"]) for r in queue], held, now,
                       budget=budget, small_n=10, batch_max_n=30, max_batch=4, max_wait=max_wait)
            if not idx:
                break
            # aging: nothing behind an old request that does not fit may start
            for j, r in enumerate(queue):
                if j >= idx[0]:
                    break
                assert not (now - r["t"] >= max_wait and held + r["est"] > budget)
            for j in sorted(idx, reverse=True):
                r = queue.pop(j)
                r["done"] = now + int(rng.integers(1, 20))
                running.append(r)
                held += r["est"]
                admitted_at[r["id"]] = now
            assert held <= budget
        if nxt == len(reqs) and not queue and not running:
            break
    assert len(admitted_at) == len(reqs)
