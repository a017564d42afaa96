"""Replica plumbing on CPU: two gloo ranks (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2401_08586_gb300 import replicas  # noqa: E402


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    try:
        w, r, lr = replicas.rank_env()
        assert (w, r, lr) == (world, rank, rank)
        if mode == "fail" and rank == 1:
            raise RuntimeError("rank 1 fails before joining")
        import datetime
        dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=10))
        replicas.barrier(w)
        items = list(range(11))
        mine = replicas.shard(items, w, r)
        t = 1.0 + rank  # rank 1 is the slowest
        rate = replicas.whole_job_rate(len(mine), t, w)
        tmax = replicas.max_over_ranks(t, w)
        allitems = [None] * w
        dist.all_gather_object(allitems, mine)
        q.put((rank, rate, tmax, sorted(x for part in allitems for x in part)))
        replicas.finish(w)
    except Exception as e:  # reported to the parent
        q.put((rank, "error", type(e).__name__, str(e)[:200]))


def run(world, mode="ok", timeout=60):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q, mode)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=timeout) for _ in range(world)]
    for p in ps:
        p.join(timeout=timeout)
    return sorted(out, key=lambda x: x[0])


def test_two_ranks_reduce_and_shard():
    out = run(2)
    for rank, rate, tmax, items in out:
        assert tmax == 2.0
        assert rate == pytest.approx(11 / 2.0)
        assert items == list(range(11))  # every item exactly once


def test_single_rank_is_identity():
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.shard(range(5), 1, 0) == [0, 1, 2, 3, 4]
    assert replicas.whole_job_rate(10, 2.0, 1) == 5.0


def test_failed_rank_is_reported_not_hung():
    """A rank that dies before the process group forms: the other rank's
    rendezvous ends with an error within its timeout instead of hanging."""
    out = run(2, mode="fail", timeout=120)
    assert out[1][1] == "error"
    assert out[0][1] == "error"
