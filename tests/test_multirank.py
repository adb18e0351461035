"""The N > 1 host path on CPU: two gloo ranks agree on the barrier-bracketed
max-over-ranks time and the weak-scaling aggregate; strong-scaling shards
cover every message once.  No GPU and no data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_24294_gb300 import multirank


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    ws, r, local = multirank.init("gloo")
    assert (ws, r, local) == (world, rank, rank)
    multirank.barrier()
    elapsed = 1.0 + rank                      # rank 1 is the slow one
    tmax = multirank.max_over_ranks(elapsed)
    total = multirank.sum_over_ranks(10 * (rank + 1))
    out[rank] = (tmax, total, multirank.weak_throughput(100.0, tmax, ws))
    multirank.finalize()


@pytest.mark.parametrize("world", [2])
def test_gloo_two_ranks(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        tmax, total, thr = out[r]
        assert tmax == 2.0 and total == 30.0
        assert thr == pytest.approx(100.0 * world / 2.0)


def test_shards_cover_once():
    for n in (0, 1, 7, 512):
        for w in (1, 2, 3, 8):
            owned = []
            for r in range(w):
                lo, hi = multirank.shard(n, r, w)
                owned += list(range(lo, hi))
                assert hi - lo in (n // w, n // w + 1)
            assert owned == list(range(n))
