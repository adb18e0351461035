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


def _shard_worker(rank, world, port, out):
    """Codes this rank's share of one plan's messages with the oracle into a
    send buffer of the full layout (the other ranks' slots left zero) and
    gathers the buffers on every rank (test-side only: the coding itself
    exchanges nothing)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import fieldgen
    from oracle import packs as op
    from oracle import plan as opl

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    multirank.init("gloo")
    x = fieldgen.t21_field()                                  # 8 lev x 32 lat x 64 lon
    nz, ny, nx = x.shape
    plan = opl.Plan(nx, ny, nz, 2, 2, 0, 3)
    res = {}
    for rate in (8, 16):
        so, _, total = plan.layout(rate)
        buf = np.zeros(total, dtype=np.uint8)
        lo, hi = multirank.shard(len(plan.messages), rank, world)
        for m in plan.messages[lo:hi]:
            s = op.message_stream(plan, rate, x, m)
            buf[so[(m.src, m.dst)]:so[(m.src, m.dst)] + s.size] = s
        parts = [torch.zeros(total, dtype=torch.uint8) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(buf))
        res[rate] = [p.numpy().tobytes() for p in parts]
    out[rank] = res
    multirank.finalize()


def test_two_ranks_code_halves_of_one_plan():
    import numpy as np

    import fieldgen
    from oracle import packs as op
    from oracle import plan as opl

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    x = fieldgen.t21_field()
    nz, ny, nx = x.shape
    plan = opl.Plan(nx, ny, nz, 2, 2, 0, 3)
    for rate in (8, 16):
        whole = op.pack(plan, rate, x)                       # one rank codes every message
        parts = [np.frombuffer(b, dtype=np.uint8) for b in out[0][rate]]
        assert out[1][rate] == out[0][rate]                   # both ranks gathered the same
        so, _, total = plan.layout(rate)
        merged = np.zeros(total, dtype=np.uint8)
        for r in range(world):
            lo, hi = multirank.shard(len(plan.messages), r, world)
            for m in plan.messages[lo:hi]:
                o, nb = so[(m.src, m.dst)], opl.message_bytes(m, rate, 3)
                assert not parts[1 - r][o:o + nb].any()       # the other rank left this slot alone
                merged[o:o + nb] = parts[r][o:o + nb]
        assert merged.tobytes() == whole.tobytes()
