"""The multi-rank side of bench.py on CPU: two gloo ranks agree on the slowest
rank's time (max) and on the total particle-steps (sum), as the replica-only
scaling needs (no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    t = bench.reduce_scalar(dist, 1.5 + rank, "max")
    u = bench.reduce_scalar(dist, 64000 * 10 * (rank + 1), "sum")
    bench.barrier(dist)
    out.put((r, w, lr, t, u))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == pytest.approx(2.5)            # the slowest rank's seconds
        assert r[4] == pytest.approx(64000 * 10 * 3)  # all ranks' particle-steps


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_scalar(None, 3.0, "max") == 3.0
    assert bench.reduce_scalar(None, 3.0, "sum") == 3.0
