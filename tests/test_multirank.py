"""The N-rank host logic of bench.py on CPU: gloo, world size 2 (weak scaling, no data exchange
besides the timing reduction; each rank its own seeded trajectory)."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = [2.0, 4.0][rank]
        units = [1000, 3000][rank]
        value, tmax = bench.aggregate_ranks(secs, units, dist)
        w = bench.make_workload("c1", seed_offset=bench.rank_seed_offset(rank), frames=4)
        q.put((rank, value, tmax, w.pos.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, _ in out:
        assert tmax == 4.0  # the slowest rank's time
        assert value == pytest.approx((1000 + 3000) / 4.0)
    assert out[0][3] != out[1][3]  # independently seeded trajectories


def test_single_rank_aggregate_is_local():
    import bench
    assert bench.aggregate_ranks(2.0, 100) == (50.0, 2.0)
