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


# ------------------------------------------------------------------------------------------
# one trajectory split by frames: partial transforms against the first frame, one all-reduce
# ------------------------------------------------------------------------------------------
def _partial_oracle(psi, f0, f1):
    """The partial transform of frames [f0, f1) against frame 0, from the oracle's direct DFT of
    the residual series with the other frames zeroed."""
    import numpy as np

    import oracle
    P, F, nq = psi.shape
    out = np.zeros((P, F, nq), dtype=np.complex128)
    for p in range(P):
        for q in range(nq):
            r = np.zeros(F, dtype=np.complex128)
            r[f0:f1] = psi[p, f0:f1, q] - psi[p, 0, q]
            out[p, :, q] = oracle.dft(r, -1)
    return out


def _sharded_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads
    from paper_2602_10064_gb300 import sharded
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        psi = workloads.random_exit_waves(2, 13, 24, seed=71).astype(np.complex128)
        f0, f1 = sharded.frame_range(13, rank, world)
        part = torch.from_numpy(_partial_oracle(psi, f0, f1).view(np.float64).copy())
        sharded.reduce_partials(part, dist)
        tot = part.numpy().view(np.complex128)
        S = np.abs(tot) ** 2
        S[:, 0] = 0.0
        q.put((rank, (f0, f1), S))
    finally:
        dist.destroy_process_group()


def test_frame_sharded_spectrum_two_ranks_equals_single_process():
    import numpy as np

    import oracle
    import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [(0, 7), (7, 13)]
    want = oracle.spectrum(workloads.random_exit_waves(2, 13, 24, seed=71))
    for _, _, S in out:
        assert np.linalg.norm(S - want) / np.linalg.norm(want) < 1e-10


def test_frame_range_covers_every_frame_once():
    from paper_2602_10064_gb300 import sharded
    for F, world in [(13, 2), (1024, 8), (7, 7), (100, 3)]:
        ranges = [sharded.frame_range(F, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == F
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
    with pytest.raises(ValueError):
        sharded.frame_range(3, 0, 4)
