"""The multi-rank bench plumbing (barrier, max over ranks, replica sharding of
independent problems) on two CPU processes with the gloo backend."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    t = bench.max_over_ranks(10.0 + rank, world)   # each rank's elapsed time
    # every rank processes its own copy of the workload: the job-wide value
    # is world * units / max time
    n = 64
    value = 2.0 * bench.triplets(n) * world / (t / 1e3)
    q.put((rank, t, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res[0][1] == res[1][1] == 11.0
    assert res[0][2] == res[1][2]


def test_triplet_count():
    import bench

    assert bench.triplets(3) == 1 and bench.triplets(4) == 4 and bench.triplets(65536) == 65536 * 65535 * 65534 // 6
