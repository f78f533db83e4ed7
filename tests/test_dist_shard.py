"""The shard plan of one matrix over several ranks, on CPU processes (gloo,
world size 2): each rank computes u and C for its own tile range with the
oracle, packs its tiles in the library's layout, the ranks all-gather the
packed buffers once, and the unpacked U and C must equal the full oracle's.
Also: the tile ranges and their mirror blocks cover the matrix exactly once,
and the split is balanced."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2307_16652_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n", [1, 63, 64, 65, 200, 777, 1000])
def test_tile_order_covers_the_upper_triangle_once(n):
    if n < 2:
        assert shard.tiles_of(2) == 1
        return
    order = shard.tile_order(n)
    T = -(-n // 64)
    assert len(order) == shard.tiles_of(n) == T * (T + 1) // 2
    assert sorted(order) == sorted((i, j) for i in range(T) for j in range(i, T))


@pytest.mark.parametrize("n,world", [(200, 2), (777, 3), (4096, 8), (65536, 8), (65536, 7)])
def test_ranges_partition_every_block_once(n, world):
    N = shard.tiles_of(n)
    ranges = [shard.shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == N
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    T = -(-n // 64)
    seen = np.zeros((T, T), dtype=np.int64)
    order = shard.tile_order(n)
    for t0, t1 in ranges:
        for t in range(t0, t1):
            bi, bj = order[t]
            seen[bi, bj] += 1
            if bi != bj:
                seen[bj, bi] += 1  # the mirror block written by the same tile
    assert np.all(seen == 1)
    if N >= 50 * world:
        assert shard.imbalance(n, world) < 1.05


def test_host_pack_roundtrip():
    rng = np.random.default_rng(3)
    n = 150
    A = rng.integers(0, 1 << 30, size=(n, n)).astype(np.int32)
    S = np.triu(A) + np.triu(A, 1).T  # symmetric
    N = shard.tiles_of(n)
    got = shard.unpack_tiles(shard.pack_tiles(S, 0, N), np.zeros_like(S), 0, N)
    assert np.array_equal(got, S)
    got = shard.unpack_tiles(shard.pack_tiles(A, 0, N, both=True), np.zeros_like(A), 0, N, both=True)
    assert np.array_equal(got, A)


def _rank_tiles_from_rows(n, t0, t1, U_rows, C_rows, rows):
    """This rank's tiles of U and C filled from the oracle's rows."""
    where = {int(r): i for i, r in enumerate(rows)}
    U = np.zeros((n, n), np.int32)
    C = np.zeros((n, n), np.float64)
    order = shard.tile_order(n)
    for t in range(t0, t1):
        bi, bj = order[t]
        for x in range(bi * 64, min(n, bi * 64 + 64)):
            U[x, bj * 64:bj * 64 + 64] = U_rows[where[x], bj * 64:bj * 64 + 64]
            C[x, bj * 64:bj * 64 + 64] = C_rows[where[x], bj * 64:bj * 64 + 64]
        for z in range(bj * 64, min(n, bj * 64 + 64)):
            C[z, bi * 64:bi * 64 + 64] = C_rows[where[z], bi * 64:bi * 64 + 64]
    return U, C


def _worker(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        D = inputs.tie_heavy_matrix(n, hi=7) if n % 2 else inputs.plain_matrix(n)
        t0, t1 = shard.shard_range(n, rank, world)
        order = shard.tile_order(n)
        blocks = sorted({b for t in range(t0, t1) for b in order[t]})
        rows = np.concatenate([np.arange(b * 64, min(n, b * 64 + 64)) for b in blocks]) if blocks else \
            np.zeros(0, np.int64)
        Ur, Cr = oracle.rows(D, rows, threads=2)  # only the rows this rank's tiles need
        U_mine, C_mine = _rank_tiles_from_rows(n, t0, t1, Ur, Cr, rows)
        width = shard.max_range(n, world)

        def exchange(M, both):
            words = shard.TILE_WORDS * (2 if both else 1)
            mine = np.zeros(width * words, dtype=M.dtype)
            p = shard.pack_tiles(M, t0, t1, both=both)
            mine[:p.size] = p
            parts = [torch.zeros(width * words, dtype=torch.from_numpy(mine).dtype) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(mine))
            full = np.zeros_like(M)
            for r in range(world):
                r0, r1 = shard.shard_range(n, r, world)
                shard.unpack_tiles(parts[r].numpy(), full, r0, r1, both=both)
            return full

        U = exchange(U_mine, both=False)
        C = exchange(C_mine, both=True)
        U_ref, C_ref = oracle.focus_and_cohesion(D, threads=2)
        q.put((rank, bool(np.array_equal(U, U_ref)), bool(np.array_equal(C, C_ref)), t1 - t0))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [200, 263])
def test_two_ranks_exchange_u_and_c_once(n):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, u_ok, c_ok, tiles in res:
        assert u_ok, f"rank {rank}: gathered U differs from the oracle"
        assert c_ok, f"rank {rank}: gathered C differs from the oracle"
        assert tiles > 0


def test_library_shard_ranges_match_the_host_plan():
    from paper_2307_16652_gb300 import binding, build

    build.build()
    for n in (2, 64, 65, 1000, 65536, 1 << 20):
        assert binding.pald_shard_tiles(n) == shard.tiles_of(n)
        for world in (1, 2, 3, 8):
            for r in range(world):
                assert binding.pald_shard_range(n, r, world) == shard.shard_range(n, r, world)
    assert binding.pald_shard_tiles(1) == 0
    with pytest.raises(binding.PaldError):
        binding.pald_shard_range(100, 2, 2)


# ---------------------------------------------------------------------------
# The batched workload over ranks: whole matrices per rank, no exchange.

@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_batched_partition_covers_every_matrix_once(world):
    ns = inputs.batched_sizes(2000)
    parts = shard.batched_partition(ns, world)
    assert len(parts) == world
    assert sorted(np.concatenate(parts).tolist()) == list(range(len(ns)))
    assert all(np.all(np.diff(p) > 0) for p in parts)  # ascending, no repeats
    assert shard.batched_imbalance(ns, world) < 1.01   # 2000 matrices balance closely by n^3


def test_batched_partition_with_more_ranks_than_matrices():
    parts = shard.batched_partition([5, 300, 9], 5)
    assert sorted(np.concatenate(parts).tolist()) == [0, 1, 2]
    assert sum(len(p) == 0 for p in parts) == 2
    assert parts[0].tolist() == [1]  # the largest goes first, to rank 0


def _batched_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = inputs.batched_sizes(12, lo=8, hi=70)
        mine = shard.batched_partition(ns, world)[rank]
        out = {}
        for i in mine:  # this rank's matrices only; nothing from the other rank is needed
            U, C = oracle.focus_and_cohesion(inputs.euclidean_fp32(inputs.batched_points(int(i), int(ns[i]))),
                                             threads=1)
            out[int(i)] = (U, C)
        everyone = [None] * world
        dist.all_gather_object(everyone, out)  # for the check only
        if rank == 0:
            merged = {}
            for part in everyone:
                assert not set(part) & set(merged), "a matrix ran on two ranks"
                merged.update(part)
            ok = sorted(merged) == list(range(len(ns)))
            for i, (U, C) in merged.items():
                Ur, Cr = oracle.focus_and_cohesion(inputs.euclidean_fp32(inputs.batched_points(i, int(ns[i]))),
                                                   threads=1)
                ok = ok and np.array_equal(U, Ur) and np.array_equal(C, Cr)
            q.put(ok)
    finally:
        dist.destroy_process_group()


def test_two_ranks_run_disjoint_batched_shares():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert q.get(timeout=10)
