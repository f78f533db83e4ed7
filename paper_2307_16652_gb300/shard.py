"""One distance matrix over several GPUs, one process per GPU.

The triplet blocks of the method are independent given D (Sec. 3.2, the
blocked triplet algorithm), so both passes split over the 64 x 64
upper-triangle super-tiles of the matrix.  Each rank takes one contiguous
range of tiles (``pald_shard_range``):

1. pass 1 on its tiles (``pald_focus_tiles``) writes u of their pairs and
   mirror pairs into the rank's U;
2. the ranks exchange u once: each packs its tiles (4096 words per tile),
   the packed buffers are all-gathered (one collective; the caller's process
   group, NCCL on GPUs), and every rank unpacks all of them, completing U;
3. pass 2 on the same tiles (``pald_cohesion_tiles``) writes C[X, Z] and
   C[Z, X] of those tiles; with ``gather_c`` C is exchanged the same way
   (8192 words per tile), so every rank ends with the full C.

Nothing here waits on another GPU inside a kernel: the only cross-rank step
is the host-issued all-gather.  Every tile gives the bits of the single-GPU
passes, so the result equals ``pald_focus`` + ``pald_cohesion`` bit for bit.

The tile order and the pack layout are restated on the host (``tile_order``,
``pack_tiles``, ``unpack_tiles``) so the partition can be checked without a
GPU.
"""
from __future__ import annotations

import numpy as np

B = 64         # tile edge
STRIP = 12     # block rows per strip of the launch order
TILE_WORDS = B * B


def tiles_of(n: int) -> int:
    t = -(-n // B)
    return t * (t + 1) // 2


def shard_range(n: int, rank: int, world: int):
    """The contiguous tile range [t0, t1) of `rank` (the formula of
    pald_shard_range)."""
    N = tiles_of(n)
    return N * rank // world, N * (rank + 1) // world


def tile_order(n: int):
    """(bi, bj), bi <= bj, of every tile in the library's launch order: the
    upper triangle walked in strips of STRIP block rows, each strip first its
    own triangle column by column, then the columns to its right."""
    T = -(-n // B)
    out = []
    k0 = 0
    while k0 < T:
        h = min(STRIP, T - k0)
        for c in range(h):                     # the strip's own triangle
            for r in range(c + 1):
                out.append((k0 + r, k0 + c))
        for col in range(k0 + h, T):           # the columns to its right
            for r in range(h):
                out.append((k0 + r, col))
        k0 += h
    return out


def pack_tiles(M: np.ndarray, t0: int, t1: int, both: bool = False) -> np.ndarray:
    """Host restatement of pald_pack_tiles for an n x n array of 4-byte words."""
    n = M.shape[0]
    order = tile_order(n)
    halves = 2 if both else 1
    out = np.zeros((t1 - t0) * TILE_WORDS * halves, dtype=M.dtype)
    for k, t in enumerate(range(t0, t1)):
        bi, bj = order[t]
        for h in range(halves):
            r0, c0 = (bi, bj) if h == 0 else (bj, bi)
            blk = np.zeros((B, B), dtype=M.dtype)
            sub = M[r0 * B:(r0 + 1) * B, c0 * B:(c0 + 1) * B]
            blk[:sub.shape[0], :sub.shape[1]] = sub
            base = (k * halves + h) * TILE_WORDS
            out[base:base + TILE_WORDS] = blk.ravel()
    return out


def unpack_tiles(packed: np.ndarray, M: np.ndarray, t0: int, t1: int, both: bool = False) -> np.ndarray:
    """Host restatement of pald_unpack_tiles (in place on M)."""
    n = M.shape[0]
    order = tile_order(n)
    halves = 2 if both else 1
    for k, t in enumerate(range(t0, t1)):
        bi, bj = order[t]
        base = k * halves * TILE_WORDS
        blk = packed[base:base + TILE_WORDS].reshape(B, B)
        rx, ry = min(B, n - bi * B), min(B, n - bj * B)
        M[bi * B:bi * B + rx, bj * B:bj * B + ry] = blk[:rx, :ry]
        if both:
            blk2 = packed[base + TILE_WORDS:base + 2 * TILE_WORDS].reshape(B, B)
            M[bj * B:bj * B + ry, bi * B:bi * B + rx] = blk2[:ry, :rx]
        else:
            M[bj * B:bj * B + ry, bi * B:bi * B + rx] = blk[:rx, :ry].T
    return M


def max_range(n: int, world: int) -> int:
    """The largest number of tiles any rank holds (all-gather buffers are
    padded to it)."""
    return max(t1 - t0 for t0, t1 in (shard_range(n, r, world) for r in range(world)))


def pald_sharded(D, U, C, *, group=None, gather_c: bool = True, accum_mode: int = 0, stream=None):
    """Both passes for one matrix over the ranks of `group` (the default
    process group): D is this rank's full copy of the distance matrix, U and
    C its full-size outputs.  Returns this rank's tile range."""
    import torch
    import torch.distributed as dist

    from . import binding

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    n = D.shape[0]
    t0, t1 = binding.pald_shard_range(n, rank, world)
    binding.pald_focus_tiles(D, U, t0, t1, stream=stream)
    width = max_range(n, world)

    def exchange(M, both):
        words = TILE_WORDS * (2 if both else 1)
        mine = torch.zeros(width * words, dtype=torch.int32, device=M.device)
        binding.pald_pack_tiles(M, t0, t1, mine, both=both, stream=stream)
        if world > 1:
            everyone = torch.empty(world * width * words, dtype=torch.int32, device=M.device)
            dist.all_gather_into_tensor(everyone, mine, group=group)
        else:
            everyone = mine
        for r in range(world):
            r0, r1 = binding.pald_shard_range(n, r, world)
            binding.pald_unpack_tiles(everyone[r * width * words:], M, r0, r1, both=both, stream=stream)

    exchange(U, both=False)
    binding.pald_cohesion_tiles(D, U, C, t0, t1, accum_mode=accum_mode, stream=stream)
    if gather_c:
        exchange(C.view(torch.int32), both=True)
    return t0, t1


def tiles_per_rank_cost(n: int, world: int):
    """Relative pass cost per rank (a diagonal tile costs about half a full
    one), to check the balance of a partition."""
    order = tile_order(n)
    cost = []
    for r in range(world):
        t0, t1 = shard_range(n, r, world)
        cost.append(sum(0.5 if order[t][0] == order[t][1] else 1.0 for t in range(t0, t1)))
    return cost


def imbalance(n: int, world: int) -> float:
    c = tiles_per_rank_cost(n, world)
    return max(c) / (sum(c) / len(c)) if sum(c) else 1.0


# ---------------------------------------------------------------------------
# The batched workload over several GPUs: the matrices are independent
# problems, so each one runs whole on one rank and no rank needs another's
# data (weak scaling, no collective on the data path).

def batched_partition(ns, world: int):
    """Matrix indices per rank: largest first (cost n^3, as both passes
    scale with C(n,3)) to the rank with the least work so far, the lowest
    rank on ties.  Deterministic; each list ascending."""
    ns = np.asarray(ns, dtype=np.int64)
    load = np.zeros(world, dtype=np.float64)
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(ns)), key=lambda k: (-int(ns[k]), k)):
        r = int(np.argmin(load))
        parts[r].append(i)
        load[r] += float(ns[i]) ** 3
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def batched_imbalance(ns, world: int) -> float:
    """Largest rank's n^3 work over the mean."""
    ns = np.asarray(ns, dtype=np.float64)
    cost = [float((ns[p] ** 3).sum()) for p in batched_partition(ns, world)]
    return max(cost) / (sum(cost) / world) if sum(cost) else 1.0


def pald_batched_sharded(ns, offs, D, U, C, *, rank: int = None, world: int = None, group=None,
                         accum_mode: int = 0, stream=None):
    """This rank's share of a batched workload: ``pald_batched`` on the
    matrices ``batched_partition`` gives it, in the caller's packed buffers
    (every rank may hold all of D; only its own matrices' U and C are
    written).  `rank` and `world` default to the process group's.  Returns
    the rank's matrix indices."""
    import torch.distributed as dist

    from . import binding

    if world is None:
        world = dist.get_world_size(group) if dist.is_initialized() else 1
    if rank is None:
        rank = dist.get_rank(group) if dist.is_initialized() else 0
    ns = np.asarray(ns, dtype=np.int64)
    offs = np.asarray(offs, dtype=np.int64)
    mine = batched_partition(ns, world)[rank]
    if len(mine):
        binding.pald_batched(ns[mine], offs[mine], D, U, C, accum_mode=accum_mode, stream=stream)
    return mine


__all__ = ["B", "TILE_WORDS", "tiles_of", "shard_range", "tile_order", "pack_tiles", "unpack_tiles", "max_range",
           "pald_sharded", "tiles_per_rank_cost", "imbalance", "batched_partition", "batched_imbalance",
           "pald_batched_sharded"]
