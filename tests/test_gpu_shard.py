"""The shard plan on one GPU: the ranks of a sharded run executed one after
another (no kernel waits on another rank), their packed tiles exchanged by
concatenation as an all-gather would, and the gathered U and C compared bit
for bit with the single-GPU passes; the device pack layout against its host
restatement."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2307_16652_gb300 import binding, build, inputs, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def _single(D):
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    return U, C


def _sharded_sequential(D, world):
    n = D.shape[0]
    width = shard.max_range(n, world)
    ranges = [binding.pald_shard_range(n, r, world) for r in range(world)]
    assert ranges == [shard.shard_range(n, r, world) for r in range(world)]
    # pass 1 per rank into its own U, packed
    packs = []
    for t0, t1 in ranges:
        Ur = torch.full((n, n), -7, dtype=torch.int32, device="cuda")
        binding.pald_focus_tiles(D, Ur, t0, t1)
        p = torch.zeros(width * 4096, dtype=torch.int32, device="cuda")
        binding.pald_pack_tiles(Ur, t0, t1, p)
        packs.append(p)
    gathered = torch.cat(packs)  # what an all-gather delivers to every rank
    U = torch.full((n, n), -9, dtype=torch.int32, device="cuda")
    for r, (t0, t1) in enumerate(ranges):
        binding.pald_unpack_tiles(gathered[r * width * 4096:], U, t0, t1)
    # pass 2 per rank, C tiles packed with both blocks
    cpacks = []
    for t0, t1 in ranges:
        Cr = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
        binding.pald_cohesion_tiles(D, U, Cr, t0, t1)
        p = torch.zeros(width * 8192, dtype=torch.int32, device="cuda")
        binding.pald_pack_tiles(Cr.view(torch.int32), t0, t1, p, both=True)
        cpacks.append(p)
    cg = torch.cat(cpacks)
    C = torch.full((n, n), -3.0, dtype=torch.float32, device="cuda")
    for r, (t0, t1) in enumerate(ranges):
        binding.pald_unpack_tiles(cg[r * width * 8192:], C.view(torch.int32), t0, t1, both=True)
    torch.cuda.synchronize()
    return U, C, packs


@pytest.mark.parametrize("n,world,kind", [(64, 2, "plain"), (130, 3, "plain"), (517, 3, "tie"), (1088, 4, "plain"),
                                          (2049, 5, "tie")])
def test_sharded_equals_single_gpu_bit_for_bit(n, world, kind):
    D_np = inputs.plain_matrix(n) if kind == "plain" else inputs.tie_heavy_matrix(n, hi=9)
    D = torch.from_numpy(D_np).cuda()
    U1, C1 = _single(D)
    U, C, packs = _sharded_sequential(D, world)
    assert torch.equal(U, U1)
    assert torch.equal(C, C1)
    # the device layout is the host restatement's
    t0, t1 = binding.pald_shard_range(n, 0, world)
    host = shard.pack_tiles(U1.cpu().numpy(), t0, t1)
    assert np.array_equal(packs[0][:host.size].cpu().numpy(), host)
    assert binding.pald_check_faults() == 0


def test_pald_sharded_on_one_rank():
    n = 300
    D = torch.from_numpy(inputs.plain_matrix(n)).cuda()
    U1, C1 = _single(D)
    U = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    C = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    t0, t1 = shard.pald_sharded(D, U, C)
    torch.cuda.synchronize()
    assert (t0, t1) == (0, shard.tiles_of(n))
    assert torch.equal(U, U1) and torch.equal(C, C1)


def test_bad_ranges_are_rejected():
    lib = binding.lib()
    n = 200
    N = binding.pald_shard_tiles(n)
    assert N == shard.tiles_of(n) == 10
    D = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    U = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    with pytest.raises(binding.PaldError):
        binding.pald_focus_tiles(D, U, 0, N + 1)
    with pytest.raises(binding.PaldError):
        binding.pald_focus_tiles(D, U, 5, 4)
    assert lib.pald_pack_tiles(U.data_ptr(), n, 0, 1, 2, U.data_ptr(), None) == 1  # both must be 0 or 1


@pytest.mark.parametrize("world", [2, 3])
def test_batched_shares_run_one_after_another_give_the_full_result(world):
    # each rank's pald_batched over its own matrices, into shared packed
    # buffers: together they must equal one pald_batched call bit for bit
    rng = np.random.default_rng(world)
    ns = np.array([int(v) for v in rng.integers(8, 300, size=40)] + [513, 1024], dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    for i, n in enumerate(ns):
        Dh[offs[i]:offs[i] + n * n] = inputs.euclidean_fp32(inputs.batched_points(i, int(n))).ravel()
    D = torch.from_numpy(Dh).cuda()
    U1 = torch.zeros(total, dtype=torch.int32, device="cuda")
    C1 = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U1, C1)
    U2 = torch.full((total,), -1, dtype=torch.int32, device="cuda")
    C2 = torch.full((total,), -1.0, dtype=torch.float32, device="cuda")
    seen = []
    for r in range(world):
        seen += shard.pald_batched_sharded(ns, offs, D, U2, C2, rank=r, world=world).tolist()
    torch.cuda.synchronize()
    assert sorted(seen) == list(range(len(ns)))
    assert binding.pald_check_faults() == 0
    for i, n in enumerate(ns):
        sl = slice(int(offs[i]), int(offs[i] + n * n))
        assert torch.equal(U2[sl], U1[sl]) and torch.equal(C2[sl], C1[sl]), f"matrix {i} (n = {n})"
