"""The tie map and pass 2's two inner loops.

Pass 2 runs a stage with a short 4-instruction loop when the tie map shows
that no one-sided tie (two equal entries in one row of D) can occur in it,
and with the long loop otherwise.  These tests check (1) the map against the
row repeats found on the host, bit for bit, (2) that the mixed loops give
exactly the bits of the long loop alone (pald_cohesion_noalloc runs without
a map), and (3) parity with the oracle on matrices with planted ties.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

DUP_CAP = 2048  # repeats per row that the map lists before flagging the block


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def expected_map(D: np.ndarray):
    """Host restatement of the map (rows of at most one hash pass, n <= 8192)."""
    n = D.shape[0]
    nb = -(-n // 64)
    wpp = -(-(-(-n // 8)) // 32)  # groups of 8 y, 32 groups per word
    words = np.zeros(nb * nb * wpp, dtype=np.uint32)
    dirty = np.zeros(nb, dtype=np.uint32)
    bits = (D + np.float32(0.0)).view(np.uint32)
    for r in range(n):
        vals, inv, cnt = np.unique(bits[r], return_inverse=True, return_counts=True)
        if n - len(vals) > DUP_CAP:
            dirty[r // 64] = 1
            continue
        for g in np.nonzero(cnt > 1)[0]:
            cols = np.nonzero(inv == g)[0]
            p, q = np.meshgrid(cols, cols, indexing="ij")
            keep = p != q
            p, q = p[keep], q[keep]
            a = np.minimum(r // 64, q // 64)
            b = np.maximum(r // 64, q // 64)
            grp = p // 8
            idx = (a * nb + b) * wpp + grp // 32
            np.bitwise_or.at(words, idx, (np.uint32(1) << (grp % 32).astype(np.uint32)))
    return words, dirty


def gpu_map(D_np):
    m = binding.pald_tie_map(torch.from_numpy(D_np).cuda())
    torch.cuda.synchronize()
    m = m.cpu().numpy().view(np.uint32)
    n = D_np.shape[0]
    nb = -(-n // 64)
    return m[:-nb], m[-nb:]


def _cases():
    rng = np.random.default_rng(11)
    return {
        "plain512": inputs.plain_matrix(512),
        "tie200": inputs.small_tie_heavy(rng, 200, hi=20),
        "dup130": inputs.small_tie_heavy(rng, 130, hi=3, dup=True),
        "planted700": inputs.planted_tie_matrix(rng, 700, ties=400),
        "planted70": inputs.planted_tie_matrix(rng, 70, ties=30),
        "tie4096": inputs.tie_heavy_matrix(4096),
        "two": np.array([[0, 1], [1, 0]], dtype=np.float32),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_tie_map_matches_host_repeats(name):
    D = _cases()[name]
    words, dirty = gpu_map(D)
    ew, ed = expected_map(D)
    assert np.array_equal(dirty != 0, ed != 0), f"dirty blocks differ: {np.nonzero((dirty != 0) != (ed != 0))}"
    diff = np.nonzero(words != ew)[0]
    assert diff.size == 0, f"{diff.size} map words differ, first at {diff[:5].tolist()}"


def test_tie_map_of_large_row_passes_flags_every_planted_tie():
    # n > 8192: rows are hashed in several passes; every planted repeat must
    # still be marked (the map may hold more, never less)
    rng = np.random.default_rng(5)
    n = 9000
    D = inputs.euclidean_fp32(rng.normal(size=(n, 6)))
    for _ in range(200):
        x, y, z = rng.choice(n, size=3, replace=False)
        D[x, z] = D[z, x] = D[x, y]
    words, dirty = gpu_map(D)
    ew, _ = expected_map(D)
    assert not np.any(dirty)
    assert np.all((words & ew) == ew)


def _cohesion_pair(D_np, schedule_id):
    D = torch.from_numpy(D_np).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    mixed = torch.empty((n, n), dtype=torch.float32, device="cuda")
    long_only = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_cohesion(D, U, mixed, schedule_id=schedule_id)
    binding.pald_cohesion_noalloc(D, U, long_only, schedule_id=schedule_id)
    torch.cuda.synchronize()
    return U, mixed, long_only


@pytest.mark.parametrize("schedule_id", list(range(8)))
@pytest.mark.parametrize("kind", ["plain2048", "planted1500", "precision1024"])
def test_short_loop_gives_the_bits_of_the_long_loop(kind, schedule_id):
    rng = np.random.default_rng(3)
    if kind == "plain2048":
        D = inputs.plain_matrix(2048)
    elif kind == "planted1500":
        D = inputs.planted_tie_matrix(rng, 1500, ties=3000)
    else:
        D = inputs.euclidean_fp32(inputs.precision_points(16384)[:1024])
    _, mixed, long_only = _cohesion_pair(D, schedule_id)
    assert torch.equal(mixed, long_only)


@pytest.mark.parametrize("n,ties", [(3, 1), (40, 20), (129, 100), (257, 300), (700, 1000)])
@pytest.mark.parametrize("schedule_id", [-1, 0, 1, 2, 6])
def test_planted_ties_parity_with_oracle(n, ties, schedule_id):
    rng = np.random.default_rng(n + ties)
    D = inputs.planted_tie_matrix(rng, n, ties=ties)
    Uref, Cref = oracle.focus_and_cohesion(D)
    Dt = torch.from_numpy(D).cuda()
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(Dt, U, schedule_id=schedule_id)
    binding.pald_cohesion(Dt, U, C, schedule_id=schedule_id)
    torch.cuda.synchronize()
    U, C = U.cpu().numpy(), C.cpu().numpy().astype(np.float64)
    assert np.array_equal(U, Uref)
    nz = Cref != 0
    assert np.all(C[~nz] == 0)
    rel = np.abs(C[nz] - Cref[nz]) / Cref[nz]
    assert rel.max() <= 2e-7, f"max relative error {rel.max():.3e}"


def test_no_kernel_gave_up_a_wait():
    # every bounded device-side wait of the runs above completed in time
    assert binding.pald_check_faults() == 0
