"""Schedule tables on the GPU: a table set by the caller is the one in force,
the passes follow it with unchanged bits, and the batched path gives the
same bits with and without the diagonal split in every bucket."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()
    yield
    binding.pald_set_schedule_table([])
    binding.pald_release()


def _run(D):
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    return U, C


def test_caller_table_is_in_force_and_keeps_the_bits():
    binding.pald_set_schedule_table([])
    D = torch.from_numpy(inputs.plain_matrix(1100)).cuda()
    U0, C0 = _run(D)
    table = [(600, 0, 2, 0), (1 << 20, 4, 6, 1)]
    binding.pald_set_schedule_table(table)
    got = binding.pald_get_schedule(1100)
    assert got["source"] == "set by the caller"
    assert (got["focus"], got["cohesion"], got["batched_split"]) == (4, 6, 1)
    assert binding.pald_get_schedule(300)["focus"] == 0
    U1, C1 = _run(D)
    assert torch.equal(U0, U1) and torch.equal(C0, C1)
    binding.pald_set_schedule_table([])
    assert binding.pald_get_schedule(1100)["source"] in ("built-in defaults", "tuned table")


@pytest.mark.parametrize("kind", ["euclid", "tie"])
def test_batched_split_choice_keeps_the_bits(kind):
    rng = np.random.default_rng(11)
    ns = np.array([3, 5, 31, 64, 65, 70, 128, 131, 200, 257, 300], dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    mats = []
    for o, n in zip(offs, ns):
        M = inputs.small_points_matrix(rng, int(n), dim=3) if kind == "euclid" else \
            inputs.small_tie_heavy(rng, int(n), hi=6)
        Dh[o:o + M.size] = M.ravel()
        mats.append(M)
    D = torch.from_numpy(Dh).cuda()
    out = {}
    for split in (0, 1):
        binding.pald_set_schedule_table([(1 << 20, 1, 1, split)])
        U = torch.zeros(total, dtype=torch.int32, device="cuda")
        C = torch.zeros(total, dtype=torch.float32, device="cuda")
        binding.pald_batched(ns, offs, D, U, C)
        torch.cuda.synchronize()
        assert binding.pald_check_faults() == 0
        out[split] = (U.cpu().numpy(), C.cpu().numpy())
    binding.pald_set_schedule_table([])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    Uh, Ch = out[0]
    for o, n, M in zip(offs, ns, mats):
        Ur, Cr = oracle.focus_and_cohesion(M)
        sl = slice(int(o), int(o) + int(n) * int(n))
        assert np.array_equal(Uh[sl].reshape(n, n), Ur)
        Cg = Ch[sl].reshape(n, n).astype(np.float64)
        nz = Cr != 0
        assert np.all(Cg[~nz] == 0)
        assert (np.abs(Cg[nz] - Cr[nz]) / Cr[nz]).max() <= 2e-7
