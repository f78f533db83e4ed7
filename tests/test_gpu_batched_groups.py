"""Diagonal tiles of the TMA tile code and the pairs inside groups of four.

A diagonal 64 x 64 TMA tile (the batched kernels, and schedule 7 of
single-matrix pass 1) runs only its 4 x 4 blocks above the diagonal on four
warps.  The pairs inside each group of four points go, in pass 1, to the
tile's other four warps and, in batched pass 2, to a kernel with one thread
per group.  Every order class that changes that split (n <= 4: group pairs
only; n % 4 != 0: a ragged last group read from the padded copies; n % 64 in
1..4: a last diagonal tile with nothing above its diagonal; dirty tie-map
blocks: the long form throughout) is checked bit for bit against tiles
without the split (the 32-wide schedule 1, and schedules 2 and 3 with
per-thread copies), in both accumulation modes and in the ignore-ties mode,
and against the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

C_RTOL = 2e-7
SIZES = [2, 3, 4, 5, 6, 7, 8, 9, 31, 32, 33, 63, 64, 65, 66, 67, 68, 69, 70, 127, 128, 129, 130, 131, 191, 193,
         255, 257, 301, 700]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()
    yield
    binding.pald_release()


def _matrices(kind, seed):
    rng = np.random.default_rng(seed)
    make = {
        "points": lambda n: inputs.small_points_matrix(rng, n, dim=3),
        "tie": lambda n: inputs.small_tie_heavy(rng, n, hi=4),  # n = 700 has dirty rows (long form)
        "dup": lambda n: inputs.small_tie_heavy(rng, n, hi=3, dup=True),
        "planted": lambda n: inputs.planted_tie_matrix(rng, n, ties=max(1, n // 8)) if n >= 8
        else inputs.small_points_matrix(rng, n, dim=2),
    }[kind]
    return [make(n) for n in SIZES]


def _batched(mats, **kw):
    ns = np.array([m.shape[0] for m in mats], dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    for o, M in zip(offs, mats):
        Dh[o:o + M.size] = M.ravel()
    D = torch.from_numpy(Dh).cuda()
    U = torch.zeros(total, dtype=torch.int32, device="cuda")
    C = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U, C, **kw)
    binding.pald_batched(ns, offs, D, U, C, **kw)  # replay of the cached graph
    torch.cuda.synchronize()
    Uh, Ch = U.cpu().numpy(), C.cpu().numpy()
    out = []
    for o, M in zip(offs, mats):
        n = M.shape[0]
        out.append((Uh[o:o + n * n].reshape(n, n), Ch[o:o + n * n].reshape(n, n)))
    return out


def _single(M, **kw):
    n = M.shape[0]
    D = torch.from_numpy(M).cuda()
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C, **kw)
    torch.cuda.synchronize()
    return U.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("accum", [binding.PALD_ACCUM_COMPENSATED, binding.PALD_ACCUM_PLAIN])
@pytest.mark.parametrize("kind", ["points", "tie", "dup", "planted"])
def test_batched_split_matches_single_path(kind, accum):
    mats = _matrices(kind, 11 + accum)
    got = _batched(mats, accum_mode=accum)
    for M, (Ub, Cb) in zip(mats, got):
        Us, Cs = _single(M, accum_mode=accum)
        n = M.shape[0]
        assert np.array_equal(Ub, Us), f"{kind} n={n}: u"
        assert np.array_equal(Cb, Cs), f"{kind} n={n}: C"
    assert binding.pald_check_faults() == 0


@pytest.mark.parametrize("kind", ["points", "tie", "dup"])
def test_batched_split_against_oracle(kind):
    mats = _matrices(kind, 23)
    got = _batched(mats)
    for M, (Ub, Cb) in zip(mats, got):
        if M.shape[0] > 301:
            continue
        Ur, Cr = oracle.focus_and_cohesion(M)
        assert np.array_equal(Ub, Ur)
        Cr = np.asarray(Cr, np.float64)
        nz = Cr != 0
        assert np.all(Cb[~nz] == 0)
        rel = np.abs(Cb[nz].astype(np.float64) - Cr[nz]) / Cr[nz]
        assert rel.max() <= C_RTOL, f"{kind} n={M.shape[0]}: max relative error {rel.max():.3e}"


@pytest.mark.parametrize("kind", ["tie", "dup"])
def test_batched_split_ignore_ties_matches_single_path(kind):
    mats = _matrices(kind, 31)
    got = _batched(mats, ignore_ties=True)
    for M, (Ub, Cb) in zip(mats, got):
        Us, Cs = _single(M, ignore_ties=True)
        assert np.array_equal(Ub, Us) and np.array_equal(Cb, Cs), f"{kind} n={M.shape[0]}"


@pytest.mark.parametrize("kind", ["points", "tie", "planted"])
@pytest.mark.parametrize("n", [64, 68, 132, 260, 1024, 1092])
def test_schedule_7_split_matches_unsplit_schedules(kind, n):
    rng = np.random.default_rng(n)
    M = {"points": lambda: inputs.small_points_matrix(rng, n, dim=3),
         "tie": lambda: inputs.small_tie_heavy(rng, n, hi=4),
         "planted": lambda: inputs.planted_tie_matrix(rng, n, ties=n // 4)}[kind]()
    D = torch.from_numpy(M).cuda()
    out = {}
    for sf, sc in ((7, 7), (2, 3), (1, 1)):
        U = torch.empty((n, n), dtype=torch.int32, device="cuda")
        C = torch.empty((n, n), dtype=torch.float32, device="cuda")
        binding.pald_focus(D, U, schedule_id=sf)
        binding.pald_cohesion(D, U, C, schedule_id=sc)
        torch.cuda.synchronize()
        out[sc] = (U.cpu().numpy(), C.cpu().numpy())
    for sc in (3, 1):
        assert np.array_equal(out[7][0], out[sc][0]), f"u: schedule 7 vs {sc}"
        assert np.array_equal(out[7][1], out[sc][1]), f"C: schedule 7 vs {sc}"
    assert binding.pald_check_faults() == 0
