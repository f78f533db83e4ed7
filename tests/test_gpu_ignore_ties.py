"""The opt-in inexact mode PALD_FLAG_IGNORE_TIES (the paper's tie-free formulas).

Pass 2 then credits z to x only when d_xz < min(d_xy, d_zy).  It must equal
the exact result bit for bit when no row of D repeats a value, and the
strict formula (checked here in float64 numpy) when rows do.
"""
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


def _distinct_matrix(n, seed):
    # every off-diagonal value distinct: no row repeats a value
    rng = np.random.default_rng(seed)
    m = n * (n - 1) // 2
    vals = (np.uint32(0x3F800000) + rng.permutation(m).astype(np.uint32)).view(np.float32)
    D = np.zeros((n, n), np.float32)
    D[np.triu_indices(n, 1)] = vals
    return D + D.T


def _run(D_np, ignore_ties, schedule_id=-1):
    D = torch.from_numpy(D_np).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U, schedule_id=schedule_id)
    binding.pald_cohesion(D, U, C, schedule_id=schedule_id, ignore_ties=ignore_ties)
    torch.cuda.synchronize()
    return U.cpu().numpy(), C.cpu().numpy()


def strict_cohesion(D, U):
    """c_xz = 1/(n-1) sum_{y != x} [d_xz < d_xy][d_xz < d_zy] / u_xy in float64."""
    n = D.shape[0]
    D = D.astype(np.float64)
    R = 1.0 / U.astype(np.float64)
    np.fill_diagonal(R, 0.0)
    C = np.zeros((n, n))
    for y in range(n):
        a1 = D[:, y][:, None]  # d_xy
        a2 = D[:, y][None, :]  # d_zy
        C += ((D < a1) & (D < a2)) * R[:, y][:, None]
    return C / (n - 1)


@pytest.mark.parametrize("n,schedule_id", [(300, -1), (1024, -1), (1024, 3), (200, 1)])
def test_ignore_ties_equals_exact_without_repeats(n, schedule_id):
    D = _distinct_matrix(n, n)
    U0, C0 = _run(D, False, schedule_id)
    U1, C1 = _run(D, True, schedule_id)
    assert np.array_equal(U0, U1) and np.array_equal(C0, C1)


@pytest.mark.parametrize("kind", ["tie", "dup", "plain"])
def test_ignore_ties_is_the_strict_formula(kind):
    rng = np.random.default_rng(17)
    D = {"tie": lambda: inputs.small_tie_heavy(rng, 160, hi=4),
         "dup": lambda: inputs.small_tie_heavy(rng, 131, hi=3, dup=True),
         "plain": lambda: inputs.plain_matrix(256)}[kind]()
    U, C = _run(D, True)
    Uref, Cexact = oracle.focus_and_cohesion(D)
    assert np.array_equal(U, Uref)  # pass 1 stays exact
    Cref = strict_cohesion(D, Uref)
    nz = Cref != 0
    assert np.all(C[~nz] == 0)
    rel = np.abs(C[nz].astype(np.float64) - Cref[nz]) / Cref[nz]
    assert rel.max() <= 2e-7, f"max relative error {rel.max():.3e}"
    if kind != "plain":
        assert not np.allclose(Cref, Cexact)  # ties matter here: the mode is inexact


def test_batched_ignore_ties_matches_single_path():
    rng = np.random.default_rng(2)
    ns = np.array([40, 97, 130, 64], dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    mats = [inputs.small_tie_heavy(rng, int(n), hi=4) for n in ns]
    for o, n, M in zip(offs, ns, mats):
        Dh[o:o + n * n] = M.ravel()
    D = torch.from_numpy(Dh).cuda()
    U = torch.zeros(total, dtype=torch.int32, device="cuda")
    C = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U, C, ignore_ties=True)
    torch.cuda.synchronize()
    Ch = C.cpu().numpy()
    for o, n, M in zip(offs, ns, mats):
        _, Cs = _run(M, True)
        assert np.array_equal(Ch[o:o + n * n].reshape(n, n), Cs)
    binding.pald_release()
