"""CUDA path against the FP64 CPU oracle, element by element.

u must match bit for bit.  C must satisfy |c - c_ref| <= 2e-7 * |c_ref| per
entry, and c == 0 exactly wherever c_ref == 0.  Every call goes through the
C ABI (via the ctypes binding); the oracle computes its own u from the same
FP32 bytes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import PALD_ACCUM_PLAIN, PaldError, binding, build, inputs

pytestmark = pytest.mark.gpu

C_RTOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def run_gpu(D_np, schedule_id=-1, accum_mode=0):
    D = torch.from_numpy(D_np).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U, schedule_id=schedule_id)
    binding.pald_cohesion(D, U, C, schedule_id=schedule_id, accum_mode=accum_mode)
    torch.cuda.synchronize()
    return U.cpu().numpy(), C.cpu().numpy()


def rel_errors(C, Cref):
    Cref = np.asarray(Cref, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    nz = Cref != 0
    rel = np.abs(C[nz] - Cref[nz]) / Cref[nz]
    return rel, nz


def assert_parity(U, C, Uref, Cref, rtol=C_RTOL):
    assert np.array_equal(U, Uref), f"u mismatch at {np.argwhere(U != Uref)[:5].tolist()}"
    rel, nz = rel_errors(C, Cref)
    assert np.all(C[~nz] == 0), "c must be exactly 0 where the oracle's is 0"
    assert rel.size == 0 or rel.max() <= rtol, f"max relative error {rel.max():.3e} > {rtol}"
    return (float(rel.max()) if rel.size else 0.0, float(rel.mean()) if rel.size else 0.0)


# ---------------------------------------------------------------------------
# small and ragged sizes, both schedules, ties and duplicate points


@pytest.mark.parametrize("n", [2, 3, 4, 5, 17, 31, 33, 64, 65, 127, 129, 130, 200])
@pytest.mark.parametrize("kind", ["euclid", "tie", "dup"])
@pytest.mark.parametrize("schedule_id", list(range(8)))
def test_ragged_sizes(n, kind, schedule_id):
    rng = np.random.default_rng(n * 7 + schedule_id)
    if kind == "euclid":
        D = inputs.small_points_matrix(rng, n, dim=3)
    elif kind == "tie":
        D = inputs.small_tie_heavy(rng, n, hi=4)
    else:
        D = inputs.small_tie_heavy(rng, n, hi=3, dup=True)
    Uref, Cref = oracle.focus_and_cohesion(D)
    U, C = run_gpu(D, schedule_id)
    assert_parity(U, C, Uref, Cref)


def test_golden_cases(golden_dir):
    import os
    from tests import pald_exact as ex

    for case in ex.load_golden(os.path.join(golden_dir, "hand_worked.txt")):
        D = np.array([[float(v) for v in r] for r in case["D"]], dtype=np.float32)
        U, C = run_gpu(D)
        assert np.array_equal(U, np.array(case["u"], dtype=np.int64)), case["name"]
        expect = np.array([[float(v) for v in r] for r in case["C"]])
        rel, nz = rel_errors(C, expect)
        assert np.all(C[~nz] == 0) and (rel.size == 0 or rel.max() <= C_RTOL), case["name"]


def test_all_zero_and_all_equal():
    for D in (np.zeros((70, 70), np.float32), np.ones((70, 70), np.float32) - np.eye(70, dtype=np.float32)):
        Uref, Cref = oracle.focus_and_cohesion(D)
        U, C = run_gpu(D)
        assert_parity(U, C, Uref, Cref)


# ---------------------------------------------------------------------------
# the workloads


def test_plain_512_full_oracle():
    D = inputs.plain_matrix(512)
    Uref, Cref = oracle.focus_and_cohesion(D)
    for sched in (0, 1):
        U, C = run_gpu(D, sched)
        mx, mean = assert_parity(U, C, Uref, Cref)
        print(f"plain-512 schedule {sched}: max rel {mx:.3e} mean {mean:.3e}")


def test_tie_heavy_4096_full_oracle():
    D = inputs.tie_heavy_matrix(4096)
    Uref, Cref = oracle.focus_and_cohesion(D)
    U, C = run_gpu(D)
    mx, mean = assert_parity(U, C, Uref, Cref)
    print(f"tie-heavy-4096: max rel {mx:.3e} mean {mean:.3e}")
    # metamorphic: D -> D^2 is exact on integers <= 20 and changes no comparison
    U2, C2 = run_gpu(D * D)
    assert np.array_equal(U2, U) and np.array_equal(C2, C)


def _sample_rows(n, k, seed):
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=k, replace=False)]))
    return rows


def test_precision_16384_sampled_rows():
    D = inputs.precision_matrix(16384)
    rows = _sample_rows(16384, 48, 5)
    Ur, Cr = oracle.rows(D, rows)
    U, C = run_gpu(D)
    mx, mean = assert_parity(U[rows], C[rows], Ur, Cr)
    _, Cp = run_gpu(D, accum_mode=PALD_ACCUM_PLAIN)
    relp, _ = rel_errors(Cp[rows], Cr)
    print(f"precision-16384 compensated: max {mx:.3e} mean {mean:.3e}; plain FP32: max {relp.max():.3e} "
          f"mean {relp.mean():.3e}")
    assert relp.max() > mx  # the plain path is the worse one


def test_invariants_on_gpu_output():
    D = inputs.precision_matrix(2048)
    U, C = run_gpu(D)
    n = D.shape[0]
    off = ~np.eye(n, dtype=bool)
    assert np.array_equal(U, U.T)
    assert U[off].min() >= 2 and U[off].max() <= n
    assert np.array_equal(np.diag(U), (D <= 0).sum(axis=1))
    assert C.min() >= 0
    assert abs(C.astype(np.float64).sum() - n / 2) < 1e-5 * n
    assert C.astype(np.float64).sum(axis=1).max() <= 1 + 1e-5


# ---------------------------------------------------------------------------
# contract, resume and the host entry point


def test_validation_statuses():
    D = inputs.plain_matrix(96)

    def status(M):
        return binding.pald_validate(torch.from_numpy(np.ascontiguousarray(M)).cuda())

    assert status(D) == 0
    A = D.copy(); A[3, 7] = np.nextafter(A[3, 7], np.float32(10))
    assert status(A) == 2
    B = D.copy(); B[5, 5] = 1.0
    assert status(B) == 3
    for bad in (np.nan, np.inf, -1.0):
        E = D.copy(); E[4, 9] = E[9, 4] = bad
        assert status(E) == 4
    E = D.copy(); E[4, 9] = E[9, 4] = np.float32(-0.0)
    assert status(E) == 4
    E = D.copy(); E[4, 9] = E[9, 4] = np.float32(2.0 ** -110)
    assert status(E) == 4
    Dt = torch.from_numpy(A).cuda()
    U = torch.empty_like(Dt, dtype=torch.int32)
    with pytest.raises(PaldError):
        binding.pald_focus(Dt, U, validate=True)


def test_resume_from_saved_u():
    D = inputs.tie_heavy_matrix(300, hi=9)
    Dg = torch.from_numpy(D).cuda()
    U = torch.empty((300, 300), dtype=torch.int32, device="cuda")
    binding.pald_focus(Dg, U)
    saved = U.cpu().numpy().copy()
    C1 = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    binding.pald_cohesion(Dg, U, C1)
    U2 = torch.from_numpy(saved).cuda()
    C2 = torch.empty_like(C1)
    binding.pald_cohesion(Dg, U2, C2)
    assert torch.equal(C1, C2)


def test_host_entry_point_matches_device_path():
    D = inputs.plain_matrix(300)
    Uh = np.empty((300, 300), np.int32)
    Ch = np.empty((300, 300), np.float32)
    binding.pald_host(D, Uh, Ch)
    U, C = run_gpu(D)
    assert np.array_equal(Uh, U) and np.array_equal(Ch, C)


def test_misaligned_buffers_take_the_copy_path():
    # TMA needs 16-byte aligned bases; views offset by one float fall back to
    # the same tiles staged with per-thread copies, with identical bits
    n = 256
    D_np = inputs.small_points_matrix(np.random.default_rng(4), n, dim=3)
    Uref, Cref = oracle.focus_and_cohesion(D_np)

    def views(dtype):
        base = torch.zeros(n * n + 4, dtype=dtype, device="cuda")
        return base[1:1 + n * n].view(n, n)

    D = views(torch.float32)
    D.copy_(torch.from_numpy(D_np).cuda())
    U, C = views(torch.int32), views(torch.float32)
    assert D.data_ptr() % 16 != 0
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    Ua, Ca = run_gpu(D_np)
    torch.cuda.synchronize()
    assert np.array_equal(U.cpu().numpy(), Ua)
    assert np.array_equal(C.cpu().numpy(), Ca)
    assert_parity(U.cpu().numpy(), C.cpu().numpy(), Uref, Cref)
