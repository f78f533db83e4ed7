"""Full-size workloads on the GPU: the n = 65536 matrix (sampled rows against
the oracle, global invariants on everything) and the batched workload (2000
matrices, one graph replay, every matrix against the full oracle and against
the single-matrix path)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
C_RTOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def check_rows(U_rows, C_rows, Ur, Cr):
    assert np.array_equal(U_rows, Ur)
    Cr = np.asarray(Cr, np.float64)
    C_rows = np.asarray(C_rows, np.float64)
    nz = Cr != 0
    assert np.all(C_rows[~nz] == 0)
    rel = np.abs(C_rows[nz] - Cr[nz]) / Cr[nz]
    assert rel.max() <= C_RTOL, f"max relative error {rel.max():.3e}"
    return rel.max(), rel.mean()


def test_paper_65536_sampled_rows_and_invariants():
    n = 65536
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    rng = np.random.default_rng(65536)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=14, replace=False)]))
    Dh = D.cpu().numpy()
    Ur, Cr = oracle.rows(Dh, rows)
    idx = torch.from_numpy(rows).cuda()
    mx, mean = check_rows(U[idx].cpu().numpy(), C[idx].cpu().numpy(), Ur, Cr)
    print(f"paper-65536 sampled {len(rows)} rows: max rel {mx:.3e} mean {mean:.3e}")
    del Dh
    # invariants on the whole output, block by block on the device
    blk = 4096
    total = torch.zeros((), dtype=torch.float64, device="cuda")
    for r0 in range(0, n, blk):
        Ub = U[r0:r0 + blk]
        assert torch.equal(Ub, U[:, r0:r0 + blk].transpose(0, 1))
        off = Ub.clone()
        ar = torch.arange(min(blk, n - r0), device="cuda")
        off[ar, ar + r0] = n  # ignore the diagonal below
        assert int(off.min()) >= 2 and int(Ub.max()) <= n
        Cb = C[r0:r0 + blk]
        assert float(Cb.min()) >= 0.0
        total += Cb.double().sum()
    assert abs(float(total) - n / 2) < 1e-6 * n


def test_past_the_fine_tie_map_order_sampled_rows():
    # beyond n = 65536 the tie map has groups of 32 y (one per stage); n % 64
    # == 4 leaves a ragged last tile row and column
    n = 65540
    nb = -(-n // 64)
    assert binding.pald_tie_map_words(n) == nb * nb * (-(-(-(-n // 32)) // 32)) + nb
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    assert binding.pald_check_faults() == 0
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([[0, 65536, n - 1], rng.choice(n, size=5, replace=False)]))
    Ur, Cr = oracle.rows(D.cpu().numpy(), rows)
    idx = torch.from_numpy(rows).cuda()
    mx, mean = check_rows(U[idx].cpu().numpy(), C[idx].cpu().numpy(), Ur, Cr)
    print(f"n={n} (coarse tie map) sampled {len(rows)} rows: max rel {mx:.3e} mean {mean:.3e}")


def _batched_inputs(count):
    ns = inputs.batched_sizes(count)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    mats = []
    for i, n, Di in inputs.batched_matrices(count):
        Dh[offs[i]:offs[i] + n * n] = Di.ravel()
        mats.append(Di)
    return ns, offs, total, Dh, mats


def test_batched_against_oracle_and_single_path():
    count = 2000
    ns, offs, total, Dh, mats = _batched_inputs(count)
    D = torch.from_numpy(Dh).cuda()
    U = torch.zeros(total, dtype=torch.int32, device="cuda")
    C = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U, C)
    binding.pald_batched(ns, offs, D, U, C)  # second call replays the cached graph
    torch.cuda.synchronize()
    Uh, Chh = U.cpu().numpy(), C.cpu().numpy()
    # every matrix against the single-matrix kernels: u and C bit for bit
    for i in range(count):
        n = int(ns[i])
        Di = torch.from_numpy(mats[i]).cuda()
        Ui = torch.empty((n, n), dtype=torch.int32, device="cuda")
        Ci = torch.empty((n, n), dtype=torch.float32, device="cuda")
        binding.pald_focus(Di, Ui)
        binding.pald_cohesion(Di, Ui, Ci)
        ub = Uh[offs[i]:offs[i] + n * n].reshape(n, n)
        cb = Chh[offs[i]:offs[i] + n * n].reshape(n, n)
        assert np.array_equal(ub, Ui.cpu().numpy()), f"matrix {i}"
        assert np.array_equal(cb, Ci.cpu().numpy()), f"matrix {i}"
    # every matrix against the full oracle (u exact, C within 2e-7, exact
    # zeros); the oracle's C code runs outside the GIL, one matrix per host
    # thread
    def against_oracle(i):
        n = int(ns[i])
        Ur, Cr = oracle.focus_and_cohesion(mats[i], threads=1)
        sl = slice(int(offs[i]), int(offs[i]) + n * n)
        try:
            mx, mean = check_rows(Uh[sl].reshape(n, n), Chh[sl].reshape(n, n), Ur, Cr)
        except AssertionError as err:
            raise AssertionError(f"matrix {i} (n={n}): {err}") from None
        return mx, mean, n * n

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        stats = list(ex.map(against_oracle, range(count)))
    worst = max(s[0] for s in stats)
    mean = sum(s[1] * s[2] for s in stats) / sum(s[2] for s in stats)
    print(f"batched: all {count} matrices vs the oracle, max rel {worst:.3e}, mean rel {mean:.3e}")
    binding.pald_release()


def test_batched_more_matrices_than_one_grid_dimension():
    # 70000 tiny matrices: more than a launch's y dimension holds, so the
    # per-matrix kernels stride over the grid; every matrix checked exactly
    rng = np.random.default_rng(7)
    count = 70000
    ns = rng.integers(2, 6, size=count).astype(np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    mats = []
    for i in range(count):
        n = int(ns[i])
        Di = inputs.small_tie_heavy(rng, n, hi=3) if i % 2 else inputs.small_points_matrix(rng, n, dim=2)
        Dh[offs[i]:offs[i] + n * n] = Di.ravel()
        mats.append(Di)
    D = torch.from_numpy(Dh).cuda()
    U = torch.zeros(total, dtype=torch.int32, device="cuda")
    C = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U, C)
    torch.cuda.synchronize()
    Uh, Ch = U.cpu().numpy(), C.cpu().numpy()
    for i in list(range(0, count, 997)) + [count - 1]:
        n = int(ns[i])
        Ur, Cr = oracle.focus_and_cohesion(mats[i])
        check_rows(Uh[offs[i]:offs[i] + n * n].reshape(n, n), Ch[offs[i]:offs[i] + n * n].reshape(n, n), Ur, Cr)
    binding.pald_release()
