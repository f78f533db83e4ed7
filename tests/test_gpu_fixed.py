"""Fixed-point cohesion (PALD_ACCUM_FIXED): exact integer sums of the
weights round(2^40 / u), so the result does not depend on the order of the
terms.  Checked against the FP64 oracle (2e-7, exact zeros); permuting the
points permutes C bit for bit (which the compensated mode only does within
rounding); tile ranges and the batched path give the same bits; the
precision-study matrix on sampled rows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import PALD_ACCUM_FIXED, binding, build, inputs, shard

pytestmark = pytest.mark.gpu
C_RTOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def _fixed(D_np_or_t):
    D = D_np_or_t if isinstance(D_np_or_t, torch.Tensor) else torch.from_numpy(D_np_or_t).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C, accum_mode=PALD_ACCUM_FIXED)
    torch.cuda.synchronize()
    assert binding.pald_check_faults() == 0
    return U, C


def _check(C, Cr):
    C = np.asarray(C, np.float64)
    nz = Cr != 0
    assert np.all(C[~nz] == 0), "c must be exactly 0 where the oracle's is 0"
    rel = np.abs(C[nz] - Cr[nz]) / Cr[nz]
    assert rel.max() <= C_RTOL, f"max relative error {rel.max():.3e}"
    return float(rel.max()), float(rel.mean())


def _matrix(kind, n, rng):
    if kind == "plain":
        return inputs.plain_matrix(n)
    if kind == "tie":
        return inputs.tie_heavy_matrix(n, hi=9)
    if kind == "dup":
        return inputs.small_tie_heavy(rng, n, hi=5, dup=True)
    return inputs.planted_tie_matrix(rng, n, ties=3 * n)


@pytest.mark.parametrize("n", [2, 3, 5, 64, 65, 130, 257])
@pytest.mark.parametrize("kind", ["plain", "tie", "dup", "planted"])
def test_fixed_against_oracle(n, kind):
    rng = np.random.default_rng(100 + n)
    D_np = _matrix(kind, n, rng)
    U, C = _fixed(D_np)
    Ur, Cr = oracle.focus_and_cohesion(D_np)
    assert np.array_equal(U.cpu().numpy(), Ur)
    _check(C.cpu().numpy(), Cr)


@pytest.mark.parametrize("n,kind", [(300, "plain"), (1027, "tie"), (513, "planted")])
def test_permuting_points_permutes_c_bit_for_bit(n, kind):
    rng = np.random.default_rng(n)
    D_np = _matrix(kind, n, rng)
    perm = rng.permutation(n)
    _, C = _fixed(D_np)
    _, Cp = _fixed(np.ascontiguousarray(D_np[np.ix_(perm, perm)]))
    assert torch.equal(Cp, C[perm][:, perm]), "fixed-point sums must not depend on the order of the terms"


def test_tile_ranges_and_batched_give_the_same_bits():
    n = 517
    D_np = inputs.tie_heavy_matrix(n, hi=11)
    D = torch.from_numpy(D_np).cuda()
    U, C = _fixed(D)
    # tiles split over three ranks, one after another on this GPU
    C3 = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
    for r in range(3):
        t0, t1 = binding.pald_shard_range(n, r, 3)
        binding.pald_cohesion_tiles(D, U, C3, t0, t1, accum_mode=PALD_ACCUM_FIXED)
    torch.cuda.synchronize()
    assert torch.equal(C3, C)
    # batched (matrix by matrix through the same path)
    rng = np.random.default_rng(5)
    ns = np.array([n, 70, 33], dtype=np.int64)
    mats = [D_np, inputs.small_points_matrix(rng, 70), inputs.small_tie_heavy(rng, 33, hi=4)]
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    for o, M in zip(offs, mats):
        Dh[o:o + M.size] = M.ravel()
    Db = torch.from_numpy(Dh).cuda()
    Ub = torch.zeros(total, dtype=torch.int32, device="cuda")
    Cb = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, Db, Ub, Cb, accum_mode=PALD_ACCUM_FIXED)
    torch.cuda.synchronize()
    for o, k, M in zip(offs, ns, mats):
        _, Ci = _fixed(M)
        assert torch.equal(Cb[o:o + k * k].view(k, k), Ci)


def test_modes_without_fixed_point_reject_it():
    n = 64
    D = torch.from_numpy(inputs.plain_matrix(n)).cuda()
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    with pytest.raises(binding.PaldError):
        binding.pald_pairwise(D, C, accum_mode=PALD_ACCUM_FIXED)
    with pytest.raises(binding.PaldError):
        binding.pald_cohesion_noalloc(D, U, C, accum_mode=PALD_ACCUM_FIXED)


def test_precision_16384_fixed_sampled_rows():
    n = 16384
    D = inputs.euclidean_fp32_torch(inputs.precision_points(n), "cuda")
    U, C = _fixed(D)
    rng = np.random.default_rng(16384)
    rows = np.unique(np.concatenate([[0, n - 1], rng.choice(n, size=30, replace=False)]))
    Ur, Cr = oracle.rows(D.cpu().numpy(), rows)
    idx = torch.from_numpy(rows).cuda()
    assert np.array_equal(U[idx].cpu().numpy(), Ur)
    mx, mean = _check(C[idx].cpu().numpy(), Cr)
    print(f"precision-16384 fixed point, {len(rows)} rows: max rel {mx:.3e} mean rel {mean:.3e}")
