"""Local depths (row sums of C, Sec. 2 eq. (LD)) and the strong-tie mask."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import PALD_ACCUM_FIXED, binding, build, inputs
from tests import pald_exact as ex

pytestmark = pytest.mark.gpu

L_RTOL = 3e-7  # the entries carry at most 2e-7 each; the sum adds one rounding


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def _gpu_C(D_np):
    D = torch.from_numpy(D_np).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    return C


@pytest.mark.parametrize("kind", ["plain512", "tie300", "dup130", "two"])
def test_local_depth_against_oracle_row_sums(kind):
    rng = np.random.default_rng(9)
    D = {"plain512": lambda: inputs.plain_matrix(512), "tie300": lambda: inputs.small_tie_heavy(rng, 300, hi=5),
         "dup130": lambda: inputs.small_tie_heavy(rng, 130, hi=3, dup=True),
         "two": lambda: np.array([[0, 1], [1, 0]], dtype=np.float32)}[kind]()
    _, Cref = oracle.focus_and_cohesion(D)
    Lref = Cref.sum(axis=1)
    L = binding.pald_local_depth(_gpu_C(D)).cpu().numpy().astype(np.float64)
    rel = np.abs(L - Lref) / Lref
    assert rel.max() <= L_RTOL, f"max relative error {rel.max():.3e}"
    assert np.all((L >= 0) & (L <= 1))


def test_local_depth_is_eq_LD_on_tiny_inputs():
    # the probability of eq. (LD), enumerated exactly, against the GPU's row sums
    rng = np.random.default_rng(21)
    for trial in range(12):
        n = int(rng.integers(2, 8))
        D = inputs.small_tie_heavy(rng, n, hi=3) if trial % 2 else inputs.small_points_matrix(rng, n, dim=2)
        L = binding.pald_local_depth(_gpu_C(D)).cpu().numpy().astype(np.float64)
        Dl = D.astype(np.float64).tolist()  # exact values for the rational enumeration
        exact = np.array([float(ex.local_depth_exact(Dl, x)) for x in range(n)])
        assert np.allclose(L, exact, rtol=L_RTOL, atol=0), (n, L, exact)


def test_local_depth_is_deterministic():
    C = _gpu_C(inputs.euclidean_fp32(inputs.precision_points(16384)[:3000]))
    a = binding.pald_local_depth(C).clone()
    b = binding.pald_local_depth(C)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_strong_ties_mask():
    C = _gpu_C(inputs.plain_matrix(512))
    Ch = C.cpu().numpy()
    diag_half = float(np.mean(np.diag(Ch))) / 2
    for tau in (0.0, diag_half, float(Ch.max()), float(Ch.max()) * 2, float(np.median(Ch[Ch > 0]))):
        T = binding.pald_strong_ties(C, tau)
        torch.cuda.synchronize()
        assert np.array_equal(T.cpu().numpy(), (Ch >= np.float32(tau)).astype(np.uint8)), tau


# ---------------------------------------------------------------------------
# pald_cohesion_depth: the row sums taken in pass 2's epilogue (eq. (LD) as
# the partition of local depth), against the oracle's row sums and against
# pald_local_depth on the same C.

def _ulps(a, b):
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    return np.abs(a.view(np.int32).astype(np.int64) - b.view(np.int32).astype(np.int64))


def _fused(D, **kw):
    D = D if isinstance(D, torch.Tensor) else torch.from_numpy(D).cuda()
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    C1 = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_cohesion(D, U, C1, **kw)
    C2 = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
    L = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    binding.pald_cohesion_depth(D, U, C2, L, **kw)
    torch.cuda.synchronize()
    assert binding.pald_check_faults() == 0
    assert torch.equal(C1, C2), "the fused call must store the same C"
    return C2, L


@pytest.mark.parametrize("n,kind", [(64, "plain"), (68, "tie"), (256, "plain"), (516, "tie"), (1000, "planted"),
                                    (1028, "plain"), (2052, "tie")])
def test_fused_depth_against_oracle_row_sums(n, kind):
    rng = np.random.default_rng(n)
    D = {"plain": lambda: inputs.plain_matrix(n), "tie": lambda: inputs.tie_heavy_matrix(n, hi=7),
         "planted": lambda: inputs.planted_tie_matrix(rng, n, ties=3 * n)}[kind]()
    C, L = _fused(D)
    _, Cref = oracle.focus_and_cohesion(D)
    Lref = Cref.sum(axis=1)
    Lg = L.cpu().numpy().astype(np.float64)
    rel = np.abs(Lg - Lref) / Lref
    assert rel.max() <= L_RTOL, f"max relative error {rel.max():.3e}"
    # both are the sum of the same stored entries, rounded once
    assert _ulps(L.cpu().numpy(), binding.pald_local_depth(C).cpu().numpy()).max() <= 1
    assert abs(Lg.sum() - n / 2) <= 1e-6 * n  # the entries of C add up to n / 2


@pytest.mark.parametrize("case", ["ragged130", "fixed", "schedule3", "ignore_ties"])
def test_fused_depth_other_paths(case):
    n = 130 if case == "ragged130" else 512
    D = inputs.tie_heavy_matrix(n, hi=5)
    kw = {"ragged130": {}, "fixed": {"accum_mode": PALD_ACCUM_FIXED}, "schedule3": {"schedule_id": 3},
          "ignore_ties": {"ignore_ties": True}}[case]
    C, L = _fused(D, **kw)
    Lsep = binding.pald_local_depth(C)
    torch.cuda.synchronize()
    if case == "ignore_ties":  # fused (TMA layout), only the tie map is empty
        assert _ulps(L.cpu().numpy(), Lsep.cpu().numpy()).max() <= 1
    else:  # separate pass over C: the same call as pald_local_depth
        assert torch.equal(L, Lsep)


def test_fused_depth_paper_8192_sampled_rows():
    n = 8192
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    C, L = _fused(D)
    Lsep = binding.pald_local_depth(C)
    torch.cuda.synchronize()
    d = _ulps(L.cpu().numpy(), Lsep.cpu().numpy())
    assert d.max() <= 1, f"{int((d > 0).sum())} rows differ, max {int(d.max())} ulp"
    rows = np.unique(np.concatenate([[0, 63, 64, n - 1], np.random.default_rng(3).choice(n, 12, replace=False)]))
    _, Cr = oracle.rows(D.cpu().numpy(), rows)
    Lg = L.cpu().numpy()[rows].astype(np.float64)
    rel = np.abs(Lg - Cr.sum(axis=1)) / Cr.sum(axis=1)
    assert rel.max() <= L_RTOL, f"max relative error {rel.max():.3e}"
    assert abs(float(L.double().sum()) - n / 2) <= 1e-6 * n


def test_fused_depth_is_deterministic():
    D = torch.from_numpy(inputs.tie_heavy_matrix(1024, hi=9)).cuda()
    _, a = _fused(D)
    _, b = _fused(D)
    assert torch.equal(a, b)
