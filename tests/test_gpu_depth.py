"""Local depths (row sums of C, Sec. 2 eq. (LD)) and the strong-tie mask."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs
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
