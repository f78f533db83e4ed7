"""The pairwise variant (pald_pairwise: both passes per strip of rows, u never
stored) against the two-pass path bit for bit and against the oracle, on
ragged sizes (strips that end inside a tile, orders not a multiple of 4),
tie-heavy matrices (the long form), duplicate points and the plain
accumulation; a large order checked on sampled rows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import PALD_ACCUM_PLAIN, binding, build, inputs

pytestmark = pytest.mark.gpu
C_RTOL = 2e-7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def _two_pass(D, **kw):
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C, **kw)
    return C


def _pairwise(D, **kw):
    n = D.shape[0]
    C = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
    binding.pald_pairwise(D, C, **kw)
    torch.cuda.synchronize()
    assert binding.pald_check_faults() == 0
    return C


def _matrix(kind, n, rng):
    if kind == "plain":
        return inputs.plain_matrix(n)
    if kind == "tie":
        return inputs.tie_heavy_matrix(n, hi=9)
    if kind == "dup":
        return inputs.small_tie_heavy(rng, n, hi=5, dup=True)
    return inputs.planted_tie_matrix(rng, n, ties=3 * n)


@pytest.mark.parametrize("n", [2, 3, 5, 64, 65, 130, 255, 256, 257, 300, 513])
@pytest.mark.parametrize("kind", ["plain", "tie", "dup", "planted"])
def test_pairwise_equals_two_pass_and_oracle(n, kind):
    rng = np.random.default_rng(n)
    D_np = _matrix(kind, n, rng)
    D = torch.from_numpy(D_np).cuda()
    C = _pairwise(D)
    assert torch.equal(C, _two_pass(D)), "not the two-pass bits"
    if n <= 300:
        _, Cr = oracle.focus_and_cohesion(D_np)
        Cg = C.cpu().numpy().astype(np.float64)
        nz = Cr != 0
        assert np.all(Cg[~nz] == 0)
        assert (np.abs(Cg[nz] - Cr[nz]) / Cr[nz]).max() <= C_RTOL


@pytest.mark.parametrize("n", [200, 1027])
def test_pairwise_plain_accumulation_and_ignore_ties(n):
    D = torch.from_numpy(inputs.tie_heavy_matrix(n, hi=12)).cuda()
    assert torch.equal(_pairwise(D, accum_mode=PALD_ACCUM_PLAIN), _two_pass(D, accum_mode=PALD_ACCUM_PLAIN))
    assert torch.equal(_pairwise(D, ignore_ties=True), _two_pass(D, ignore_ties=True))


def test_pairwise_scratch_is_small():
    # strip buffer (256 x n floats) + the tie map: a few percent of the 8 n^2
    # bytes that U and R take on the two-pass path
    for n in (8192, 65536, 147456):
        assert binding.pald_pairwise_scratch_bytes(n) < 0.04 * 8 * n * n, n
    assert binding.pald_pairwise_scratch_bytes(1) == 0


def test_pairwise_paper_8192_sampled_rows():
    n = 8192
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    C = _pairwise(D)
    assert torch.equal(C, _two_pass(D))
    rows = np.array([0, 1, 4095, 8191])
    _, Cr = oracle.rows(D.cpu().numpy(), rows)
    Cg = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    nz = Cr != 0
    assert np.all(Cg[~nz] == 0)
    assert (np.abs(Cg[nz] - Cr[nz]) / Cr[nz]).max() <= C_RTOL
