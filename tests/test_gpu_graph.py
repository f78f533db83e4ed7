"""The graph-distance workload on the GPU: hop counts of seeded
collaboration graphs (the stand-in for the networks of Sec. 7).  Every row
repeats a handful of values thousands of times, so the tie map marks its
blocks dirty and pass 2 runs the long form throughout."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")

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
    yield
    binding.pald_release()


def _single(M):
    n = M.shape[0]
    D = torch.from_numpy(M).cuda()
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    return U.cpu().numpy(), C.cpu().numpy()


@pytest.mark.parametrize("n", [700, 1026, 1500])
def test_graph_distances_against_oracle(n):
    M = inputs.graph_matrix(n)
    U, C = _single(M)
    Ur, Cr = oracle.focus_and_cohesion(M)
    assert np.array_equal(U, Ur)
    nz = Cr != 0
    assert np.all(C[~nz] == 0)
    rel = np.abs(C[nz].astype(np.float64) - Cr[nz]) / Cr[nz]
    assert rel.max() <= C_RTOL, f"n={n}: max relative error {rel.max():.3e}"
    assert binding.pald_check_faults() == 0


def test_batched_graph_distances_match_single_path():
    mats = [inputs.graph_matrix(n, index=i) for i, n in enumerate((97, 260, 513, 1024))]
    ns = np.array([m.shape[0] for m in mats], dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    Dh = np.zeros(total, np.float32)
    for o, M in zip(offs, mats):
        Dh[o:o + M.size] = M.ravel()
    D = torch.from_numpy(Dh).cuda()
    U = torch.zeros(total, dtype=torch.int32, device="cuda")
    C = torch.zeros(total, dtype=torch.float32, device="cuda")
    binding.pald_batched(ns, offs, D, U, C)
    torch.cuda.synchronize()
    Uh, Ch = U.cpu().numpy(), C.cpu().numpy()
    for o, M in zip(offs, mats):
        k = M.shape[0]
        Us, Cs = _single(M)
        assert np.array_equal(Uh[o:o + k * k].reshape(k, k), Us), f"n={k}: u"
        assert np.array_equal(Ch[o:o + k * k].reshape(k, k), Cs), f"n={k}: C"
