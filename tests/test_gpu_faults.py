"""The give-up path of the bounded device-side waits, run for real.

Every mbarrier wait of the pass kernels gives up after a time limit, records
a fault word and lets its CTA stop instead of hanging the GPU.  Here one CTA
runs the same TMA pipeline with no copy ever issued, so its waits run out
after one millisecond; nothing faults and the context stays usable.  The
test checks that the fault reaches the host exactly once through
pald_check_faults, and that the passes still run correctly afterwards.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

PALD_OK, PALD_ERR_INVALID_ARG, PALD_ERR_TIMEOUT = 0, 1, 7


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def test_a_wait_that_runs_out_is_reported_once():
    assert binding.pald_check_faults() == PALD_OK  # nothing pending from earlier work
    binding.pald_test_bounded_wait(1_000_000)      # 1 ms limit
    assert binding.pald_check_faults() == PALD_ERR_TIMEOUT
    assert binding.pald_check_faults() == PALD_OK  # the record was cleared
    # the context is still usable: a small matrix still matches the oracle
    D_np = inputs.plain_matrix(192)
    D = torch.from_numpy(D_np).cuda()
    U = torch.empty((192, 192), dtype=torch.int32, device="cuda")
    C = torch.empty((192, 192), dtype=torch.float32, device="cuda")
    binding.pald_focus(D, U)
    binding.pald_cohesion(D, U, C)
    torch.cuda.synchronize()
    Ur, Cr = oracle.focus_and_cohesion(D_np)
    assert np.array_equal(U.cpu().numpy(), Ur)
    rel = np.abs(C.cpu().numpy().astype(np.float64) - Cr)[Cr != 0] / Cr[Cr != 0]
    assert rel.max() <= 2e-7
    assert binding.pald_check_faults() == PALD_OK


def test_limit_out_of_range_is_rejected():
    lib = binding.lib()
    assert lib.pald_test_bounded_wait(10, None) == PALD_ERR_INVALID_ARG
    assert lib.pald_test_bounded_wait(3_000_000_000, None) == PALD_ERR_INVALID_ARG
