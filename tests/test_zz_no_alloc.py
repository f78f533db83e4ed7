"""pald_cohesion_noalloc, the pass-2 entry point for callers that must not
allocate device memory (for example because their own pool already owns the
device memory, or because an allocation's implicit synchronisation is not
acceptable in their loop).  It keeps its scratch in a fixed array built into
the library, so it is limited to n <= 2048.

The file name makes pytest collect it last.  It must pass on its own in a
fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu

C_RTOL = 2e-7  # the tolerance of the other cohesion parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    binding.lib()


def _close(C, ref):
    C = C.double().cpu().numpy()
    ref = ref.double().cpu().numpy()
    nz = ref != 0
    assert np.all(C[~nz] == 0)
    rel = np.abs(C[nz] - ref[nz]) / ref[nz]
    assert rel.max() <= C_RTOL, f"max relative error {rel.max():.3e}"


@pytest.mark.parametrize("n,kind", [(2048, "plain"), (701, "tie")])
def test_noalloc_matches_pald_cohesion_on_two_calls(n, kind):
    D_np = inputs.plain_matrix(n) if kind == "plain" else inputs.tie_heavy_matrix(n, hi=9)
    D = torch.from_numpy(D_np).cuda()
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    ref = torch.empty((n, n), dtype=torch.float32, device="cuda")
    binding.pald_cohesion(D, U, ref)
    for _ in range(2):  # the fixed scratch keeps the previous call's contents
        C = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
        binding.pald_cohesion_noalloc(D, U, C)
        torch.cuda.synchronize()
        _close(C, ref)


def test_noalloc_rejects_orders_beyond_its_array():
    o = binding.PaldOpts(0, 0, -1, 0)
    fake = ctypes.c_void_p(256)  # never touched: the size check comes first
    st = binding.lib().pald_cohesion_noalloc(fake, fake, 2049, fake, ctypes.byref(o), None)
    assert st == 8  # PALD_ERR_UNSUPPORTED
    assert "unsupported" in binding.pald_status_string(st)
