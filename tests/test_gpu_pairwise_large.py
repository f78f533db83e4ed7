"""pald_pairwise at an order where the two-pass path cannot run on one GPU:
n = 147456, so D, U, R and C would take 348 GB, more than the device holds,
while D + C take 174 GB.  Sampled rows against the FP64 oracle, and the
global invariants (C >= 0, sum of C = n / 2) over the whole output.

About a quarter of an hour of GPU time, so the test runs only when
PALD_LARGE=1.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import binding, build, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
N_LARGE = 147456


@pytest.mark.skipif(os.environ.get("PALD_LARGE") != "1", reason="set PALD_LARGE=1 (about 15 min of GPU time)")
def test_pairwise_beyond_the_two_pass_memory():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    n = N_LARGE
    with open("/proc/meminfo") as f:
        avail = {l.split(":")[0]: int(l.split()[1]) * 1024 for l in f}.get("MemAvailable", 0)
    if avail < 2 * 4 * n * n:  # the oracle's rows read all of D from host memory
        pytest.skip(f"{avail / 1e9:.0f} GB of host memory available, {8 * n * n / 1e9:.0f} GB wanted")
    _, total = torch.cuda.mem_get_info()
    assert 16 * n * n > total, "D, U, R and C would fit: not the order this test is about"
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    binding.pald_pairwise(D, C)
    b.record()
    torch.cuda.synchronize()
    assert binding.pald_check_faults() == 0
    ms = a.elapsed_time(b)
    rows = np.array([0, 1, n // 2, n - 1] + list(np.random.default_rng(n).choice(n, size=12, replace=False)))
    rows = np.unique(rows)
    Dfull = D.cpu().numpy()  # the oracle's rows need all of D (87 GB of host memory)
    _, Cr = oracle.rows(Dfull, rows)
    del Dfull
    Cg = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    nz = Cr != 0
    assert np.all(Cg[~nz] == 0)
    rel = np.abs(Cg[nz] - Cr[nz]) / Cr[nz]
    assert rel.max() <= 2e-7, f"max relative error {rel.max():.3e}"
    total_c = torch.zeros((), dtype=torch.float64, device="cuda")
    for r0 in range(0, n, 8192):
        blk = C[r0:r0 + 8192]
        assert float(blk.min()) >= 0.0
        total_c += blk.double().sum()
    assert abs(float(total_c) - n / 2) < 1e-6 * n
    T = n * (n - 1) * (n - 2) // 6
    print(f"pald_pairwise n={n}: {ms / 1e3:.1f} s, {2 * T / (ms / 1e3):.3e} triplet-visits/s, "
          f"{len(rows)} rows: max rel {rel.max():.3e} mean {rel.mean():.3e}")
