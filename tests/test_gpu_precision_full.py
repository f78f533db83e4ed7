"""The precision study against the FULL FP64 oracle (every entry of the
16384 x 16384 precision-study matrix): the compensated FP32 path, the plain
FP32 sum and the fixed-point mode, max and mean relative error each.

The oracle needs about half an hour of 16 host cores here, so the test runs
only when PALD_FULL_PRECISION=1; PALD_PRECISION_OUT names a JSON file for
the numbers.  The default GPU run covers the same matrix on sampled rows
(test_gpu_parity.py, test_gpu_fixed.py).
"""
import json
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2307_16652_gb300 import PALD_ACCUM_COMPENSATED, PALD_ACCUM_FIXED, PALD_ACCUM_PLAIN, binding, build, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.skipif(os.environ.get("PALD_FULL_PRECISION") != "1", reason="set PALD_FULL_PRECISION=1 (about 30 min)")
def test_precision_16384_against_the_full_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    n = 16384
    D = inputs.euclidean_fp32_torch(inputs.precision_points(n), "cuda")
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    binding.pald_focus(D, U)
    outs = {}
    for name, mode in (("compensated", PALD_ACCUM_COMPENSATED), ("plain_fp32", PALD_ACCUM_PLAIN),
                       ("fixed_point", PALD_ACCUM_FIXED)):
        C = torch.empty((n, n), dtype=torch.float32, device="cuda")
        binding.pald_cohesion(D, U, C, accum_mode=mode)
        torch.cuda.synchronize()
        outs[name] = C.cpu().numpy()
        del C
    Ug = U.cpu().numpy()
    Dh = D.cpu().numpy()
    del D, U
    torch.cuda.empty_cache()
    t0 = time.time()
    U_ref, C_ref = oracle.focus_and_cohesion(Dh)
    oracle_s = time.time() - t0
    assert np.array_equal(Ug, U_ref), "focus sizes differ from the oracle"
    nz = C_ref != 0
    ref = C_ref[nz]
    res = {"n": n, "entries": int(n * n), "nonzero": int(nz.sum()), "oracle_seconds": round(oracle_s, 1),
           "threads": oracle.default_threads()}
    for name, C in outs.items():
        Cg = C.astype(np.float64)
        zeros_ok = bool(np.all(Cg[~nz] == 0))
        rel = np.abs(Cg[nz] - ref) / ref
        res[name] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                     "p99_rel": float(np.quantile(rel, 0.99)), "exact_zeros": zeros_ok}
        del Cg, rel
    out = os.environ.get("PALD_PRECISION_OUT")
    if out:
        with open(out, "w") as f:
            json.dump(res, f, indent=1)
    print(json.dumps(res))
    for name in ("compensated", "fixed_point"):
        assert res[name]["exact_zeros"]
        assert res[name]["max_rel"] <= 2e-7, f"{name}: {res[name]}"
