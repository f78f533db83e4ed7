"""Host logic of bench.py: the traffic record written from an ncu CSV, its
digest guard, and its scaling to other orders (no GPU)."""
import json
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",'
          '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _row(i, kernel, metric, unit, value):
    return (f'"{i}","1","python3","h","{kernel}","1","7","(256, 1, 1)","(8256, 1, 1)","0","10.3",'
            f'"Command line profiler metrics","{metric}","{unit}","{value}"')


def _csv(tmp_path):
    lines = ["==PROF== Connected to process 1", HEADER]
    k1 = "void unnamed>::focus_tma_kernel<TileGeom<64, 1, 1, 1, 4, 32, 32>>(CUtensorMap_st, const float *, long)"
    k2 = "void unnamed>::cohesion_tma_kernel<0, 0>(CUtensorMap_st, CUtensorMap_st, const float *, long)"
    lines += [_row(0, k1, "dram__bytes_read.sum", "byte", "1,000"), _row(0, k1, "dram__bytes_write.sum", "Kbyte", "2"),
              _row(0, k1, "gpu__time_duration.sum", "ns", "23738592"),
              _row(1, k2, "dram__bytes_read.sum", "Mbyte", "5"), _row(1, k2, "dram__bytes_write.sum", "byte", "7"),
              _row(1, k2, "gpu__time_duration.sum", "us", "45356.2")]
    p = tmp_path / "traffic.csv"
    p.write_text("\n".join(lines) + "\n")
    return p


def test_traffic_record_from_an_ncu_csv(tmp_path):
    out = tmp_path / "traffic.json"
    rec = bench.write_traffic_record(str(_csv(tmp_path)), str(out))
    assert rec == json.loads(out.read_text())
    assert rec["csrc_digest"] == bench.csrc_digest()
    f, c = rec["kernels"]["focus_tma_kernel"], rec["kernels"]["cohesion_tma_kernel"]
    assert (f["read"], f["write"], f["dram_bytes"]) == (1000, 2000, 3000)
    assert (c["read"], c["write"], c["dram_bytes"]) == (5_000_000, 7, 5_000_007)
    assert f["ms_under_ncu"] == pytest.approx(23.739, abs=1e-3)
    assert c["ms_under_ncu"] == pytest.approx(45.356, abs=1e-3)
    assert f["n"] == c["n"] == bench.TRAFFIC_N


def test_committed_traffic_record_scales_and_guards(monkeypatch, tmp_path):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    k = rec["kernels"]["cohesion_tma_kernel"]
    if rec["csrc_digest"] == bench.csrc_digest():
        # scaled by unique triplets C(n,3) from the captured order
        got = bench.traffic_for("cohesion_tma_kernel", 2 * k["n"])
        assert got == pytest.approx(k["dram_bytes"] * bench.triplets(2 * k["n"]) / bench.triplets(k["n"]))
    # a record taken on other sources is never used
    monkeypatch.setattr(bench, "csrc_digest", lambda: "not-the-captured-sources")
    assert bench.traffic_for("cohesion_tma_kernel", 65536) is None
