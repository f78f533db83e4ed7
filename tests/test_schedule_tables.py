"""Schedule tables: the autotuner's buckets, the C++ the build generates from
tuned_schedules.json, and the host-side checks of pald_set_schedule_table
(all without a GPU)."""
import ctypes
import json

import pytest

from paper_2307_16652_gb300 import autotune, binding, build

INVALID = 1


def test_bucket_bounds_are_geometric_midpoints():
    assert autotune.bucket_bounds([256, 512, 1024]) == [362, 724, 1 << 20]
    assert autotune.bucket_bounds([8192, 1024]) == [2896, 1 << 20]


def test_generated_tables(tmp_path, monkeypatch):
    doc = {"tables": [{"gpu": "GPU A", "sms": 10, "buckets": [
        {"n_max": 100, "focus": 1, "cohesion": 2, "batched_split": 0},
        {"n_max": 1 << 20, "focus": 2, "cohesion": 7, "batched_split": 1}]}]}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(doc))
    monkeypatch.setattr(build, "TUNED", str(path))
    src = build.tuned_tables_source()
    assert '{"GPU A", 10, 2, {{100, 1, 2, 0}, {1048576, 2, 7, 1}}},' in src
    assert "kTunedTableCount = 1;" in src
    path.write_text(json.dumps({"tables": []}))
    assert "kTunedTableCount = 1;" in build.tuned_tables_source()  # the placeholder that never matches


def test_install_replaces_the_same_gpu(tmp_path):
    path = tmp_path / "t.json"
    t1 = {"gpu": "G", "sms": 1, "buckets": [{"n_max": 4, "focus": 0, "cohesion": 0, "batched_split": 0}]}
    t2 = dict(t1, buckets=[{"n_max": 8, "focus": 1, "cohesion": 1, "batched_split": 1}])
    other = dict(t1, sms=2)
    autotune.install(t1, str(path))
    autotune.install(other, str(path))
    autotune.install(t2, str(path))
    tables = json.loads(path.read_text())["tables"]
    assert len(tables) == 2
    assert [t["buckets"][0]["n_max"] for t in tables if t["sms"] == 1] == [8]


def test_the_committed_tables_are_well_formed():
    with open(build.TUNED) as f:
        doc = json.load(f)
    for t in doc.get("tables", []):
        b = t["buckets"]
        assert 1 <= len(b) <= 16
        assert all(x["n_max"] < y["n_max"] for x, y in zip(b, b[1:]))
        assert b[-1]["n_max"] >= 1 << 20
        for x in b:
            assert 0 <= x["focus"] < 8 and 0 <= x["cohesion"] < 8 and x["batched_split"] in (0, 1)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def _table(rows):
    arr = (binding.PaldScheduleBucket * max(1, len(rows)))()
    for i, r in enumerate(rows):
        arr[i] = binding.PaldScheduleBucket(*r)
    return arr


@pytest.mark.parametrize("rows", [
    [(100, 1, 1, 1, 0), (100, 2, 2, 1, 0)],      # n_max not increasing
    [(100, 8, 1, 1, 0)],                          # no schedule 8
    [(100, 1, -1, 1, 0)],
    [(100, 1, 1, 2, 0)],                          # split is 0 or 1
    [(100, 1, 1, 1, 5)],                          # reserved must be 0
    [(1, 1, 1, 1, 0)],                            # n_max >= 2
])
def test_bad_tables_are_rejected_on_the_host(lib, rows):
    assert lib.pald_set_schedule_table(_table(rows), len(rows)) == INVALID


def test_bad_counts_are_rejected(lib):
    assert lib.pald_set_schedule_table(None, 1) == INVALID
    assert lib.pald_set_schedule_table(_table([(100, 1, 1, 1, 0)] * 17), 17) == INVALID
    assert lib.pald_set_schedule_table(_table([]), -1) == INVALID
    out = binding.PaldScheduleBucket()
    assert lib.pald_get_schedule(1, ctypes.byref(out), None) == INVALID
    assert lib.pald_get_schedule(100, None, None) == INVALID
