"""Tile-schedule autotuner for the two passes (the GPU counterpart of the
block-size tuning of Sec. 5).

For each order n of ``--n`` it times every built-in schedule
(``pald_schedule_count()`` of them, see ``csrc/schedules.cuh``) of pass 1 and
pass 2 on a seeded paper-recipe matrix, with CUDA events on the launching
stream after a warm-up call, and checks that every schedule gives the
default's bits.  The orders are turned into size buckets (bucket i covers
the orders up to the geometric mean of n_i and n_{i+1}); each bucket takes
the fastest schedule of each pass at its order.

For the buckets within the batched range (orders up to 4096) it then times
``pald_batched`` on a set of batched-recipe matrices whose orders fall in the
bucket, once with diagonal tiles splitting off their in-group pairs and once
without, checks that both give the same bits, and keeps the split unless the
whole tiles are faster by more than 1% (``choose_split``).

The result is one table keyed by GPU name and SM count.  ``--install``
merges it into ``tuned_schedules.json`` beside this file, from which
``build.py`` compiles it into the library (``pald_get_schedule`` reports it
as the "tuned table"); ``pald_set_schedule_table`` applies a table at run
time without rebuilding.

    python -m paper_2307_16652_gb300.autotune --n 256 512 1024 2048 4096 8192 --install
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED = os.path.join(HERE, "tuned_schedules.json")
MAX_N = 1 << 20
BATCHED_MAX_N = 4096


def _time(fn, reps, stream):
    import torch

    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def bucket_bounds(ns):
    """Upper bounds of the buckets around the tuned orders."""
    ns = sorted(ns)
    bounds = [int(math.sqrt(a * b)) for a, b in zip(ns, ns[1:])]
    return bounds + [MAX_N]


def tune_single(ns, reps, log):
    import torch

    from . import binding, inputs

    stream = torch.cuda.current_stream()
    count = binding.pald_schedule_count()
    rows = []
    for n in sorted(ns):
        D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
        U = torch.empty((n, n), dtype=torch.int32, device="cuda")
        C = torch.empty((n, n), dtype=torch.float32, device="cuda")
        binding.pald_focus(D, U)
        ref_u = U.clone()
        binding.pald_cohesion(D, U, C)
        ref_c = C.clone()
        row = {"n": n, "focus_ms": {}, "cohesion_ms": {}}
        for s in range(count):
            tf = _time(lambda: binding.pald_focus(D, U, schedule_id=s), reps, stream)
            ok_u = bool(torch.equal(U, ref_u))
            tc = _time(lambda: binding.pald_cohesion(D, ref_u, C, schedule_id=s), reps, stream)
            ok_c = bool(torch.equal(C, ref_c))
            if not (ok_u and ok_c):
                raise RuntimeError(f"schedule {s} at n={n} does not reproduce the default's bits")
            row["focus_ms"][s] = round(tf, 4)
            row["cohesion_ms"][s] = round(tc, 4)
            log(f"n={n:6d} schedule {s}: focus {tf:9.3f} ms  cohesion {tc:9.3f} ms")
        row["best_focus"] = min(row["focus_ms"], key=row["focus_ms"].get)
        row["best_cohesion"] = min(row["cohesion_ms"], key=row["cohesion_ms"].get)
        rows.append(row)
        del D, U, C, ref_u, ref_c
        torch.cuda.empty_cache()
    return rows


def batched_set(lo, hi, work, seed):
    """Orders drawn uniformly in [lo, hi] until sum n^3 reaches `work`, with
    batched-recipe matrices of those orders packed back to back."""
    import numpy as np

    from . import inputs

    rng = np.random.default_rng(seed)
    ns = []
    while sum(n ** 3 for n in ns) < work and len(ns) < 20000:
        ns.append(int(rng.integers(lo, hi + 1)))
    ns = np.array(ns, dtype=np.int64)
    offs, total = inputs.packed_offsets(ns)
    D = np.zeros(total, np.float32)
    for i, n in enumerate(ns):
        D[offs[i]:offs[i] + n * n] = inputs.euclidean_fp32(inputs.batched_points(i, int(n))).ravel()
    return ns, offs, D


SPLIT_MARGIN = 0.01  # the whole-tile choice must win by more than this fraction (measurement noise)


def choose_split(ms_split: float, ms_whole: float) -> int:
    """Keep the default (diagonal tiles split, in pairs) unless whole tiles
    are faster by more than SPLIT_MARGIN: a bucket's test set is a small
    sample of the orders, and on the full batched workload a choice within
    noise on its bucket set measured slower."""
    return 0 if ms_whole < ms_split * (1.0 - SPLIT_MARGIN) else 1


def rederive(table):
    """Re-apply choose_split to a table's own batched measurements."""
    for m in table.get("measured", {}).get("batched", []):
        table["buckets"][m["bucket"]]["batched_split"] = choose_split(m["ms_split"], m["ms_whole"])
    return table


def tune_batched(buckets, reps, work, log):
    import torch

    from . import binding

    stream = torch.cuda.current_stream()
    lo = 2
    results = []
    for k, b in enumerate(buckets):
        hi = min(b["n_max"], BATCHED_MAX_N)
        if lo > hi:
            break
        ns, offs, Dh = batched_set(max(lo, 8), hi, work, seed=100 + k)
        D = torch.from_numpy(Dh).cuda()
        U = torch.zeros_like(D, dtype=torch.int32)
        C = torch.zeros_like(D)
        ms, bits = {}, {}
        for split in (1, 0):
            table = [dict(bb) for bb in buckets]
            table[k]["batched_split"] = split
            binding.pald_set_schedule_table(table)
            ms[split] = _time(lambda: binding.pald_batched(ns, offs, D, U, C), reps, stream)
            bits[split] = (U.clone(), C.clone())
            binding.pald_release()
        if not (torch.equal(bits[0][0], bits[1][0]) and torch.equal(bits[0][1], bits[1][1])):
            raise RuntimeError(f"batched split and whole diagonal tiles differ in bucket {k}")
        b["batched_split"] = choose_split(ms[1], ms[0])
        results.append({"bucket": k, "orders": [int(ns.min()), int(ns.max())], "matrices": len(ns),
                        "ms_split": round(ms[1], 4), "ms_whole": round(ms[0], 4)})
        log(f"batched bucket {k} (n {lo}..{hi}, {len(ns)} matrices): split {ms[1]:.3f} ms, whole {ms[0]:.3f} ms")
        lo = b["n_max"] + 1
        del D, U, C, bits
        torch.cuda.empty_cache()
    binding.pald_set_schedule_table([])
    return results


def tune(ns, reps=3, batched_reps=5, batched_work=2e11, verbose=True):
    import torch

    from . import binding, build

    build.build()
    binding.lib()
    log = (lambda m: print(m, file=sys.stderr, flush=True)) if verbose else (lambda m: None)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    binding.pald_set_schedule_table([])  # measure from the built-in state
    single = tune_single(ns, reps, log)
    buckets = [{"n_max": nmax, "focus": int(r["best_focus"]), "cohesion": int(r["best_cohesion"]),
                "batched_split": 1} for nmax, r in zip(bucket_bounds(ns), single)]
    batched = tune_batched(buckets, batched_reps, batched_work, log)
    return {"gpu": props.name, "sms": props.multi_processor_count,
            "source": f"autotune.py, n = {sorted(ns)}, {time.strftime('%Y-%m-%d')}",
            "buckets": buckets, "measured": {"single": single, "batched": batched}}


def install(table, path=TUNED):
    """Merge `table` into the tuned tables (replacing one for the same GPU)."""
    doc = {"tables": []}
    if os.path.exists(path):
        with open(path) as f:
            doc = json.load(f)
    doc["tables"] = [t for t in doc.get("tables", []) if (t["gpu"], t["sms"]) != (table["gpu"], table["sms"])]
    doc["tables"].append(table)
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, nargs="+", default=[256, 512, 1024, 2048, 4096, 8192])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batched-work", type=float, default=2e11, help="sum of n^3 per batched bucket set")
    ap.add_argument("--out", default=None, help="also write the table to this file")
    ap.add_argument("--install", action="store_true", help="merge the table into tuned_schedules.json")
    args = ap.parse_args()
    table = tune(args.n, args.reps, batched_work=args.batched_work)
    text = json.dumps(table, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    if args.install:
        install(table)
    print(text)


if __name__ == "__main__":
    main()
