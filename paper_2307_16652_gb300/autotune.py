"""Tile-schedule autotuner for the two passes.

Times every built-in schedule (``pald_schedule_count()`` of them, see
``csrc/schedules.cuh``) of pass 1 and pass 2 on seeded matrices of several
orders, with CUDA events on the launching stream after warm-up, and writes a
JSON table keyed by GPU name, SM count and matrix order.  The library's
built-in defaults are set from such a table; ``pald_opts.schedule_id``
(``schedule_id=`` in the binding) picks a schedule explicitly.

    python -m paper_2307_16652_gb300.autotune --n 2048 4096 8192 --out tune.json
"""
from __future__ import annotations

import argparse
import json
import sys


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


def tune(ns, reps=3, verbose=True):
    import torch

    from . import binding, build, inputs

    build.build()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    count = binding.pald_schedule_count()
    table = {"gpu": props.name, "sms": props.multi_processor_count, "schedules": {}, "results": []}
    for s in range(count):
        table["schedules"][s] = binding.pald_schedule_name(s)
    for n in ns:
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
            row["focus_ms"][s] = tf if ok_u else None
            row["cohesion_ms"][s] = tc if ok_c else None
            if verbose:
                print(f"n={n:6d} schedule {s}: focus {tf:9.3f} ms{'' if ok_u else ' (MISMATCH)'}  "
                      f"cohesion {tc:9.3f} ms{'' if ok_c else ' (MISMATCH)'}", file=sys.stderr)
        for key in ("focus", "cohesion"):
            ms = {s: t for s, t in row[f"{key}_ms"].items() if t is not None}
            row[f"best_{key}"] = min(ms, key=ms.get)
        table["results"].append(row)
        del D, U, C, ref_u, ref_c
        torch.cuda.empty_cache()
    return table


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, nargs="+", default=[1024, 2048, 4096, 8192])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    table = tune(args.n, args.reps)
    text = json.dumps(table, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
