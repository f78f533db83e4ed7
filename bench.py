#!/usr/bin/env python3
"""Benchmark of the PaLD triplet passes on GB300.

One step = both passes (scan + local focus sizes, then cohesion) over one
seeded synthetic distance matrix that is already resident in HBM.  The
default workload is the paper-scale matrix, n = 65536 (points in R^32 from a
64-component Gaussian mixture, D = 17.2 GB, far larger than L2, so no L2
flush is needed between steps).

Metric: unique triplets C(n,3) processed per second per pass, i.e.
2*C(n,3) / (step time), summed over ranks.  Under torchrun every rank runs
its own copy of the workload (independent problems, weak scaling, no
collective on the data path).

Printed: one JSON line with the device-timed value, the roofline of the
dominant kernel (CUDA-core issue peak), the end-to-end number through the C
ABI with host buffers (pald_host), and the CPU oracle timed on a bounded
row sample of the same matrix.  ``--impl reference`` times that oracle alone.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triplets/sec per pass, % of CUDA-core peak; batched vs plain at stated error"
UNIT = "triplets/s"
LAUNCHES_PER_STEP = 6          # scan + focus | scan + tie map + reciprocal + cohesion
OPS_PER_TRIPLET = {"focus": 9, "cohesion": 18}   # lane-op budget per unique triplet
LANES_PER_SM_CLK = 128                            # 4 SMSPs x 1 warp-instruction x 32 lanes


def triplets(n: int) -> int:
    return n * (n - 1) * (n - 2) // 6


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU under torchrun)

def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.lines: list[str] = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        rows = [[c.strip() for c in ln.split(",")] for ln in self.lines if ln.count(",") >= 8]
        if self.bus_id:
            mine = [r for r in rows if r[0].lower() == self.bus_id]
            rows = mine or rows
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(self.NAMES, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def bus_id_of(device: int):
    import torch

    p = torch.cuda.get_device_properties(device)
    if hasattr(p, "pci_bus_id"):
        return f"{getattr(p, 'pci_domain_id', 0):08x}:{p.pci_bus_id:02x}:{getattr(p, 'pci_device_id', 0):02x}.0"
    return None


# ---------------------------------------------------------------------------
# workloads

def make_matrix(workload: str):
    """Device-resident FP32 D for a single-matrix workload."""
    import torch

    from paper_2307_16652_gb300 import inputs

    if workload == inputs.PAPER_65536:
        return inputs.euclidean_fp32_torch(inputs.paper_points(65536), "cuda")
    if workload == inputs.PRECISION_16384:
        return inputs.euclidean_fp32_torch(inputs.precision_points(16384), "cuda")
    if workload == inputs.TIE_HEAVY_4096:
        return torch.from_numpy(inputs.tie_heavy_matrix(4096)).cuda()
    if workload == inputs.PLAIN_512:
        return torch.from_numpy(inputs.plain_matrix(512)).cuda()
    if workload.startswith("paper-"):
        n = int(workload.split("-")[1])
        return inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    raise SystemExit(f"unknown workload {workload}")


# The sources that build the two single-matrix pass kernels and choose
# their launches: a change to any of them voids the recorded DRAM traffic.
TRAFFIC_SOURCES = ["include/pald.h", "paper_2307_16652_gb300/tuned_schedules.json"] + [
    f"paper_2307_16652_gb300/csrc/{f}" for f in (
        "pald_internal.cuh", "tile_geom.cuh", "tma_ring.cuh", "focus_core.cuh", "cohesion_core.cuh", "schedules.cuh",
        "pald_focus.cu", "pald_cohesion.cu", "pald_api.cu")]


def csrc_digest() -> str:
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


# The capture the traffic record comes from: one launch of each pass kernel
# at n = 8192 (inputs larger than L2, a few GB on the device), DRAM counters
# only (a single-pass capture), after the same bench command exited 0.
TRAFFIC_N = 8192
TRAFFIC_CAPTURE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                   "--clock-control none -k regex:'focus_tma_kernel|cohesion_tma_kernel' -s 6 -c 2 --csv "
                   "--log-file traffic8192.csv python bench.py --workload paper-8192 --steps 1 --warmup 3 "
                   "--no-e2e --no-cpu-baseline --no-batched --no-extras")
UNITS = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1e-9, "us": 1e-6, "ms": 1e-3,
         "nsecond": 1e-9, "usecond": 1e-6, "msecond": 1e-3}


def write_traffic_record(csv_path: str, out_path: str):
    """profiles/traffic.json from the CSV of TRAFFIC_CAPTURE, stamped with the
    digest of the sources it ran on (run this beside the capture)."""
    import collections
    import csv

    with open(csv_path) as f:
        rows = list(csv.reader(f))
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, ui = (h.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    per = collections.defaultdict(dict)
    for r in rows[hdr + 1:]:
        if len(r) <= vi:
            continue
        name = next((k for k in ("focus_tma_kernel", "cohesion_tma_kernel") if k in r[ki]), None)
        if name:
            per[name][r[mi]] = float(r[vi].replace(",", "")) * UNITS.get(r[ui], 1)
    rec = {"csrc_digest": csrc_digest(), "source": TRAFFIC_CAPTURE,
           "scaling": "dram bytes per launch at n, scaled to other n by unique triplets C(n,3)",
           "digest_of": "bench.TRAFFIC_SOURCES at the time of the capture", "kernels": {}}
    for k, m in sorted(per.items()):
        rd, wr = m["dram__bytes_read.sum"], m["dram__bytes_write.sum"]
        rec["kernels"][k] = {"n": TRAFFIC_N, "dram_bytes": int(rd + wr), "read": int(rd), "write": int(wr),
                             "ms_under_ncu": round(m["gpu__time_duration.sum"] * 1e3, 3)}
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def traffic_for(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to n by
    the units processed; None when absent or taken on different kernel code."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("csrc_digest") != csrc_digest():
        return None
    k = rec.get("kernels", {}).get(kernel)
    if not k:
        return None
    return k["dram_bytes"] * triplets(n) / triplets(k["n"])


def oracle_rows_rate(D_host, n: int, k: int, seed: int):
    """Time the oracle on k rows of D (both passes for those rows)."""
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    rows = np.random.default_rng(seed).choice(n, size=k, replace=False)
    t0 = time.perf_counter()
    oracle.rows(D_host, rows, threads=cores)
    dt = time.perf_counter() - t0
    # k rows are k/n of each pass; the metric counts both passes
    value = 2.0 * triplets(n) * (k / n) / dt
    return value, dt, cores


def workload_config(args, n: int, world: int) -> dict:
    """The `config` of both arms' JSON lines (the same keys and values)."""
    return {"workload": args.workload, "n": n, "accum_mode": "compensated", "schedule": "auto",
            "l2": "inputs larger than L2 (D is %.1f GB), no flush" % (4 * n * n / 1e9),
            "parallelism": f"replicas x{world} (independent matrices)"}


# ---------------------------------------------------------------------------
# our arm

def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2307_16652_gb300 as pald

    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    D = make_matrix(args.workload)
    n = D.shape[0]
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        pald.pald_focus(D, U)
        if ev:
            ev[1].record(stream)
        pald.pald_cohesion(D, U, C)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(bus_id_of(dev))
    clocks.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), world)
    t_focus = [e[0].elapsed_time(e[1]) for e in evs]
    t_coh = [e[1].elapsed_time(e[2]) for e in evs]
    ms_step = elapsed_ms / args.steps
    T = triplets(n)
    value = 2.0 * T * world / (ms_step / 1e3)

    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * LANES_PER_SM_CLK * sm_max * 1e6
    per_pass = {}
    for name, ts in (("focus", t_focus), ("cohesion", t_coh)):
        mean_s = statistics.mean(ts) / 1e3
        ops = OPS_PER_TRIPLET[name] * T / mean_s
        per_pass[name] = {"ms": round(statistics.mean(ts), 3), "triplets_per_s": T / mean_s,
                          "budget_ops_per_s": ops, "frac_of_issue_peak": ops / peak_ops}
    dom = max(per_pass, key=lambda k: per_pass[k]["ms"])
    tma = n % 4 == 0 and n >= 1024  # the default schedules stage operands with TMA when the row pitch allows it
    kernel_name = {"focus": "focus_tma_kernel" if tma else "focus_kernel",
                   "cohesion": "cohesion_tma_kernel" if tma else "cohesion_kernel"}[dom]
    roofline = {"bound": "alu", "kernel": kernel_name,
                "achieved": per_pass[dom]["budget_ops_per_s"] / 1e12, "peak": peak_ops / 1e12,
                "unit": "Tops/s", "frac": per_pass[dom]["frac_of_issue_peak"],
                "traffic": traffic_for(kernel_name, n),
                "peak_basis": f"{props.multi_processor_count} SMs x {LANES_PER_SM_CLK} lane-ops/clk x "
                              f"{sm_max:.0f} MHz (issue peak derived from unit counts and max SM clock)",
                "ops_per_triplet": OPS_PER_TRIPLET[dom]}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(args, n, world),
           "per_pass": per_pass, "roofline": roofline, "gpu_launches": LAUNCHES_PER_STEP * args.steps,
           "clocks": clk}

    D_host = None
    if rank == 0 and not args.no_e2e:
        # end to end through the C ABI on host buffers: H2D of D, both passes,
        # D2H of U and C, inside the timed region
        D_host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        D_host.copy_(D)
        U_host = torch.empty((n, n), dtype=torch.int32, pin_memory=True)
        C_host = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        del U, C
        torch.cuda.empty_cache()
        e2e_steps = max(1, min(args.steps, args.e2e_steps))
        ts = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            pald.pald_host(D_host, U_host, C_host)
            ts.append(time.perf_counter() - t0)
        t = statistics.mean(ts)
        out["e2e"] = {"value": 2.0 * triplets(n) / t, "unit": UNIT, "h2d_bytes_per_step": 4 * n * n,
                      "d2h_bytes_per_step": 8 * n * n, "steps": e2e_steps, "api": "pald_host",
                      "s_per_step": [round(x, 3) for x in ts]}
    if rank == 0 and not args.no_cpu_baseline:
        if D_host is None:
            D_host = D.cpu()
        Dh = D_host.numpy()
        k = args.oracle_rows or (os.cpu_count() or 1)
        v, dt, cores = oracle_rows_rate(Dh, n, k, seed=1)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{k} random rows of the same n={n} matrix, both passes "
                                         f"({dt:.1f} s), scaled by n/{k}",
                               # the whole matrix at the sampled rate (the oracle's work grows as n^3)
                               "full_extrapolated_s": round(2.0 * triplets(n) / v, 1)}
    if rank == 0 and not args.no_batched:
        out["batched"] = run_batched_compare(args)
    if rank == 0 and not args.no_extras:
        out["other_workloads"] = run_other_workloads(props, (clk or {}).get("sm_max_mhz") or 2070.0)
    return out


def run_other_workloads(props, sm_max):
    """Per-pass rates on the other single-matrix configs: tie-heavy-4096 (a
    tie in nearly every 8-y group: pass 2 runs its 8-slot long form
    throughout) and precision-16384; on the paper recipe at n = 8192, pass 2
    with the fused local depth, pass 2 in each accumulation mode and the
    pairwise strip variant (u never stored)."""
    import torch

    import paper_2307_16652_gb300 as pald
    from paper_2307_16652_gb300 import inputs

    stream = torch.cuda.current_stream()
    peak_ops = props.multi_processor_count * LANES_PER_SM_CLK * sm_max * 1e6

    def timed(fn, reps):
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

    out = {}
    for wl, reps in ((inputs.TIE_HEAVY_4096, 5), (inputs.PRECISION_16384, 2)):
        D = make_matrix(wl)
        n = D.shape[0]
        U = torch.empty((n, n), dtype=torch.int32, device="cuda")
        C = torch.empty((n, n), dtype=torch.float32, device="cuda")
        T = triplets(n)
        rec = {"n": n}
        for name, fn in (("focus", lambda: pald.pald_focus(D, U)), ("cohesion", lambda: pald.pald_cohesion(D, U, C))):
            ms = timed(fn, reps)
            rec[name] = {"ms": round(ms, 3), "triplets_per_s": T / (ms / 1e3),
                         "frac_of_issue_peak": OPS_PER_TRIPLET[name] * T / (ms / 1e3) / peak_ops}
        words = pald.pald_tie_map_words(n)
        tmap = pald.pald_tie_map(D)
        nb = -(-n // 64)
        import numpy as np

        cells = tmap[:words - nb].cpu().numpy().view(np.uint8)
        marked = int(np.unpackbits(cells).sum())
        dirty = int((tmap[words - nb:] != 0).sum())
        rec["tie_map"] = {"marked_bits": marked, "dirty_blocks": dirty, "blocks": nb}
        out[wl] = rec
        del D, U, C
        torch.cuda.empty_cache()
    n = 8192
    D = inputs.euclidean_fp32_torch(inputs.paper_points(n), "cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    U = torch.empty((n, n), dtype=torch.int32, device="cuda")
    L = torch.empty(n, dtype=torch.float32, device="cuda")
    pald.pald_focus(D, U)
    ms_c = timed(lambda: pald.pald_cohesion(D, U, C), 2)
    ms_sep = timed(lambda: pald.pald_local_depth(C, L), 5)
    ms_f = timed(lambda: pald.pald_cohesion_depth(D, U, C, L), 2)
    out["depth-paper-8192"] = {"n": n, "cohesion_ms": round(ms_c, 3), "cohesion_depth_ms": round(ms_f, 3),
                               "local_depth_pass_ms": round(ms_sep, 3),
                               "note": "pass 2 with the row sums in its epilogue vs pass 2 alone and the "
                                       "separate O(n^2) pass over C"}
    modes = {"compensated": ms_c}
    for name, mode in (("plain_fp32", pald.PALD_ACCUM_PLAIN), ("fixed_point", pald.PALD_ACCUM_FIXED)):
        modes[name] = timed(lambda: pald.pald_cohesion(D, U, C, accum_mode=mode), 2)
    out["accum-modes-paper-8192"] = {
        "n": n, **{f"{k}_ms": round(v, 3) for k, v in modes.items()},
        **{f"{k}_frac_of_issue_peak": OPS_PER_TRIPLET["cohesion"] * triplets(n) / (v / 1e3) / peak_ops
           for k, v in modes.items()}}
    del U, L
    ms = timed(lambda: pald.pald_pairwise(D, C), 2)
    out["pairwise-paper-8192"] = {"n": n, "ms_both_passes": round(ms, 3),
                                  "triplets_per_s_per_pass": 2 * triplets(n) / (ms / 1e3) / 2,
                                  "scratch_bytes": pald.pald_pairwise_scratch_bytes(n),
                                  "note": "u never stored; every pair's u counted in both orientations"}
    del D, C
    torch.cuda.empty_cache()
    return out


def run_batched_compare(args):
    """Batched workload: one graph replay vs looping the single-matrix calls."""
    import numpy as np
    import torch

    import paper_2307_16652_gb300 as pald
    from paper_2307_16652_gb300 import inputs

    count = args.batched_count
    ns = inputs.batched_sizes(count)
    offs, total = inputs.packed_offsets(ns)
    D = torch.zeros(total, dtype=torch.float32, device="cuda")
    for i, n in enumerate(ns):
        Di = inputs.euclidean_fp32_torch(inputs.batched_points(i, int(n)), "cuda", block=int(n))
        D[offs[i]:offs[i] + n * n] = Di.reshape(-1)
    U = torch.empty(total, dtype=torch.int32, device="cuda")
    C = torch.empty(total, dtype=torch.float32, device="cuda")
    views = [(D[o:o + n * n].view(n, n), U[o:o + n * n].view(n, n), C[o:o + n * n].view(n, n))
             for o, n in zip(offs.tolist(), ns.tolist())]
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(2):
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

    def batched():
        pald.pald_batched(ns, offs, D, U, C)

    def loop():
        for Dv, Uv, Cv in views:
            pald.pald_focus(Dv, Uv)
            pald.pald_cohesion(Dv, Uv, Cv)

    t_b = timed(batched, 5)
    Ub, Cb = U.clone(), C.clone()
    t_l = timed(loop, 2)
    same = bool(torch.equal(Ub, U) and torch.equal(Cb, C))
    T = sum(triplets(int(n)) for n in ns)
    pald.pald_release()
    return {"workload": inputs.BATCHED_2000 if count == 2000 else f"batched-{count}", "matrices": count,
            "ms_batched": t_b, "ms_plain_loop": t_l, "value": 2.0 * T / (t_b / 1e3), "unit": UNIT,
            "speedup_vs_plain_loop": t_l / t_b, "bit_identical_to_plain_loop": same}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle, as it stands

def run_reference(args, rank, world):
    import numpy as np
    import torch

    if rank != 0:
        return None
    D = make_matrix(args.workload) if torch.cuda.is_available() else None
    if D is None:
        raise SystemExit("the reference arm generates its input on the GPU")
    n = D.shape[0]
    Dh = D.cpu().numpy()
    del D
    k = args.oracle_rows or (os.cpu_count() or 1)
    for w in range(args.warmup):
        oracle_rows_rate(Dh, n, k, seed=100 + w)
    times = []
    cores = os.cpu_count() or 1
    for s in range(args.steps):
        _, dt, cores = oracle_rows_rate(Dh, n, k, seed=200 + s)
        times.append(dt)
    t = statistics.mean(times)
    value = 2.0 * triplets(n) * (k / n) / t
    sample = f"{k} random rows of the n={n} matrix per step, both passes, scaled by n/{k}"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, n, world),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper-65536")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="pald_host calls timed for the end-to-end number (at most --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other single-matrix workloads")
    ap.add_argument("--batched-count", type=int, default=2000)
    ap.add_argument("--oracle-rows", type=int, default=0)
    ap.add_argument("--traffic-from", metavar="CSV",
                    help="write the traffic record from the CSV of TRAFFIC_CAPTURE and exit (no GPU work)")
    ap.add_argument("--traffic-out", default=os.path.join(ROOT, "profiles", "traffic.json"))
    args = ap.parse_args()
    if args.traffic_from:
        print(json.dumps(write_traffic_record(args.traffic_from, args.traffic_out), indent=1))
        return
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    rank, world, local = dist_setup(args)
    if rank == 0 or world == 1:
        if args.impl == "reference":
            import oracle  # the reference arm builds and loads the oracle only

            oracle.build()
        else:
            import __graft_entry__

            __graft_entry__.build()
    barrier(world)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
