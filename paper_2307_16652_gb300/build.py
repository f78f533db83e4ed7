"""Build libpald.so in-tree for sm_103a (GB300).

Every translation unit is compiled by nvcc in parallel with
``-gencode arch=compute_103a,code=sm_103a``, then linked into
``paper_2307_16652_gb300/_build/libpald.so``.  No CMake, no torch extension
machinery: the library is a plain C-ABI shared object.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpald.so")

SOURCES = ["pald_api.cu", "pald_scan.cu", "pald_focus.cu", "pald_cohesion.cu", "pald_batched.cu",
           "pald_noalloc.cu", "pald_ties.cu", "pald_depth.cu", "pald_shard.cu", "pald_pairwise.cu", "pald_fixed.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", f"-I{INCLUDE}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpald")


TUNED = os.path.join(HERE, "tuned_schedules.json")


def tuned_tables_source() -> str:
    """C++ initialiser of the autotuned schedule tables (tuned_schedules.json,
    written by the autotuner) that pald_api.cu includes."""
    import json

    tables = []
    if os.path.exists(TUNED):
        with open(TUNED) as f:
            tables = json.load(f).get("tables", [])
    rows = []
    for t in tables:
        bs = t["buckets"]
        if not 1 <= len(bs) <= 16:
            raise ValueError(f"{TUNED}: a table needs 1 to 16 buckets")
        cells = ", ".join("{%d, %d, %d, %d}" % (int(b["n_max"]), int(b["focus"]), int(b["cohesion"]),
                                                int(b["batched_split"])) for b in bs)
        name = str(t["gpu"]).replace("\\", "").replace('"', "")
        rows.append('  {"%s", %d, %d, {%s}},' % (name, int(t["sms"]), len(bs), cells))
    if not rows:  # keep the array non-empty; a table of 0 buckets never matches
        rows.append('  {"", 0, 0, {}},')
    return ("// Generated by build.py from tuned_schedules.json: do not edit.\n"
            "static const TunedTable kTunedTables[] = {\n" + "\n".join(rows) + "\n};\n"
            "static const int kTunedTableCount = %d;\n" % len(rows))


def _inputs_digest(extra: list[str]) -> str:
    h = hashlib.sha256()
    if os.path.exists(TUNED):
        with open(TUNED, "rb") as f:
            h.update(f.read())
    for root in (CSRC, INCLUDE):
        for name in sorted(os.listdir(root)):
            p = os.path.join(root, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + extra).encode())
    return h.hexdigest()


def build(verbose: bool = False, extra_flags: list[str] | None = None, force: bool = False,
          out_dir: str | None = None) -> str:
    """Compile (if sources changed) and return the path of libpald.so
    (in ``out_dir`` when given, for builds with other compile-time options)."""
    extra = list(extra_flags or [])
    build_dir = out_dir or BUILD
    lib_path = os.path.join(build_dir, "libpald.so")
    os.makedirs(build_dir, exist_ok=True)
    digest = _inputs_digest(extra)
    stamp = os.path.join(build_dir, "libpald.digest")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return lib_path
    cc = nvcc()
    with open(os.path.join(build_dir, "tuned_schedules.inc"), "w") as f:
        f.write(tuned_tables_source())

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, f"-I{build_dir}", *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
