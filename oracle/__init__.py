"""Plain FP64 CPU oracle for the PaLD passes (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library's product path never does: it shares no code with the oracle.

The arithmetic lives in ``pald_oracle.c`` (plain C, compiled with gcc on the
machine that runs it); this module only builds it and marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pald_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict[int, ctypes.CDLL] = {}


def build(mutant: int = 0, out_dir: str | None = None) -> str:
    """Compile the oracle (``mutant`` > 0 plants one deliberate mistake)."""
    out_dir = out_dir or (_BUILD if mutant == 0 else tempfile.mkdtemp(prefix="pald_oracle_mut"))
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"libpald_oracle{'' if mutant == 0 else '_m%d' % mutant}.so")
    if mutant == 0 and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    tmp = so + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           f"-DPALD_ORACLE_MUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def _lib(mutant: int = 0) -> ctypes.CDLL:
    with _lock:
        if mutant not in _libs:
            lib = ctypes.CDLL(build(mutant))
            i64, i32p, f32p, f64p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            lib.pald_oracle.argtypes = [f32p, i64, i32p, f64p, ctypes.c_int]
            lib.pald_oracle_cohesion.argtypes = [f32p, i32p, i64, f64p, ctypes.c_int]
            lib.pald_oracle_rows.argtypes = [f32p, i64, ctypes.c_void_p, i64, i32p, f64p, ctypes.c_int]
            for f in (lib.pald_oracle, lib.pald_oracle_cohesion, lib.pald_oracle_rows):
                f.restype = ctypes.c_int
            lib.pald_oracle_mutant.restype = ctypes.c_int
            _libs[mutant] = lib
        return _libs[mutant]


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _as_d(D) -> np.ndarray:
    D = np.ascontiguousarray(D, dtype=np.float32)
    if D.ndim != 2 or D.shape[0] != D.shape[1] or D.shape[0] < 2:
        raise ValueError("D must be a square matrix of order >= 2")
    return D


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def focus_and_cohesion(D, threads: int | None = None, mutant: int = 0, cohesion: bool = True):
    """Return (u int32 n x n, C float64 n x n or None) for the whole matrix."""
    D = _as_d(D)
    n = D.shape[0]
    U = np.empty((n, n), dtype=np.int32)
    C = np.empty((n, n), dtype=np.float64) if cohesion else None
    rc = _lib(mutant).pald_oracle(_ptr(D), n, _ptr(U), _ptr(C) if C is not None else None,
                                 threads or default_threads())
    if rc != 0:
        raise RuntimeError("oracle failed")
    return U, C


def focus(D, threads: int | None = None, mutant: int = 0) -> np.ndarray:
    return focus_and_cohesion(D, threads, mutant, cohesion=False)[0]


def cohesion_from_u(D, U, threads: int | None = None, mutant: int = 0) -> np.ndarray:
    """C from the oracle's own u (used to time the second pass alone)."""
    D = _as_d(D)
    n = D.shape[0]
    U = np.ascontiguousarray(U, dtype=np.int32)
    C = np.empty((n, n), dtype=np.float64)
    if _lib(mutant).pald_oracle_cohesion(_ptr(D), _ptr(U), n, _ptr(C), threads or default_threads()) != 0:
        raise RuntimeError("oracle failed")
    return C


def rows(D, row_ids, threads: int | None = None, mutant: int = 0, cohesion: bool = True):
    """u and C restricted to the rows ``row_ids``: O(k n^2) work."""
    D = _as_d(D)
    n = D.shape[0]
    r = np.ascontiguousarray(np.asarray(row_ids, dtype=np.int64))
    k = r.shape[0]
    U = np.empty((k, n), dtype=np.int32)
    C = np.empty((k, n), dtype=np.float64) if cohesion else None
    rc = _lib(mutant).pald_oracle_rows(_ptr(D), n, _ptr(r), k, _ptr(U),
                                      _ptr(C) if C is not None else None, threads or default_threads())
    if rc != 0:
        raise RuntimeError("oracle failed")
    return U, C
