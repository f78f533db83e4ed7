"""ctypes binding of libpald (argument marshalling only).

Each function has the name of the C entry point it calls.  Device tensors
are passed as raw pointers together with the current torch CUDA stream, so
the kernels are ordered with the caller's other work.  Loading the library
does not build it: run ``python -m paper_2307_16652_gb300.build`` (or
``__graft_entry__.build()``) first.  A missing library raises; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PALD_ACCUM_COMPENSATED = 0
PALD_ACCUM_PLAIN = 1
PALD_ACCUM_FIXED = 2
PALD_FLAG_IGNORE_TIES = 1

_STATUS = {
    0: "PALD_OK", 1: "PALD_ERR_INVALID_ARG", 2: "PALD_ERR_NOT_SYMMETRIC", 3: "PALD_ERR_BAD_DIAGONAL",
    4: "PALD_ERR_BAD_VALUE", 5: "PALD_ERR_CUDA", 6: "PALD_ERR_NO_MEMORY", 7: "PALD_ERR_TIMEOUT",
    8: "PALD_ERR_UNSUPPORTED",
}


class PaldError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = _STATUS.get(status, str(status))
        msg = f"{where}: {name} ({_lib().pald_status_string(status).decode()})"
        if status == 5:
            msg += f", cudaError={_lib().pald_last_cuda_error()}"
        super().__init__(msg)


class PaldOpts(ctypes.Structure):
    _fields_ = [("validate", ctypes.c_int32), ("accum_mode", ctypes.c_int32),
                ("schedule_id", ctypes.c_int32), ("flags", ctypes.c_int32)]


class PaldScheduleBucket(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("focus", ctypes.c_int32), ("cohesion", ctypes.c_int32),
                ("batched_split", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_handle: ctypes.CDLL | None = None


def library_path() -> str:
    return _build.LIB


def _lib() -> ctypes.CDLL:
    global _handle
    with _lock:
        if _handle is not None:
            return _handle
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libpald is not built ({path} missing); run paper_2307_16652_gb300.build.build()")
        h = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        op = ctypes.POINTER(PaldOpts)
        h.pald_focus.argtypes = [vp, i64, vp, op, vp]
        h.pald_cohesion.argtypes = [vp, vp, i64, vp, op, vp]
        h.pald_cohesion_noalloc.argtypes = [vp, vp, i64, vp, op, vp]
        h.pald_cohesion_depth.argtypes = [vp, vp, i64, vp, vp, op, vp]
        h.pald_batched.argtypes = [i32, vp, vp, vp, vp, vp, op, vp]
        h.pald_host.argtypes = [vp, i64, vp, vp, op]
        h.pald_validate.argtypes = [vp, i64, vp]
        h.pald_tie_map.argtypes = [vp, i64, vp, vp]
        h.pald_check_faults.argtypes = [vp]
        h.pald_test_bounded_wait.argtypes = [i64, vp]
        h.pald_set_schedule_table.argtypes = [ctypes.POINTER(PaldScheduleBucket), i32]
        h.pald_pairwise.argtypes = [vp, i64, vp, op, vp]
        h.pald_pairwise_scratch_bytes.argtypes = [i64]
        h.pald_pairwise_scratch_bytes.restype = i64
        h.pald_shard_tiles.argtypes = [i64]
        h.pald_shard_tiles.restype = i64
        h.pald_shard_range.argtypes = [i64, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        h.pald_focus_tiles.argtypes = [vp, i64, i64, i64, vp, op, vp]
        h.pald_cohesion_tiles.argtypes = [vp, vp, i64, i64, i64, vp, op, vp]
        h.pald_pack_tiles.argtypes = [vp, i64, i64, i64, i32, vp, vp]
        h.pald_unpack_tiles.argtypes = [vp, i64, i64, i64, i32, vp, vp]
        h.pald_get_schedule.argtypes = [i64, ctypes.POINTER(PaldScheduleBucket), ctypes.POINTER(i32)]
        h.pald_local_depth.argtypes = [vp, i64, vp, vp]
        h.pald_strong_ties.argtypes = [vp, i64, ctypes.c_float, vp, vp]
        h.pald_tie_map_words.argtypes = [i64]
        h.pald_tie_map_words.restype = i64
        for f in (h.pald_focus, h.pald_cohesion, h.pald_cohesion_noalloc, h.pald_cohesion_depth, h.pald_batched,
                  h.pald_host,
                  h.pald_validate, h.pald_tie_map, h.pald_check_faults, h.pald_local_depth, h.pald_strong_ties,
                  h.pald_test_bounded_wait, h.pald_set_schedule_table, h.pald_get_schedule, h.pald_shard_range,
                  h.pald_focus_tiles, h.pald_cohesion_tiles, h.pald_pack_tiles, h.pald_unpack_tiles,
                  h.pald_pairwise):
            f.restype = ctypes.c_int
        h.pald_status_string.argtypes = [ctypes.c_int]
        h.pald_status_string.restype = ctypes.c_char_p
        h.pald_schedule_name.argtypes = [i32]
        h.pald_schedule_name.restype = ctypes.c_char_p
        h.pald_schedule_count.restype = i32
        h.pald_last_cuda_error.restype = i32
        h.pald_version.restype = i32
        h.pald_release.restype = None
        _handle = h
        return h


def lib() -> ctypes.CDLL:
    """The loaded libpald handle (raises if it is not built)."""
    return _lib()


def _opts(validate=False, accum_mode=PALD_ACCUM_COMPENSATED, schedule_id=-1, ignore_ties=False):
    return PaldOpts(int(bool(validate)), int(accum_mode), int(schedule_id),
                    PALD_FLAG_IGNORE_TIES if ignore_ties else 0)


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(t, dtype, n=None, name="tensor"):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and tuple(t.shape) != (n, n):
        raise ValueError(f"{name} must have shape ({n}, {n}), got {tuple(t.shape)}")
    return t.data_ptr()


def _raise(st, where):
    if st != 0:
        raise PaldError(st, where)


def pald_focus(D, U, *, validate=False, schedule_id=-1, stream=None):
    """Pass 1: U[x, y] = u_xy (int32) from the FP32 distance matrix D."""
    import torch

    n = D.shape[0]
    o = _opts(validate, PALD_ACCUM_COMPENSATED, schedule_id)
    st = _lib().pald_focus(_check(D, torch.float32, n, "D"), n, _check(U, torch.int32, n, "U"),
                           ctypes.byref(o), _stream_ptr(stream))
    _raise(st, "pald_focus")
    return U


def pald_cohesion(D, U, C, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, schedule_id=-1, ignore_ties=False,
                  stream=None):
    """Pass 2: C[x, z] = c_xz (FP32) from D and the focus sizes U.

    ignore_ties=True is the paper's inexact fast mode (PALD_FLAG_IGNORE_TIES)."""
    import torch

    n = D.shape[0]
    o = _opts(validate, accum_mode, schedule_id, ignore_ties)
    st = _lib().pald_cohesion(_check(D, torch.float32, n, "D"), _check(U, torch.int32, n, "U"), n,
                              _check(C, torch.float32, n, "C"), ctypes.byref(o), _stream_ptr(stream))
    _raise(st, "pald_cohesion")
    return C


def pald_cohesion_depth(D, U, C, L=None, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, schedule_id=-1,
                        ignore_ties=False, stream=None):
    """Pass 2 with the local depths L[x] = sum_z C[x, z] from its epilogue;
    returns (C, L).  C gets the same bits as :func:`pald_cohesion`."""
    import torch

    n = D.shape[0]
    if L is None:
        L = torch.empty(n, dtype=torch.float32, device=D.device)
    if not (isinstance(L, torch.Tensor) and L.is_cuda and L.dtype == torch.float32 and L.is_contiguous()
            and tuple(L.shape) == (n,)):
        raise ValueError(f"L must be a contiguous float32 CUDA tensor of shape ({n},)")
    o = _opts(validate, accum_mode, schedule_id, ignore_ties)
    st = _lib().pald_cohesion_depth(_check(D, torch.float32, n, "D"), _check(U, torch.int32, n, "U"), n,
                                    _check(C, torch.float32, n, "C"), L.data_ptr(), ctypes.byref(o),
                                    _stream_ptr(stream))
    _raise(st, "pald_cohesion_depth")
    return C, L


def pald_cohesion_noalloc(D, U, C, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, schedule_id=-1,
                          stream=None):
    """Pass 2 for callers that must not allocate device memory (n <= 2048).

    Same result as :func:`pald_cohesion`; the scratch is a fixed array inside
    the library, shared by every call on a device, so calls must not overlap
    on the GPU."""
    import torch

    n = D.shape[0]
    o = _opts(validate, accum_mode, schedule_id)
    st = _lib().pald_cohesion_noalloc(_check(D, torch.float32, n, "D"), _check(U, torch.int32, n, "U"), n,
                                      _check(C, torch.float32, n, "C"), ctypes.byref(o), _stream_ptr(stream))
    _raise(st, "pald_cohesion_noalloc")
    return C


def pald_batched(ns, offs, D, U, C, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, ignore_ties=False,
                 stream=None):
    """Both passes for packed matrices: matrix i is ns[i] x ns[i] at element offs[i]."""
    import numpy as np
    import torch

    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.int64))
    offs = np.ascontiguousarray(np.asarray(offs, dtype=np.int64))
    if ns.shape != offs.shape or ns.ndim != 1:
        raise ValueError("ns and offs must be 1-D arrays of equal length")
    for t, dt, nm in ((D, torch.float32, "D"), (U, torch.int32, "U"), (C, torch.float32, "C")):
        _check(t, dt, None, nm)
    need = int((offs + ns * ns).max())
    if min(D.numel(), U.numel(), C.numel()) < need:
        raise ValueError("packed buffers are smaller than the last matrix")
    o = _opts(validate, accum_mode, -1, ignore_ties)
    st = _lib().pald_batched(len(ns), ns.ctypes.data, offs.ctypes.data, D.data_ptr(), U.data_ptr(),
                             C.data_ptr(), ctypes.byref(o), _stream_ptr(stream))
    _raise(st, "pald_batched")


def pald_host(D, U, C, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED):
    """Both passes on host (numpy or CPU torch) buffers; copies in and out."""
    import numpy as np

    def ptr(a, dtype):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU tensors")
            return a.data_ptr()
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous of the right dtype")
        return a.ctypes.data

    n = D.shape[0]
    o = _opts(validate, accum_mode, -1)
    st = _lib().pald_host(ptr(D, np.float32), n, ptr(U, np.int32), ptr(C, np.float32), ctypes.byref(o))
    _raise(st, "pald_host")


def pald_validate(D, *, stream=None):
    """Check the input contract of D; returns the status code (0 = valid)."""
    import torch

    n = D.shape[0]
    return _lib().pald_validate(_check(D, torch.float32, n, "D"), n, _stream_ptr(stream))


def pald_local_depth(C, L=None, *, stream=None):
    """Local depths L[x] = sum_z C[x, z] (FP32 CUDA tensors); returns L."""
    import torch

    n = C.shape[0]
    if L is None:
        L = torch.empty(n, dtype=torch.float32, device=C.device)
    if not (isinstance(L, torch.Tensor) and L.is_cuda and L.dtype == torch.float32 and L.is_contiguous()
            and tuple(L.shape) == (n,)):
        raise ValueError(f"L must be a contiguous float32 CUDA tensor of shape ({n},)")
    st = _lib().pald_local_depth(_check(C, torch.float32, n, "C"), n, L.data_ptr(), _stream_ptr(stream))
    _raise(st, "pald_local_depth")
    return L


def pald_strong_ties(C, threshold, T=None, *, stream=None):
    """Mask T[x, z] = (C[x, z] >= threshold) as uint8 (CUDA tensors); returns T."""
    import torch

    n = C.shape[0]
    if T is None:
        T = torch.empty((n, n), dtype=torch.uint8, device=C.device)
    st = _lib().pald_strong_ties(_check(C, torch.float32, n, "C"), n, float(threshold),
                                 _check(T, torch.uint8, n, "T"), _stream_ptr(stream))
    _raise(st, "pald_strong_ties")
    return T


def pald_tie_map_words(n: int) -> int:
    return _lib().pald_tie_map_words(n)


def pald_tie_map(D, *, stream=None):
    """The tie map pass 2 uses for D (int32 view of the uint32 words; see pald.h)."""
    import torch

    n = D.shape[0]
    words = pald_tie_map_words(n)
    if words <= 0:
        raise ValueError(f"n={n} out of range")
    out = torch.empty(words, dtype=torch.int32, device=D.device)
    st = _lib().pald_tie_map(_check(D, torch.float32, n, "D"), n, out.data_ptr(), _stream_ptr(stream))
    _raise(st, "pald_tie_map")
    return out


def pald_check_faults(*, stream=None) -> int:
    """Synchronise and return 0, or 7 (PALD_ERR_TIMEOUT) if a kernel gave up a bounded wait."""
    return _lib().pald_check_faults(_stream_ptr(stream))


def pald_test_bounded_wait(limit_ns: int, *, stream=None) -> None:
    """Diagnostic: launch one CTA whose bounded waits give up after limit_ns
    (pald_check_faults then reports PALD_ERR_TIMEOUT once)."""
    _raise(_lib().pald_test_bounded_wait(int(limit_ns), _stream_ptr(stream)), "pald_test_bounded_wait")


SCHEDULE_SOURCES = {0: "built-in defaults", 1: "tuned table", 2: "set by the caller"}


def pald_set_schedule_table(buckets) -> None:
    """Replace the current device's schedule table.  ``buckets`` is a list of
    dicts (or tuples) n_max, focus, cohesion, batched_split sorted by n_max;
    an empty list restores the table the library was built with."""
    rows = [b if isinstance(b, dict) else dict(zip(("n_max", "focus", "cohesion", "batched_split"), b))
            for b in buckets]
    arr = (PaldScheduleBucket * max(1, len(rows)))()
    for i, b in enumerate(rows):
        arr[i] = PaldScheduleBucket(int(b["n_max"]), int(b["focus"]), int(b["cohesion"]),
                                    int(b["batched_split"]), 0)
    _raise(_lib().pald_set_schedule_table(arr, len(rows)), "pald_set_schedule_table")


def pald_get_schedule(n: int) -> dict:
    """The schedule bucket that applies to order n on the current device."""
    out = PaldScheduleBucket()
    src = ctypes.c_int32()
    _raise(_lib().pald_get_schedule(int(n), ctypes.byref(out), ctypes.byref(src)), "pald_get_schedule")
    return {"n_max": out.n_max, "focus": out.focus, "cohesion": out.cohesion, "batched_split": out.batched_split,
            "source": SCHEDULE_SOURCES.get(src.value, str(src.value))}


def pald_pairwise(D, C, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, ignore_ties=False, stream=None):
    """Both passes by strips of rows, u never stored: device memory for D, C and
    pald_pairwise_scratch_bytes(n) only.  Same C as pald_focus + pald_cohesion."""
    import torch

    n = D.shape[0]
    o = _opts(validate, accum_mode, -1, ignore_ties)
    _raise(_lib().pald_pairwise(_check(D, torch.float32, n, "D"), n, _check(C, torch.float32, n, "C"),
                                ctypes.byref(o), _stream_ptr(stream)), "pald_pairwise")
    return C


def pald_pairwise_scratch_bytes(n: int) -> int:
    return _lib().pald_pairwise_scratch_bytes(int(n))


def pald_shard_tiles(n: int) -> int:
    """Number of 64 x 64 upper-triangle super-tiles of order n (the shard units)."""
    return _lib().pald_shard_tiles(int(n))


def pald_shard_range(n: int, rank: int, world: int):
    """The contiguous tile range [t0, t1) of `rank` out of `world`."""
    t0, t1 = ctypes.c_int64(), ctypes.c_int64()
    _raise(_lib().pald_shard_range(int(n), int(rank), int(world), ctypes.byref(t0), ctypes.byref(t1)),
           "pald_shard_range")
    return t0.value, t1.value


def pald_focus_tiles(D, U, t0, t1, *, validate=False, stream=None):
    """Pass 1 on the tiles [t0, t1): u of their pairs (and mirrors) into U."""
    import torch

    n = D.shape[0]
    o = _opts(validate, PALD_ACCUM_COMPENSATED, -1)
    _raise(_lib().pald_focus_tiles(_check(D, torch.float32, n, "D"), n, int(t0), int(t1),
                                   _check(U, torch.int32, n, "U"), ctypes.byref(o), _stream_ptr(stream)),
           "pald_focus_tiles")
    return U


def pald_cohesion_tiles(D, U, C, t0, t1, *, validate=False, accum_mode=PALD_ACCUM_COMPENSATED, ignore_ties=False,
                        stream=None):
    """Pass 2 on the tiles [t0, t1) (U complete): C[X, Z] and C[Z, X] of those tiles."""
    import torch

    n = D.shape[0]
    o = _opts(validate, accum_mode, -1, ignore_ties)
    _raise(_lib().pald_cohesion_tiles(_check(D, torch.float32, n, "D"), _check(U, torch.int32, n, "U"), n,
                                      int(t0), int(t1), _check(C, torch.float32, n, "C"), ctypes.byref(o),
                                      _stream_ptr(stream)), "pald_cohesion_tiles")
    return C


def _words(t, name):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.element_size() == 4):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of 4-byte elements")
    return t.data_ptr()


def pald_pack_tiles(M, t0, t1, packed, *, both=False, stream=None):
    """Tiles [t0, t1) of the n x n matrix M into `packed` (4096 or 8192 words per tile)."""
    n = M.shape[0]
    need = (int(t1) - int(t0)) * 4096 * (2 if both else 1)
    if packed.numel() < need:
        raise ValueError(f"packed holds {packed.numel()} words, {need} needed")
    _raise(_lib().pald_pack_tiles(_words(M, "M"), n, int(t0), int(t1), int(bool(both)), _words(packed, "packed"),
                                  _stream_ptr(stream)), "pald_pack_tiles")
    return packed


def pald_unpack_tiles(packed, M, t0, t1, *, both=False, stream=None):
    """The inverse of pald_pack_tiles (with both=False each block's transpose is written too)."""
    n = M.shape[0]
    need = (int(t1) - int(t0)) * 4096 * (2 if both else 1)
    if packed.numel() < need:
        raise ValueError(f"packed holds {packed.numel()} words, {need} needed")
    _raise(_lib().pald_unpack_tiles(_words(packed, "packed"), n, int(t0), int(t1), int(bool(both)), _words(M, "M"),
                                    _stream_ptr(stream)), "pald_unpack_tiles")
    return M


def pald_schedule_count() -> int:
    return _lib().pald_schedule_count()


def pald_schedule_name(i: int):
    s = _lib().pald_schedule_name(i)
    return s.decode() if s is not None else None


def pald_status_string(status: int) -> str:
    return _lib().pald_status_string(status).decode()


def pald_version() -> int:
    return _lib().pald_version()


def pald_release() -> None:
    _lib().pald_release()
