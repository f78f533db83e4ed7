"""GB300-native PaLD: the two triplet passes of partitioned local depths.

The compute lives in ``libpald.so`` (hand-written sm_103a CUDA kernels behind
the C ABI of ``include/pald.h``).  This package is a thin binding over that
ABI: it checks tensors, passes raw device pointers and the current CUDA
stream, and turns status codes into exceptions.  There is no CPU fallback:
every call fails loudly if the library is not built or no GPU is present.

    from paper_2307_16652_gb300 import pald_focus, pald_cohesion
    pald_focus(D, U)          # D: (n, n) float32 CUDA tensor, U: (n, n) int32
    pald_cohesion(D, U, C)    # C: (n, n) float32

The seeded workload generators are in :mod:`paper_2307_16652_gb300.inputs`.
"""
from __future__ import annotations

from .binding import (  # noqa: F401
    PALD_ACCUM_COMPENSATED,
    PALD_ACCUM_FIXED,
    PALD_ACCUM_PLAIN,
    PALD_FLAG_IGNORE_TIES,
    PaldError,
    lib,
    pald_check_faults,
    library_path,
    pald_batched,
    pald_cohesion,
    pald_cohesion_depth,
    pald_cohesion_noalloc,
    pald_cohesion_tiles,
    pald_focus,
    pald_focus_tiles,
    pald_get_schedule,
    pald_host,
    pald_local_depth,
    pald_pack_tiles,
    pald_pairwise,
    pald_pairwise_scratch_bytes,
    pald_release,
    pald_schedule_count,
    pald_schedule_name,
    pald_set_schedule_table,
    pald_shard_range,
    pald_shard_tiles,
    pald_status_string,
    pald_strong_ties,
    pald_test_bounded_wait,
    pald_tie_map,
    pald_tie_map_words,
    pald_unpack_tiles,
    pald_validate,
    pald_version,
)

__all__ = [
    "PALD_ACCUM_COMPENSATED", "PALD_ACCUM_FIXED", "PALD_ACCUM_PLAIN", "PALD_FLAG_IGNORE_TIES", "PaldError", "lib", "library_path", "pald_check_faults",
    "pald_batched", "pald_cohesion", "pald_cohesion_depth", "pald_cohesion_noalloc", "pald_focus", "pald_host", "pald_local_depth",
    "pald_release", "pald_strong_ties", "pald_test_bounded_wait",
    "pald_schedule_count", "pald_schedule_name", "pald_set_schedule_table", "pald_get_schedule", "pald_status_string", "pald_tie_map", "pald_tie_map_words",
    "pald_validate", "pald_version", "pald_cohesion_tiles", "pald_focus_tiles", "pald_pack_tiles",
    "pald_unpack_tiles", "pald_shard_range", "pald_shard_tiles", "pald_pairwise", "pald_pairwise_scratch_bytes",
]
