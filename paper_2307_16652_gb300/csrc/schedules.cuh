// Tile schedules of both passes and the default choice per matrix order.
//
// A schedule is a tile geometry (see tile_geom.cuh).  The defaults below
// come from timing every schedule on GB300 (the project's autotuner,
// paper_2307_16652_gb300/autotune.py); pald_opts.schedule_id overrides them.
#pragma once

#include "tile_geom.cuh"

namespace pald {

constexpr int kScheduleCount = 8;

//                       B    H  GX GY CW  BK  unroll
using FocusS0 = TileGeom<64, 1, 1, 1, 4, 16>;    // 4x4 pairs/thread, 256 threads
using FocusS1 = TileGeom<32, 1, 1, 1, 4, 16>;    // small matrices, 64 threads
using FocusS2 = TileGeom<64, 1, 1, 1, 4, 32>;    // deeper stages
using FocusS3 = TileGeom<128, 2, 2, 1, 4, 16>;   // 8x4 pairs/thread, 128x64 CTA tiles
using FocusS4 = TileGeom<64, 2, 1, 1, 4, 32>;    // 64x32 CTA tiles, 128 threads
using FocusS5 = TileGeom<64, 1, 1, 1, 4, 64, 16>;  // 64-deep stages, partly unrolled
using FocusS6 = TileGeom<128, 2, 2, 1, 4, 32>;   // 8x4 pairs/thread, 32-deep
using FocusS7 = FocusS2;                         // S2's tile, TMA-staged

using CohesionS0 = TileGeom<64, 1, 1, 1, 4, 16>;  // 4x4 pairs/thread, 256 threads
using CohesionS1 = TileGeom<32, 1, 1, 1, 4, 16>;  // small matrices, 64 threads
using CohesionS2 = TileGeom<64, 2, 1, 1, 2, 16>;  // 4x2 pairs/thread: more warps per SM
using CohesionS3 = TileGeom<64, 1, 1, 1, 4, 32>;  // deeper stages
using CohesionS4 = TileGeom<64, 2, 1, 1, 2, 32>;  // 4x2 pairs/thread, deeper stages
using CohesionS5 = TileGeom<64, 1, 1, 1, 4, 32, 4>;  // 32-deep, loop unrolled by 4 (smaller code)
using CohesionS6 = TileGeom<64, 1, 1, 1, 4, 64, 8>;  // 64-deep stages, unrolled by 8
using CohesionS7 = TileGeom<64, 1, 1, 1, 4, 32, 16>;  // S3's tile, TMA-staged, two CTAs per SM

inline int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Defaults from the GB300 autotune table (times in ms, best per order):
//   focus    n=1024: s7 0.117 | 2048: s4 0.515 | 4096: s2/s7 3.52 | 8192: s2/s7 27.1
//   cohesion n=1024: s7 0.229 | 2048: s7 1.118 | 4096: s7 7.17   | 8192: s7 54.6
// Orders below 1024 take the 32-wide tiles so that the launch still covers
// the GPU.
inline int default_focus_schedule(int64_t n) { return n < 1024 ? 1 : 2; }

// Schedule 7 (TMA) needs n % 4 == 0 and aligned buffers; otherwise it runs
// schedule 3's tile with per-thread copies.
inline int default_cohesion_schedule(int64_t n) { return n < 1024 ? 1 : (n % 4 == 0 ? 7 : (n < 4096 ? 4 : 3)); }

}  // namespace pald
