// Tile schedules of both passes and the default choice per matrix order.
//
// A schedule is a tile geometry (see tile_geom.cuh).  The defaults below
// come from timing every schedule on GB300 (the project's autotuner,
// paper_2307_16652_gb300/autotune.py); pald_opts.schedule_id overrides them.
#pragma once

#include <type_traits>

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
using CohesionS5 = TileGeom<64, 1, 1, 1, 4, 32, kMergeEvery>;  // 32-deep, loop unrolled by one merge chunk
using CohesionS6 = TileGeom<64, 1, 1, 1, 4, 64, (kMergeEvery > 8 ? kMergeEvery : 8)>;  // 64-deep stages, unrolled by 8
// S3's tile, TMA-staged, two CTAs per SM, packed stage (cohesion_stage_packed).
// Measured at n = 8192 / 16384 on GB300: a whole stage unrolled (32 y) 47.98
// / 375.3 ms, 16 y 49.37 / 386.5, 8 y 56.8 / 445.5; the scalar stage with 16 y
// 49.70 / 389.0.
// PALD_ACCUM_PLAIN keeps 16 y: unrolled by 32 its build spills 640 bytes.
#ifndef PALD_COH_UNR
#define PALD_COH_UNR 32
#endif
using CohesionS7 = TileGeom<64, 1, 1, 1, 4, 32, PALD_COH_UNR>;
using CohesionS7Plain = TileGeom<64, 1, 1, 1, 4, 32, 16>;
template <int MODE>
using CohesionTmaGeo = std::conditional_t<MODE == PALD_ACCUM_PLAIN, CohesionS7Plain, CohesionS7>;

inline int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// The schedule choices for one range of orders (pald_schedule_bucket).
struct ScheduleBucket {
  int64_t n_max;
  int32_t focus, cohesion, batched_split;
};
constexpr int kMaxBuckets = 16;

// The bucket in force for order n on the current device: the caller's table
// (pald_set_schedule_table), else the autotuned table built into the library
// for this GPU (name and SM count), else the built-in defaults below.
// Returns 0, 1 or 2 for defaults, tuned, caller (pald_get_schedule).
int schedule_for(int64_t n, ScheduleBucket* out);
// Changes whenever a device's table changes (batched plans depend on it).
uint64_t schedule_generation();

// Built-in defaults when no tuned table matches the GPU.  Orders below 1024
// take the 32-wide tiles so that the launch still covers the GPU.
// Schedule 7 (TMA) needs n % 4 == 0 and aligned buffers; otherwise it runs
// the same tile with per-thread copies (schedule 2's tile for pass 1).
inline ScheduleBucket builtin_schedule(int64_t n) {
  return ScheduleBucket{n < 1024 ? 1023 : (int64_t(1) << 20), n < 1024 ? 1 : (n % 4 == 0 ? 7 : 2),
                        n < 1024 ? 1 : (n % 4 == 0 ? 7 : (n < 4096 ? 4 : 3)), 1};
}

inline int default_focus_schedule(int64_t n) {
  ScheduleBucket b;
  schedule_for(n, &b);
  return b.focus;
}
inline int default_cohesion_schedule(int64_t n) {
  ScheduleBucket b;
  schedule_for(n, &b);
  // a tuned TMA choice for an order the TMA tile cannot take runs schedule 3
  // or 4's tile (see launch_cohesion); keep the built-in rule's choice there
  return (b.cohesion == 7 && n % 4 != 0) ? builtin_schedule(n).cohesion : b.cohesion;
}

}  // namespace pald
