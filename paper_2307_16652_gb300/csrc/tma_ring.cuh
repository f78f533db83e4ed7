// Operand staging by TMA for both passes.
//
// A ring of kTmaStages shared-memory buffers; each buffer holds P panels of
// BK rows x 64 columns (FP32) and has one mbarrier.  One thread issues a
// stage's P tensor copies (2-D boxes of the n x n matrix, rows y0..y0+BK-1,
// 64 columns from an x that is a multiple of 64, zero-filled outside the
// matrix) with one expect-tx arrival; the copies complete the barrier's
// phase.  Every thread waits on the phase with a time limit.  One CTA
// barrier per stage tells the issuing thread that the buffer it refills next
// (the one read in the previous stage) is free, and keeps all warps on the
// same stage.
#pragma once

#include "pald_internal.cuh"

namespace pald {

constexpr int kTmaStages = 3;

template <int P, int BK>
struct TmaRing {
  static constexpr int PANEL = BK * 64;                 // floats of one panel
  static constexpr int FLOATS = kTmaStages * P * PANEL;
  static constexpr int BYTES = FLOATS * 4 + 8 * kTmaStages;
  static constexpr uint32_t STAGE_BYTES = P * PANEL * 4u;

  float* panels;   // [kTmaStages][P][BK][64], 128-byte aligned
  uint64_t* bars;  // [kTmaStages]
  uint64_t limit_ns = kWaitLimitNs;  // how long a wait may take before it gives up

  // Places the ring at the first 128-byte boundary of `smem` (a shared
  // array; offsets keep the compiler on shared-memory loads).  Returns the
  // first float after the ring.
  __device__ __forceinline__ float* carve(float* smem) {
    const int pad = static_cast<int>((128u - (smem_u32(smem) & 127u)) & 127u) / 4;
    panels = smem + pad;
    bars = reinterpret_cast<uint64_t*>(panels + FLOATS);
    return reinterpret_cast<float*>(bars + kTmaStages);
  }
  __device__ __forceinline__ float* panel(int buf, int k) const { return panels + (buf * P + k) * PANEL; }

  // One thread: fresh barriers (the ring's previous user, if any, called inval).
  __device__ __forceinline__ void init() const {
#pragma unroll
    for (int b = 0; b < kTmaStages; ++b) mbar_init(smem_u32(bars + b), 1);
    mbar_fence_init();
  }
  // One thread, after every wait of the ring's last use has returned.
  __device__ __forceinline__ void inval() const {
#pragma unroll
    for (int b = 0; b < kTmaStages; ++b)
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bars + b)) : "memory");
  }
  // One thread: stage q's panels k = 0..P-1 from maps[k] at column cols[k].
  __device__ __forceinline__ void issue(int q, const CUtensorMap* const (&maps)[P], const int (&cols)[P]) const {
    const int buf = q % kTmaStages;
    const uint32_t bar = smem_u32(bars + buf);
    mbar_expect_tx(bar, STAGE_BYTES);
#pragma unroll
    for (int k = 0; k < P; ++k) tma_load_2d(smem_u32(panel(buf, k)), maps[k], cols[k], q * BK, bar);
  }
  __device__ __forceinline__ bool wait(int st) const {
    return mbar_wait_bounded(smem_u32(bars + st % kTmaStages), static_cast<uint32_t>((st / kTmaStages) & 1),
                             limit_ns);
  }
};

// Runs stages 0..nstages-1 through `ring`: `issue(q)` (called by thread 0)
// starts stage q's copies, `compute(st, buf)` consumes stage st from buffer
// buf.  Returns false when a wait ran out of time: every thread then stops,
// and thread 0 first waits (bounded again) for the copies it had issued.
template <class Ring, class Issue, class Compute>
__device__ __forceinline__ bool tma_pipeline(const Ring& ring, int nstages, Issue issue, Compute compute) {
  if (threadIdx.x == 0)
    for (int q = 0; q < kTmaStages - 1 && q < nstages; ++q) issue(q);
  int st = 0;
  for (; st < nstages; ++st) {
    const bool ok = ring.wait(st);
    // stage st has landed for every thread (or some thread gave up), and
    // every thread is done with stage st-1's buffer, which is refilled next
    if (__syncthreads_or(!ok)) break;
    if (threadIdx.x == 0 && st + kTmaStages - 1 < nstages) issue(st + kTmaStages - 1);
    compute(st, st % kTmaStages);
  }
  if (st < nstages) {
    if (threadIdx.x == 0)
      for (int q = st; q < st + kTmaStages - 1 && q < nstages; ++q) ring.wait(q);
    __syncthreads();
    return false;
  }
  return true;
}

}  // namespace pald
