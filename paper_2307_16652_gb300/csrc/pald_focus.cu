// Pass 1 (local focus sizes) for one matrix: one CTA per upper-triangle
// super-tile slice (X <= Y); off-diagonal super-tiles also write the mirror.
// Schedule 7 stages the operands with TMA (tma_ring.cuh).
#include "focus_core.cuh"
#include "schedules.cuh"

namespace pald {

namespace {

template <class Geo, int MINB>
__global__ void __launch_bounds__(Geo::NT, MINB)
    focus_kernel(const float* __restrict__ D, int64_t n, int32_t* __restrict__ U,
                 const ScanResult* __restrict__ scan, int64_t T, int64_t t0) {
  extern __shared__ __align__(16) float smem[];
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0 * Geo::H, T, Geo::H, &bi, &bj, &slice);
  const float scale = focus_scale(scan->inv_min_pos_bits);
  focus_tile<Geo>(D, n, U, bi, bj, slice, scale, smem);
}

// Set by a CTA whose bounded wait gave up (never in normal operation).
__device__ uint32_t g_focus_faults;

// Three CTAs per SM (80 registers): measured 12% faster than two CTAs with
// 128 registers at n = 8192 on GB300 (23.9 against 27.1 ms).
#ifndef PALD_FOCUS_TMA_MINB
#define PALD_FOCUS_TMA_MINB 3
#endif

template <class Geo>
__global__ void __launch_bounds__(Geo::NT, PALD_FOCUS_TMA_MINB)
    focus_tma_kernel(const __grid_constant__ CUtensorMap tmD, const float* __restrict__ D, int64_t n,
                     int32_t* __restrict__ U, const ScanResult* __restrict__ scan, int64_t T, int64_t t0) {
  extern __shared__ __align__(128) float smem_tma[];
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0, T, 1, &bi, &bj, &slice);
  TmaRing<2, Geo::BK> ring;
  ring.carve(smem_tma);
  const float scale = focus_scale(scan->inv_min_pos_bits);
  if (!focus_tile_tma<Geo>(&tmD, D, n, U, bi, bj, scale, true, ring, nullptr, 0, true) && threadIdx.x == 0)
    atomicOr(&g_focus_faults, 1u);
}

// The TMA path needs the row pitch and the base addresses 16-byte aligned.
bool focus_tma_ok(const float* D, const int32_t* U, int64_t n) {
  return n >= 64 && n % 4 == 0 && reinterpret_cast<uintptr_t>(D) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(U) % 16 == 0;
}

template <class Geo>
cudaError_t launch_tma(const float* D, int64_t n, int32_t* U, const ScanResult* scan, cudaStream_t s, int64_t t0,
                       int64_t t1) {
  const int64_t T = (n + 63) / 64;
  if (t1 < 0) t1 = T * (T + 1) / 2;
  const int64_t ctas = t1 - t0;
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  CUtensorMap mD;
  cudaError_t e = encode_panel_map(&mD, D, n, n, Geo::BK);
  if (e != cudaSuccess) return e;
  const int smem = TmaRing<2, Geo::BK>::BYTES + 128;
  if ((e = smem_opt_in(reinterpret_cast<const void*>(focus_tma_kernel<Geo>), smem)) != cudaSuccess) return e;
  focus_tma_kernel<Geo><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(mD, D, n, U, scan, T, t0);
  return cudaGetLastError();
}

template <class Geo, int MINB>
cudaError_t launch_t(const float* D, int64_t n, int32_t* U, const ScanResult* scan, cudaStream_t s, int64_t t0 = 0,
                     int64_t t1 = -1) {
  const int64_t T = (n + Geo::B - 1) / Geo::B;
  if (t1 < 0) t1 = T * (T + 1) / 2;
  const int64_t ctas = (t1 - t0) * Geo::H;
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  const int smem = FocusSmem<Geo>::FLOATS * static_cast<int>(sizeof(float));
  const cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(focus_kernel<Geo, MINB>), smem);
  if (e != cudaSuccess) return e;
  focus_kernel<Geo, MINB><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(D, n, U, scan, T, t0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t take_focus_faults(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_focus_faults, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out != 0u)
    e = cudaMemcpyToSymbolAsync(g_focus_faults, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t launch_focus(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int schedule,
                         cudaStream_t s) {
  if (schedule < 0) schedule = default_focus_schedule(n);
  switch (schedule) {
    case 0: return launch_t<FocusS0, 2>(D, n, U, scan, s);
    case 1: return launch_t<FocusS1, 8>(D, n, U, scan, s);
    case 2: return launch_t<FocusS2, 2>(D, n, U, scan, s);
    case 3: return launch_t<FocusS3, 1>(D, n, U, scan, s);
    case 4: return launch_t<FocusS4, 4>(D, n, U, scan, s);
    case 5: return launch_t<FocusS5, 2>(D, n, U, scan, s);
    case 6: return launch_t<FocusS6, 1>(D, n, U, scan, s);
    case 7:
      if (focus_tma_ok(D, U, n)) return launch_tma<FocusS7>(D, n, U, scan, s, 0, -1);
      return launch_t<FocusS2, 2>(D, n, U, scan, s);  // same tile with per-thread copies
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_focus_range(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int64_t t0, int64_t t1,
                               cudaStream_t s) {
  // the 64 x 64 tiles of the shard plan: TMA-staged when the layout allows
  if (focus_tma_ok(D, U, n)) return launch_tma<FocusS7>(D, n, U, scan, s, t0, t1);
  return launch_t<FocusS2, 2>(D, n, U, scan, s, t0, t1);
}

}  // namespace pald
