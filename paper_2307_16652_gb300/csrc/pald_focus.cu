// Pass 1 (local focus sizes) for one matrix: one CTA per upper-triangle
// super-tile slice (X <= Y); off-diagonal super-tiles also write the mirror.
#include "focus_core.cuh"
#include "schedules.cuh"

namespace pald {

namespace {

template <class Geo, int MINB>
__global__ void __launch_bounds__(Geo::NT, MINB)
    focus_kernel(const float* __restrict__ D, int64_t n, int32_t* __restrict__ U,
                 const ScanResult* __restrict__ scan, int64_t T) {
  extern __shared__ __align__(16) float smem[];
  int bi, bj, slice;
  decode_tile(blockIdx.x, T, Geo::H, &bi, &bj, &slice);
  const float scale = focus_scale(scan->inv_min_pos_bits);
  focus_tile<Geo>(D, n, U, bi, bj, slice, scale, smem);
}

template <class Geo, int MINB>
cudaError_t launch_t(const float* D, int64_t n, int32_t* U, const ScanResult* scan, cudaStream_t s) {
  const int64_t T = (n + Geo::B - 1) / Geo::B;
  const int64_t ctas = T * (T + 1) / 2 * Geo::H;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  const int smem = FocusSmem<Geo>::FLOATS * static_cast<int>(sizeof(float));
  static bool attr_set = false;  // idempotent: racing setters write the same value
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(focus_kernel<Geo, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  focus_kernel<Geo, MINB><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(D, n, U, scan, T);
  return cudaGetLastError();
}

}  // namespace

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
    case 7: return launch_t<FocusS7, 2>(D, n, U, scan, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pald
