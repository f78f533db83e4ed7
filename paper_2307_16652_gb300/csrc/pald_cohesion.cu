// Pass 2 (cohesion) for one matrix: a row-parallel kernel forms R = 1/u with
// a zero diagonal, then one CTA per upper-triangle super-tile slice (X <= Z)
// computes both C[X, Z] and C[Z, X] from the same comparisons.
#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

namespace {

__global__ void __launch_bounds__(256) reciprocal_kernel(const int32_t* __restrict__ U, float* __restrict__ R,
                                                         int64_t n) {
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(U) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(R) % 16) == 0;
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) reciprocal_rows(U, R, n, row, vec);
}

template <class Geo, int MODE, int MINB>
__global__ void __launch_bounds__(Geo::NT, MINB)
    cohesion_kernel(const float* __restrict__ D, const float* __restrict__ R, int64_t n, float* __restrict__ C,
                    int64_t T) {
  extern __shared__ __align__(16) float smem[];
  int bi, bj, slice;
  decode_tile(blockIdx.x, T, Geo::H, &bi, &bj, &slice);
  cohesion_tile<Geo, MODE>(D, R, n, C, bi, bj, slice, smem);
}

template <class Geo, int MODE, int MINB>
cudaError_t launch_t(const float* D, const float* R, int64_t n, float* C, cudaStream_t s) {
  const int64_t T = (n + Geo::B - 1) / Geo::B;
  const int64_t ctas = T * (T + 1) / 2 * Geo::H;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  const int smem = CohesionSmem<Geo>::FLOATS * static_cast<int>(sizeof(float));
  static bool attr_set = false;  // idempotent: racing setters write the same value
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(cohesion_kernel<Geo, MODE, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cohesion_kernel<Geo, MODE, MINB><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(D, R, n, C, T);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const float* D, const float* R, int64_t n, float* C, int schedule, cudaStream_t s) {
  switch (schedule) {
    case 0: return launch_t<CohesionS0, MODE, 1>(D, R, n, C, s);
    case 1: return launch_t<CohesionS1, MODE, 4>(D, R, n, C, s);
    case 2: return launch_t<CohesionS2, MODE, 2>(D, R, n, C, s);
    case 3: return launch_t<CohesionS3, MODE, 1>(D, R, n, C, s);
    case 4: return launch_t<CohesionS4, MODE, 2>(D, R, n, C, s);
    case 5: return launch_t<CohesionS5, MODE, 1>(D, R, n, C, s);
    case 6: return launch_t<CohesionS6, MODE, 1>(D, R, n, C, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_reciprocal(const int32_t* U, float* R, int64_t n, cudaStream_t s) {
  const int64_t cap = int64_t(sm_count()) * 16;
  const int64_t grid = n < cap ? n : cap;
  reciprocal_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(U, R, n);
  return cudaGetLastError();
}

cudaError_t launch_cohesion(const float* D, const float* R, int64_t n, float* C, int accum_mode, int schedule,
                            cudaStream_t s) {
  if (schedule < 0) schedule = default_cohesion_schedule(n);
  if (accum_mode == PALD_ACCUM_PLAIN) return launch_mode<PALD_ACCUM_PLAIN>(D, R, n, C, schedule, s);
  return launch_mode<PALD_ACCUM_COMPENSATED>(D, R, n, C, schedule, s);
}

}  // namespace pald
