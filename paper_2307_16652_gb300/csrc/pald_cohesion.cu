// Pass 2 (cohesion) for one matrix: a row-parallel kernel forms R = 1/u with
// a zero diagonal, then one CTA per upper-triangle tile pair (X <= Z)
// computes both C[X, Z] and C[Z, X] from the same comparisons.
#include "cohesion_core.cuh"

namespace pald {

namespace {

__global__ void __launch_bounds__(256) reciprocal_kernel(const int32_t* __restrict__ U, float* __restrict__ R,
                                                         int64_t n) {
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(U) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(R) % 16) == 0;
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) reciprocal_rows(U, R, n, row, vec);
}

template <int BM, int G, int MODE>
__global__ void __launch_bounds__(CohesionGeom<BM, G>::NT, 1)
    cohesion_kernel(const float* __restrict__ D, const float* __restrict__ R, int64_t n, float* __restrict__ C,
                    int64_t T) {
  __shared__ __align__(16) float smem[CohesionGeom<BM, G>::SMEM_FLOATS];
  int bi, bj;
  tri_decode(blockIdx.x, T, &bi, &bj);
  cohesion_tile<BM, G, MODE>(D, R, n, C, bi, bj, smem);
}

template <int BM, int G, int MODE>
cudaError_t launch_t(const float* D, const float* R, int64_t n, float* C, cudaStream_t s) {
  const int64_t T = (n + BM - 1) / BM;
  const int64_t tiles = T * (T + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  cohesion_kernel<BM, G, MODE><<<static_cast<unsigned>(tiles), CohesionGeom<BM, G>::NT, 0, s>>>(D, R, n, C, T);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reciprocal(const int32_t* U, float* R, int64_t n, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = n < int64_t(sms) * 16 ? n : int64_t(sms) * 16;
  reciprocal_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(U, R, n);
  return cudaGetLastError();
}

// schedule: 0 = 64-tile (4x4 per thread, 256 threads), 1 = 32-tile (4x4 per
// thread, 64 threads); -1 = automatic (32 when 64-tiles cannot fill the GPU).
cudaError_t launch_cohesion(const float* D, const float* R, int64_t n, float* C, int accum_mode, int schedule,
                            cudaStream_t s) {
  if (schedule < 0) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t T = (n + 63) / 64;
    schedule = (T * (T + 1) / 2 >= 2 * sms) ? 0 : 1;
  }
  const bool plain = accum_mode == PALD_ACCUM_PLAIN;
  if (schedule == 0)
    return plain ? launch_t<64, 1, PALD_ACCUM_PLAIN>(D, R, n, C, s)
                 : launch_t<64, 1, PALD_ACCUM_COMPENSATED>(D, R, n, C, s);
  return plain ? launch_t<32, 1, PALD_ACCUM_PLAIN>(D, R, n, C, s)
               : launch_t<32, 1, PALD_ACCUM_COMPENSATED>(D, R, n, C, s);
}

}  // namespace pald
