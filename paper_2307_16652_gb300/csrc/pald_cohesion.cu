// Pass 2 (cohesion) for one matrix: one CTA per upper-triangle tile pair
// (X <= Z) computes both C[X, Z] and C[Z, X] from the same comparisons.
#include "cohesion_core.cuh"

namespace pald {

namespace {

template <int BM, int G, int MODE>
__global__ void __launch_bounds__(CohesionGeom<BM, G>::NT, 1)
    cohesion_kernel(const float* __restrict__ D, const int32_t* __restrict__ U, int64_t n, float* __restrict__ C,
                    int64_t T) {
  __shared__ __align__(16) float smem[CohesionGeom<BM, G>::SMEM_FLOATS];
  int bi, bj;
  tri_decode(blockIdx.x, T, &bi, &bj);
  cohesion_tile<BM, G, MODE>(D, U, n, C, bi, bj, smem);
}

template <int BM, int G, int MODE>
cudaError_t launch_t(const float* D, const int32_t* U, int64_t n, float* C, cudaStream_t s) {
  const int64_t T = (n + BM - 1) / BM;
  const int64_t tiles = T * (T + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  cohesion_kernel<BM, G, MODE><<<static_cast<unsigned>(tiles), CohesionGeom<BM, G>::NT, 0, s>>>(D, U, n, C, T);
  return cudaGetLastError();
}

}  // namespace

// schedule: 0 = 64-tile (4x4 per thread, 256 threads), 1 = 32-tile (4x4 per
// thread, 64 threads); -1 = automatic (32 when 64-tiles cannot fill the GPU).
cudaError_t launch_cohesion(const float* D, const int32_t* U, int64_t n, float* C, int accum_mode, int schedule,
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
    return plain ? launch_t<64, 1, PALD_ACCUM_PLAIN>(D, U, n, C, s)
                 : launch_t<64, 1, PALD_ACCUM_COMPENSATED>(D, U, n, C, s);
  return plain ? launch_t<32, 1, PALD_ACCUM_PLAIN>(D, U, n, C, s)
               : launch_t<32, 1, PALD_ACCUM_COMPENSATED>(D, U, n, C, s);
}

}  // namespace pald
