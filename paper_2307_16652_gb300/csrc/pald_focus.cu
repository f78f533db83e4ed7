// Pass 1 (local focus sizes) for one matrix: one CTA per upper-triangle tile
// pair (X <= Y); off-diagonal tiles also write the mirrored tile.
#include "focus_core.cuh"

namespace pald {

namespace {

template <int BM, int G, int MINB>
__global__ void __launch_bounds__(FocusGeom<BM, G>::NT, MINB)
    focus_kernel(const float* __restrict__ D, int64_t n, int32_t* __restrict__ U,
                 const ScanResult* __restrict__ scan, int64_t T) {
  __shared__ __align__(16) float smem[FocusGeom<BM, G>::SMEM_FLOATS];
  int bi, bj;
  tri_decode(blockIdx.x, T, &bi, &bj);
  const float scale = focus_scale(scan->inv_min_pos_bits);
  focus_tile<BM, G>(D, n, U, bi, bj, scale, smem);
}

template <int BM, int G, int MINB>
cudaError_t launch_focus_t(const float* D, int64_t n, int32_t* U, const ScanResult* scan, cudaStream_t s) {
  const int64_t T = (n + BM - 1) / BM;
  const int64_t tiles = T * (T + 1) / 2;
  if (tiles > 0x7fffffff) return cudaErrorInvalidValue;
  focus_kernel<BM, G, MINB><<<static_cast<unsigned>(tiles), FocusGeom<BM, G>::NT, 0, s>>>(D, n, U, scan, T);
  return cudaGetLastError();
}

}  // namespace

// schedule: 0 = 64-tile (4x4 per thread, 256 threads, 2 CTAs per SM),
// 1 = 32-tile (4x4 per thread, 64 threads); -1 = automatic (the 32 tile when
// 64-tiles cannot fill the GPU three times over).
cudaError_t launch_focus(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int schedule,
                         cudaStream_t s) {
  if (schedule < 0) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t T = (n + 63) / 64;
    schedule = (T * (T + 1) / 2 >= 3 * sms) ? 0 : 1;
  }
  if (schedule == 0) return launch_focus_t<64, 1, 2>(D, n, U, scan, s);
  return launch_focus_t<32, 1, 8>(D, n, U, scan, s);
}

}  // namespace pald
