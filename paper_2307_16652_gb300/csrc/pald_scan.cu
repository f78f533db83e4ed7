// Input scan and validation of a distance matrix.
//
// The scan finds the smallest positive entry and the largest entry; pass 1
// derives from them the single power-of-two scale that turns "m > t" into one
// saturating FFMA for every threshold of the matrix.  Validation checks the
// input contract stated in pald.h (symmetry bit for bit, +0.0 diagonal,
// finite non-negative entries, positive entries >= 2^-100) with a tiled
// transpose so that both reads stay coalesced.
#include "pald_internal.cuh"

namespace pald {

namespace {

constexpr uint32_t kTinyBits = 0x0d800000u;  // bit pattern of 2^-100
constexpr int kScanThreads = 256;

__device__ __forceinline__ void scan_value(uint32_t b, uint32_t& inv_min, uint32_t& mx) {
  // non-negative finite values order like their bit patterns
  const bool finite_nonneg = b < 0x7f800000u;
  if (finite_nonneg && b != 0u) inv_min = max(inv_min, ~b);
  if (finite_nonneg) mx = max(mx, b);
}

__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// min positive and max over `count` consecutive elements (vectorised body)
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const float* __restrict__ D, int64_t count,
                                                            ScanResult* __restrict__ out) {
  uint32_t inv_min = 0u, mx = 0u;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t nvec = (reinterpret_cast<uintptr_t>(D) % 16 == 0) ? count / 4 : 0;
  const uint4* D4 = reinterpret_cast<const uint4*>(D);
  for (int64_t i = tid; i < nvec; i += stride) {
    uint4 v = __ldg(D4 + i);
    scan_value(v.x, inv_min, mx);
    scan_value(v.y, inv_min, mx);
    scan_value(v.z, inv_min, mx);
    scan_value(v.w, inv_min, mx);
  }
  for (int64_t i = nvec * 4 + tid; i < count; i += stride) scan_value(__float_as_uint(__ldg(D + i)), inv_min, mx);
  inv_min = warp_max(inv_min);
  mx = warp_max(mx);
  __shared__ uint32_t s_inv[kScanThreads / 32], s_mx[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_inv[warp] = inv_min;
    s_mx[warp] = mx;
  }
  __syncthreads();
  if (warp == 0) {
    inv_min = lane < kScanThreads / 32 ? s_inv[lane] : 0u;
    mx = lane < kScanThreads / 32 ? s_mx[lane] : 0u;
    inv_min = warp_max(inv_min);
    mx = warp_max(mx);
    if (lane == 0) {
      if (inv_min) atomicMax(&out->inv_min_pos_bits, inv_min);
      if (mx) atomicMax(&out->max_bits, mx);
    }
  }
}

// Validation over 32 x 32 tile pairs (bi <= bj).
__global__ void __launch_bounds__(256) validate_kernel(const float* __restrict__ D, int64_t n,
                                                       ScanResult* __restrict__ out) {
  const int64_t bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  __shared__ uint32_t tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  uint32_t flags = 0u;
  // load the (bj, bi) tile transposed into smem
  for (int r = ty; r < 32; r += 8) {
    const int64_t row = bj * 32 + r, col = bi * 32 + tx;
    tile[r][tx] = (row < n && col < n) ? __float_as_uint(__ldg(D + row * n + col)) : 0u;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t row = bi * 32 + r, col = bj * 32 + tx;
    if (row >= n || col >= n) continue;
    const uint32_t b = __float_as_uint(__ldg(D + row * n + col));
    if (b != tile[tx][r]) flags |= kFlagAsymmetric;
    if (row == col) {
      if (b != 0u) flags |= kFlagBadDiagonal;
    } else {
      if (b >= 0x7f800000u) flags |= kFlagBadValue;          // NaN, inf or sign bit set
      if (b != 0u && b < kTinyBits) flags |= kFlagBadValue;  // positive below 2^-100
    }
  }
  flags = __reduce_or_sync(0xffffffffu, flags);
  if ((threadIdx.x & 31) == 0 && flags) atomicOr(&out->flags, flags);
}

}  // namespace

cudaError_t launch_scan(const float* D, int64_t n, ScanResult* out, bool validate, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(ScanResult), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t count = n * n;
  int64_t want = (count / 4 + kScanThreads - 1) / kScanThreads;
  int grid = static_cast<int>(want < int64_t(sms) * 8 ? (want > 0 ? want : 1) : int64_t(sms) * 8);
  scan_kernel<<<grid, kScanThreads, 0, s>>>(D, count, out);
  e = cudaGetLastError();
  if (e != cudaSuccess || !validate) return e;
  const int64_t T = (n + 31) / 32;
  if (T > 65535) return cudaErrorInvalidValue;
  dim3 g(static_cast<unsigned>(T), static_cast<unsigned>(T));
  validate_kernel<<<g, 256, 0, s>>>(D, n, out);
  return cudaGetLastError();
}

}  // namespace pald
