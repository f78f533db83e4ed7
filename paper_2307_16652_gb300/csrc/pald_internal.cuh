// Internal declarations shared by the libpald translation units.
//
// Everything here is device plumbing for the CUDA path: PTX wrappers, tile
// geometry, the scan summary the passes read, and host launch helpers.  None
// of it is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pald.h"

namespace pald {

// ---------------------------------------------------------------------------
// Scan summary of one matrix, produced on the device before pass 1.
struct ScanResult {
  uint32_t inv_min_pos_bits;  // ~(bit pattern of the smallest positive entry); 0 if none
  uint32_t max_bits;          // bit pattern of the largest entry
  uint32_t flags;             // validation flags (kFlag* below), 0 when valid
  uint32_t pad;
};

// Scale 2^(23 - e) with e the exponent of the smallest positive entry: for
// every threshold t of the matrix, sat(m * s - t * s) is exactly [m > t].
__host__ __device__ __forceinline__ float focus_scale(uint32_t inv_min_pos_bits) {
  if (inv_min_pos_bits == 0u) return 1.0f;
  const int e = static_cast<int>(((~inv_min_pos_bits) >> 23) & 0xffu) - 127;
  int k = 23 - e;
  if (k > 127) k = 127;
  if (k < -126) k = -126;
  union { uint32_t u; float f; } v;
  v.u = static_cast<uint32_t>(k + 127) << 23;
  return v.f;
}

enum : uint32_t {
  kFlagAsymmetric = 1u,
  kFlagBadDiagonal = 2u,
  kFlagBadValue = 4u,  // NaN, inf, sign bit set, or a positive value below 2^-100
  kFlagRange = 8u,     // max / min_pos too large for the exact step construction
};

// ---------------------------------------------------------------------------
// PTX wrappers.  The passes decide every comparison on the FP32 inputs; the
// helpers only pin the instruction forms that keep the work on the FMA pipe.

// sat(a * s + c): one FFMA with saturation to [0, 1].
__device__ __forceinline__ float ffma_sat(float a, float s, float c) {
  float r;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(s), "f"(c));
  return r;
}

__device__ __forceinline__ float fmin_(float a, float b) {
  float r;
  asm("min.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// 16-byte async copy global -> shared; src_bytes < 16 zero-fills the rest.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float exp2i(int e) { return __uint_as_float(static_cast<uint32_t>(e + 127) << 23); }

// Unbiased exponent of a positive normal float.
__device__ __forceinline__ int exponent_of(float v) {
  return static_cast<int>((__float_as_uint(v) >> 23) & 0xffu) - 127;
}

// ---------------------------------------------------------------------------
// Upper-triangle tile enumeration: linear index -> (bi, bj), bi <= bj, with
// all tiles of block-row bi consecutive (consecutive CTAs share the bi panel).
__host__ __device__ __forceinline__ void tri_decode(int64_t t, int64_t T, int* bi, int* bj) {
  // row r holds T - r tiles; start(r) = r*T - r*(r-1)/2
  double tt = static_cast<double>(T) + 0.5;
  int64_t r = static_cast<int64_t>(tt - sqrt(tt * tt - 2.0 * static_cast<double>(t)));
  if (r < 0) r = 0;
  if (r > T - 1) r = T - 1;
  auto start = [T](int64_t q) { return q * T - q * (q - 1) / 2; };
  while (r > 0 && start(r) > t) --r;
  while (r + 1 < T && start(r + 1) <= t) ++r;
  *bi = static_cast<int>(r);
  *bj = static_cast<int>(r + (t - start(r)));
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).

cudaError_t launch_scan(const float* D, int64_t n, ScanResult* out, bool validate, cudaStream_t s);
cudaError_t launch_focus(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int schedule,
                         cudaStream_t s);
cudaError_t launch_reciprocal(const int32_t* U, float* R, int64_t n, cudaStream_t s);
cudaError_t launch_cohesion(const float* D, const float* R, int64_t n, float* C, int accum_mode, int schedule,
                            cudaStream_t s);

// Batched: descriptors of every matrix, and a flat list of tile work items.
struct MatrixDesc {
  int64_t off;  // element offset of the matrix in D, U and C
  int32_t n;
  int32_t tiles_focus;     // number of upper-triangle tiles of the pass-1 schedule
  int32_t tiles_cohesion;  // same for pass 2
  int32_t pad;
};
struct WorkItem {
  int32_t matrix;
  int32_t bi, bj;
  int32_t slice;  // column slice of the super-tile
};

}  // namespace pald
