// Pass 2 (cohesion) for one matrix: a row-parallel kernel forms R = 1/u with
// a zero diagonal, then one CTA per upper-triangle super-tile slice (X <= Z)
// computes both C[X, Z] and C[Z, X] from the same comparisons, each stage in
// the short or the long form as the tie map says.
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

namespace {

#ifndef PALD_COH_PACKED
#define PALD_COH_PACKED 1
#endif
// The TMA pass-2 tile runs the packed stage (cohesion_stage_packed), which
// reads R in the paired column order.
constexpr bool kPackedTma = PALD_COH_PACKED != 0;

__global__ void __launch_bounds__(256) reciprocal_kernel(const int32_t* __restrict__ U, float* __restrict__ R,
                                                         int64_t n, bool paired) {
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(U) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(R) % 16) == 0;
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) reciprocal_rows(U, n, R, n, row, vec, paired);
}

template <class Geo, int MODE, int MINB>
__global__ void __launch_bounds__(Geo::NT, MINB)
    cohesion_kernel(const float* __restrict__ D, const float* __restrict__ R, int64_t n, float* __restrict__ C,
                    const uint32_t* __restrict__ tmap, const ScanResult* __restrict__ scan, int64_t T,
                    int64_t t0) {
  extern __shared__ __align__(16) float smem[];
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0 * Geo::H, T, Geo::H, &bi, &bj, &slice);
  cohesion_tile<Geo, MODE>(D, R, n, C, tmap, focus_scale(scan->inv_min_pos_bits), bi, bj, slice, smem);
}

template <class Geo, int MODE, int MINB>
cudaError_t launch_t(const float* D, const float* R, int64_t n, float* C, const uint32_t* tmap,
                     const ScanResult* scan, cudaStream_t s, int64_t t0 = 0, int64_t t1 = -1) {
  const int64_t T = (n + Geo::B - 1) / Geo::B;
  if (t1 < 0) t1 = T * (T + 1) / 2;
  const int64_t ctas = (t1 - t0) * Geo::H;
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  const int smem = CohesionSmem<Geo>::FLOATS * static_cast<int>(sizeof(float));
  const cudaError_t e = smem_opt_in(reinterpret_cast<const void*>(cohesion_kernel<Geo, MODE, MINB>), smem);
  if (e != cudaSuccess) return e;
  cohesion_kernel<Geo, MODE, MINB><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(D, R, n, C, tmap, scan, T,
                                                                                    t0);
  return cudaGetLastError();
}

// Set by a CTA whose bounded wait gave up (never in normal operation).
__device__ uint32_t g_cohesion_faults;

#ifndef PALD_COHESION_TMA_MINB
#define PALD_COHESION_TMA_MINB 2
#endif

// With DEPTH the tiles also write their row sums to P (the fused local
// depth, depth_partials).
template <int MODE, bool DEPTH>
__global__ void __launch_bounds__(CohesionTmaGeo<MODE>::NT, PALD_COHESION_TMA_MINB)
    cohesion_tma_kernel(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmR,
                        const float* __restrict__ D, int64_t n, float* __restrict__ C,
                        const uint32_t* __restrict__ tmap, const ScanResult* __restrict__ scan, int64_t T,
                        int64_t t0, double* __restrict__ P) {
  extern __shared__ __align__(128) float smem_tma[];
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0, T, 1, &bi, &bj, &slice);
  using Geo = CohesionTmaGeo<MODE>;
  TmaRing<4, Geo::BK> ring;
  uint32_t* tie_words = reinterpret_cast<uint32_t*>(ring.carve(smem_tma));
  const float S = focus_scale(scan->inv_min_pos_bits);
  if (!cohesion_tile_tma<Geo, MODE, DEPTH, kPackedTma>(&tmD, &tmR, D, n, C, tmap, S, bi, bj, true, ring,
                                                              tie_words, false, P) &&
      threadIdx.x == 0)
    atomicOr(&g_cohesion_faults, 1u);
}

// Self-test of the bounded waits: one CTA runs the TMA pipeline of the pass
// kernels over a few stages whose copies are never issued, so nothing ever
// arrives on the ring's barriers.  Its first wait gives up after `limit_ns`,
// every thread leaves the loop, thread 0 waits (bounded again) for the copies
// it would have had in flight, and the CTA records the fault word exactly as
// a pass-2 kernel does.  Nothing faults or hangs: the kernel ends after
// about three limits.
__global__ void __launch_bounds__(128) wait_selftest_kernel(uint64_t limit_ns) {
  __shared__ __align__(128) float smem_ring[TmaRing<1, 16>::BYTES / 4 + 32];
  TmaRing<1, 16> ring;
  ring.limit_ns = limit_ns;
  ring.carve(smem_ring);
  if (threadIdx.x == 0) ring.init();
  __syncthreads();
  const bool ok = tma_pipeline(ring, kTmaStages + 1, [](int) {}, [](int, int) {});
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  if (!ok && threadIdx.x == 0) atomicOr(&g_cohesion_faults, 1u);
}

// The TMA path needs the row pitch and the base addresses 16-byte aligned.
bool tma_ok(const float* D, const float* R, const float* C, int64_t n) {
  return n >= 64 && n % 4 == 0 && reinterpret_cast<uintptr_t>(D) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(R) % 16 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0;
}

template <int MODE, bool DEPTH = false>
cudaError_t launch_tma(const float* D, const float* R, int64_t n, float* C, const uint32_t* tmap,
                       const ScanResult* scan, cudaStream_t s, int64_t t0 = 0, int64_t t1 = -1,
                       double* P = nullptr) {
  using Geo = CohesionTmaGeo<MODE>;
  const int64_t T = (n + 63) / 64;
  if (t1 < 0) t1 = T * (T + 1) / 2;
  const int64_t ctas = t1 - t0;
  if (ctas <= 0) return cudaSuccess;
  if (ctas > 0x7fffffff) return cudaErrorInvalidValue;
  CUtensorMap mD, mR;
  cudaError_t e = encode_panel_map(&mD, D, n, n, Geo::BK);
  if (e == cudaSuccess) e = encode_panel_map(&mR, R, n, n, Geo::BK);
  if (e != cudaSuccess) return e;
  const int smem = CohesionTmaSmem<Geo>::bytes(n);  // TMA ring + tie words
  e = smem_opt_in(reinterpret_cast<const void*>(cohesion_tma_kernel<MODE, DEPTH>), CohesionTmaSmem<Geo>::MAX_BYTES);
  if (e != cudaSuccess) return e;
  cohesion_tma_kernel<MODE, DEPTH><<<static_cast<unsigned>(ctas), Geo::NT, smem, s>>>(mD, mR, D, n, C, tmap, scan, T,
                                                                                     t0, P);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_mode(const float* D, const float* R, int64_t n, float* C, const uint32_t* tmap,
                        const ScanResult* scan, int schedule, cudaStream_t s) {
  switch (schedule) {
    case 0: return launch_t<CohesionS0, MODE, 1>(D, R, n, C, tmap, scan, s);
    case 1: return launch_t<CohesionS1, MODE, 4>(D, R, n, C, tmap, scan, s);
    case 2: return launch_t<CohesionS2, MODE, 2>(D, R, n, C, tmap, scan, s);
    case 3: return launch_t<CohesionS3, MODE, 1>(D, R, n, C, tmap, scan, s);
    case 4: return launch_t<CohesionS4, MODE, 2>(D, R, n, C, tmap, scan, s);
    case 5: return launch_t<CohesionS5, MODE, 1>(D, R, n, C, tmap, scan, s);
    case 6: return launch_t<CohesionS6, MODE, 1>(D, R, n, C, tmap, scan, s);
    case 7:
      if (tma_ok(D, R, C, n)) return launch_tma<MODE>(D, R, n, C, tmap, scan, s);
      return launch_t<CohesionS3, MODE, 1>(D, R, n, C, tmap, scan, s);  // same tile with per-thread copies
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_reciprocal(const int32_t* U, float* R, int64_t n, cudaStream_t s, bool paired) {
  const int64_t cap = int64_t(sm_count()) * 16;
  const int64_t grid = n < cap ? n : cap;
  reciprocal_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(U, R, n, paired);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 128, 0, s>>>(limit_ns);
  return cudaGetLastError();
}

cudaError_t take_cohesion_faults(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_cohesion_faults, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out != 0u)
    e = cudaMemcpyToSymbolAsync(g_cohesion_faults, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

cudaError_t encode_panel_map(CUtensorMap* map, const float* base, int64_t n, int64_t pitch, int rows) {
  return encode_rect_map(map, base, n, n, pitch, rows);
}

cudaError_t encode_rect_map(CUtensorMap* map, const float* base, int64_t cols, int64_t nrows, int64_t pitch,
                            int rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(nrows)};  // {columns, rows}
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch) * sizeof(float)};       // row pitch, bytes
  const cuuint32_t box[2] = {64u, static_cast<cuuint32_t>(rows)};
  const cuuint32_t elem[2] = {1u, 1u};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
                            elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_cohesion_range(const float* D, const int32_t* U, float* R, int64_t n, float* C,
                                  const uint32_t* tmap, const ScanResult* scan, int accum_mode, int64_t t0, int64_t t1,
                                  cudaStream_t s) {
  // the 64 x 64 tiles of the shard plan: TMA-staged when the layout allows
  const bool tma = tma_ok(D, R, C, n);
  const cudaError_t e = launch_reciprocal(U, R, n, s, tma && kPackedTma);
  if (e != cudaSuccess) return e;
  if (accum_mode == PALD_ACCUM_PLAIN)
    return tma ? launch_tma<PALD_ACCUM_PLAIN>(D, R, n, C, tmap, scan, s, t0, t1)
               : launch_t<CohesionS3, PALD_ACCUM_PLAIN, 1>(D, R, n, C, tmap, scan, s, t0, t1);
  return tma ? launch_tma<PALD_ACCUM_COMPENSATED>(D, R, n, C, tmap, scan, s, t0, t1)
             : launch_t<CohesionS3, PALD_ACCUM_COMPENSATED, 1>(D, R, n, C, tmap, scan, s, t0, t1);
}

// R comes from the stream-ordered allocator (256-byte aligned).
bool cohesion_depth_fused_ok(const float* D, const float* C, int64_t n) { return tma_ok(D, D, C, n); }

cudaError_t launch_cohesion_depth(const float* D, const int32_t* U, float* R, int64_t n, float* C,
                                  const uint32_t* tmap, const ScanResult* scan, int accum_mode, double* P,
                                  cudaStream_t s) {
  if (!tma_ok(D, R, C, n)) return cudaErrorInvalidValue;
  const cudaError_t e = launch_reciprocal(U, R, n, s, kPackedTma);
  if (e != cudaSuccess) return e;
  if (accum_mode == PALD_ACCUM_PLAIN) return launch_tma<PALD_ACCUM_PLAIN, true>(D, R, n, C, tmap, scan, s, 0, -1, P);
  return launch_tma<PALD_ACCUM_COMPENSATED, true>(D, R, n, C, tmap, scan, s, 0, -1, P);
}

cudaError_t launch_cohesion(const float* D, const int32_t* U, float* R, int64_t n, float* C, const uint32_t* tmap,
                            const ScanResult* scan, int accum_mode, int schedule, cudaStream_t s) {
  if (schedule < 0) schedule = default_cohesion_schedule(n);
  const cudaError_t e = launch_reciprocal(U, R, n, s, schedule == 7 && tma_ok(D, R, C, n) && kPackedTma);
  if (e != cudaSuccess) return e;
  if (accum_mode == PALD_ACCUM_PLAIN) return launch_mode<PALD_ACCUM_PLAIN>(D, R, n, C, tmap, scan, schedule, s);
  return launch_mode<PALD_ACCUM_COMPENSATED>(D, R, n, C, tmap, scan, schedule, s);
}

}  // namespace pald
