// Internal declarations shared by the libpald translation units.
//
// Everything here is device plumbing for the CUDA path: PTX wrappers, tile
// geometry, the scan summary the passes read, and host launch helpers.  None
// of it is shared with the CPU oracle.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pald.h"

namespace pald {

// y per FP32 partial of the compensated cohesion sums (pass 2): every
// kMergeEvery consecutive y the partial is folded into the running sum.
#ifndef PALD_MERGE_EVERY
#define PALD_MERGE_EVERY 8
#endif
constexpr int kMergeEvery = PALD_MERGE_EVERY;
static_assert(kMergeEvery == 4 || kMergeEvery == 8 || kMergeEvery == 16,
              "partials span 4, 8 or 16 y (the bias is then a power of two)");

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

// ---------------------------------------------------------------------------
// mbarrier and TMA (tensor copy) wrappers.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// Makes initialised mbarriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n\tfence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival that also announces `bytes` of incoming transaction data.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One plain arrival.
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0u;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Every wait on an mbarrier is bounded: after this long the waiter gives up
// and reports a fault instead of hanging the GPU.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// 2-D tensor copy global -> shared of one box at coordinates (x = column,
// y = row); completes `bar`'s transaction count.  x * 4 must be a multiple
// of 16 bytes; rows and columns outside the tensor read as zero.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

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
// Tie map of one matrix, read by pass 2 to choose its per-stage inner loop.
//
// Pass 2 has a 4-instruction form that is exact unless a one-sided tie
// d_xy == d_xz (or d_zy == d_zx) occurs; such a tie is two equal entries in
// one row of D.  The map holds one bit per (pair of 64-blocks {X, Z}, group
// of `group` consecutive y): set when some row r of X or Z has two equal
// entries at columns p and q with the block of q being the other side of the
// pair and p in the y group.  `dirty[b]` marks a block with a row whose
// repeats were too many to list; every stage of a tile touching it takes the
// exact loop.  Layout: words[nb][nb][wpp] then dirty[nb], all uint32.
// Groups are 8 y up to n = 65536 (a sparse tie marks a quarter of a 32-y
// stage, and a stage with some marked groups runs the long form on those
// groups only), 32 y beyond, where the map's n^3 / 2^18 bytes would grow
// past 1 GB.
constexpr int kTieBlock = 64;        // rows / columns per block of the map
constexpr int kTieGroupFine = 8;     // y per group for n <= kTieFineMaxN
constexpr int kTieGroupCoarse = 32;  // y per group beyond
constexpr int64_t kTieFineMaxN = 65536;

struct TieMapDims {
  int64_t nb;   // blocks per side, ceil(n / 64)
  int64_t wpp;  // words per block pair, ceil(ceil(n / group) / 32)
  int group;    // y per group
  int gshift;   // log2(group): every group index is a shift, not a 64-bit division
};

__host__ __device__ __forceinline__ TieMapDims tie_map_dims(int64_t n) {
  TieMapDims d;
  static_assert(kTieGroupFine == 8 && kTieGroupCoarse == 32, "group sizes are powers of two");
  d.group = n <= kTieFineMaxN ? kTieGroupFine : kTieGroupCoarse;
  d.gshift = n <= kTieFineMaxN ? 3 : 5;
  d.nb = (n + kTieBlock - 1) / kTieBlock;
  d.wpp = ((n + d.group - 1) / d.group + 31) / 32;
  return d;
}

// The map bits of stage st (BK consecutive y) of one block pair: group g
// onwards, `mask` wide (low bit first; they never straddle two words).  A
// nonzero value means some y of the stage need the long form.
struct TieStage {
  int64_t g;
  uint32_t mask;
};
__host__ __device__ __forceinline__ TieStage tie_stage(int64_t st, int BK, int gshift) {
  const int gps = BK >= (1 << gshift) ? BK >> gshift : 1;  // groups per stage (a stage inside one group: 1)
  return {BK >= (1 << gshift) ? st * (BK >> gshift) : (st * BK) >> gshift, gps >= 32 ? ~0u : (1u << gps) - 1u};
}

// Words of the map including the dirty flags.
__host__ __device__ __forceinline__ int64_t tie_map_words(int64_t n) {
  const TieMapDims d = tie_map_dims(n);
  return d.nb * d.nb * d.wpp + d.nb;
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files).

// Opts kernel `fn` in to `bytes` of dynamic shared memory on the CURRENT
// device (the attribute is per device), once per (kernel, device) and size;
// thread-safe.
cudaError_t smem_opt_in(const void* fn, int bytes);

cudaError_t launch_scan(const float* D, int64_t n, ScanResult* out, bool validate, cudaStream_t s);
cudaError_t launch_focus(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int schedule,
                         cudaStream_t s);
// R = 1/u with a zero diagonal; `paired`: the column order of the packed
// pass-2 stage (reciprocal_rows).
cudaError_t launch_reciprocal(const int32_t* U, float* R, int64_t n, cudaStream_t s, bool paired = false);
// The 64 x 64 super-tiles [t0, t1) of a pass, in the launch order of
// decode_tile (the units of a shard plan); TMA-staged when the layout allows.
cudaError_t launch_focus_range(const float* D, int64_t n, int32_t* U, const ScanResult* scan, int64_t t0, int64_t t1,
                               cudaStream_t s);
cudaError_t launch_cohesion_range(const float* D, const int32_t* U, float* R, int64_t n, float* C,
                                  const uint32_t* tmap, const ScanResult* scan, int accum_mode, int64_t t0, int64_t t1,
                                  cudaStream_t s);
// Clears and fills the tie map (tie_map_words(n) words at `map`).
cudaError_t launch_tie_map(const float* D, int64_t n, uint32_t* map, cudaStream_t s);
// Pass 2: first R = 1/u from U into the scratch R (n x n FP32, in the
// layout the chosen kernel reads), then the tiles.
// `tmap` null: every stage takes the long loop (same result, slower).
// `scan` is the matrix's scan summary (launch_scan), for the pass-1 scale.
cudaError_t launch_cohesion(const float* D, const int32_t* U, float* R, int64_t n, float* C, const uint32_t* tmap,
                            const ScanResult* scan, int accum_mode, int schedule, cudaStream_t s);
// Pass 2 on the TMA tiles (all of them) with the fused local depth: the
// tiles also write their row sums to P ([ceil(n/64)][n] FP64, every entry
// written once), which launch_depth_merge then adds up in order.  Needs the
// TMA layout (cohesion_depth_fused_ok; R 16-byte aligned).
bool cohesion_depth_fused_ok(const float* D, const float* C, int64_t n);
cudaError_t launch_cohesion_depth(const float* D, const int32_t* U, float* R, int64_t n, float* C,
                                  const uint32_t* tmap, const ScanResult* scan, int accum_mode, double* P,
                                  cudaStream_t s);
cudaError_t launch_depth_merge(const double* P, int64_t n, float* L, cudaStream_t s);
// Read and clear the device fault words of the pass-1, pass-2 and batched
// kernels (nonzero: a bounded wait gave up).  Synchronise `s`.
cudaError_t take_cohesion_faults(uint32_t* out, cudaStream_t s);
cudaError_t take_focus_faults(uint32_t* out, cudaStream_t s);
cudaError_t take_batched_faults(uint32_t* out, cudaStream_t s);
cudaError_t take_pairwise_faults(uint32_t* out, cudaStream_t s);
cudaError_t take_fixed_faults(uint32_t* out, cudaStream_t s);
// Fixed-point pass 2 (PALD_ACCUM_FIXED) on the upper-triangle tiles
// [t0, t1) (t1 < 0: all), with `scratch` of fixed_scratch_bytes(D, n) bytes.
size_t fixed_scratch_bytes(const float* D, int64_t n);
cudaError_t launch_fixed_cohesion(const float* D, const int32_t* U, int64_t n, float* C, const uint32_t* tmap,
                                  const ScanResult* scan, void* scratch, int64_t t0, int64_t t1, cudaStream_t s);
// One CTA whose bounded waits run out after limit_ns (the give-up path of
// the TMA pipeline); it records the pass-2 fault word.
cudaError_t launch_wait_selftest(uint64_t limit_ns, cudaStream_t s);
// Tensor map of an n x n FP32 row-major matrix stored with row pitch `pitch`
// elements (a multiple of 4), with boxes of `rows` x 64.
cudaError_t encode_panel_map(CUtensorMap* map, const float* base, int64_t n, int64_t pitch, int rows);
// The same for a `cols` x `nrows` matrix (row pitch `pitch` elements).
cudaError_t encode_rect_map(CUtensorMap* map, const float* base, int64_t cols, int64_t nrows, int64_t pitch,
                            int rows);

// Batched: descriptors of every matrix, and a flat list of tile work items.
struct MatrixDesc {
  int64_t off;  // element offset of the matrix in D, U and C
  int32_t n;
  int32_t tiles_focus;     // number of upper-triangle tiles of the pass-1 schedule
  int32_t tiles_cohesion;  // same for pass 2
  int32_t pad;
  int64_t tmap_off;        // word offset of the matrix's tie map
};
struct WorkItem {
  int32_t matrix;
  int32_t a, b;  // block row and column of the tile (a <= b); for kItemDiagPair the two diagonal blocks
  int32_t kind;  // kItemTile, kItemTileWhole or kItemDiagPair
};
enum : int32_t {
  kItemTile = 0,       // one 64 x 64 upper-triangle tile off the diagonal
  kItemTileWhole = 1,  // one 64 x 64 upper-triangle tile; a diagonal one computes all of its pairs
  kItemDiagPair = 2,   // diagonal tiles (a, a) and (b, b) of one matrix (b < 0: only a): pass 1
                       // runs them on the two halves of a CTA, pass 2 one after the other;
                       // their in-group pairs (x / 4 == z / 4) come from the group kernels
};

}  // namespace pald
