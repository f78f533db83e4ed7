// The pairwise variant (Sec. 3.1, Alg. 1) for matrices too large to hold u:
// both passes per strip of rows, with only D, C and one strip buffer in HBM.
//
// Alg. 1 takes one pair (x, y) at a time: it counts u_xy over z, then
// sweeps z again and credits c_xz and c_yz with 1/u_xy.  Here the pairs are
// taken a strip of h rows x at a time (h = 256):
//   1. strip pass 1: u_xy for every x of the strip and every y (rectangular
//      64 x 64 tiles, both triangles), written only as 1/u into the strip
//      buffer Rt[y][x - x0] (n x h floats, 64 MB at n = 65536: it stays in
//      L2 between its writer and its reader; u itself is never stored);
//   2. strip pass 2: for every x of the strip and every z, the credit that
//      c_xz receives over all y (the c_yz side of each pair is credited when
//      y's strip comes, from its own recount of u_yx = u_xy).
// Every row of C therefore has one writer and is written once, in a fixed
// order: no atomics, deterministic.  The one-sided sums repeat, operation for
// operation, the c_xz lane of the two-pass kernel (the same FFMA forms, the
// same y order, the same fold points), so C equals pald_cohesion's bit for
// bit.  The cost: every pair's u is counted twice (once per orientation)
// and pass 2 runs n^3 one-sided steps instead of n^3/2 two-sided ones.
#include <algorithm>

#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

pald_status cuda_fail(cudaError_t e);
bool opts_ok(const pald_opts* o);
pald_opts opts_or_default(const pald_opts* o);
pald_status scan_and_check(const float* D, int64_t n, ScanResult* scratch, bool validate, cudaStream_t s);

namespace {

using PG = FocusS7;     // 64 x 64 tiles, 4 x 4 pairs per thread, 32-deep stages
constexpr int kStripRows = 256;
constexpr int64_t kMaxN = int64_t(1) << 20;

// Set by a CTA whose bounded wait gave up (never in normal operation).
__device__ uint32_t g_pairwise_faults;

// Thread placement in a rectangular 64 x 64 tile (both triangles, also when
// bi == bj): thread t takes 4 x 4 block (t % ax, t / ax) of the blocks that
// hold pairs of the matrix.  Returns whether thread t owns a block.
__device__ __forceinline__ bool tile_block_rect(int bi, int bj, int64_t n, int t, int* a, int* b) {
  const int64_t rx = n - int64_t(bi) * 64, rz = n - int64_t(bj) * 64;
  const int ax = rx >= 64 ? 16 : static_cast<int>((rx + 3) / 4);
  const int az = rz >= 64 ? 16 : static_cast<int>((rz + 3) / 4);
  *a = 0;
  *b = 0;
  if (t >= ax * az) return false;
  *a = t % ax;
  *b = t / ax;
  return true;
}

// Strip pass 1: tile (bx, by) of the strip, bx in [x0/64, x0/64 + bxs).
__global__ void __launch_bounds__(PG::NT, 3)
    strip_focus_kernel(const __grid_constant__ CUtensorMap tmD, const float* __restrict__ D, int64_t n, int64_t x0,
                       int bxs, float* __restrict__ Rt, int64_t h, const ScanResult* __restrict__ scan) {
  extern __shared__ __align__(128) float smem[];
  constexpr int BK = PG::BK, TX = PG::TX, TY = PG::TY;
  const int bx = static_cast<int>(x0 / 64) + static_cast<int>(blockIdx.x) % bxs;
  const int by = static_cast<int>(blockIdx.x) / bxs;
  TmaRing<2, BK> ring;
  ring.carve(smem);
  int tx, ty;
  const bool active = tile_block_rect(bx, by, n, threadIdx.x, &tx, &ty);
  const int64_t X0 = int64_t(bx) * 64, Y0 = int64_t(by) * 64;
  const float scale = focus_scale(scan->inv_min_pos_bits);
  const int nstages = static_cast<int>((n + BK - 1) / BK);
  if (threadIdx.x == 0) ring.init();
  __syncthreads();
  float cst[TX][TY];
  uint64_t acc[TX][TY];
  focus_init<PG>(D, n, X0, Y0, tx, ty, scale, cst, acc);
  const CUtensorMap* const maps[2] = {&tmD, &tmD};
  const int cols[2] = {bx * 64, by * 64};
  const bool ok = tma_pipeline(ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
                               [&](int st, int buf) {
                                 if (active)
                                   focus_stage<PG, 16>(ring.panel(buf, 0), ring.panel(buf, 1), tx, ty, scale, cst,
                                                       acc, stage_extent<BK, 16>(n, st));
                               });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(&g_pairwise_faults, 1u);
    return;
  }
  if (!active) return;
  // 1/u into the strip buffer, transposed: Rt[y][x - x0], four x per store
  const int nn = static_cast<int>(n);
#pragma unroll
  for (int j = 0; j < TY; ++j) {
    const int64_t y = Y0 + PG::col_off(ty, j);
    if (y >= n) continue;
    const int64_t xb = X0 + PG::row_off(tx, 0);
    float r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = recip_entry(nn - count_of(acc[i][j]), xb + i, y);
    float* dst = Rt + y * h + (xb - x0);
    if (xb + 3 < n) {
      *reinterpret_cast<float4*>(dst) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (xb + i < n) dst[i] = r[i];
    }
  }
}

// One-sided steps: the c_xz lane of cohesion_step / cohesion_step_short,
// instruction for instruction, on half L of a packed pair of partials.
template <int L>
__device__ __forceinline__ void one_sided_short(uint64_t& s2, float a1, float a2, float S, float c, float r1) {
  float lo, hi;
  unpack2(s2, lo, hi);
  float& s = L == 0 ? lo : hi;
  asm("{\n\t.reg .f32 m, v;\n\t"
      "min.f32 m, %1, %2;\n\t"
      "fma.rn.sat.f32 v, m, %3, %4;\n\t"
      "fma.rn.f32 %0, v, %5, %0;\n\t}"
      : "+f"(s)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(r1));
  s2 = pack2(lo, hi);
}

// Long form: credit w(d_xz, d_zy) * r_xy when d_xz <= d_xy.  (When also
// d_zy < d_xz the weight is 0 and the add is of +0, as in the two-sided
// form, whose predicate also asks d_xz <= d_zy.)
template <int L>
__device__ __forceinline__ void one_sided_long(uint64_t& s2, float a1, float a2, float S, float c, float r1) {
  float lo, hi;
  unpack2(s2, lo, hi);
  float& s = L == 0 ? lo : hi;
  asm("{\n\t.reg .pred p;\n\t.reg .f32 t1, t2, v2;\n\t"
      "fma.rn.f32 t2, %2, %3, %4;\n\t"
      "fma.rn.sat.f32 v2, t2, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.f32 t1, %1, %3, %4;\n\t"
      "setp.ge.f32 p, t1, 0f00000000;\n\t"
      "@p fma.rn.f32 %0, v2, %5, %0;\n\t}"
      : "+f"(s)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(r1));
  s2 = pack2(lo, hi);
}

// One stage of strip pass 2: panels D[y][X], Rt[y][X - x0], D[y][Z].  The
// thread's partials are packed as {S(i, j), S(i, j + 2)} (the same fold
// phase: x + z keeps its parity), jj = 0, 1.
template <int MODE, bool SHORT>
__device__ __forceinline__ void strip_cohesion_stage(const float* ad, const float* ar, const float* bd, int tx, int tz,
                                                     float S, const float (&cv)[4][4], uint64_t (&sacc)[4][2],
                                                     uint64_t (&hacc)[4][2], int kend) {
  constexpr int UNR = 16;
  static_assert(UNR % kMergeEvery == 0, "chunks hold whole merge chunks");
#pragma unroll 1
  for (int k0 = 0; k0 < kend; k0 += UNR) {
#pragma unroll
    for (int k = 0; k < UNR; ++k) {
      const int kk = k0 + k;
      float a1[4], r1[4], a2[4];
      lds<4>(ad + kk * 64 + 4 * tx, a1);
      lds<4>(ar + kk * 64 + 4 * tx, r1);
      lds<4>(bd + kk * 64 + 4 * tz, a2);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (SHORT) {
            if (j < 2)
              one_sided_short<0>(sacc[i][j], a1[i], a2[j], S, cv[i][j], r1[i]);
            else
              one_sided_short<1>(sacc[i][j - 2], a1[i], a2[j], S, cv[i][j], r1[i]);
          } else {
            if (j < 2)
              one_sided_long<0>(sacc[i][j], a1[i], a2[j], S, cv[i][j], r1[i]);
            else
              one_sided_long<1>(sacc[i][j - 2], a1[i], a2[j], S, cv[i][j], r1[i]);
          }
        }
      if (MODE == PALD_ACCUM_COMPENSATED) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
            if ((k % kMergeEvery) == fold_phase(i, jj)) fast2sum_fold(hacc[i][jj], sacc[i][jj]);
      }
    }
  }
}


template <int MODE>
__global__ void __launch_bounds__(PG::NT, 2)
    strip_cohesion_kernel(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmR,
                          const float* __restrict__ D, int64_t n, int64_t x0, int bxs, float* __restrict__ C,
                          const uint32_t* __restrict__ tmap, const ScanResult* __restrict__ scan) {
  extern __shared__ __align__(128) float smem[];
  constexpr int BK = PG::BK;
  const int bx = static_cast<int>(x0 / 64) + static_cast<int>(blockIdx.x) % bxs;
  const int bz = static_cast<int>(blockIdx.x) / bxs;
  TmaRing<3, BK> ring;
  uint32_t* tie_words = reinterpret_cast<uint32_t*>(ring.carve(smem));
  int tx, tz;
  const bool active = tile_block_rect(bx, bz, n, threadIdx.x, &tx, &tz);
  const int64_t X0 = int64_t(bx) * 64, Z0 = int64_t(bz) * 64;
  const float S = focus_scale(scan->inv_min_pos_bits);
  const int nstages = static_cast<int>((n + BK - 1) / BK);
  if (threadIdx.x == 0) ring.init();
  {
    const TieMapDims dm = tie_map_dims(n);
    const int64_t lo = bx < bz ? bx : bz, hi = bx < bz ? bz : bx;  // the map is kept for lo <= hi
    const bool all_long = tmap == nullptr || __ldg(tmap + dm.nb * dm.nb * dm.wpp + bx) != 0u ||
                          __ldg(tmap + dm.nb * dm.nb * dm.wpp + bz) != 0u;
    const uint32_t* row = tmap + (lo * dm.nb + hi) * dm.wpp;
    for (int w = threadIdx.x; w < dm.wpp; w += PG::NT) tie_words[w] = all_long ? ~0u : __ldg(row + w);
  }
  __syncthreads();
  float cv[4][4];
  uint64_t sacc[4][2], hacc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t x = X0 + 4 * tx + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t z = Z0 + 4 * tz + j;
      cv[i][j] = __fmul_rn(-((x < n && z < n) ? __ldg(D + x * n + z) : 0.f), S);  // exact: power of two
    }
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      sacc[i][jj] = pack2(0.f, 0.f);
      hacc[i][jj] = pack2(kMergeBias, kMergeBias);
    }
  }
  const int gshift = tie_map_dims(n).gshift;
  const CUtensorMap* const maps[3] = {&tmD, &tmR, &tmD};
  const int cols[3] = {bx * 64, static_cast<int>(X0 - x0), bz * 64};
  const bool ok = tma_pipeline(
      ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
      [&](int st, int buf) {
        if (!active) return;
        const TieStage ts = tie_stage(st, BK, gshift);  // any group of the stage marked: long form
        const int kend = stage_extent<BK, 16>(n, st);
        if ((tie_words[ts.g >> 5] >> (ts.g & 31)) & ts.mask)
          strip_cohesion_stage<MODE, false>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2), tx, tz, S,
                                            cv, sacc, hacc, kend);
        else
          strip_cohesion_stage<MODE, true>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2), tx, tz, S,
                                           cv, sacc, hacc, kend);
      });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(&g_pairwise_faults, 1u);
    return;
  }
  if (!active) return;
  float ih, il;
  inverse_pair(n - 1, ih, il);
  const bool vec = (n % 4) == 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t x = X0 + 4 * tx + i;
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = cohesion_value<MODE>(hacc[i][j % 2], sacc[i][j % 2], j >= 2, ih, il);
    storew<4>(C, n, x, Z0 + 4 * tz, v, vec);
  }
}

constexpr int kFocusSmem = TmaRing<2, PG::BK>::BYTES + 128;
constexpr int kCohesionSmemMax = TmaRing<3, PG::BK>::BYTES + 128 + 4 * kTieWordsMax;

// Padded copy of D (row pitch a multiple of 4) for the TMA copies.
__global__ void __launch_bounds__(256) pad_rows_kernel(const float* __restrict__ D, int64_t n, int64_t pitch,
                                                       float* __restrict__ Dp) {
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x)
    for (int64_t c = threadIdx.x; c < pitch; c += blockDim.x) Dp[row * pitch + c] = c < n ? D[row * n + c] : 0.f;
}

struct Scratch {
  void* p = nullptr;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

cudaError_t take_pairwise_faults(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_pairwise_faults, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out != 0u)
    e = cudaMemcpyToSymbolAsync(g_pairwise_faults, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace pald

using namespace pald;

extern "C" {

int64_t pald_pairwise_scratch_bytes(int64_t n) {
  if (n < 2 || n > kMaxN) return 0;
  const int64_t pitch = (n + 3) / 4 * 4;
  size_t b = align256(static_cast<size_t>(n) * kStripRows * sizeof(float));     // strip buffer
  b += align256(static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t));     // tie map
  b += 256;                                                                     // scan summary
  if (pitch != n) b += align256(static_cast<size_t>(n) * pitch * sizeof(float));  // padded D
  return static_cast<int64_t>(b);
}

pald_status pald_pairwise(const float* D, int64_t n, float* C, const pald_opts* opts, pald_stream_t stream) {
  if (!D || !C || n < 2 || n > kMaxN || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  if (opts && opts->accum_mode == PALD_ACCUM_FIXED) return PALD_ERR_INVALID_ARG;  // compensated or plain only
  if (reinterpret_cast<uintptr_t>(D) % 16 || reinterpret_cast<uintptr_t>(C) % 16) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t pitch = (n + 3) / 4 * 4;
  const size_t rbytes = align256(static_cast<size_t>(n) * kStripRows * sizeof(float));
  const size_t tbytes = align256(static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t));
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(static_cast<size_t>(pald_pairwise_scratch_bytes(n)));
  if (e != cudaSuccess) return cuda_fail(e);
  char* base = static_cast<char*>(scratch.p);
  float* Rt = reinterpret_cast<float*>(base);
  auto* tmap = reinterpret_cast<uint32_t*>(base + rbytes);
  auto* scan = reinterpret_cast<ScanResult*>(base + rbytes + tbytes);
  const float* Dt = D;  // what the tensor copies read (D itself when its rows are 16-byte aligned)
  if (pitch != n) {
    float* Dp = reinterpret_cast<float*>(base + rbytes + tbytes + 256);
    const int64_t grid = n < 4096 ? n : 4096;
    pad_rows_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(D, n, pitch, Dp);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    Dt = Dp;
  }
  pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if (o.flags & PALD_FLAG_IGNORE_TIES)
    e = cudaMemsetAsync(tmap, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  else
    e = launch_tie_map(D, n, tmap, s);
  if (e != cudaSuccess) return cuda_fail(e);

  CUtensorMap mD, mR;
  if ((e = encode_rect_map(&mD, Dt, n, n, pitch, PG::BK)) != cudaSuccess) return cuda_fail(e);
  if ((e = encode_rect_map(&mR, Rt, kStripRows, n, kStripRows, PG::BK)) != cudaSuccess) return cuda_fail(e);
  if ((e = smem_opt_in(reinterpret_cast<const void*>(strip_focus_kernel), kFocusSmem)) != cudaSuccess)
    return cuda_fail(e);
  const bool plain = o.accum_mode == PALD_ACCUM_PLAIN;
  const void* cfn = plain ? reinterpret_cast<const void*>(strip_cohesion_kernel<PALD_ACCUM_PLAIN>)
                          : reinterpret_cast<const void*>(strip_cohesion_kernel<PALD_ACCUM_COMPENSATED>);
  if ((e = smem_opt_in(cfn, kCohesionSmemMax)) != cudaSuccess) return cuda_fail(e);
  const int csmem = TmaRing<3, PG::BK>::BYTES + 128 + 4 * static_cast<int>(tie_map_dims(n).wpp);
  const int64_t T = (n + 63) / 64;
  for (int64_t x0 = 0; x0 < n; x0 += kStripRows) {
    const int bxs = static_cast<int>(std::min<int64_t>(kStripRows / 64, T - x0 / 64));
    const unsigned grid = static_cast<unsigned>(bxs * T);
    strip_focus_kernel<<<grid, PG::NT, kFocusSmem, s>>>(mD, D, n, x0, bxs, Rt, kStripRows, scan);
    if (plain)
      strip_cohesion_kernel<PALD_ACCUM_PLAIN><<<grid, PG::NT, csmem, s>>>(mD, mR, D, n, x0, bxs, C, tmap, scan);
    else
      strip_cohesion_kernel<PALD_ACCUM_COMPENSATED><<<grid, PG::NT, csmem, s>>>(mD, mR, D, n, x0, bxs, C, tmap,
                                                                               scan);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  }
  return PALD_OK;
}

}  // extern "C"
