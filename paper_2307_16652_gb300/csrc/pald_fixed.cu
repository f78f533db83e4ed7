// Fixed-point cohesion (PALD_ACCUM_FIXED): pass 2 with exact integer sums, so
// C does not depend on the order in which the terms of Sec. 2 eq. (fxz) are
// added (any tiling, any split of y or of the tiles over GPUs gives the
// same bits).
//
// Each weight 1/u_xy is replaced by the integer Q = round(2^40 / u_xy) and
// every credit w in {0, 1/2, 1} (Sec. 5 tie split) by 2w, so the sum for
// c_xz is the integer A = sum_y 2w * Q < n * 2^40, and c_xz = A / 2^41 /
// (n - 1) with one FP64 scaling and one rounding to FP32 at the end.  The
// sum is exact: Q is split into two pieces hi = Q >> 20 and lo = Q & (2^20
// - 1), the tile streams the FP32 values 2 hi and 2 lo (even integers below
// 2^21, so w times either is an integer), FP32 partials over 8 y stay below
// 2^24 and are therefore exact, and every 8 y they are converted (exactly)
// and added into int64 accumulators A = 2^20 * sum(hi part) + sum(lo part).
// The comparisons are the two-pass kernel's (short and long forms chosen by
// the tie map).  Error against the definition: each Q is off by at most 1/2,
// i.e. by u / 2^41 relative, so |c - c_exact| <= (max u) / 2^41 * c_exact.
#include <algorithm>

#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

namespace {

using FX = CohesionS7;  // 64 x 64 tiles, 4 x 4 pairs per thread, 32-deep stages, 256 threads
constexpr int kFixedShift = 40;  // Q = round(2^40 / u)
constexpr int kPieceBits = 20;   // Q = hi * 2^20 + lo

// Set by a CTA whose bounded wait gave up (never in normal operation).
__device__ uint32_t g_fixed_faults;

// Rh[y][x] = 2 (Q >> 20), Rl[y][x] = 2 (Q & (2^20 - 1)) for Q = round(2^40 /
// u_xy), 0 on the diagonal and for u <= 0; U has row pitch n, the pieces
// row pitch `pitch`.  (u is symmetric, so row y of the pieces is column y.)
__global__ void __launch_bounds__(256) fixed_pieces_kernel(const int32_t* __restrict__ U, int64_t n, int64_t pitch,
                                                           float* __restrict__ Rh, float* __restrict__ Rl) {
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x)
    for (int64_t c = threadIdx.x; c < pitch; c += blockDim.x) {
      float h = 0.f, l = 0.f;
      if (c < n && c != row) {
        const int32_t u = __ldg(U + row * n + c);
        if (u > 0) {
          const uint64_t q = ((uint64_t(1) << (kFixedShift + 1)) / static_cast<uint64_t>(u) + 1) >> 1;
          h = static_cast<float>(2 * (q >> kPieceBits));
          l = static_cast<float>(2 * (q & ((uint64_t(1) << kPieceBits) - 1)));
        }
      }
      Rh[row * pitch + c] = h;
      Rl[row * pitch + c] = l;
    }
}

// Row-padded copy of D (pitch a multiple of 4) for the tensor copies.
__global__ void __launch_bounds__(256) fixed_pad_kernel(const float* __restrict__ D, int64_t n, int64_t pitch,
                                                        float* __restrict__ Dp) {
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x)
    for (int64_t c = threadIdx.x; c < pitch; c += blockDim.x) Dp[row * pitch + c] = c < n ? D[row * n + c] : 0.f;
}

// The exact partials of one pair: hi and lo pieces for c_xz and c_zx.
struct FixedPartial {
  float hx, lx, hz, lz;
};

__device__ __forceinline__ void fixed_step_short(FixedPartial& p, float a1, float a2, float S, float c, float rh1,
                                                 float rl1, float rh2, float rl2) {
  asm("{\n\t.reg .f32 m, v;\n\t"
      "min.f32 m, %4, %5;\n\t"
      "fma.rn.sat.f32 v, m, %6, %7;\n\t"
      "fma.rn.f32 %0, v, %8, %0;\n\t"
      "fma.rn.f32 %1, v, %9, %1;\n\t"
      "fma.rn.f32 %2, v, %10, %2;\n\t"
      "fma.rn.f32 %3, v, %11, %3;\n\t}"
      : "+f"(p.hx), "+f"(p.lx), "+f"(p.hz), "+f"(p.lz)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(rh1), "f"(rl1), "f"(rh2), "f"(rl2));
}

__device__ __forceinline__ void fixed_step_long(FixedPartial& p, float a1, float a2, float S, float c, float rh1,
                                                float rl1, float rh2, float rl2) {
  asm("{\n\t.reg .pred q;\n\t.reg .f32 m, t1, t2, v1, v2;\n\t"
      "fma.rn.f32 t2, %5, %6, %7;\n\t"
      "fma.rn.f32 t1, %4, %6, %7;\n\t"
      "fma.rn.sat.f32 v2, t2, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.sat.f32 v1, t1, 0f3F000000, 0f3F000000;\n\t"
      "min.f32 m, v1, v2;\n\t"
      "setp.gt.f32 q, m, 0f00000000;\n\t"
      "@q fma.rn.f32 %0, v2, %8, %0;\n\t"
      "@q fma.rn.f32 %1, v2, %9, %1;\n\t"
      "@q fma.rn.f32 %2, v1, %10, %2;\n\t"
      "@q fma.rn.f32 %3, v1, %11, %3;\n\t}"
      : "+f"(p.hx), "+f"(p.lx), "+f"(p.hz), "+f"(p.lz)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(rh1), "f"(rl1), "f"(rh2), "f"(rl2));
}

// Moves an exact FP32 partial pair (hi piece, lo piece) into A and clears it.
__device__ __forceinline__ void fixed_fold(int64_t& A, float& h, float& l) {
  A += (static_cast<int64_t>(__float2int_rz(h)) << kPieceBits) + static_cast<int64_t>(__float2int_rz(l));
  h = 0.f;
  l = 0.f;
}

constexpr int kFixedFold = 8;  // y per exact FP32 partial (8 * 2^21 <= 2^24)

template <bool SHORT>
__device__ __forceinline__ void fixed_stage(const float* dX, const float* hX, const float* lX, const float* dZ,
                                            const float* hZ, const float* lZ, int tx, int tz, float S,
                                            const float (&cv)[4][4], FixedPartial (&p)[4][4],
                                            int64_t (&Ax)[4][4], int64_t (&Az)[4][4], int kend) {
  constexpr int UNR = 16;
  static_assert(UNR % kFixedFold == 0, "chunks hold whole fold periods");
#pragma unroll 1
  for (int k0 = 0; k0 < kend; k0 += UNR) {
#pragma unroll
    for (int k = 0; k < UNR; ++k) {
      const int kk = k0 + k;
      float a1[4], h1[4], l1[4], a2[4], h2[4], l2[4];
      lds<4>(dX + kk * 64 + 4 * tx, a1);
      lds<4>(hX + kk * 64 + 4 * tx, h1);
      lds<4>(lX + kk * 64 + 4 * tx, l1);
      lds<4>(dZ + kk * 64 + 4 * tz, a2);
      lds<4>(hZ + kk * 64 + 4 * tz, h2);
      lds<4>(lZ + kk * 64 + 4 * tz, l2);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (SHORT)
            fixed_step_short(p[i][j], a1[i], a2[j], S, cv[i][j], h1[i], l1[i], h2[j], l2[j]);
          else
            fixed_step_long(p[i][j], a1[i], a2[j], S, cv[i][j], h1[i], l1[i], h2[j], l2[j]);
        }
      if (k % kFixedFold == kFixedFold - 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            fixed_fold(Ax[i][j], p[i][j].hx, p[i][j].lx);
            fixed_fold(Az[i][j], p[i][j].hz, p[i][j].lz);
          }
      }
    }
  }
}

// c = A / 2^41 / (n - 1), one FP64 scaling, one rounding to FP32.
__device__ __forceinline__ float fixed_value(int64_t A, double inv) {
  return __double2float_rn(__dmul_rn(static_cast<double>(A), inv));
}

// One upper-triangle tile (decode_tile order from t0): D, 2 hi and 2 lo
// panels of X and of Z per 32-y stage (six panels, 144 KB of ring: one CTA
// per SM), both C[X, Z] and C[Z, X] written.
__global__ void __launch_bounds__(FX::NT, 1)
    fixed_tile_kernel(const __grid_constant__ CUtensorMap tmD, const __grid_constant__ CUtensorMap tmH,
                      const __grid_constant__ CUtensorMap tmL, const float* __restrict__ D, int64_t n,
                      float* __restrict__ C, const uint32_t* __restrict__ tmap, const ScanResult* __restrict__ scan,
                      int64_t T, int64_t t0, bool vec) {
  extern __shared__ __align__(128) float smem[];
  constexpr int BK = FX::BK;
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0, T, 1, &bi, &bj, &slice);
  TmaRing<6, BK> ring;
  uint32_t* tie_words = reinterpret_cast<uint32_t*>(ring.carve(smem));
  int tx, tz;
  const bool active = tile_block_64(bi, bj, n, threadIdx.x, &tx, &tz, false);
  const int64_t X0 = int64_t(bi) * 64, Z0 = int64_t(bj) * 64;
  const float S = focus_scale(scan->inv_min_pos_bits);
  const int nstages = static_cast<int>((n + BK - 1) / BK);
  if (threadIdx.x == 0) ring.init();
  {
    const TieMapDims dm = tie_map_dims(n);
    const bool all_long = tmap == nullptr || __ldg(tmap + dm.nb * dm.nb * dm.wpp + bi) != 0u ||
                          __ldg(tmap + dm.nb * dm.nb * dm.wpp + bj) != 0u;
    const uint32_t* row = tmap + (int64_t(bi) * dm.nb + bj) * dm.wpp;
    for (int w = threadIdx.x; w < dm.wpp; w += FX::NT) tie_words[w] = all_long ? ~0u : __ldg(row + w);
  }
  __syncthreads();
  float cv[4][4];
  FixedPartial p[4][4];
  int64_t Ax[4][4], Az[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t x = X0 + 4 * tx + i, z = Z0 + 4 * tz + j;
      cv[i][j] = __fmul_rn(-((x < n && z < n) ? __ldg(D + x * n + z) : 0.f), S);  // exact: power of two
      p[i][j] = FixedPartial{0.f, 0.f, 0.f, 0.f};
      Ax[i][j] = 0;
      Az[i][j] = 0;
    }
  const int gshift = tie_map_dims(n).gshift;
  const CUtensorMap* const maps[6] = {&tmD, &tmH, &tmL, &tmD, &tmH, &tmL};
  const int cols[6] = {bi * 64, bi * 64, bi * 64, bj * 64, bj * 64, bj * 64};
  const bool ok = tma_pipeline(
      ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
      [&](int st, int buf) {
        if (!active) return;
        const TieStage ts = tie_stage(st, BK, gshift);  // any group of the stage marked: long form
        const int kend = stage_extent<BK, 16>(n, st);
        if ((tie_words[ts.g >> 5] >> (ts.g & 31)) & ts.mask)
          fixed_stage<false>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2), ring.panel(buf, 3),
                             ring.panel(buf, 4), ring.panel(buf, 5), tx, tz, S, cv, p, Ax, Az, kend);
        else
          fixed_stage<true>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2), ring.panel(buf, 3),
                            ring.panel(buf, 4), ring.panel(buf, 5), tx, tz, S, cv, p, Ax, Az, kend);
      });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(&g_fixed_faults, 1u);
    return;
  }
  if (!active) return;
  const double inv = 1.0 / (static_cast<double>(int64_t(1) << (kFixedShift + 1)) * static_cast<double>(n - 1));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = fixed_value(Ax[i][j], inv);
    storew<4>(C, n, X0 + 4 * tx + i, Z0 + 4 * tz, v, vec);
  }
  if (tx != tz || bi != bj) {  // the block's mirror
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = fixed_value(Az[i][j], inv);
      storew<4>(C, n, Z0 + 4 * tz + j, X0 + 4 * tx, v, vec);
    }
  }
}

constexpr int kFixedSmemMax = TmaRing<6, FX::BK>::BYTES + 128 + 4 * kTieWordsMax;

}  // namespace

// The tensor copies need D's rows 16-byte aligned; otherwise they read a
// row-padded copy.
bool fixed_needs_pad(const float* D, int64_t n) { return n % 4 != 0 || reinterpret_cast<uintptr_t>(D) % 16 != 0; }

size_t fixed_scratch_bytes(const float* D, int64_t n) {
  const int64_t pitch = (n + 3) / 4 * 4;
  const size_t piece = (static_cast<size_t>(n) * static_cast<size_t>(pitch) * sizeof(float) + 255) / 256 * 256;
  return 2 * piece + (fixed_needs_pad(D, n) ? piece : 0);  // hi and lo pieces, and a padded D
}

cudaError_t launch_fixed_cohesion(const float* D, const int32_t* U, int64_t n, float* C, const uint32_t* tmap,
                                  const ScanResult* scan, void* scratch, int64_t t0, int64_t t1, cudaStream_t s) {
  const int64_t pitch = (n + 3) / 4 * 4;
  const size_t piece = (static_cast<size_t>(n) * static_cast<size_t>(pitch) * sizeof(float) + 255) / 256 * 256;
  float* Rh = static_cast<float*>(scratch);
  float* Rl = reinterpret_cast<float*>(static_cast<char*>(scratch) + piece);
  const float* Dt = D;
  const int64_t grid = std::min<int64_t>(n, 16 * sm_count());
  if (fixed_needs_pad(D, n)) {
    float* Dp = reinterpret_cast<float*>(static_cast<char*>(scratch) + 2 * piece);
    fixed_pad_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(D, n, pitch, Dp);
    Dt = Dp;
  }
  fixed_pieces_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(U, n, pitch, Rh, Rl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t T = (n + 63) / 64;
  if (t1 < 0) t1 = T * (T + 1) / 2;
  if (t1 <= t0) return cudaSuccess;
  CUtensorMap mD, mH, mL;
  if ((e = encode_rect_map(&mD, Dt, n, n, pitch, FX::BK)) != cudaSuccess) return e;
  if ((e = encode_rect_map(&mH, Rh, n, n, pitch, FX::BK)) != cudaSuccess) return e;
  if ((e = encode_rect_map(&mL, Rl, n, n, pitch, FX::BK)) != cudaSuccess) return e;
  if ((e = smem_opt_in(reinterpret_cast<const void*>(fixed_tile_kernel), kFixedSmemMax)) != cudaSuccess) return e;
  const int smem = TmaRing<6, FX::BK>::BYTES + 128 + 4 * static_cast<int>(tie_map_dims(n).wpp);
  const bool vec = n % 4 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0;
  fixed_tile_kernel<<<static_cast<unsigned>(t1 - t0), FX::NT, smem, s>>>(mD, mH, mL, D, n, C, tmap, scan, T, t0,
                                                                          vec);
  return cudaGetLastError();
}

cudaError_t take_fixed_faults(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_fixed_faults, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out != 0u)
    e = cudaMemcpyToSymbolAsync(g_fixed_faults, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace pald
