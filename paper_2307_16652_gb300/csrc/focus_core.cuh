// Pass 1 core: local focus sizes of one BM x BM tile of U.
//
// For every pair (x, y) of the tile,
//     u_xy = #{ z : min(d_xz, d_yz) <= d_xy }                 (Sec. 2, U_xy)
// computed as n - #{ z : min(d_xz, d_yz) > d_xy }.  The strict test is one
// saturating FFMA: with a power-of-two scale s shared by the whole matrix
// (2^(23 - e), e the exponent of its smallest positive entry) and c = -t*s,
//     sat(m*s + c) = sat((m - t)*s) = [m > t]   exactly,
// because m > t implies m - t >= ulp(t) >= 2^(e-23), and t*s is a pure
// power-of-two scaling, so no rounding can move the result across 0 or 1.
//
// Two consecutive z are handled together:
//     m0 = min(d_xz0, d_yz0), m1 = min(d_xz1, d_yz1)     2 x FMNMX   (ALU pipe)
//     h0 = sat(m0*s + c),     h1 = sat(m1*s + c)         2 x FFMA    (FMA pipe)
//     {acc0, acc1} += {h0, h1}                           1 x FADD2   (FMA pipe, 2 cycles)
// i.e. 2.5 issue slots per (x, y, z) with the ALU and FMA pipes equally
// loaded (4 cycles each per two z).  The two partial counts are exact
// integers in FP32 (n < 2^24) and are added at the end.
//
// Layout: the CTA streams z through shared memory in chunks of BK.  Because
// D is symmetric, column block D[X, z-chunk] is read as rows D[z-chunk, X],
// so every global read is a contiguous row segment (the "transpose" is
// free).  Thread (tx, ty) owns x in {g*BM/G + 4*tx + i} and y in
// {g*BM/G + 4*ty + j} (g < G, i, j < 4): its shared-memory reads are
// 16-byte vectors with no bank conflicts, and its global stores of u (and of
// the mirrored tile u_YX) are 16-byte vectors too.
#pragma once

#include "pald_internal.cuh"

namespace pald {

template <int BM, int G>
struct FocusGeom {
  static constexpr int BK = 16;                 // z per pipeline stage
  static constexpr int TPD = BM / (4 * G);      // threads per tile dimension
  static constexpr int NT = TPD * TPD;          // threads per CTA
  static constexpr int TM = 4 * G;              // rows (and columns) per thread
  static constexpr int STAGE = BK * BM;         // floats per operand per stage
  static constexpr int SMEM_FLOATS = 2 * 2 * STAGE;
};

// Copy rows z0..z0+BK-1, columns c0..c0+BM-1 of the n x n matrix at M into
// dst[BK][BM]; out-of-range elements are zero-filled.
template <int BM, int NT, int BK>
__device__ __forceinline__ void stage_rows(float* dst, const float* __restrict__ M, int64_t n, int64_t z0,
                                           int64_t c0, bool vec) {
  if (vec) {
    constexpr int V = BK * BM / 4;
#pragma unroll
    for (int k = threadIdx.x; k < V; k += NT) {
      const int r = k / (BM / 4), c = (k % (BM / 4)) * 4;
      const int64_t row = z0 + r, col = c0 + c;
      int bytes = 0;
      const float* src = M;
      if (row < n && col < n) {
        const int64_t left = n - col;
        bytes = left >= 4 ? 16 : static_cast<int>(left) * 4;
        src = M + row * n + col;
      }
      cp_async16(dst + r * BM + c, src, bytes);
    }
  } else {
    constexpr int V = BK * BM;
#pragma unroll 4
    for (int k = threadIdx.x; k < V; k += NT) {
      const int r = k / BM, c = k % BM;
      const int64_t row = z0 + r, col = c0 + c;
      const bool ok = row < n && col < n;
      cp_async4(dst + r * BM + c, ok ? M + row * n + col : M, ok ? 4 : 0);
    }
  }
}

// Load 4 consecutive floats of row `row` starting at column `col` (zeros
// outside the matrix).
__device__ __forceinline__ float4 load4(const float* __restrict__ M, int64_t n, int64_t row, int64_t col, bool vec) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (row >= n) return v;
  const float* p = M + row * n + col;
  if (vec && col + 3 < n) return __ldg(reinterpret_cast<const float4*>(p));
  if (col + 0 < n) v.x = __ldg(p + 0);
  if (col + 1 < n) v.y = __ldg(p + 1);
  if (col + 2 < n) v.z = __ldg(p + 2);
  if (col + 3 < n) v.w = __ldg(p + 3);
  return v;
}

__device__ __forceinline__ void store4i(int32_t* __restrict__ M, int64_t n, int64_t row, int64_t col, int4 v,
                                        bool vec) {
  if (row >= n) return;
  int32_t* p = M + row * n + col;
  if (vec && col + 3 < n) {
    *reinterpret_cast<int4*>(p) = v;
    return;
  }
  if (col + 0 < n) p[0] = v.x;
  if (col + 1 < n) p[1] = v.y;
  if (col + 2 < n) p[2] = v.z;
  if (col + 3 < n) p[3] = v.w;
}

// {acc0, acc1} += {[min(a0, b0) > t], [min(a1, b1) > t]} for two consecutive z.
__device__ __forceinline__ void focus_step2(uint64_t& acc, float a0, float b0, float a1, float b1, float s, float c) {
  asm("{\n\t.reg .f32 m0, m1, h0, h1;\n\t.reg .b64 hh;\n\t"
      "min.f32 m0, %1, %2;\n\t"
      "min.f32 m1, %3, %4;\n\t"
      "fma.rn.sat.f32 h0, m0, %5, %6;\n\t"
      "fma.rn.sat.f32 h1, m1, %5, %6;\n\t"
      "mov.b64 hh, {h0, h1};\n\t"
      "add.rn.f32x2 %0, %0, hh;\n\t}"
      : "+l"(acc)
      : "f"(a0), "f"(b0), "f"(a1), "f"(b1), "f"(s), "f"(c));
}

__device__ __forceinline__ int count_of(uint64_t acc) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc));
  return static_cast<int>(lo) + static_cast<int>(hi);
}

// Computes and stores U[X, Y] (and U[Y, X] when bi != bj) for tile (bi, bj).
// `smem` holds Geom::SMEM_FLOATS floats.  Must be called by all NT threads.
template <int BM, int G>
__device__ __forceinline__ void focus_tile(const float* __restrict__ D, int64_t n, int32_t* __restrict__ U, int bi,
                                           int bj, float scale, float* smem) {
  using Geo = FocusGeom<BM, G>;
  constexpr int BK = Geo::BK, TM = Geo::TM, TPD = Geo::TPD, NT = Geo::NT;
  const int64_t X0 = static_cast<int64_t>(bi) * BM, Y0 = static_cast<int64_t>(bj) * BM;
  const int tx = threadIdx.x % TPD, ty = threadIdx.x / TPD;
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(D) % 16) == 0;

  float* As = smem;                    // [2][BK][BM]  D[z][X0 + .]
  float* Bs = smem + 2 * Geo::STAGE;   // [2][BK][BM]  D[z][Y0 + .]

  const int64_t nstages = (n + BK - 1) / BK;
  stage_rows<BM, NT, BK>(As, D, n, 0, X0, vec);
  stage_rows<BM, NT, BK>(Bs, D, n, 0, Y0, vec);
  cp_async_commit();

  // thresholds t = d_xy -> c = -t * scale (exact: power-of-two scaling)
  float cst[TM][TM];
  uint64_t acc[TM][TM];
#pragma unroll
  for (int gi = 0; gi < G; ++gi)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t x = X0 + gi * (BM / G) + 4 * tx + i;
#pragma unroll
      for (int gj = 0; gj < G; ++gj) {
        const float4 t = load4(D, n, x, Y0 + gj * (BM / G) + 4 * ty, vec);
        cst[gi * 4 + i][gj * 4 + 0] = -t.x * scale;
        cst[gi * 4 + i][gj * 4 + 1] = -t.y * scale;
        cst[gi * 4 + i][gj * 4 + 2] = -t.z * scale;
        cst[gi * 4 + i][gj * 4 + 3] = -t.w * scale;
      }
    }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = 0ull;

  for (int64_t st = 0; st < nstages; ++st) {
    const int buf = static_cast<int>(st & 1);
    if (st + 1 < nstages) {
      stage_rows<BM, NT, BK>(As + (buf ^ 1) * Geo::STAGE, D, n, (st + 1) * BK, X0, vec);
      stage_rows<BM, NT, BK>(Bs + (buf ^ 1) * Geo::STAGE, D, n, (st + 1) * BK, Y0, vec);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* as = As + buf * Geo::STAGE;
    const float* bs = Bs + buf * Geo::STAGE;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 2) {
      float a0[TM], b0[TM], a1[TM], b1[TM];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const float4 va0 = *reinterpret_cast<const float4*>(as + kk * BM + g * (BM / G) + 4 * tx);
        const float4 vb0 = *reinterpret_cast<const float4*>(bs + kk * BM + g * (BM / G) + 4 * ty);
        const float4 va1 = *reinterpret_cast<const float4*>(as + (kk + 1) * BM + g * (BM / G) + 4 * tx);
        const float4 vb1 = *reinterpret_cast<const float4*>(bs + (kk + 1) * BM + g * (BM / G) + 4 * ty);
        a0[4 * g + 0] = va0.x; a0[4 * g + 1] = va0.y; a0[4 * g + 2] = va0.z; a0[4 * g + 3] = va0.w;
        b0[4 * g + 0] = vb0.x; b0[4 * g + 1] = vb0.y; b0[4 * g + 2] = vb0.z; b0[4 * g + 3] = vb0.w;
        a1[4 * g + 0] = va1.x; a1[4 * g + 1] = va1.y; a1[4 * g + 2] = va1.z; a1[4 * g + 3] = va1.w;
        b1[4 * g + 0] = vb1.x; b1[4 * g + 1] = vb1.y; b1[4 * g + 2] = vb1.z; b1[4 * g + 3] = vb1.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) focus_step2(acc[i][j], a0[i], b0[j], a1[i], b1[j], scale, cst[i][j]);
    }
    __syncthreads();
  }

  // u = n - #{z : min > t}; zero-filled z beyond n never count (m = 0 <= t)
  const int nn = static_cast<int>(n);
#pragma unroll
  for (int gi = 0; gi < G; ++gi)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t x = X0 + gi * (BM / G) + 4 * tx + i;
      const int r = gi * 4 + i;
#pragma unroll
      for (int gj = 0; gj < G; ++gj) {
        const int c = gj * 4;
        int4 v = make_int4(nn - count_of(acc[r][c + 0]), nn - count_of(acc[r][c + 1]),
                           nn - count_of(acc[r][c + 2]), nn - count_of(acc[r][c + 3]));
        store4i(U, n, x, Y0 + gj * (BM / G) + 4 * ty, v, vec);
      }
    }
  if (bi != bj) {
#pragma unroll
    for (int gj = 0; gj < G; ++gj)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t y = Y0 + gj * (BM / G) + 4 * ty + j;
        const int c = gj * 4 + j;
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
          const int r = gi * 4;
          int4 v = make_int4(nn - count_of(acc[r + 0][c]), nn - count_of(acc[r + 1][c]),
                             nn - count_of(acc[r + 2][c]), nn - count_of(acc[r + 3][c]));
          store4i(U, n, y, X0 + gi * (BM / G) + 4 * tx, v, vec);
        }
      }
  }
}

}  // namespace pald
