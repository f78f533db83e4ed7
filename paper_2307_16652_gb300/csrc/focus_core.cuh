// Pass 1 core: local focus sizes of one CTA tile of U.
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
// Layout: the CTA streams z through shared memory in stages of BK.  Because
// D is symmetric, the column block D[X, z-stage] is read as the rows
// D[z-stage, X], so every global read is a contiguous row segment (the
// "transpose" is free).  See tile_geom.cuh for the thread ownership.
#pragma once

#include <type_traits>

#include "tile_geom.cuh"

namespace pald {

// Copy rows z0..z0+BK-1, columns c0..c0+W-1 of the n x n matrix at M into
// dst[BK][W]; out-of-range elements are zero-filled.
template <int W, int NT, int BK>
__device__ __forceinline__ void stage_rows(float* dst, const float* __restrict__ M, int64_t n, int64_t z0,
                                           int64_t c0, bool vec) {
  if (vec) {
    constexpr int V = BK * W / 4;
#pragma unroll
    for (int k = threadIdx.x; k < V; k += NT) {
      const int r = k / (W / 4), c = (k % (W / 4)) * 4;
      const int64_t row = z0 + r, col = c0 + c;
      const bool ok = row < n && col < n;  // n % 4 == 0: a vector is all in or all out
      cp_async16(dst + r * W + c, ok ? M + row * n + col : M, ok ? 16 : 0);
    }
  } else {
    constexpr int V = BK * W;
#pragma unroll 4
    for (int k = threadIdx.x; k < V; k += NT) {
      const int r = k / W, c = k % W;
      const int64_t row = z0 + r, col = c0 + c;
      const bool ok = row < n && col < n;
      cp_async4(dst + r * W + c, ok ? M + row * n + col : M, ok ? 4 : 0);
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

// W (4 or 2) consecutive floats of a shared-memory operand row.
template <int W = 4>
__device__ __forceinline__ void lds(const float* p, float* out) {
  if (W == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    out[0] = v.x;
    out[1] = v.y;
  }
}

// Store W (4 or 2) consecutive values of row `row` at column `col`.
template <int W, typename T>
__device__ __forceinline__ void storew(T* __restrict__ M, int64_t n, int64_t row, int64_t col, const T* v, bool vec) {
  if (row >= n) return;
  T* p = M + row * n + col;
  if (W == 4 && vec && col + 3 < n) {
    if constexpr (sizeof(T) == 4) {
      using V4 = typename std::conditional<std::is_same<T, float>::value, float4, int4>::type;
      V4 q;
      q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
      *reinterpret_cast<V4*>(p) = q;
    }
    return;
  }
  if (W == 2 && vec && col + 1 < n) {
    using V2 = typename std::conditional<std::is_same<T, float>::value, float2, int2>::type;
    V2 q;
    q.x = v[0]; q.y = v[1];
    *reinterpret_cast<V2*>(p) = q;
    return;
  }
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (col + k < n) p[k] = v[k];
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

// Stages in flight: the buffer refilled while stage s is computed is the one
// stage s-1 used, so one barrier per stage orders reuse and visibility.
constexpr int kPipe = 3;

template <class Geo>
struct FocusSmem {
  static constexpr int FLOATS = kPipe * (Geo::SX + Geo::SY);  // kPipe stages of both operands
};

// Computes and stores U[X, Y] (and U[Y, X] off the diagonal) for super-tile
// (bi, bj), column slice `slice`.  `smem` holds FocusSmem<Geo>::FLOATS
// floats.  Must be called by all Geo::NT threads.
template <class Geo>
__device__ __forceinline__ void focus_tile(const float* __restrict__ D, int64_t n, int32_t* __restrict__ U, int bi,
                                           int bj, int slice, float scale, float* smem) {
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY, NT = Geo::NT;
  const int64_t X0 = static_cast<int64_t>(bi) * Geo::B;
  const int64_t Y0 = static_cast<int64_t>(bj) * Geo::B + static_cast<int64_t>(slice) * Geo::BY;
  const int tx = threadIdx.x % Geo::TPX, ty = threadIdx.x / Geo::TPX;
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(D) % 16) == 0;

  float* As = smem;                       // [kPipe][BK][BX]  D[z][X0 + .]
  float* Bs = smem + kPipe * Geo::SX;     // [kPipe][BK][BY]  D[z][Y0 + .]

  const int64_t nstages = (n + BK - 1) / BK;
#pragma unroll
  for (int p = 0; p < kPipe - 1; ++p) {
    if (p < nstages) {
      stage_rows<Geo::BX, NT, BK>(As + p * Geo::SX, D, n, p * BK, X0, vec);
      stage_rows<Geo::BY, NT, BK>(Bs + p * Geo::SY, D, n, p * BK, Y0, vec);
    }
    cp_async_commit();
  }

  // thresholds t = d_xy -> c = -t * scale (exact: power-of-two scaling)
  float cst[TX][TY];
  uint64_t acc[TX][TY];
#pragma unroll
  for (int i = 0; i < TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int j = 0; j < TY; ++j) {
      const int64_t y = Y0 + Geo::col_off(ty, j);
      cst[i][j] = (x < n && y < n) ? -__ldg(D + x * n + y) * scale : 0.f;
    }
  }
#pragma unroll
  for (int i = 0; i < TX; ++i)
#pragma unroll
    for (int j = 0; j < TY; ++j) acc[i][j] = 0ull;

  for (int64_t st = 0; st < nstages; ++st) {
    const int buf = static_cast<int>(st % kPipe);
    cp_async_wait<kPipe - 2>();  // stage st has landed (later ones may be in flight)
    __syncthreads();             // ... for every thread, and stage st-1's buffer is free
    if (st + kPipe - 1 < nstages) {
      const int nb = static_cast<int>((st + kPipe - 1) % kPipe);
      stage_rows<Geo::BX, NT, BK>(As + nb * Geo::SX, D, n, (st + kPipe - 1) * BK, X0, vec);
      stage_rows<Geo::BY, NT, BK>(Bs + nb * Geo::SY, D, n, (st + kPipe - 1) * BK, Y0, vec);
    }
    cp_async_commit();  // possibly empty: keeps one group per stage
    const float* as = As + buf * Geo::SX;
    const float* bs = Bs + buf * Geo::SY;
#pragma unroll Geo::UNR / 2
    for (int kk = 0; kk < BK; kk += 2) {
      float a0[TX], b0[TY], a1[TX], b1[TY];
#pragma unroll
      for (int g = 0; g < Geo::GX; ++g) {
        lds<4>(as + kk * Geo::BX + Geo::row_off(tx, 4 * g), a0 + 4 * g);
        lds<4>(as + (kk + 1) * Geo::BX + Geo::row_off(tx, 4 * g), a1 + 4 * g);
      }
#pragma unroll
      for (int g = 0; g < Geo::GY; ++g) {
        lds<Geo::CW>(bs + kk * Geo::BY + Geo::col_off(ty, Geo::CW * g), b0 + Geo::CW * g);
        lds<Geo::CW>(bs + (kk + 1) * Geo::BY + Geo::col_off(ty, Geo::CW * g), b1 + Geo::CW * g);
      }
#pragma unroll
      for (int i = 0; i < TX; ++i)
#pragma unroll
        for (int j = 0; j < TY; ++j) focus_step2(acc[i][j], a0[i], b0[j], a1[i], b1[j], scale, cst[i][j]);
    }
  }

  // u = n - #{z : min > t}; zero-filled z beyond n never count (m = 0 <= t)
  const int nn = static_cast<int>(n);
#pragma unroll
  for (int i = 0; i < TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int gj = 0; gj < Geo::GY; ++gj) {
      int32_t v[Geo::CW];
#pragma unroll
      for (int k = 0; k < Geo::CW; ++k) v[k] = nn - count_of(acc[i][Geo::CW * gj + k]);
      storew<Geo::CW>(U, n, x, Y0 + Geo::col_off(ty, Geo::CW * gj), v, vec);
    }
  }
  if (bi != bj) {
#pragma unroll
    for (int j = 0; j < TY; ++j) {
      const int64_t y = Y0 + Geo::col_off(ty, j);
#pragma unroll
      for (int gi = 0; gi < Geo::GX; ++gi) {
        int32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = nn - count_of(acc[4 * gi + k][j]);
        storew<4>(U, n, y, X0 + Geo::row_off(tx, 4 * gi), v, vec);
      }
    }
  }
}

}  // namespace pald
