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
#include "tma_ring.cuh"

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

// Thresholds c = -d_xy * scale (exact: power-of-two scaling) and zeroed counts.
template <class Geo>
__device__ __forceinline__ void focus_init(const float* __restrict__ D, int64_t n, int64_t X0, int64_t Y0, int tx,
                                           int ty, float scale, float (&cst)[Geo::TX][Geo::TY],
                                           uint64_t (&acc)[Geo::TX][Geo::TY]) {
#pragma unroll
  for (int i = 0; i < Geo::TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int j = 0; j < Geo::TY; ++j) {
      const int64_t y = Y0 + Geo::col_off(ty, j);
      cst[i][j] = (x < n && y < n) ? -__ldg(D + x * n + y) * scale : 0.f;
      acc[i][j] = 0ull;
    }
  }
}

// Valid streamed indices of stage st, rounded up to a whole chunk of CH:
// the zero-filled rows past n add nothing to either pass, so whole chunks of
// them are skipped.
template <int BK, int CH>
__device__ __forceinline__ int stage_extent(int64_t n, int st) {
  const int64_t nk = n - static_cast<int64_t>(st) * BK;
  return nk >= BK ? BK : static_cast<int>((nk + CH - 1) / CH) * CH;
}

// One pipeline stage (BK consecutive z): as = D[z-stage][X], bs = D[z-stage][Y].
// The stage runs in chunks of CH z (the first `kend` z, a multiple of CH).
template <class Geo, int CH = Geo::BK>
__device__ __forceinline__ void focus_stage(const float* as, const float* bs, int tx, int ty, float scale,
                                            const float (&cst)[Geo::TX][Geo::TY],
                                            uint64_t (&acc)[Geo::TX][Geo::TY], int kend = Geo::BK) {
  constexpr int TX = Geo::TX, TY = Geo::TY;
  constexpr int U2 = (CH == Geo::BK ? Geo::UNR : CH) / 2;
  static_assert(Geo::BK % CH == 0 && CH % 2 == 0, "chunks must tile the stage in pairs of z");
#pragma unroll 1
  for (int k0 = 0; k0 < kend; k0 += CH) {
#pragma unroll U2
    for (int k = 0; k < CH; k += 2) {
      const int kk = k0 + k;
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
}

// 1/u as pass 2 reads it: correctly rounded, 0 on the diagonal (which
// removes the y == x term) and for u <= 0.
__device__ __forceinline__ float recip_entry(int32_t u, int64_t row, int64_t col) {
  return (u <= 0 || row == col) ? 0.f : __frcp_rn(static_cast<float>(u));
}

// Stores W consecutive values of row `row` at column `col` of a matrix of
// order n stored with row pitch `pitch`.
template <int W>
__device__ __forceinline__ void storew_pitched(float* __restrict__ M, int64_t n, int64_t pitch, int64_t row,
                                               int64_t col, const float* v, bool vec) {
  if (row >= n) return;
  float* p = M + row * pitch + col;
  if (W == 4 && vec && col + 3 < n) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    return;
  }
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (col + k < n) p[k] = v[k];
}

// u = n - #{z : min > t} (zero-filled z beyond n never count: m = 0 <= t);
// stores U[X, Y] and, when `mirror`, U[Y, X].  U has row pitch n.  With a
// non-null R it also stores R = 1/u (recip_entry) there, row pitch `rpitch`
// (a multiple of 4), so that pass 2 needs no reciprocal kernel.
template <class Geo>
__device__ __forceinline__ void focus_finish(int32_t* __restrict__ U, int64_t n, int64_t X0, int64_t Y0, int tx,
                                             int ty, bool mirror, bool vec, const uint64_t (&acc)[Geo::TX][Geo::TY],
                                             float* __restrict__ R = nullptr, int64_t rpitch = 0) {
  const int nn = static_cast<int>(n);
#pragma unroll
  for (int i = 0; i < Geo::TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int gj = 0; gj < Geo::GY; ++gj) {
      const int64_t y0 = Y0 + Geo::col_off(ty, Geo::CW * gj);
      int32_t v[Geo::CW];
#pragma unroll
      for (int k = 0; k < Geo::CW; ++k) v[k] = nn - count_of(acc[i][Geo::CW * gj + k]);
      storew<Geo::CW>(U, n, x, y0, v, vec);
      if (R) {
        float r[Geo::CW];
#pragma unroll
        for (int k = 0; k < Geo::CW; ++k) r[k] = recip_entry(v[k], x, y0 + k);
        storew_pitched<Geo::CW>(R, n, rpitch, x, y0, r, true);
      }
    }
  }
  if (mirror) {
#pragma unroll
    for (int j = 0; j < Geo::TY; ++j) {
      const int64_t y = Y0 + Geo::col_off(ty, j);
#pragma unroll
      for (int gi = 0; gi < Geo::GX; ++gi) {
        const int64_t x0 = X0 + Geo::row_off(tx, 4 * gi);
        int32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = nn - count_of(acc[4 * gi + k][j]);
        storew<4>(U, n, y, x0, v, vec);
        if (R) {
          float r[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) r[k] = recip_entry(v[k], y, x0 + k);
          storew_pitched<4>(R, n, rpitch, y, x0, r, true);
        }
      }
    }
  }
}

// Computes and stores U[X, Y] (and U[Y, X] off the diagonal) for super-tile
// (bi, bj), column slice `slice`, staging operands with per-thread cp.async
// copies.  `smem` holds FocusSmem<Geo>::FLOATS floats.  Must be called by
// all Geo::NT threads.
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
  float cst[TX][TY];
  uint64_t acc[TX][TY];
  focus_init<Geo>(D, n, X0, Y0, tx, ty, scale, cst, acc);

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
    focus_stage<Geo>(As + buf * Geo::SX, Bs + buf * Geo::SY, tx, ty, scale, cst, acc);
  }
  focus_finish<Geo>(U, n, X0, Y0, tx, ty, bi != bj, vec, acc);
}

// ---------------------------------------------------------------------------
// Group pairs of a diagonal pass-1 TMA tile.
//
// A diagonal 64 x 64 tile of focus_tile_tma with `skip_diag` hands threads
// only its 4 x 4 blocks strictly above the diagonal (120 blocks: threads
// 0..119, warps 0..3, one per scheduler).  The pairs (x, z) with
// x / 4 == z / 4, which its sixteen diagonal blocks would hold, go to the
// four warps that are left (threads 128..255): ten pairs per group (i <= j;
// u is symmetric), pair slot p = 10 g + k of group g, slots t - 128 and t for
// thread t (the second only for threads below 160, so 160 slots in all).
// Each of those warps carries one or two pairs per lane instead of a block's
// sixteen, so a diagonal tile costs about half a full one instead of a whole
// one, and reads only the tile's own panel.  The counts are exact, so the
// bits are the block code's.  (Pass 2 leaves these pairs to cohesion_group,
// a kernel of its own: beside pass 2's long unrolled loops the extra
// shared-memory reads of in-tile group warps cost more than they save.)

__device__ __forceinline__ float comp4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Row y, columns x0 .. x0+3 of a matrix of order n with row pitch `pitch`
// (a multiple of 4, 16-byte aligned rows; the columns up to the pitch
// exist); zeros for y >= n.
__device__ __forceinline__ float4 group_row(const float* __restrict__ M, int64_t pitch, int64_t n, int64_t y,
                                            int64_t x0) {
  if (y >= n) return make_float4(0.f, 0.f, 0.f, 0.f);
  return __ldg(reinterpret_cast<const float4*>(M + y * pitch + x0));
}

// Pair k = 0..9 of a group: (i, j) with i <= j, row by row.
__host__ __device__ constexpr int group_pair_i(int k) { return k < 4 ? 0 : (k < 7 ? 1 : (k < 9 ? 2 : 3)); }
__host__ __device__ constexpr int group_pair_j(int k) {
  return k < 4 ? k : (k < 7 ? k - 3 : (k < 9 ? k - 5 : 3));
}

constexpr int kGroupThread0 = 128;  // first thread of the group warps

// The (up to two) pairs of thread t on a diagonal tile whose rows are
// X0 .. X0 + rows - 1 (rows >= 1; the tile's ragged end included).
struct GroupPairs {
  int cnt;          // pairs of this thread: 0, 1 or 2
  int ci[2], cj[2]; // tile columns 4g + i, 4g + j of the pair's points
  __device__ __forceinline__ GroupPairs(int t, int64_t rows) {
    const int ax = rows >= 64 ? 16 : static_cast<int>((rows + 3) / 4);  // groups holding rows
    const int total = 10 * ax;
    cnt = 0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int p = t - kGroupThread0 + kGroupThread0 * s;
      const bool on = t >= kGroupThread0 && p < total;
      const int g = p / 10, k = p - 10 * (p / 10);
      ci[s] = on ? 4 * g + group_pair_i(k) : 0;
      cj[s] = on ? 4 * g + group_pair_j(k) : 0;
      if (on) cnt = s + 1;
    }
  }
};

// Pass 1, one stage: the group pairs' counts in acc[0][0] and acc[0][1]
// (the packed counts of z even / odd, as focus_step2 keeps them).  as is
// the stage's panel D[z-stage][X].
template <class Geo, int CH>
__device__ __forceinline__ void focus_group_stage(const float* as, const GroupPairs& gp, float scale,
                                                  const float (&cst)[Geo::TX][Geo::TY],
                                                  uint64_t (&acc)[Geo::TX][Geo::TY], int kend) {
#pragma unroll 1
  for (int k0 = 0; k0 < kend; k0 += 4) {  // a short loop body, as in cohesion_group_stage
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const float* a = as + (k0 + k) * Geo::BX;
      const float* b = a + Geo::BX;
      focus_step2(acc[0][0], a[gp.ci[0]], a[gp.cj[0]], b[gp.ci[0]], b[gp.cj[0]], scale, cst[0][0]);
      if (gp.cnt > 1)
        focus_step2(acc[0][1], a[gp.ci[1]], a[gp.cj[1]], b[gp.ci[1]], b[gp.cj[1]], scale, cst[0][1]);
    }
  }
}

// Stores u (and 1/u into R when given, recip_entry) of the group pairs,
// both orders; a[s] is pair s's packed count.
__device__ __forceinline__ void focus_group_finish(int32_t* __restrict__ U, int64_t n, int64_t X0,
                                                   const GroupPairs& gp, const uint64_t (&a)[2],
                                                   float* __restrict__ R, int64_t rpitch) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int64_t x = X0 + gp.ci[s], z = X0 + gp.cj[s];
    if (s < gp.cnt && x < n && z < n) {
      const int32_t u = static_cast<int32_t>(n) - count_of(a[s]);
      U[x * n + z] = u;
      U[z * n + x] = u;
      if (R) {
        R[x * rpitch + z] = recip_entry(u, x, z);
        R[z * rpitch + x] = recip_entry(u, z, x);
      }
    }
  }
}

// TMA-staged pass-1 tile (64 x 64, see tma_ring.cuh): the X and Y panels of
// each stage come from the tensor map `tmD` of the n x n matrix (which may
// be a row-padded copy); thresholds are read from D (row pitch n), U is
// written with row pitch n, and R = 1/u too when R is given (focus_finish).
// With `skip_diag` a diagonal tile runs its pairs inside the groups of four
// points on the threads from 128 on (GroupPairs above).  Returns false when
// a wait ran out of time.
template <class Geo>
__device__ __forceinline__ bool focus_tile_tma(const CUtensorMap* tmD, const float* __restrict__ D, int64_t n,
                                               int32_t* __restrict__ U, int bi, int bj, float scale, bool vec,
                                               TmaRing<2, Geo::BK>& ring, float* __restrict__ R = nullptr,
                                               int64_t rpitch = 0, bool skip_diag = false) {
  static_assert(Geo::BX == 64 && Geo::BY == 64 && Geo::TPX == 16 && Geo::TPY == 16 && Geo::GX == 1 &&
                    Geo::GY == 1 && Geo::CW == 4,
                "TMA tiles are 64 x 64 with 4 x 4 pairs per thread");
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY;
  int tx, ty;
  const bool active = tile_block_64(bi, bj, n, threadIdx.x, &tx, &ty, skip_diag);
  const bool grp = skip_diag && bi == bj && threadIdx.x >= kGroupThread0;  // a group-pair thread
  const int64_t X0 = int64_t(bi) * 64, rows = n - X0;
  const int nstages = static_cast<int>((n + BK - 1) / BK);
  constexpr int CH = 16;  // the last stage runs only its chunks that hold rows of the matrix
  if (threadIdx.x == 0) ring.init();
  __syncthreads();
  float cst[TX][TY];
  uint64_t acc[TX][TY];
  focus_init<Geo>(D, n, X0, int64_t(bj) * 64, tx, ty, scale, cst, acc);
  if (grp) {  // the group pairs' thresholds take slots [0][0] and [0][1]
    const GroupPairs gp(threadIdx.x, rows);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int64_t x = X0 + gp.ci[s], z = X0 + gp.cj[s];
      cst[0][s] = (s < gp.cnt && x < n && z < n) ? -__ldg(D + x * n + z) * scale : 0.f;
    }
  }
  const CUtensorMap* const maps[2] = {tmD, tmD};
  const int cols[2] = {bi * 64, bj * 64};
  const bool ok = tma_pipeline(ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
                               [&](int st, int buf) {
                                 const int kend = stage_extent<BK, CH>(n, st);
                                 if (grp)
                                   focus_group_stage<Geo, CH>(ring.panel(buf, 0), GroupPairs(threadIdx.x, rows),
                                                              scale, cst, acc, kend);
                                 else if (active)
                                   focus_stage<Geo, CH>(ring.panel(buf, 0), ring.panel(buf, 1), tx, ty, scale, cst,
                                                        acc, kend);
                               });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  // off the diagonal, or for an above-diagonal block of a diagonal tile,
  // the block's mirror is written too
  if (ok && active)
    focus_finish<Geo>(U, n, X0, int64_t(bj) * 64, tx, ty, tx != ty || bi != bj, vec, acc, R, rpitch);
  if (ok && grp) focus_group_finish(U, n, X0, GroupPairs(threadIdx.x, rows), {acc[0][0], acc[0][1]}, R, rpitch);
  return ok;
}

// ---------------------------------------------------------------------------
// Two diagonal tiles in one CTA (batched pass 1).  A diagonal 64 x 64 tile
// without its in-group pairs has 120 4 x 4 blocks strictly above its
// diagonal: four warps' worth.  Alone it would leave half of a CTA's warps
// idle for a whole tile; here threads 0..127 take the blocks of diagonal
// tile (ba, ba) and threads 128..255 those of (bb, bb) of the same matrix
// (bb < 0: the second half idles), each half reading its own panel of the
// stage (D[z][Xa] and D[z][Xb]).  The pairs inside the groups of four
// points are left to focus_group.  Counts are exact, so the bits are the
// single tile's.  Returns false when a wait ran out of time.
template <class Geo>
__device__ __forceinline__ bool focus_diag_pair_tma(const CUtensorMap* tmD, const float* __restrict__ D, int64_t n,
                                                    int32_t* __restrict__ U, int ba, int bb, float scale, bool vec,
                                                    TmaRing<2, Geo::BK>& ring, float* __restrict__ R,
                                                    int64_t rpitch) {
  static_assert(Geo::BX == 64 && Geo::BY == 64 && Geo::NT == 256, "pairs of 64 x 64 tiles on 256 threads");
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY;
  const int half = static_cast<int>(threadIdx.x) / 128;  // warp-uniform
  const int bi = half == 0 ? ba : bb;
  int tx = 0, ty = 0;  // an idle half keeps a valid placement (its setup loads stay in the matrix)
  const bool active = bi >= 0 && tile_block_64(bi, bi, n, threadIdx.x % 128, &tx, &ty, true);
  const int64_t X0 = int64_t(bi >= 0 ? bi : ba) * 64;
  const int nstages = static_cast<int>((n + BK - 1) / BK);
  constexpr int CH = 16;
  if (threadIdx.x == 0) ring.init();
  __syncthreads();
  float cst[TX][TY];
  uint64_t acc[TX][TY];
  focus_init<Geo>(D, n, X0, X0, tx, ty, scale, cst, acc);
  const CUtensorMap* const maps[2] = {tmD, tmD};
  const int cols[2] = {ba * 64, (bb >= 0 ? bb : ba) * 64};
  const bool ok = tma_pipeline(ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
                               [&](int st, int buf) {
                                 if (active)
                                   focus_stage<Geo, CH>(ring.panel(buf, half), ring.panel(buf, half), tx, ty, scale,
                                                        cst, acc, stage_extent<BK, CH>(n, st));
                               });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  // every block is strictly above the diagonal: its mirror is written too
  if (ok && active) focus_finish<Geo>(U, n, X0, X0, tx, ty, true, vec, acc, R, rpitch);
  return ok;
}

// The pairs inside group q of four points x0 .. x0+3 (x0 = 4q), both orders
// and the diagonal, for pass 1: one thread streams z through the group's
// four columns of row z (one 16-byte vector of the row-padded copy Dp:
// d_zx = d_xz by symmetry) and counts [min(d_xz, d_x'z) > d_xx'] for the ten
// pairs x <= x'.  Writes u to U (row pitch n) and 1/u (recip_entry) to R
// (row pitch `rpitch`).  Exact counts: the bits of the tile code.  (Its cost
// is one read of Dp from HBM: the matrix's data has left L2 by then.)
__device__ __forceinline__ void focus_group(const float* __restrict__ Dp, int64_t pitch, int64_t n, int64_t q,
                                            float scale, int32_t* __restrict__ U, float* __restrict__ R,
                                            int64_t rpitch) {
  const int64_t x0 = 4 * q;
  float cst[10];
  {
    float4 row[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = group_row(Dp, pitch, n, x0 + i, x0);
#pragma unroll
    for (int k = 0; k < 10; ++k) cst[k] = -comp4(row[group_pair_i(k)], group_pair_j(k)) * scale;  // exact
  }
  float cnt[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) cnt[k] = 0.f;
#pragma unroll 4
  for (int64_t z = 0; z < n; ++z) {
    const float4 d = group_row(Dp, pitch, n, z, x0);
#pragma unroll
    for (int k = 0; k < 10; ++k)
      cnt[k] += ffma_sat(fmin_(comp4(d, group_pair_i(k)), comp4(d, group_pair_j(k))), scale, cst[k]);
  }
  const int nn = static_cast<int>(n);
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const int64_t x = x0 + group_pair_i(k), y = x0 + group_pair_j(k);
    if (x >= n || y >= n) continue;
    const int32_t u = nn - static_cast<int32_t>(cnt[k]);  // an exact count below 2^24
    U[x * n + y] = u;
    U[y * n + x] = u;
    R[x * rpitch + y] = recip_entry(u, x, y);
    R[y * rpitch + x] = recip_entry(u, y, x);
  }
}

}  // namespace pald
