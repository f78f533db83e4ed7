// Pass 2 core: cohesion of one CTA tile of the pair of blocks (X, Z), X <= Z.
//
// For an output pair (x, z) and every third point y the paper's cohesion
// (Sec. 2 eq. (cohesion), written out as eq. (fxz)) with the half-credit tie
// split of Sec. 5 contributes
//     to c_xz:  [d_xz <= min(d_xy, d_zy)] * w(d_xz, d_zy) * r_xy
//     to c_zx:  [d_xz <= min(d_xy, d_zy)] * w(d_xz, d_xy) * r_zy
// with r = 1/u and w(b, a) = 0, 1/2, 1 for a < b, a == b, a > b.  (z in U_xy
// together with d_zx <= d_zy is the same as d_xz <= min(d_xy, d_zy).)  R has
// a zero diagonal, which removes the excluded y == x term exactly, duplicate
// points included.  R = 1/u is precomputed once per matrix (the reciprocal
// loop between the passes, Sec. 6 figures), not in this kernel.
//
// Exact comparisons.  S = 2^(23 - e) is the matrix-wide power of two of
// pass 1 (e the exponent of the smallest positive entry) and c = -b*S, with
// b = d_xz, is the only per-pair constant.  For any entries a, b of the
// matrix, t = a*S + c (one FFMA) is exactly 0 when a == b and at least 1 in
// magnitude otherwise (a != b differ by at least one unit in the last place
// of the smaller, which S scales to >= 1; a*S and b*S are exact).  Hence
//     sat(t)             = [a > b]
//     sat(t * 1/2 + 1/2) = w(b, a)        (0, 1/2 or 1, exactly)
//
// Long form, per (x, z, y), eight instructions:
//     t2 = d_zy * S + c ;  t1 = d_xy * S + c        2 x FFMA     (FMA pipe)
//     v2 = sat(t2/2 + 1/2) = w(b, d_zy) ; v1 = w(b, d_xy)
//                                                  2 x FFMA.SAT (FMA pipe)
//     m  = min(v1, v2) ;  p = m > 0                FMNMX, FSETP (ALU pipe)
//       (w(b, a) is 0 exactly when a < b, so p is d_xz <= min(d_xy, d_zy))
//     @p S_xz += v2 * r_xy ;  @p S_zx += v1 * r_zy 2 x FFMA     (FMA pipe)
//
// Short form, four instructions, for stages in which no one-sided tie
// (d_xy == d_xz < d_zy, or d_zy == d_zx < d_xy) can occur:
//     m  = min(d_xy, d_zy)                         FMNMX        (ALU pipe)
//     v  = sat(m * S + c) = [m > b]                FFMA.SAT     (FMA pipe)
//     S_xz += v * r_xy ;  S_zx += v * r_zy         2 x FFMA     (FMA pipe)
// Without one-sided ties, b < m gives weight 1 to both sums and b > m gives
// 0 to both.  b == m then needs d_xy == d_zy == d_xz with two equal entries
// in row x or z (a marked tie, so not here), or y == z or y == x with
// b == 0, where x == z and both r vanish (r_xx = 0) or the points are
// duplicates (a marked tie again).  So every add that differs from the long
// form adds +0, and both forms give the same bits.  Which y may use the
// short form comes from the tie map (one bit per 64 x 64 block pair and
// 8 y; tie_map_core.cuh builds it).
//
// Accumulation (PALD_ACCUM_COMPENSATED): the pair {S_xz, S_zx} is an FP32
// partial over kMergeEvery = 8 consecutive y (fold_phase below places the
// chunk ends).  Every 8 y it is folded into the running sums {H_xz, H_zx},
// which start at the bias B = 8: a partial never exceeds 8 * 1/2 plus the
// carried error, so |H| >= |S| always holds and Fast2Sum (three adds, done as
// packed f32x2 ops on both accumulators at once) is error-free.  (Chunks of
// 8 y instead of 4 halve the fold's share of the FMA pipe; on the paper-scale
// and precision-study matrices the measured max and mean errors against the
// FP64 oracle did not change.)  Its exact error becomes the start of the next partial, so
// nothing is lost between chunks.  At the end H - B + S is formed exactly as
// a two-float value, multiplied by 1/(n-1) (also two floats) and rounded once
// to FP32: the precision of an FP64 merge, without the FP64 pipe (two_sum,
// mul_pair below).  PALD_ACCUM_PLAIN keeps one FP32 running sum (the
// precision baseline), normalised the same way.
#pragma once

#include <type_traits>

#include "focus_core.cuh"

namespace pald {

constexpr float kMergeBias = static_cast<float>(kMergeEvery);  // >= kMergeEvery * 1/2 + carried error

template <class Geo>
struct CohesionSmem {
  static constexpr int FLOATS = kPipe * 2 * (Geo::SX + Geo::SY);  // kPipe stages of D_X, R_X, D_Z, R_Z
};

// Long form of one (x, z, y) step on the packed partial {S_xz, S_zx}.
__device__ __forceinline__ void cohesion_step(uint64_t& sacc, float a1, float a2, float S, float c, float r1,
                                              float r2) {
  asm("{\n\t.reg .pred p;\n\t.reg .f32 m, t1, t2, v1, v2, sx, sz;\n\t"
      "mov.b64 {sx, sz}, %0;\n\t"
      "fma.rn.f32 t2, %2, %3, %4;\n\t"
      "fma.rn.f32 t1, %1, %3, %4;\n\t"
      "fma.rn.sat.f32 v2, t2, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.sat.f32 v1, t1, 0f3F000000, 0f3F000000;\n\t"
      "min.f32 m, v1, v2;\n\t"
      "setp.gt.f32 p, m, 0f00000000;\n\t"
      "@p fma.rn.f32 sx, v2, %5, sx;\n\t"
      "@p fma.rn.f32 sz, v1, %6, sz;\n\t"
      "mov.b64 %0, {sx, sz};\n\t}"
      : "+l"(sacc)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(r1), "f"(r2));
}

// Short form of one (x, z, y) step (no one-sided tie possible).
__device__ __forceinline__ void cohesion_step_short(uint64_t& sacc, float a1, float a2, float S, float c, float r1,
                                                    float r2) {
  asm("{\n\t.reg .f32 m, v, sx, sz;\n\t"
      "mov.b64 {sx, sz}, %0;\n\t"
      "min.f32 m, %1, %2;\n\t"
      "fma.rn.sat.f32 v, m, %3, %4;\n\t"
      "fma.rn.f32 sx, v, %5, sx;\n\t"
      "fma.rn.f32 sz, v, %6, sz;\n\t"
      "mov.b64 %0, {sx, sz};\n\t}"
      : "+l"(sacc)
      : "f"(a1), "f"(a2), "f"(S), "f"(c), "f"(r1), "f"(r2));
}

// Fold phase of the pair in row slot i and column slot j of a thread tile:
// kMergeEvery - 1 when x + z is even, kMergeEvery / 2 - 1 when it is odd,
// for the pair's global (x, z).
// Every geometry puts x == i and z == j (mod 2) (tile_geom.cuh), so this is
// a compile-time constant per slot.  It must be symmetric in x and z:
// depending on the tile size, c_zx is the zx lane of pair (x, z) or the xz
// lane of pair (z, x), and a symmetric phase gives both the same chunking,
// so every schedule, both forms and the batched path stay bit-identical.
__host__ __device__ constexpr int fold_phase(int i, int j) {
  return ((i + j) & 1) ? kMergeEvery / 2 - 1 : kMergeEvery - 1;
}

// ---------------------------------------------------------------------------
// Final merge in two-float arithmetic.  GB300 runs FP64 at about two
// operations per clock per SM, so a per-entry FP64 merge costs more than the
// inner loop of a short tile; these error-free transformations give the same
// result (the exact merge rounded once to FP32, up to 2^-46 relative).

// TwoSum (Knuth): s + e == a + b exactly, s = RN(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// 1/m as hi + lo for a positive integer m < 2^24: hi = RN(1/m), and
// lo = (1 - hi*m) * hi, where 1 - hi*m comes out of one FMA exactly (the
// residual of a correctly rounded reciprocal), so hi + lo = 1/m to about
// 2^-47 relative.
__device__ __forceinline__ void inverse_pair(int64_t m, float& hi, float& lo) {
  const float mf = static_cast<float>(m);
  hi = __frcp_rn(mf);
  lo = __fmul_rn(__fmaf_rn(-hi, mf, 1.0f), hi);
}

// RN((a + b) * (ih + il)) for a two-float a + b (|b| <= ulp(a)) and a
// two-float ih + il, up to 2^-46 relative: a*ih is split exactly by an FMA,
// the small cross terms are added to its error, and one final add rounds.
__device__ __forceinline__ float mul_pair(float a, float b, float ih, float il) {
  const float m = __fmul_rn(a, ih);
  const float t = __fmaf_rn(a, ih, -m);
  return __fadd_rn(m, __fmaf_rn(a, il, __fmaf_rn(b, ih, t)));
}

// Packed f32x2 add and subtract (one instruction for both lanes).
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// Fast2Sum on both lanes: h + s == old h + old s exactly when |h| >= |s|;
// h takes the rounded sum and s the exact rounding error.
__device__ __forceinline__ void fast2sum_fold(uint64_t& h, uint64_t& s) {
  const uint64_t t = add2(h, s);
  const uint64_t z = sub2(t, h);
  s = sub2(s, z);
  h = t;
}

__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// One pipeline stage (BK consecutive y) of a CTA tile, long or short form,
// in chunks of U y: y kbeg .. kend-1 of the stage (multiples of U; the
// zero-filled y past n add +0, so whole chunks of them are skipped).
template <class Geo, int MODE, bool SHORT, int U = Geo::UNR>
__device__ __forceinline__ void cohesion_stage(const float* ad, const float* ar, const float* bd, const float* br,
                                               int tx, int tz, float S, const float (&cv)[Geo::TX][Geo::TY],
                                               uint64_t (&sacc)[Geo::TX][Geo::TY],
                                               uint64_t (&hacc)[Geo::TX][Geo::TY], int kend = Geo::BK,
                                               int kbeg = 0) {
  constexpr int TX = Geo::TX, TY = Geo::TY;
  static_assert(U % kMergeEvery == 0, "chunks hold whole merge chunks");
#pragma unroll 1
  for (int k0 = kbeg; k0 < kend; k0 += U) {
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int kk = k0 + k;
      float a1[TX], r1[TX], a2[TY], r2[TY];
#pragma unroll
      for (int g = 0; g < Geo::GX; ++g) {
        lds<4>(ad + kk * Geo::BX + Geo::row_off(tx, 4 * g), a1 + 4 * g);
        lds<4>(ar + kk * Geo::BX + Geo::row_off(tx, 4 * g), r1 + 4 * g);
      }
#pragma unroll
      for (int g = 0; g < Geo::GY; ++g) {
        lds<Geo::CW>(bd + kk * Geo::BY + Geo::col_off(tz, Geo::CW * g), a2 + Geo::CW * g);
        lds<Geo::CW>(br + kk * Geo::BY + Geo::col_off(tz, Geo::CW * g), r2 + Geo::CW * g);
      }
#pragma unroll
      for (int q = 0; q < TX * TY; ++q) {
        const int i = q / TY, j = q % TY;
        if (SHORT)
          cohesion_step_short(sacc[i][j], a1[i], a2[j], S, cv[i][j], r1[i], r2[j]);
        else
          cohesion_step(sacc[i][j], a1[i], a2[j], S, cv[i][j], r1[i], r2[j]);
      }
      if (MODE == PALD_ACCUM_COMPENSATED) {
        // pair (x, z) folds after the y with y mod kMergeEvery ==
        // fold_phase(i, j) (k0 and every stage start are multiples of
        // kMergeEvery): half of a thread's pairs fold at each of two y per
        // chunk, spreading the packed adds over the FMA pipe
#pragma unroll
        for (int i = 0; i < TX; ++i)
#pragma unroll
          for (int j = 0; j < TY; ++j)
            if ((k % kMergeEvery) == fold_phase(i, j)) fast2sum_fold(hacc[i][j], sacc[i][j]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Packed stage of the 64 x 64 TMA tile (4 x 4 pairs per thread).  The
// partials of pairs (i, j) and (i, j + 2) fold at the same y (x + z keeps
// its parity), so they share one 64-bit register per side:
//   sx[i][jj] = {S_xz(i, jj), S_xz(i, jj + 2)},  sz[i][jj] = {S_zx(i, jj), S_zx(i, jj + 2)}
// (hx, hz the same for H).  The short form then credits both pairs of a
// side with one packed FMA: 3 issue slots per pair instead of 4, with the
// same FMA-pipe work.  Every lane performs exactly the FMA of the scalar
// form, so the bits do not change.  The R panels must hold the columns of
// each group of four in the order 0, 2, 1, 3 (reciprocal_rows with
// `paired`): {r_zy(jj), r_zy(jj + 2)} is then one aligned register pair,
// and {r_xy, r_xy} costs one move per row slot and y.

// Short form of pairs (i, jj) and (i, jj + 2).
__device__ __forceinline__ void cohesion_step2_short(uint64_t& sx, uint64_t& sz, float a1, float a2lo, float a2hi,
                                                     float S, float clo, float chi, uint64_t r1d, uint64_t r2p) {
  asm("{\n\t.reg .f32 m0, m1, v0, v1;\n\t.reg .b64 v;\n\t"
      "min.f32 m0, %2, %3;\n\t"
      "min.f32 m1, %2, %4;\n\t"
      "fma.rn.sat.f32 v0, m0, %5, %6;\n\t"
      "fma.rn.sat.f32 v1, m1, %5, %7;\n\t"
      "mov.b64 v, {v0, v1};\n\t"
      "fma.rn.f32x2 %0, v, %8, %0;\n\t"
      "fma.rn.f32x2 %1, v, %9, %1;\n\t}"
      : "+l"(sx), "+l"(sz)
      : "f"(a1), "f"(a2lo), "f"(a2hi), "f"(S), "f"(clo), "f"(chi), "l"(r1d), "l"(r2p));
}

// Long form of pairs (i, jj) and (i, jj + 2) on the packed partials: per
// lane the operations of cohesion_step, with both lanes of sx and sz
// updated in place.
__device__ __forceinline__ void cohesion_step2_long(uint64_t& sx, uint64_t& sz, float a1, float a2lo, float a2hi,
                                                    float S, float clo, float chi, float r1, float r2lo,
                                                    float r2hi) {
  asm("{\n\t.reg .pred p0, p1;\n\t"
      ".reg .f32 m0, m1, t10, t11, t20, t21, v10, v11, v20, v21, x0, x1, z0, z1;\n\t"
      "mov.b64 {x0, x1}, %0;\n\t"
      "mov.b64 {z0, z1}, %1;\n\t"
      "fma.rn.f32 t20, %3, %5, %6;\n\t"
      "fma.rn.f32 t21, %4, %5, %7;\n\t"
      "fma.rn.f32 t10, %2, %5, %6;\n\t"
      "fma.rn.f32 t11, %2, %5, %7;\n\t"
      "fma.rn.sat.f32 v20, t20, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.sat.f32 v21, t21, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.sat.f32 v10, t10, 0f3F000000, 0f3F000000;\n\t"
      "fma.rn.sat.f32 v11, t11, 0f3F000000, 0f3F000000;\n\t"
      "min.f32 m0, v10, v20;\n\t"
      "min.f32 m1, v11, v21;\n\t"
      "setp.gt.f32 p0, m0, 0f00000000;\n\t"
      "setp.gt.f32 p1, m1, 0f00000000;\n\t"
      "@p0 fma.rn.f32 x0, v20, %8, x0;\n\t"
      "@p1 fma.rn.f32 x1, v21, %8, x1;\n\t"
      "@p0 fma.rn.f32 z0, v10, %9, z0;\n\t"
      "@p1 fma.rn.f32 z1, v11, %10, z1;\n\t"
      "mov.b64 %0, {x0, x1};\n\t"
      "mov.b64 %1, {z0, z1};\n\t}"
      : "+l"(sx), "+l"(sz)
      : "f"(a1), "f"(a2lo), "f"(a2hi), "f"(S), "f"(clo), "f"(chi), "f"(r1), "f"(r2lo), "f"(r2hi));
}

template <class Geo, int MODE, bool SHORT, int U = Geo::UNR>
__device__ __forceinline__ void cohesion_stage_packed(const float* ad, const float* ar, const float* bd,
                                                      const float* br, int tx, int tz, float S,
                                                      const float (&cv)[4][4], uint64_t (&sx)[4][2],
                                                      uint64_t (&sz)[4][2], uint64_t (&hx)[4][2],
                                                      uint64_t (&hz)[4][2], int kend, int kbeg = 0) {
  static_assert(Geo::TX == 4 && Geo::TY == 4 && Geo::GX == 1 && Geo::GY == 1 && Geo::BX == 64 && Geo::BY == 64,
                "the packed stage is for 64 x 64 tiles with 4 x 4 pairs per thread");
  static_assert(U % kMergeEvery == 0, "chunks hold whole merge chunks");
  constexpr int kSlot[4] = {0, 2, 1, 3};  // register of r_xy(i) in the paired order
#pragma unroll 1
  for (int k0 = kbeg; k0 < kend; k0 += U) {
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int kk = k0 + k;
      float a1[4], rx[4], a2[4];
      lds<4>(ad + kk * 64 + 4 * tx, a1);
      lds<4>(ar + kk * 64 + 4 * tx, rx);
      lds<4>(bd + kk * 64 + 4 * tz, a2);
      const ulonglong2 rz = *reinterpret_cast<const ulonglong2*>(br + kk * 64 + 4 * tz);
      const uint64_t r2p[2] = {rz.x, rz.y};  // {r_zy(0), r_zy(2)}, {r_zy(1), r_zy(3)}
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float r1 = rx[kSlot[i]];
        if (SHORT) {
          const uint64_t r1d = pack2(r1, r1);
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
            cohesion_step2_short(sx[i][jj], sz[i][jj], a1[i], a2[jj], a2[jj + 2], S, cv[i][jj], cv[i][jj + 2], r1d,
                                 r2p[jj]);
        } else {
#pragma unroll
          for (int jj = 0; jj < 2; ++jj) {
            float r2lo, r2hi;
            unpack2(r2p[jj], r2lo, r2hi);
            cohesion_step2_long(sx[i][jj], sz[i][jj], a1[i], a2[jj], a2[jj + 2], S, cv[i][jj], cv[i][jj + 2], r1,
                                r2lo, r2hi);
          }
        }
      }
      if (MODE == PALD_ACCUM_COMPENSATED) {
        // the fold points of cohesion_stage: pairs (i, jj) and (i, jj + 2) share fold_phase(i, jj)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 2; ++jj)
            if ((k % kMergeEvery) == fold_phase(i, jj)) {
              fast2sum_fold(hx[i][jj], sx[i][jj]);
              fast2sum_fold(hz[i][jj], sz[i][jj]);
            }
      }
    }
  }
}

// The packed partials of cohesion_stage_packed back in the per-pair layout
// {xz, zx} of cohesion_finish.
__device__ __forceinline__ void unpair_partials(const uint64_t (&sx)[4][2], const uint64_t (&sz)[4][2],
                                                uint64_t (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      float x0, x1, z0, z1;
      unpack2(sx[i][jj], x0, x1);
      unpack2(sz[i][jj], z0, z1);
      acc[i][jj] = pack2(x0, z0);
      acc[i][jj + 2] = pack2(x1, z1);
    }
}

// Reads the tie-map row of one tile's block pair: tied(st) is nonzero when
// stage st (y = st*BK .. st*BK+BK-1) must take the long form.  Uniform over
// the CTA.  A null map, or a dirty block on either side, means "always".
template <int BK>
struct TieCursor {
  const uint32_t* row;
  int64_t nstages;
  int gshift;
  bool all_long;
  __device__ __forceinline__ TieCursor(const uint32_t* tmap, int64_t n, int64_t X0, int64_t Z0) {
    const TieMapDims dm = tie_map_dims(n);
    gshift = dm.gshift;
    const int64_t bx = X0 / kTieBlock, bz = Z0 / kTieBlock;
    row = tmap + (bx * dm.nb + bz) * dm.wpp;
    nstages = (n + BK - 1) / BK;
    all_long = tmap == nullptr || __ldg(tmap + dm.nb * dm.nb * dm.wpp + bx) != 0u ||
               __ldg(tmap + dm.nb * dm.nb * dm.wpp + bz) != 0u;
  }
  __device__ __forceinline__ uint32_t tied(int64_t st) const {
    if (all_long) return 1u;
    if (st >= nstages) return 0u;
    const TieStage ts = tie_stage(st, BK, gshift);
    return (__ldg(row + (ts.g >> 5)) >> (ts.g & 31)) & ts.mask;
  }
};

// Per-pair constants c = -d_xz * S and the zeroed accumulators.
template <class Geo>
__device__ __forceinline__ void cohesion_init(const float* __restrict__ D, int64_t n, int64_t X0, int64_t Z0, int tx,
                                              int tz, float S, float (&cv)[Geo::TX][Geo::TY],
                                              uint64_t (&sacc)[Geo::TX][Geo::TY],
                                              uint64_t (&hacc)[Geo::TX][Geo::TY]) {
#pragma unroll
  for (int i = 0; i < Geo::TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int j = 0; j < Geo::TY; ++j) {
      const int64_t z = Z0 + Geo::col_off(tz, j);
      cv[i][j] = __fmul_rn(-((x < n && z < n) ? __ldg(D + x * n + z) : 0.f), S);  // exact: power of two
    }
  }
  const uint64_t zero2 = pack2(0.f, 0.f);
  const uint64_t bias2 = pack2(kMergeBias, kMergeBias);
#pragma unroll
  for (int i = 0; i < Geo::TX; ++i)
#pragma unroll
    for (int j = 0; j < Geo::TY; ++j) {
      sacc[i][j] = zero2;
      hacc[i][j] = bias2;
    }
}

// Value of the xz (or zx) lane of a pair: compensated (H - B) + S, or plain
// S, times 1/(n-1) = ih + il, formed exactly as a two-float value and
// rounded once.
template <int MODE>
__device__ __forceinline__ float cohesion_value(uint64_t h2, uint64_t s2, bool zx, float ih, float il) {
  float hl, hh, sl, sh;
  unpack2(h2, hl, hh);
  unpack2(s2, sl, sh);
  const float h = zx ? hh : hl, s = zx ? sh : sl;
  if (MODE == PALD_ACCUM_COMPENSATED) {
    float p, e;
    two_sum(__fsub_rn(h, kMergeBias), s, p, e);  // H - B is exact: B is a multiple of H's unit
    return mul_pair(p, e, ih, il);
  }
  return mul_pair(s, 0.f, ih, il);
}

// Final merge and stores of C[X, Z] (and of C[Z, X] when `mirror`).  With
// DEPTH, rs[i] also receives the sum (in FP64, in column order) of the
// stored values of row X0 + row_off(tx, i) inside the matrix, and ms[j]
// that of mirror row Z0 + col_off(tz, j); both start at 0.
template <class Geo, int MODE, bool DEPTH = false>
__device__ __forceinline__ void cohesion_finish(float* __restrict__ C, int64_t n, int64_t X0, int64_t Z0, int tx,
                                                int tz, bool mirror, bool vec,
                                                const uint64_t (&sacc)[Geo::TX][Geo::TY],
                                                const uint64_t (&hacc)[Geo::TX][Geo::TY],
                                                double (*rs)[Geo::TX] = nullptr, double (*ms)[Geo::TY] = nullptr) {
  float ih, il;
  inverse_pair(n - 1, ih, il);
  auto finish = [&](uint64_t h2, uint64_t s2, bool zx) -> float { return cohesion_value<MODE>(h2, s2, zx, ih, il); };
#pragma unroll
  for (int i = 0; i < Geo::TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int gj = 0; gj < Geo::GY; ++gj) {
      float v[Geo::CW];
#pragma unroll
      for (int k = 0; k < Geo::CW; ++k) v[k] = finish(hacc[i][Geo::CW * gj + k], sacc[i][Geo::CW * gj + k], false);
      const int64_t z0 = Z0 + Geo::col_off(tz, Geo::CW * gj);
      storew<Geo::CW>(C, n, x, z0, v, vec);
      if constexpr (DEPTH) {
#pragma unroll
        for (int k = 0; k < Geo::CW; ++k)
          if (x < n && z0 + k < n) (*rs)[i] += static_cast<double>(v[k]);
      }
    }
  }
  if (mirror) {
#pragma unroll
    for (int j = 0; j < Geo::TY; ++j) {
      const int64_t z = Z0 + Geo::col_off(tz, j);
#pragma unroll
      for (int gi = 0; gi < Geo::GX; ++gi) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = finish(hacc[4 * gi + k][j], sacc[4 * gi + k][j], true);
        const int64_t x0 = X0 + Geo::row_off(tx, 4 * gi);
        storew<4>(C, n, z, x0, v, vec);
        if constexpr (DEPTH) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (z < n && x0 + k < n) (*ms)[j] += static_cast<double>(v[k]);
        }
      }
    }
  }
}

template <class Geo>
__device__ __forceinline__ void cohesion_tile_checks() {
  static_assert(Geo::BK % kMergeEvery == 0 && Geo::UNR % kMergeEvery == 0, "stages must hold whole merge chunks");
  static_assert(Geo::B <= kTieBlock && kTieBlock % Geo::B == 0, "a tile must lie in one tie-map block pair");
  static_assert(Geo::BK == 16 || Geo::BK == 32 || Geo::BK == 64, "stage depth must tile the tie-map y groups");
}

// Computes C[X, Z] (and C[Z, X] off the diagonal) for super-tile (bi, bj),
// column slice `slice`, staging operands with per-thread cp.async copies.
// `smem` holds CohesionSmem<Geo>::FLOATS floats.  `tmap` is the matrix's
// tie map (null: long form everywhere); S its pass-1 scale (focus_scale).
// Must be called by all Geo::NT threads.
template <class Geo, int MODE>
__device__ __forceinline__ void cohesion_tile(const float* __restrict__ D, const float* __restrict__ R, int64_t n,
                                              float* __restrict__ C, const uint32_t* __restrict__ tmap, float S,
                                              int bi, int bj, int slice, float* smem) {
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY, NT = Geo::NT;
  cohesion_tile_checks<Geo>();
  const int64_t X0 = static_cast<int64_t>(bi) * Geo::B;
  const int64_t Z0 = static_cast<int64_t>(bj) * Geo::B + static_cast<int64_t>(slice) * Geo::BY;
  const int tx = threadIdx.x % Geo::TPX, tz = threadIdx.x / Geo::TPX;
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(D) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(R) % 16) == 0;

  float* Ad = smem;                                   // [kPipe][BK][BX]  d_xy  (row y, column x)
  float* Ar = Ad + kPipe * Geo::SX;                   // [kPipe][BK][BX]  r_xy
  float* Bd = Ar + kPipe * Geo::SX;                   // [kPipe][BK][BY]  d_zy
  float* Br = Bd + kPipe * Geo::SY;                   // [kPipe][BK][BY]  r_zy

  const int64_t nstages = (n + BK - 1) / BK;
  auto stage = [&](int buf, int64_t y0) {
    stage_rows<Geo::BX, NT, BK>(Ad + buf * Geo::SX, D, n, y0, X0, vec);
    stage_rows<Geo::BX, NT, BK>(Ar + buf * Geo::SX, R, n, y0, X0, vec);
    stage_rows<Geo::BY, NT, BK>(Bd + buf * Geo::SY, D, n, y0, Z0, vec);
    stage_rows<Geo::BY, NT, BK>(Br + buf * Geo::SY, R, n, y0, Z0, vec);
  };
#pragma unroll
  for (int p = 0; p < kPipe - 1; ++p) {
    if (p < nstages) stage(p, p * BK);
    cp_async_commit();
  }

  const TieCursor<BK> ties(tmap, n, X0, Z0);
  uint32_t tie_next = ties.tied(0);

  float cv[TX][TY];
  uint64_t sacc[TX][TY], hacc[TX][TY];
  cohesion_init<Geo>(D, n, X0, Z0, tx, tz, S, cv, sacc, hacc);

  for (int64_t st = 0; st < nstages; ++st) {
    const int buf = static_cast<int>(st % kPipe);
    const uint32_t tie_now = tie_next;
    tie_next = ties.tied(st + 1);  // loaded a stage ahead of its use
    cp_async_wait<kPipe - 2>();    // stage st has landed (later ones may be in flight)
    __syncthreads();               // ... for every thread, and stage st-1's buffer is free
    if (st + kPipe - 1 < nstages) stage(static_cast<int>((st + kPipe - 1) % kPipe), (st + kPipe - 1) * BK);
    cp_async_commit();  // possibly empty: keeps one group per stage
    const float* ad = Ad + buf * Geo::SX;
    const float* ar = Ar + buf * Geo::SX;
    const float* bd = Bd + buf * Geo::SY;
    const float* br = Br + buf * Geo::SY;
    if (tie_now)
      cohesion_stage<Geo, MODE, false>(ad, ar, bd, br, tx, tz, S, cv, sacc, hacc);
    else
      cohesion_stage<Geo, MODE, true>(ad, ar, bd, br, tx, tz, S, cv, sacc, hacc);
  }
  cohesion_finish<Geo, MODE>(C, n, X0, Z0, tx, tz, bi != bj, vec, sacc, hacc);
}

// ---------------------------------------------------------------------------
// TMA-staged tile (64 x 64, see tma_ring.cuh): the D and R panels of X and Z
// come from the tensor maps tmD and tmR of the n x n matrices (which may be
// row-padded copies); the per-pair constants are read from D (row pitch n)
// and C is written with row pitch n.  No per-thread copy arithmetic remains
// in the loop, and the kernel fits two CTAs per SM (four warps per
// scheduler).

// tie-map words of one block pair for any n <= 2^20
constexpr int kTieWordsMax = ((1 << 20) / kTieGroupCoarse + 31) / 32;
static_assert((kTieFineMaxN / kTieGroupFine + 31) / 32 <= kTieWordsMax, "fine maps fit too");

template <class Geo>
struct CohesionTmaSmem {
  using Ring = TmaRing<4, Geo::BK>;
  // ring (128-byte aligned), then the tile's tie-map words
  static constexpr int bytes(int64_t n) { return Ring::BYTES + 128 + 4 * static_cast<int>(tie_map_dims(n).wpp); }
  static constexpr int MAX_BYTES = Ring::BYTES + 128 + 4 * kTieWordsMax;
};

// Row sums of one finished 64 x 64 tile for the fused local depth (Sec. 2,
// eq. (LD): l_x is the sum of row x of C).  P is [T][n] FP64 with T = the
// number of 64-wide column blocks: P[bj * n + x] receives the sum of c_xz
// over the tile's columns z (block bj) for each row x of X, and, off the
// diagonal, P[bi * n + z] that of c_zx over block bi for each row z of Z.
// Every entry of P is written by exactly one tile.  The order is fixed: a
// thread's four columns (cohesion_finish), then the 16 column groups of
// four in order.  `sh` holds 2 x 16 x 64 doubles of shared memory; all NT
// threads call this together.
template <class Geo>
__device__ __forceinline__ void depth_partials(double* __restrict__ P, int64_t n, int bi, int bj, int tx, int tz,
                                               bool active, bool mirror, const double (&rs)[Geo::TX],
                                               const double (&ms)[Geo::TY], double* sh) {
  static_assert(Geo::TX == 4 && Geo::TY == 4 && Geo::GX == 1 && Geo::GY == 1, "4 x 4 pairs per thread");
  // SX[g][r]: columns 4g..4g+3 of row r of X.  On the diagonal the rows of
  // Z are those of X, and block (a, b) with a < b writes row part (b, 4a+i)
  // and mirror part (a, 4b+j): every (group, row) slot exactly once.
  double* SX = sh;
  double* SZ = bi == bj ? sh : sh + 16 * 64;
  for (int k = threadIdx.x; k < 2 * 16 * 64; k += Geo::NT) sh[k] = 0.0;  // groups past n stay 0
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < 4; ++i) SX[tz * 64 + 4 * tx + i] = rs[i];
    if (mirror) {
#pragma unroll
      for (int j = 0; j < 4; ++j) SZ[tx * 64 + 4 * tz + j] = ms[j];
    }
  }
  __syncthreads();
  const int t = static_cast<int>(threadIdx.x);
  const bool zpart = t >= 64;
  if (t < 128 && !(zpart && bi == bj)) {
    const double* S = zpart ? SZ : SX;
    const int r = t & 63;
    const int64_t row = int64_t(zpart ? bj : bi) * 64 + r;
    if (row < n) {
      double sum = 0.0;
#pragma unroll
      for (int g = 0; g < 16; ++g) sum += S[g * 64 + r];
      P[int64_t(zpart ? bi : bj) * n + row] = sum;
    }
  }
}

// Returns false when a wait ran out of time; the CTA then stops early and
// its outputs are unspecified.  `tie_words` holds tie_map_dims(n).wpp words
// of shared memory.  With `skip_diag` a diagonal tile leaves out its 4 x 4
// blocks on the diagonal (the pairs inside the groups of four points), for
// cohesion_group below to compute: four warps instead of five.  With DEPTH
// (and no `skip_diag`) the tile also writes its row sums to P
// (depth_partials), reusing the ring's panels once the last stage is done.
// With PACKED the stages run cohesion_stage_packed, which needs tmR to map
// an R in the paired column order (the result is the same).
template <class Geo, int MODE, bool DEPTH = false, bool PACKED = false>
__device__ __forceinline__ bool cohesion_tile_tma(const CUtensorMap* tmD, const CUtensorMap* tmR,
                                                  const float* __restrict__ D, int64_t n, float* __restrict__ C,
                                                  const uint32_t* __restrict__ tmap, float S, int bi, int bj,
                                                  bool vec, TmaRing<4, Geo::BK>& ring, uint32_t* tie_words,
                                                  bool skip_diag = false, double* __restrict__ P = nullptr) {
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY, NT = Geo::NT;
  static_assert(Geo::BX == 64 && Geo::BY == 64 && Geo::TPX == 16 && Geo::TPY == 16 && Geo::GX == 1 &&
                    Geo::GY == 1 && Geo::CW == 4,
                "TMA tiles are 64 x 64 with 4 x 4 pairs per thread");
  cohesion_tile_checks<Geo>();
  int tx, tz;
  const bool active = tile_block_64(bi, bj, n, threadIdx.x, &tx, &tz, skip_diag);
  const int64_t X0 = int64_t(bi) * 64;
  const int nstages = static_cast<int>((n + BK - 1) / BK);

  if (threadIdx.x == 0) ring.init();
  // the tile's tie-map row (all ones when there is no map or a block is dirty)
  const int gshift = tie_map_dims(n).gshift;
  {
    const TieMapDims dm = tie_map_dims(n);
    const int64_t bx = bi, bz = bj;  // 64-wide tiles are the map's blocks
    const bool all_long = tmap == nullptr || __ldg(tmap + dm.nb * dm.nb * dm.wpp + bx) != 0u ||
                          __ldg(tmap + dm.nb * dm.nb * dm.wpp + bz) != 0u;
    const uint32_t* row = tmap + (bx * dm.nb + bz) * dm.wpp;
    for (int w = threadIdx.x; w < dm.wpp; w += NT) tie_words[w] = all_long ? ~0u : __ldg(row + w);
  }
  __syncthreads();

  float cv[TX][TY];
  uint64_t sacc[TX][TY], hacc[TX][TY];
  cohesion_init<Geo>(D, n, X0, int64_t(bj) * 64, tx, tz, S, cv, sacc, hacc);
  uint64_t sx[4][2], sz[4][2], hx[4][2], hz[4][2];  // the packed partials (PACKED only)
  if constexpr (PACKED) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        sx[i][jj] = sz[i][jj] = sacc[i][jj];
        hx[i][jj] = hz[i][jj] = hacc[i][jj];
      }
  }

  // y [kb, ke) of the stage in buffer buf, in one form, in chunks of U y
  auto run = [&](auto short_form, auto unroll, int buf, int kb, int ke) {
    constexpr bool SHORT = decltype(short_form)::value;
    constexpr int U = decltype(unroll)::value;
    if constexpr (PACKED)
      cohesion_stage_packed<Geo, MODE, SHORT, U>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2),
                                                 ring.panel(buf, 3), tx, tz, S, cv, sx, sz, hx, hz, ke, kb);
    else
      cohesion_stage<Geo, MODE, SHORT, U>(ring.panel(buf, 0), ring.panel(buf, 1), ring.panel(buf, 2),
                                          ring.panel(buf, 3), tx, tz, S, cv, sacc, hacc, ke, kb);
  };
  using Short = std::true_type;
  using Long = std::false_type;
  // a stage with some of its tie groups marked runs chunks of CH y, each in
  // the form its groups need (CH: whole fine groups and whole merge chunks;
  // coarse groups cover a stage, so their stages are never mixed)
  constexpr int CH = kTieGroupFine > kMergeEvery ? kTieGroupFine : kMergeEvery;
  static_assert(BK % CH == 0 && CH % kTieGroupFine == 0, "a stage holds whole chunks");
  static_assert(BK <= kTieGroupCoarse, "a stage lies inside one coarse group (never mixed)");
  const CUtensorMap* const maps[4] = {tmD, tmR, tmD, tmR};
  const int cols[4] = {bi * 64, bi * 64, bj * 64, bj * 64};
  const bool ok = tma_pipeline(
      ring, nstages, [&](int q) { ring.issue(q, maps, cols); },
      [&](int st, int buf) {
        if (!active) return;
        const TieStage ts = tie_stage(st, BK, gshift);
        const uint32_t bits = (tie_words[ts.g >> 5] >> (ts.g & 31)) & ts.mask;
        if (bits == 0u) {
          run(Short(), std::integral_constant<int, Geo::UNR>(), buf, 0, stage_extent<BK, Geo::UNR>(n, st));
        } else if (bits == ts.mask) {
          run(Long(), std::integral_constant<int, Geo::UNR>(), buf, 0, stage_extent<BK, Geo::UNR>(n, st));
        } else {  // fine groups only
          const int ke = stage_extent<BK, CH>(n, st);
          const int gpc = CH >> gshift;  // groups per chunk
          const uint32_t cmask = (1u << gpc) - 1u;
#pragma unroll 1
          for (int c = 0; c * CH < ke; ++c) {
            if ((bits >> (c * gpc)) & cmask)
              run(Long(), std::integral_constant<int, CH>(), buf, c * CH, c * CH + CH);
            else
              run(Short(), std::integral_constant<int, CH>(), buf, c * CH, c * CH + CH);
          }
        }
      });
  __syncthreads();
  if (threadIdx.x == 0) ring.inval();
  if constexpr (PACKED) {
    unpair_partials(sx, sz, sacc);
    unpair_partials(hx, hz, hacc);
  }
  // off the diagonal, or for an above-diagonal block of a diagonal tile,
  // the block's mirror (the zx lanes) is written too
  const bool mirror = tx != tz || bi != bj;
  if constexpr (DEPTH) {
    static_assert(Geo::BK * 64 * 4 * kTmaStages >= 2 * 16 * 64 * 2, "row sums fit in the ring's panels");
    double rs[TX] = {}, ms[TY] = {};
    if (ok && active) cohesion_finish<Geo, MODE, true>(C, n, X0, int64_t(bj) * 64, tx, tz, mirror, vec, sacc, hacc,
                                                       &rs, &ms);
    // every copy has landed and every stage has been read: the panels are free
    if (ok) depth_partials<Geo>(P, n, bi, bj, tx, tz, active, mirror, rs, ms, reinterpret_cast<double*>(ring.panels));
  } else {
    if (ok && active) cohesion_finish<Geo, MODE>(C, n, X0, int64_t(bj) * 64, tx, tz, mirror, vec, sacc, hacc);
  }
  return ok;
}

// ---------------------------------------------------------------------------
// The pairs inside one group of four points x0 .. x0+3 (x0 = 4q), which a
// diagonal TMA tile with `skip_diag` leaves out: one thread per group,
// streaming y straight from global memory (the group's four columns of row
// y are one 16-byte vector).  Only the ten pairs i <= j are formed (pair
// (j, i) repeats pair (i, j) with the two lanes swapped).  Each lane repeats
// the tile's operations on its pair in the same order: the same step in the
// form the tile takes (the tie map's bit of block pair (x0 / 64, x0 / 64)
// per group of 8 y), the fold after the same y, the same final merge.  The
// tile also runs zero-filled y past n; those add +0, and folding the last
// partial into H leaves H + S, and so the merged value, unchanged: stopping
// at the first multiple of 4 past n gives the same bits.

// One y of the ten pairs, then the folds due after it (y mod kMergeEvery == K).
template <int MODE, bool SHORT, int K>
__device__ __forceinline__ void cohesion_group_y(const float4& d, const float4& r, float S, const float (&cv)[10],
                                                 uint64_t (&sacc)[10], uint64_t (&hacc)[10]) {
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int i = group_pair_i(p), j = group_pair_j(p);
    if (SHORT)
      cohesion_step_short(sacc[p], comp4(d, i), comp4(d, j), S, cv[p], comp4(r, i), comp4(r, j));
    else
      cohesion_step(sacc[p], comp4(d, i), comp4(d, j), S, cv[p], comp4(r, i), comp4(r, j));
  }
  if (MODE == PALD_ACCUM_COMPENSATED) {
#pragma unroll
    for (int p = 0; p < 10; ++p)
      if (K == fold_phase(group_pair_i(p), group_pair_j(p))) fast2sum_fold(hacc[p], sacc[p]);
  }
}

// Four consecutive y starting at phase P (y mod kMergeEvery == P).
template <int MODE, bool SHORT, int P>
__device__ __forceinline__ void cohesion_group_4y(const float4 (&d)[4], const float4 (&r)[4], float S,
                                                  const float (&cv)[10], uint64_t (&sacc)[10],
                                                  uint64_t (&hacc)[10]) {
  cohesion_group_y<MODE, SHORT, P + 0>(d[0], r[0], S, cv, sacc, hacc);
  cohesion_group_y<MODE, SHORT, P + 1>(d[1], r[1], S, cv, sacc, hacc);
  cohesion_group_y<MODE, SHORT, P + 2>(d[2], r[2], S, cv, sacc, hacc);
  cohesion_group_y<MODE, SHORT, P + 3>(d[3], r[3], S, cv, sacc, hacc);
}

// Four y from y0 (a multiple of 4), with their phase in the merge chunk.
template <int MODE, bool SHORT>
__device__ __forceinline__ void cohesion_group_step(int64_t y0, const float4 (&d)[4], const float4 (&r)[4], float S,
                                                    const float (&cv)[10], uint64_t (&sacc)[10],
                                                    uint64_t (&hacc)[10]) {
  switch (static_cast<int>(y0 % kMergeEvery) / 4) {
    case 0: cohesion_group_4y<MODE, SHORT, 0>(d, r, S, cv, sacc, hacc); break;
    case 1: cohesion_group_4y<MODE, SHORT, 4 % kMergeEvery>(d, r, S, cv, sacc, hacc); break;
    case 2: cohesion_group_4y<MODE, SHORT, 8 % kMergeEvery>(d, r, S, cv, sacc, hacc); break;
    default: cohesion_group_4y<MODE, SHORT, 12 % kMergeEvery>(d, r, S, cv, sacc, hacc); break;
  }
}

// C of the sixteen pairs of group q.  Dp, Rp: D and R = 1/u with row pitch
// `pitch` (16-byte aligned rows, finite values in the pad columns); C: row
// pitch n (vector stores when `vecC`); tmap: the matrix's tie map (null:
// long form everywhere).
template <int MODE>
__device__ __forceinline__ void cohesion_group(const float* __restrict__ Dp, const float* __restrict__ Rp,
                                               int64_t pitch, int64_t n, int64_t q, float S, float* __restrict__ C,
                                               bool vecC, const uint32_t* __restrict__ tmap) {
  const int64_t x0 = 4 * q;
  float cv[10];
  uint64_t sacc[10], hacc[10];
  {
    float4 row[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) row[i] = group_row(Dp, pitch, n, x0 + i, x0);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      cv[k] = __fmul_rn(-comp4(row[group_pair_i(k)], group_pair_j(k)), S);  // exact: power of two
      sacc[k] = pack2(0.f, 0.f);
      hacc[k] = pack2(kMergeBias, kMergeBias);
    }
  }
  const TieMapDims dm = tie_map_dims(n);
  const int64_t bx = x0 / kTieBlock;
  const bool all_long = tmap == nullptr || __ldg(tmap + dm.nb * dm.nb * dm.wpp + bx) != 0u;
  const uint32_t* trow = tmap + (bx * dm.nb + bx) * dm.wpp;
  static_assert(kTieGroupFine % 4 == 0 && kTieGroupCoarse % 4 == 0, "tie groups hold whole 4-y steps");

  // the tile stops after a whole merge chunk; folding the last partial
  // early or late does not change H + S
  const int64_t n4 = (n + 3) / 4 * 4;
  float4 d[4], r[4], dn[4], rn[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d[k] = group_row(Dp, pitch, n, k, x0);
    r[k] = group_row(Rp, pitch, n, k, x0);
  }
  bool tied = true;
  for (int64_t y0 = 0; y0 < n4; y0 += 4) {
    if ((y0 & (dm.group - 1)) == 0) {
      const int64_t g = y0 >> dm.gshift;
      tied = all_long || ((__ldg(trow + (g >> 5)) >> (g & 31)) & 1u);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // the next four rows, loaded while these are used
      dn[k] = group_row(Dp, pitch, n, y0 + 4 + k, x0);
      rn[k] = group_row(Rp, pitch, n, y0 + 4 + k, x0);
    }
    if (tied)
      cohesion_group_step<MODE, false>(y0, d, r, S, cv, sacc, hacc);
    else
      cohesion_group_step<MODE, true>(y0, d, r, S, cv, sacc, hacc);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      d[k] = dn[k];
      r[k] = rn[k];
    }
  }
  float ih, il;
  inverse_pair(n - 1, ih, il);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = i <= j ? (i == 0 ? j : (i == 1 ? j + 3 : (i == 2 ? j + 5 : 9)))
                           : (j == 0 ? i : (j == 1 ? i + 3 : (j == 2 ? i + 5 : 9)));
      v[j] = cohesion_value<MODE>(hacc[p], sacc[p], i > j, ih, il);
    }
    storew<4>(C, n, x0 + i, x0, v, vecC);
  }
}

// R[row][col] = 1/u (correctly rounded FP32), 0 on the diagonal and where
// u <= 0, for one row of an n x n matrix; U has row pitch n, R row pitch
// `rp` (a multiple of 4 when `vec`).  The CTA's threads share the row.
// With `paired` (n % 4 == 0) the columns of each group of four are stored
// in the order 0, 2, 1, 3: the layout the packed pass-2 stage reads.
__device__ __forceinline__ void reciprocal_rows(const int32_t* __restrict__ U, int64_t n, float* __restrict__ R,
                                                int64_t rp, int64_t row, bool vec, bool paired = false) {
  const int32_t* u = U + row * n;
  float* r = R + row * rp;
  if (vec) {
    const int64_t n4 = n / 4;
    for (int64_t k = threadIdx.x; k < n4; k += blockDim.x) {
      const int4 q = __ldg(reinterpret_cast<const int4*>(u) + k);
      const int64_t c = 4 * k;
      float4 o;
      o.x = (q.x <= 0 || c + 0 == row) ? 0.f : __frcp_rn(static_cast<float>(q.x));
      o.y = (q.y <= 0 || c + 1 == row) ? 0.f : __frcp_rn(static_cast<float>(q.y));
      o.z = (q.z <= 0 || c + 2 == row) ? 0.f : __frcp_rn(static_cast<float>(q.z));
      o.w = (q.w <= 0 || c + 3 == row) ? 0.f : __frcp_rn(static_cast<float>(q.w));
      if (paired) {
        const float t = o.y;
        o.y = o.z;
        o.z = t;
      }
      reinterpret_cast<float4*>(r)[k] = o;
    }
  } else {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      const int32_t q = __ldg(u + c);
      const int64_t m = c & 3;
      const int64_t to = paired && (m == 1 || m == 2) ? (c ^ 3) : c;  // 1 <-> 2 within the group
      r[to] = (q <= 0 || c == row) ? 0.f : __frcp_rn(static_cast<float>(q));
    }
  }
}

}  // namespace pald
