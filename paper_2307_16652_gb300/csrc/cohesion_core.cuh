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
// Per (x, z, y) the inner loop issues six instructions, all of them exact
// FP32 decisions on the input values:
//     v2 = sat(d_zy * s + c) = w(b, d_zy)          FFMA.SAT     (FMA pipe)
//     v1 = sat(d_xy * s + c) = w(b, d_xy)          FFMA.SAT     (FMA pipe)
//     m  = min(v1, v2)                             FMNMX        (ALU pipe)
//     p  = m > 0   (d_xz <= min(d_xy, d_zy))       FSETP        (ALU pipe)
//     @p S_xz += v2 * r_xy                         FFMA         (FMA pipe)
//     @p S_zx += v1 * r_zy                         FFMA         (FMA pipe)
// (w(b, a) is 0 exactly when a < b, so the focus/support test needs no
// separate copy of b.)
// where (s, c) are per-pair constants built from b = d_xz so that
// sat(a*s + c) = w(b, a) exactly: s = 2^(22-e) (2^(23-e) if b is a power of
// two), c = 1/2 - b*s.  Then a == b gives exactly 1/2, and any other float a
// is at least half a unit away from b*s after scaling, so saturation maps it
// to 0 or 1.  b = 0 uses s = 2^127, c = 1/2 (inputs have no positive entry
// below 2^-100).
//
// Accumulation (PALD_ACCUM_COMPENSATED): the pair {S_xz, S_zx} is an FP32
// partial over 4 consecutive y.  Every 4 y it is folded into the running sums
// {H_xz, H_zx}, which start at the bias B = 4: a partial never exceeds
// 4 * 1/2 plus the carried error, so |H| >= |S| always holds and Fast2Sum
// (three adds, done as packed f32x2 ops on both accumulators at once) is
// error-free.  Its exact error becomes the start of the next partial, so
// nothing is lost between chunks.  At the end H - B + S is formed in FP64,
// multiplied by 1/(n-1) in FP64 and rounded once to FP32.
// PALD_ACCUM_PLAIN keeps one FP32 running sum (the precision baseline).
#pragma once

#include "focus_core.cuh"

namespace pald {

constexpr int kMergeEvery = 4;      // y per FP32 partial
constexpr float kMergeBias = 4.0f;  // >= kMergeEvery * 1/2 + carried error

template <class Geo>
struct CohesionSmem {
  static constexpr int FLOATS = kPipe * 2 * (Geo::SX + Geo::SY);  // kPipe stages of D_X, R_X, D_Z, R_Z
};

__device__ __forceinline__ void tie_constants(float b, float& s, float& c) {
  const uint32_t bits = __float_as_uint(b);
  if (bits == 0u) {
    s = exp2i(127);
    c = 0.5f;
    return;
  }
  const int e = exponent_of(b);
  const bool pow2 = (bits & 0x7fffffu) == 0u;
  int k = (pow2 ? 23 : 22) - e;
  k = k > 127 ? 127 : (k < -126 ? -126 : k);
  s = exp2i(k);
  c = __fsub_rn(0.5f, __fmul_rn(b, s));  // b*s is exact (power-of-two scaling)
}

// One (x, z, y) step on the packed partial {S_xz, S_zx}; see the header.
__device__ __forceinline__ void cohesion_step(uint64_t& sacc, float a1, float a2, float s, float c, float r1,
                                              float r2) {
  asm("{\n\t.reg .pred p;\n\t.reg .f32 m, v1, v2, sx, sz;\n\t"
      "mov.b64 {sx, sz}, %0;\n\t"
      "fma.rn.sat.f32 v2, %2, %3, %4;\n\t"
      "fma.rn.sat.f32 v1, %1, %3, %4;\n\t"
      "min.f32 m, v1, v2;\n\t"
      "setp.gt.f32 p, m, 0f00000000;\n\t"
      "@p fma.rn.f32 sx, v2, %5, sx;\n\t"
      "@p fma.rn.f32 sz, v1, %6, sz;\n\t"
      "mov.b64 %0, {sx, sz};\n\t}"
      : "+l"(sacc)
      : "f"(a1), "f"(a2), "f"(s), "f"(c), "f"(r1), "f"(r2));
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

// Computes C[X, Z] (and C[Z, X] off the diagonal) for super-tile (bi, bj),
// column slice `slice`.  `smem` holds CohesionSmem<Geo>::FLOATS floats.
// Must be called by all Geo::NT threads.
template <class Geo, int MODE>
__device__ __forceinline__ void cohesion_tile(const float* __restrict__ D, const float* __restrict__ R, int64_t n,
                                              float* __restrict__ C, int bi, int bj, int slice, float* smem) {
  constexpr int BK = Geo::BK, TX = Geo::TX, TY = Geo::TY, NT = Geo::NT;
  static_assert(BK % kMergeEvery == 0, "stages must hold whole merge chunks");
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

  float sv[TX][TY], cv[TX][TY];
  uint64_t sacc[TX][TY], hacc[TX][TY];
#pragma unroll
  for (int i = 0; i < TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int j = 0; j < TY; ++j) {
      const int64_t z = Z0 + Geo::col_off(tz, j);
      tie_constants((x < n && z < n) ? __ldg(D + x * n + z) : 0.f, sv[i][j], cv[i][j]);
    }
  }
  const uint64_t zero2 = pack2(0.f, 0.f);
  const uint64_t bias2 = pack2(kMergeBias, kMergeBias);
#pragma unroll
  for (int i = 0; i < TX; ++i)
#pragma unroll
    for (int j = 0; j < TY; ++j) {
      sacc[i][j] = zero2;
      hacc[i][j] = bias2;
    }

  for (int64_t st = 0; st < nstages; ++st) {
    const int buf = static_cast<int>(st % kPipe);
    cp_async_wait<kPipe - 2>();  // stage st has landed (later ones may be in flight)
    __syncthreads();             // ... for every thread, and stage st-1's buffer is free
    if (st + kPipe - 1 < nstages) stage(static_cast<int>((st + kPipe - 1) % kPipe), (st + kPipe - 1) * BK);
    cp_async_commit();  // possibly empty: keeps one group per stage
    const float* ad = Ad + buf * Geo::SX;
    const float* ar = Ar + buf * Geo::SX;
    const float* bd = Bd + buf * Geo::SY;
    const float* br = Br + buf * Geo::SY;
#pragma unroll Geo::UNR
    for (int kk = 0; kk < BK; ++kk) {
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
      for (int i = 0; i < TX; ++i)
#pragma unroll
        for (int j = 0; j < TY; ++j)
          cohesion_step(sacc[i][j], a1[i], a2[j], sv[i][j], cv[i][j], r1[i], r2[j]);
      if (MODE == PALD_ACCUM_COMPENSATED) {
        // every pair folds at the same y (y mod 4 == 3): the chunking is
        // then the same for every schedule, for both lanes of a pair and
        // for the batched path, so all of them give bit-identical C
        if ((kk % kMergeEvery) == kMergeEvery - 1) {
#pragma unroll
          for (int i = 0; i < TX; ++i)
#pragma unroll
            for (int j = 0; j < TY; ++j) fast2sum_fold(hacc[i][j], sacc[i][j]);
        }
      }
    }
  }

  const double inv = 1.0 / static_cast<double>(n - 1);
  // value of the (xz or zx) lane: compensated (H - B) + S in FP64, or plain S
  auto finish = [&](uint64_t h2, uint64_t s2, bool zx) -> float {
    float hl, hh, sl, sh;
    unpack2(h2, hl, hh);
    unpack2(s2, sl, sh);
    const float h = zx ? hh : hl, s = zx ? sh : sl;
    if (MODE == PALD_ACCUM_COMPENSATED)
      return static_cast<float>(((static_cast<double>(h) - static_cast<double>(kMergeBias)) +
                                 static_cast<double>(s)) * inv);
    return static_cast<float>(static_cast<double>(s) * inv);
  };
#pragma unroll
  for (int i = 0; i < TX; ++i) {
    const int64_t x = X0 + Geo::row_off(tx, i);
#pragma unroll
    for (int gj = 0; gj < Geo::GY; ++gj) {
      float v[Geo::CW];
#pragma unroll
      for (int k = 0; k < Geo::CW; ++k) v[k] = finish(hacc[i][Geo::CW * gj + k], sacc[i][Geo::CW * gj + k], false);
      storew<Geo::CW>(C, n, x, Z0 + Geo::col_off(tz, Geo::CW * gj), v, vec);
    }
  }
  if (bi != bj) {
#pragma unroll
    for (int j = 0; j < TY; ++j) {
      const int64_t z = Z0 + Geo::col_off(tz, j);
#pragma unroll
      for (int gi = 0; gi < Geo::GX; ++gi) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = finish(hacc[4 * gi + k][j], sacc[4 * gi + k][j], true);
        storew<4>(C, n, z, X0 + Geo::row_off(tx, 4 * gi), v, vec);
      }
    }
  }
}

// R[row][col] = 1/u (correctly rounded FP32), 0 on the diagonal and where
// u <= 0; rows [r0, r1) of one n x n matrix, one warp per row stretch.
__device__ __forceinline__ void reciprocal_rows(const int32_t* __restrict__ U, float* __restrict__ R, int64_t n,
                                                int64_t row, bool vec) {
  const int32_t* u = U + row * n;
  float* r = R + row * n;
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
      reinterpret_cast<float4*>(r)[k] = o;
    }
  } else {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      const int32_t q = __ldg(u + c);
      r[c] = (q <= 0 || c == row) ? 0.f : __frcp_rn(static_cast<float>(q));
    }
  }
}

}  // namespace pald
