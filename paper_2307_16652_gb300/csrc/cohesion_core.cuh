// Pass 2 core: cohesion of one BM x BM tile pair (X, Z), X <= Z.
//
// For an output pair (x, z) and every third point y the paper's cohesion
// (Sec. 2 eq. (cohesion), written out as eq. (fxz)) with the half-credit tie
// split of Sec. 5 contributes
//     to c_xz:  [d_xz <= min(d_xy, d_zy)] * w(d_xz, d_zy) * r_xy
//     to c_zx:  [d_xz <= min(d_xy, d_zy)] * w(d_xz, d_xy) * r_zy
// with r = 1/u and w(b, a) = 0, 1/2, 1 for a < b, a == b, a > b.  (z in U_xy
// together with d_zx <= d_zy is the same as d_xz <= min(d_xy, d_zy).)  The
// diagonal of R is set to 0, which removes the excluded y == x term exactly,
// duplicate points included.
//
// Per (x, z, y) the inner loop issues six instructions, all of them exact
// FP32 decisions on the input values:
//     m  = min(d_xy, d_zy)                FMNMX        (ALU pipe)
//     p  = m >= b                         FSETP        (ALU pipe)
//     v2 = sat(d_zy * s + c)              FFMA.SAT     (FMA pipe)
//     v1 = sat(d_xy * s + c)              FFMA.SAT     (FMA pipe)
//     @p S_xz += v2 * r_xy                FFMA         (FMA pipe)
//     @p S_zx += v1 * r_zy                FFMA         (FMA pipe)
// where (s, c) are per-pair constants built from b = d_xz so that
// sat(a*s + c) = w(b, a) exactly: s = 2^(22-e) (2^(23-e) if b is a power of
// two), c = 1/2 - b*s.  Then a == b gives exactly 1/2, and any other float a
// is at least half a unit away from b*s after scaling, so saturation maps it
// to 0 or 1.  b = 0 uses s = 2^127, c = 1/2 (inputs have no positive entry
// below 2^-100).
//
// Accumulation (PALD_ACCUM_COMPENSATED): S holds an FP32 partial over one
// 16-y stage; after each stage it is folded into the running FP32 sum H with
// an error-free TwoSum, and the exact rounding error becomes the start of the
// next partial, so nothing is lost between stages.  At the end H + S is
// formed in FP64, multiplied by 1/(n-1) in FP64 and rounded once to FP32.
// PALD_ACCUM_PLAIN keeps one FP32 running sum (the precision baseline).
#pragma once

#include "focus_core.cuh"

namespace pald {

template <int BM, int G>
struct CohesionGeom {
  static constexpr int BK = 16;                // y per stage (= compensation chunk)
  static constexpr int TPD = BM / (4 * G);
  static constexpr int NT = TPD * TPD;
  static constexpr int TM = 4 * G;
  static constexpr int STAGE = BK * BM;        // floats per operand per stage
  static constexpr int SMEM_FLOATS = 2 * 4 * STAGE;  // two stages of D_X, R_X, D_Z, R_Z
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

// One (x, z, y) step; see the header comment.
__device__ __forceinline__ void cohesion_step(float& sxz, float& szx, float a1, float a2, float b, float s, float c,
                                              float r1, float r2) {
  asm("{\n\t.reg .pred p;\n\t.reg .f32 m, v1, v2;\n\t"
      "min.f32 m, %2, %3;\n\t"
      "setp.ge.f32 p, m, %4;\n\t"
      "fma.rn.sat.f32 v2, %3, %5, %6;\n\t"
      "fma.rn.sat.f32 v1, %2, %5, %6;\n\t"
      "@p fma.rn.f32 %0, v2, %7, %0;\n\t"
      "@p fma.rn.f32 %1, v1, %8, %1;\n\t}"
      : "+f"(sxz), "+f"(szx)
      : "f"(a1), "f"(a2), "f"(b), "f"(s), "f"(c), "f"(r1), "f"(r2));
}

// Error-free TwoSum: h + e == old h + old e exactly; e carries the error.
__device__ __forceinline__ void two_sum_fold(float& h, float& e) {
  const float s = __fadd_rn(h, e);
  const float bb = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(e, bb));
  h = s;
  e = err;
}

// r = 1/u for the staged u values of this stage; 0 on the diagonal (y == x)
// and outside the matrix (where u was zero-filled).
template <int BM, int NT, int BK>
__device__ __forceinline__ void reciprocal_stage(float* buf, int64_t y0, int64_t c0) {
  uint32_t* ub = reinterpret_cast<uint32_t*>(buf);
#pragma unroll
  for (int k = threadIdx.x; k < BK * BM; k += NT) {
    const int r = k / BM, cc = k % BM;
    const int u = static_cast<int>(ub[k]);
    const bool zero = (u <= 0) || (y0 + r == c0 + cc);
    buf[k] = zero ? 0.f : __frcp_rn(static_cast<float>(u));
  }
}

template <int BM, int G, int MODE>
__device__ __forceinline__ void cohesion_tile(const float* __restrict__ D, const int32_t* __restrict__ U, int64_t n,
                                              float* __restrict__ C, int bi, int bj, float* smem) {
  using Geo = CohesionGeom<BM, G>;
  constexpr int BK = Geo::BK, TM = Geo::TM, TPD = Geo::TPD, NT = Geo::NT;
  const int64_t X0 = static_cast<int64_t>(bi) * BM, Z0 = static_cast<int64_t>(bj) * BM;
  const int tx = threadIdx.x % TPD, tz = threadIdx.x / TPD;
  const bool vec = (n % 4) == 0 && (reinterpret_cast<uintptr_t>(D) % 16) == 0 &&
                   (reinterpret_cast<uintptr_t>(U) % 16) == 0;

  float* Ad = smem;                   // [2][BK][BM]  d_xy  (row y, column x)
  float* Ar = smem + 2 * Geo::STAGE;  // [2][BK][BM]  u_xy -> r_xy
  float* Bd = smem + 4 * Geo::STAGE;  // [2][BK][BM]  d_zy
  float* Br = smem + 6 * Geo::STAGE;  // [2][BK][BM]  u_zy -> r_zy
  const float* Uf = reinterpret_cast<const float*>(U);

  const int64_t nstages = (n + BK - 1) / BK;
  stage_rows<BM, NT, BK>(Ad, D, n, 0, X0, vec);
  stage_rows<BM, NT, BK>(Ar, Uf, n, 0, X0, vec);
  stage_rows<BM, NT, BK>(Bd, D, n, 0, Z0, vec);
  stage_rows<BM, NT, BK>(Br, Uf, n, 0, Z0, vec);
  cp_async_commit();

  float bv[TM][TM], sv[TM][TM], cv[TM][TM];
  float sxz[TM][TM], szx[TM][TM], hxz[TM][TM], hzx[TM][TM];
#pragma unroll
  for (int gi = 0; gi < G; ++gi)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t x = X0 + gi * (BM / G) + 4 * tx + i;
#pragma unroll
      for (int gj = 0; gj < G; ++gj) {
        const float4 t = load4(D, n, x, Z0 + gj * (BM / G) + 4 * tz, vec);
        const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = gi * 4 + i, q = gj * 4 + j;
          bv[r][q] = tv[j];
          tie_constants(tv[j], sv[r][q], cv[r][q]);
        }
      }
    }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) sxz[i][j] = szx[i][j] = hxz[i][j] = hzx[i][j] = 0.f;

  for (int64_t st = 0; st < nstages; ++st) {
    const int buf = static_cast<int>(st & 1);
    if (st + 1 < nstages) {
      const int nb = (buf ^ 1) * Geo::STAGE;
      stage_rows<BM, NT, BK>(Ad + nb, D, n, (st + 1) * BK, X0, vec);
      stage_rows<BM, NT, BK>(Ar + nb, Uf, n, (st + 1) * BK, X0, vec);
      stage_rows<BM, NT, BK>(Bd + nb, D, n, (st + 1) * BK, Z0, vec);
      stage_rows<BM, NT, BK>(Br + nb, Uf, n, (st + 1) * BK, Z0, vec);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    reciprocal_stage<BM, NT, BK>(Ar + buf * Geo::STAGE, st * BK, X0);
    reciprocal_stage<BM, NT, BK>(Br + buf * Geo::STAGE, st * BK, Z0);
    __syncthreads();
    const float* ad = Ad + buf * Geo::STAGE;
    const float* ar = Ar + buf * Geo::STAGE;
    const float* bd = Bd + buf * Geo::STAGE;
    const float* br = Br + buf * Geo::STAGE;
#pragma unroll 2
    for (int kk = 0; kk < BK; ++kk) {
      float a1[TM], r1[TM], a2[TM], r2[TM];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int ox = kk * BM + g * (BM / G) + 4 * tx, oz = kk * BM + g * (BM / G) + 4 * tz;
        const float4 va = *reinterpret_cast<const float4*>(ad + ox);
        const float4 vr = *reinterpret_cast<const float4*>(ar + ox);
        const float4 vb = *reinterpret_cast<const float4*>(bd + oz);
        const float4 vs = *reinterpret_cast<const float4*>(br + oz);
        a1[4 * g + 0] = va.x; a1[4 * g + 1] = va.y; a1[4 * g + 2] = va.z; a1[4 * g + 3] = va.w;
        r1[4 * g + 0] = vr.x; r1[4 * g + 1] = vr.y; r1[4 * g + 2] = vr.z; r1[4 * g + 3] = vr.w;
        a2[4 * g + 0] = vb.x; a2[4 * g + 1] = vb.y; a2[4 * g + 2] = vb.z; a2[4 * g + 3] = vb.w;
        r2[4 * g + 0] = vs.x; r2[4 * g + 1] = vs.y; r2[4 * g + 2] = vs.z; r2[4 * g + 3] = vs.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j)
          cohesion_step(sxz[i][j], szx[i][j], a1[i], a2[j], bv[i][j], sv[i][j], cv[i][j], r1[i], r2[j]);
    }
    if (MODE == PALD_ACCUM_COMPENSATED) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) {
          two_sum_fold(hxz[i][j], sxz[i][j]);
          two_sum_fold(hzx[i][j], szx[i][j]);
        }
    }
    __syncthreads();
  }

  const double inv = 1.0 / static_cast<double>(n - 1);
  auto finish = [&](float h, float s) -> float {
    if (MODE == PALD_ACCUM_COMPENSATED) return static_cast<float>((static_cast<double>(h) + static_cast<double>(s)) * inv);
    return static_cast<float>(static_cast<double>(s) * inv);
  };
#pragma unroll
  for (int gi = 0; gi < G; ++gi)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t x = X0 + gi * (BM / G) + 4 * tx + i;
      const int r = gi * 4 + i;
      if (x >= n) continue;
#pragma unroll
      for (int gj = 0; gj < G; ++gj) {
        const int q = gj * 4;
        const int64_t z = Z0 + gj * (BM / G) + 4 * tz;
        float4 v = make_float4(finish(hxz[r][q], sxz[r][q]), finish(hxz[r][q + 1], sxz[r][q + 1]),
                               finish(hxz[r][q + 2], sxz[r][q + 2]), finish(hxz[r][q + 3], sxz[r][q + 3]));
        float* p = C + x * n + z;
        if (vec && z + 3 < n) {
          *reinterpret_cast<float4*>(p) = v;
        } else {
          if (z + 0 < n) p[0] = v.x;
          if (z + 1 < n) p[1] = v.y;
          if (z + 2 < n) p[2] = v.z;
          if (z + 3 < n) p[3] = v.w;
        }
      }
    }
  if (bi != bj) {
#pragma unroll
    for (int gj = 0; gj < G; ++gj)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t z = Z0 + gj * (BM / G) + 4 * tz + j;
        const int q = gj * 4 + j;
        if (z >= n) continue;
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
          const int r = gi * 4;
          const int64_t x = X0 + gi * (BM / G) + 4 * tx;
          float4 v = make_float4(finish(hzx[r][q], szx[r][q]), finish(hzx[r + 1][q], szx[r + 1][q]),
                                 finish(hzx[r + 2][q], szx[r + 2][q]), finish(hzx[r + 3][q], szx[r + 3][q]));
          float* p = C + z * n + x;
          if (vec && x + 3 < n) {
            *reinterpret_cast<float4*>(p) = v;
          } else {
            if (x + 0 < n) p[0] = v.x;
            if (x + 1 < n) p[1] = v.y;
            if (x + 2 < n) p[2] = v.z;
            if (x + 3 < n) p[3] = v.w;
          }
        }
      }
  }
}

}  // namespace pald
