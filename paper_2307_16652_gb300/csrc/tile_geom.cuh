// Tile geometry shared by both passes.
//
// A pass computes an n x n output that is split into square "super-tiles"
// of edge B.  Only super-tiles (bi, bj) with bi <= bj are launched; an
// off-diagonal super-tile also writes its mirror image.  A super-tile may be
// cut into H column slices (H = 1 or 2), one CTA each, so that the CTA tile
// is B x (B/H).
//
// Inside a CTA tile each thread owns TX = 4*GX rows and TY = CW*GY columns
// (CW = 4 or 2): row group g covers rows g*(BX/GX) + 4*tx + {0..3}, column
// group g covers columns g*(BY/GY) + CW*ty + {0..CW-1}.  Every shared-memory
// operand read is then one 16- or 8-byte vector, the reads of a warp are
// free of bank conflicts, and global stores of the tile (CW-wide) and of its
// mirror (4-wide) are vectors too.
#pragma once

#include "pald_internal.cuh"

namespace pald {

template <int B_, int H_, int GX_, int GY_, int CW_, int BK_, int UNR_ = BK_>
struct TileGeom {
  static constexpr int B = B_;            // super-tile edge
  static constexpr int H = H_;            // column slices per super-tile
  static constexpr int BX = B;            // CTA tile rows
  static constexpr int BY = B / H;        // CTA tile columns
  static constexpr int GX = GX_, GY = GY_;
  static constexpr int CW = CW_;          // column vector width (4 or 2)
  static constexpr int TX = 4 * GX, TY = CW * GY;
  static constexpr int TPX = BX / TX;     // threads along rows
  static constexpr int TPY = BY / TY;     // threads along columns
  static constexpr int NT = TPX * TPY;
  static constexpr int BK = BK_;          // streamed index per pipeline stage
  static constexpr int UNR = UNR_;        // unroll factor of the streamed loop (a divisor of BK)
  static constexpr int SX = BK * BX;      // floats of one row-side operand stage
  static constexpr int SY = BK * BY;      // floats of one column-side operand stage
  static_assert(BX % TX == 0 && BY % TY == 0, "tile must divide into thread tiles");
  static_assert((BX / GX) % 4 == 0 && (BY / GY) % CW == 0, "groups must be vector aligned");
  static_assert(CW == 4 || CW == 2, "column vectors are 4 or 2 wide");
  static_assert(BK % 4 == 0, "stage depth must be a multiple of 4");
  static_assert(BK % UNR == 0 && UNR % 4 == 0, "unroll must divide the stage and keep 4-y phases");

  // global row / column of row i and column j of thread (tx, ty)
  __device__ static __forceinline__ int row_off(int tx, int i) { return (i / 4) * (BX / GX) + 4 * tx + (i % 4); }
  __device__ static __forceinline__ int col_off(int ty, int j) { return (j / CW) * (BY / GY) + CW * ty + (j % CW); }
};

// Launch index -> (bi, bj, slice), bi <= bj.  The upper triangle of
// super-tiles is walked in strips of kStrip block-rows: strip k first covers
// its own triangle (columns k*S .. k*S+S-1), then the columns to its right,
// S tiles per column.  CTAs that run together therefore touch about
// kStrip + (resident CTAs / kStrip) distinct row panels instead of one panel
// per CTA, and the panels they stream stay in L2 for each other.
constexpr int kStrip = 12;

__host__ __device__ __forceinline__ void decode_tile(int64_t t, int64_t T, int H, int* bi, int* bj, int* slice) {
  int64_t st = t / H;
  *slice = static_cast<int>(t - st * H);
  const int64_t S = kStrip;
  int64_t k0 = 0;
  for (;;) {
    const int64_t h = (T - k0) < S ? (T - k0) : S;  // rows in this strip
    const int64_t tri = h * (h + 1) / 2;            // its own triangle
    const int64_t total = tri + (T - k0 - h) * h;   // plus the columns to the right
    if (st < total) {
      if (st < tri) {  // column c of the triangle holds c + 1 tiles
        int64_t c = static_cast<int64_t>((sqrt(8.0 * static_cast<double>(st) + 1.0) - 1.0) / 2.0);
        while (c * (c + 1) / 2 > st) --c;
        while ((c + 1) * (c + 2) / 2 <= st) ++c;
        *bj = static_cast<int>(k0 + c);
        *bi = static_cast<int>(k0 + (st - c * (c + 1) / 2));
      } else {
        const int64_t r = st - tri;
        *bj = static_cast<int>(k0 + h + r / h);
        *bi = static_cast<int>(k0 + r % h);
      }
      return;
    }
    st -= total;
    k0 += h;
  }
}

// Thread placement in a 64 x 64 tile of 16 x 16 thread blocks (4 x 4 pairs
// each) of an n x n matrix.  A full off-diagonal tile gives thread t block
// (t % 16, t / 16).  Otherwise only the blocks that hold pairs of the matrix
// are handed out, to threads 0, 1, ... in order, so that whole warps drop
// out: on a ragged edge tile the blocks inside the matrix, and on a diagonal
// tile (X == Z) only the blocks (a, b) with a <= b, since a block below the
// diagonal repeats, with rows and columns swapped, what its mirror above
// computes.  With `skip_diag` a diagonal tile also leaves out its blocks
// (a, a): 120 blocks instead of 136, four warps instead of five (their
// pairs go to the other four warps, GroupPairs in focus_core.cuh).
// Threads without a block only take part in the barriers.  Returns whether
// thread t owns a block.
__device__ __forceinline__ bool tile_block_64(int bi, int bj, int64_t n, int t, int* a, int* b,
                                                       bool skip_diag = false) {
  const int64_t rx = n - int64_t(bi) * 64, rz = n - int64_t(bj) * 64;
  const int ax = rx >= 64 ? 16 : static_cast<int>((rx + 3) / 4);  // blocks holding rows of the matrix
  const int az = rz >= 64 ? 16 : static_cast<int>((rz + 3) / 4);
  *a = 0;
  *b = 0;  // placement of a thread without a block (its setup work is harmless)
  if (bi != bj) {
    if (ax == 16 && az == 16) {
      *a = t % 16;
      *b = t / 16;
      return true;
    }
    if (t >= ax * az) return false;
    *a = t % ax;
    *b = t / ax;
    return true;
  }
  // upper triangle of the ax x ax blocks, row by row; row r holds blocks
  // (r, r + d) .. (r, ax - 1)
  const int d = skip_diag ? 1 : 0;
  int r = 0;
  while (r < ax && t >= ax - r - d) {
    t -= ax - r - d;
    ++r;
  }
  if (r == ax) return false;
  *a = r;
  *b = r + d + t;
  return true;
}

}  // namespace pald
