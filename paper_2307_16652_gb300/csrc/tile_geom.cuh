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

template <int B_, int H_, int GX_, int GY_, int CW_, int BK_>
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
  static constexpr int SX = BK * BX;      // floats of one row-side operand stage
  static constexpr int SY = BK * BY;      // floats of one column-side operand stage
  static_assert(BX % TX == 0 && BY % TY == 0, "tile must divide into thread tiles");
  static_assert((BX / GX) % 4 == 0 && (BY / GY) % CW == 0, "groups must be vector aligned");
  static_assert(CW == 4 || CW == 2, "column vectors are 4 or 2 wide");
  static_assert(BK % 4 == 0, "stage depth must be a multiple of 4");

  // global row / column of row i and column j of thread (tx, ty)
  __device__ static __forceinline__ int row_off(int tx, int i) { return (i / 4) * (BX / GX) + 4 * tx + (i % 4); }
  __device__ static __forceinline__ int col_off(int ty, int j) { return (j / CW) * (BY / GY) + CW * ty + (j % CW); }
};

// Launch index -> (bi, bj, slice).  Super-tiles of one block-row are
// consecutive so that CTAs running together share the row panel in L2.
__device__ __forceinline__ void decode_tile(int64_t t, int64_t T, int H, int* bi, int* bj, int* slice) {
  const int64_t st = t / H;
  *slice = static_cast<int>(t - st * H);
  tri_decode(st, T, bi, bj);
}

}  // namespace pald
