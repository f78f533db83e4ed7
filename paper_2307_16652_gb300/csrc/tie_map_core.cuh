// Tie map construction: finds, row by row, every pair of equal entries of D
// and marks the (block pair, y group) cells of the map that pass 2 must run
// with its exact inner loop.  See pald_internal.cuh for the map layout.
//
// Why rows: pass 2's short form computes, per (x, z, y), the weight
// w(d_xz, min(d_xy, d_zy)) and credits it to both c_xz and c_zx.  Against
// the definition (z in U_xy, support w(d_zx, d_zy); Sec. 2 eq. (fxz) with the
// tie split of Sec. 5) it is wrong only when
//     d_xy == d_xz < d_zy   (c_xz should get 1, gets 1/2), or
//     d_zy == d_zx < d_xy   (c_zx should get 1, gets 1/2),
// i.e. when row x (or row z) of D holds the same value at two columns
// {y, z} (or {y, x}).  So for every row r and every ordered pair (p, q),
// p != q, of columns with d_rp == d_rq, the cell ({block(r), block(q)},
// group(p)) is marked; a tile (X, Z) whose stage y-range meets no marked
// cell can use the short form with a result identical bit for bit.
//
// Per row, one CTA hashes the row's values into a shared-memory table
// (open addressing, linear probing); an insert that finds its value already
// present is a repeat and is listed with its slot.  After a barrier, each
// listed repeat marks its pairs with the slot's first column and with every
// other repeat of the same slot.  Rows longer than half the table are processed in
// ceil(n / (slots / 2)) passes, each taking the values whose hash falls in
// its share, so the table never fills beyond one half.  A row with more than
// DUPCAP repeats in one pass (e.g. small-integer distances) is not listed:
// its block is flagged dirty instead.
#pragma once

#include "pald_internal.cuh"

namespace pald {

constexpr uint32_t kTieEmpty = 0xffffffffu;  // a NaN pattern: never a valid entry

// Shared-memory sizes of one row's scan: THREADS threads, a table of SLOTS
// hash slots (a power of two; each pass takes at most SLOTS / 2 values) and
// room to list DUPCAP repeated values per pass.
template <int THREADS, int SLOTS, int DUPCAP>
struct TieConfig {
  static constexpr int kThreads = THREADS;
  static constexpr int kSlots = SLOTS;
  static constexpr int kPart = SLOTS / 2;
  static constexpr int kDupCap = DUPCAP;
  static_assert((SLOTS & (SLOTS - 1)) == 0, "hash slots must be a power of two");
  struct Smem {
    uint32_t key[SLOTS];    // value bits
    int32_t first[SLOTS];   // column of the first occurrence
    int32_t dslot[DUPCAP];  // repeats: slot ...
    int32_t dcol[DUPCAP];   // ... and column
    int32_t ndup;
    int32_t overflow;
  };
};
using TieLarge = TieConfig<1024, 16384, 2048>;  // one matrix, any order: 147 KB, one CTA per SM
using TieSmall = TieConfig<256, 2048, 512>;     // batched orders <= 4096: 20 KB, many CTAs per SM

// 32-bit finalizer of MurmurHash3 (Appleby, public domain): mixes all input
// bits into all output bits, so the table slot and the pass share are
// independent of the float's exponent structure.
__device__ __forceinline__ uint32_t tie_hash(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// Marks cell ({block(row), block(q)}, group(p)).
__device__ __forceinline__ void tie_mark(uint32_t* map, const TieMapDims& dm, int64_t brow, int64_t p, int64_t q) {
  int64_t a = brow, b = q / kTieBlock;
  if (a > b) {
    const int64_t t = a;
    a = b;
    b = t;
  }
  const int64_t g = p >> dm.gshift;
  atomicOr(map + (a * dm.nb + b) * dm.wpp + (g >> 5), 1u << (g & 31));
}

struct NoVisit {
  __device__ __forceinline__ void operator()(int64_t, float) const {}
};

// All Cfg::kThreads threads of the CTA process row `row` of the n x n matrix
// at `Dm` into `map` (already zeroed).  `visit(c, d_row,c)` sees every entry
// of the row once (during the first hash pass).  Contains barriers: call
// uniformly.
template <class Cfg, class Visit = NoVisit>
__device__ __forceinline__ void tie_map_row(const float* __restrict__ Dm, int64_t n, int64_t row, uint32_t* map,
                                            const TieMapDims& dm, typename Cfg::Smem& sm, Visit visit = Visit()) {
  constexpr int NT = Cfg::kThreads, SLOTS = Cfg::kSlots, CAP = Cfg::kDupCap;
  const float* drow = Dm + row * n;
  const int64_t brow = row / kTieBlock;
  const int parts = static_cast<int>((n + Cfg::kPart - 1) / Cfg::kPart);
  bool dirty = false;
  for (int part = 0; part < parts && !dirty; ++part) {  // part 0 always runs
    for (int i = threadIdx.x; i < SLOTS; i += NT) sm.key[i] = kTieEmpty;
    if (threadIdx.x == 0) {
      sm.ndup = 0;
      sm.overflow = 0;
    }
    __syncthreads();
    for (int64_t c = threadIdx.x; c < n; c += NT) {
      const float d = __ldg(drow + c);
      if (part == 0) visit(c, d);
      // +0.0f turns a stray -0.0 into +0.0 (equal under comparison)
      const uint32_t v = __float_as_uint(__fadd_rn(d, 0.0f));
      const uint32_t h = tie_hash(v);
      if (parts > 1 && static_cast<int>((static_cast<uint64_t>(h) * static_cast<uint64_t>(parts)) >> 32) != part)
        continue;
      uint32_t slot = h & (SLOTS - 1);
      int k = 0;
      for (; k < SLOTS; ++k) {
        const uint32_t old = atomicCAS(&sm.key[slot], kTieEmpty, v);
        if (old == kTieEmpty) {
          sm.first[slot] = static_cast<int32_t>(c);
          break;
        }
        if (old == v) {
          const int i = atomicAdd(&sm.ndup, 1);
          if (i < CAP) {
            sm.dslot[i] = static_cast<int32_t>(slot);
            sm.dcol[i] = static_cast<int32_t>(c);
          }
          break;
        }
        slot = (slot + 1) & (SLOTS - 1);
      }
      if (k == SLOTS) sm.overflow = 1;  // only for values outside the input contract
    }
    __syncthreads();
    const int nd = sm.ndup;
    dirty = nd > CAP || sm.overflow != 0;
    if (!dirty) {
      for (int i = threadIdx.x; i < nd; i += NT) {
        const int s = sm.dslot[i];
        const int64_t ci = sm.dcol[i];
        const int64_t f = sm.first[s];
        tie_mark(map, dm, brow, f, ci);
        tie_mark(map, dm, brow, ci, f);
        for (int j = 0; j < nd; ++j)
          if (j != i && sm.dslot[j] == s) tie_mark(map, dm, brow, ci, sm.dcol[j]);
      }
    }
    __syncthreads();  // the table is cleared again by the next pass or row
  }
  if (dirty && threadIdx.x == 0) atomicOr(map + dm.nb * dm.nb * dm.wpp + brow, 1u);
}

}  // namespace pald
