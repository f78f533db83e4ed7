// Batched PaLD: many independent matrices of uneven order in one persistent
// launch per pass.
//
// Host side: the orders and offsets are checked, every matrix is cut into
// upper-triangle 64 x 64 tile pairs, and the tiles of all matrices are put in
// one work list ordered by cost (largest matrices first: a tile's cost is
// proportional to its matrix order, and longest-first keeps the tail short).
// Every matrix gets a row-padded copy of D (row pitch rounded up to a
// multiple of 4 floats, the 16-byte pitch TMA needs) and a row-padded R, and
// one TMA tensor map for each.  The list, the descriptors, scan results, tie
// maps, tensor maps and padded buffers live in one device allocation owned by
// a cached plan; the launches (plus the resets) are captured once into a CUDA
// graph and replayed on later calls with the same arguments.
//
// Device side: each persistent CTA takes the next work item from a global
// atomic counter (claiming the one after it while the tile runs) and runs
// the TMA tile code of the single-matrix kernels on the item's matrix.  A
// CTA that finds the list exhausted exits; the only waits are the bounded
// mbarrier waits of the TMA ring.  A diagonal tile without the pairs inside
// its groups of four points has four warps' worth of 4 x 4 blocks, so the
// diagonal tiles of a matrix come in pairs: pass 1 runs the two on the two
// halves of one CTA (focus_diag_pair_tma), pass 2 one after the other.  The
// in-group pairs go to a kernel with one thread per group after each pass
// (focus_group, cohesion_group).  Measured choices: tie maps as work items at
// pass 1's tail were 6.6 ms slower than in the prep kernel, parallel graph
// branches for the side kernels no faster than one chain, a pass-2 pair on
// two CTA halves no faster than in sequence.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "cohesion_core.cuh"
#include "schedules.cuh"
#include "tie_map_core.cuh"

namespace pald {

pald_status cuda_fail(cudaError_t e);
bool opts_ok(const pald_opts* o);
pald_opts opts_or_default(const pald_opts* o);

namespace {

using FG = FocusS7;     // 64 x 64 tiles, 32-deep TMA stages
// 64 x 64 tiles, 32-deep TMA stages, the scalar stage unrolled by 16 y (the
// packed stage needs R in its paired column order, which the padded copies
// of uneven order do not have)
using CG = TileGeom<64, 1, 1, 1, 4, 32, 16>;
static_assert(FG::B == 64 && CG::B == 64 && FG::H == 1 && CG::H == 1, "both passes share one tile list");
constexpr int kB = 64;
constexpr int kMaxGridY = 65535;  // matrices beyond it are strided over blockIdx.y
constexpr int kMaxBatchedN = 4096;
static_assert(kMaxBatchedN <= kTieFineMaxN, "batched tie maps have fine groups");
constexpr int kTieWordsBatched = ((kMaxBatchedN + kTieGroupFine - 1) / kTieGroupFine + 31) / 32;
constexpr int kGroupThreads = 128;  // groups of four points per CTA of the group kernels

// Set by a CTA whose bounded wait gave up (never in normal operation).
__device__ uint32_t g_batched_faults;

// Descriptor of matrix m beyond MatrixDesc: where its padded copies and its
// tensor maps are.
struct PadDesc {
  int64_t off_p;  // element offset of the padded D and R copies
  int64_t pitch;  // their row pitch (n rounded up to a multiple of 4)
};

// Before pass 1 when ties are ignored (no tie maps): every row of every
// matrix is copied into the padded layout (the TMA copies need a 16-byte row
// pitch) while the smallest positive and the largest entry go into the
// matrix's scan summary (zeroed before; pass 1 takes its scale from it).
// Matrices along blockIdx.y, one warp per row, rows strided over the CTAs of
// the matrix: a plain HBM-bound copy.
constexpr int kCopyThreads = 256;
constexpr int kCopyBlocksPerMatrix = 8;

__global__ void __launch_bounds__(kCopyThreads) batched_copy_kernel(const float* __restrict__ D,
                                                                    const MatrixDesc* __restrict__ mats,
                                                                    const PadDesc* __restrict__ pads,
                                                                    float* __restrict__ Dp,
                                                                    ScanResult* __restrict__ scans, int count) {
  constexpr int kWarps = kCopyThreads / 32;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int m = blockIdx.y; m < count; m += gridDim.y) {
    const MatrixDesc md = mats[m];
    const PadDesc pd = pads[m];
    uint32_t inv_min = 0u, mx = 0u;
    for (int64_t row = int64_t(blockIdx.x) * kWarps + warp; row < md.n; row += int64_t(gridDim.x) * kWarps) {
      const float* src = D + md.off + row * md.n;
      float* dst = Dp + pd.off_p + row * pd.pitch;
      for (int64_t c0 = 0; c0 < md.n; c0 += 4 * 32) {  // four loads in flight per lane
        float d[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t c = c0 + 32 * k + lane;
          d[k] = c < md.n ? __ldg(src + c) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t c = c0 + 32 * k + lane;
          if (c >= md.n) continue;
          dst[c] = d[k];
          const uint32_t b = __float_as_uint(d[k]);
          if (b < 0x7f800000u) {  // finite, not negative
            if (b != 0u) inv_min = max(inv_min, ~b);
            mx = max(mx, b);
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      inv_min = max(inv_min, __shfl_xor_sync(0xffffffffu, inv_min, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
      if (inv_min) atomicMax(&scans[m].inv_min_pos_bits, inv_min);
      if (mx) atomicMax(&scans[m].max_bits, mx);
    }
  }
}

// The prep before pass 1: the same copy and scan, plus every row's repeats
// into the matrix's tie map (zeroed before), at the prep's own occupancy
// (many CTAs per SM: the per-row hashing is latency-bound; as work items of
// the persistent pass-1 kernel it measured 6.6 ms slower on the batched
// workload).  Matrices along blockIdx.y, one CTA per row at a time.
struct PrepVisit {
  float* dst;  // padded row
  uint32_t* inv_min;
  uint32_t* mx;
  __device__ __forceinline__ void operator()(int64_t c, float d) const {
    dst[c] = d;
    const uint32_t b = __float_as_uint(d);
    if (b < 0x7f800000u) {
      if (b != 0u) *inv_min = max(*inv_min, ~b);
      *mx = max(*mx, b);
    }
  }
};

constexpr int kTieBlocksPerMatrix = 16;
#ifndef PALD_PREP_THREADS
#define PALD_PREP_THREADS 256
#endif
// The prep's per-row hashing is latency-bound: what counts is how many rows
// are in flight per SM (shared memory and threads per CTA bound it).
using TiePrep = TieConfig<PALD_PREP_THREADS, 2048, 512>;

__global__ void __launch_bounds__(TiePrep::kThreads) batched_prep_kernel(const float* __restrict__ D,
                                                                          const MatrixDesc* __restrict__ mats,
                                                                          const PadDesc* __restrict__ pads,
                                                                          float* __restrict__ Dp,
                                                                          ScanResult* __restrict__ scans,
                                                                          uint32_t* __restrict__ tmaps, int count) {
  __shared__ TiePrep::Smem sm;
  for (int m = blockIdx.y; m < count; m += gridDim.y) {
    const MatrixDesc md = mats[m];
    const PadDesc pd = pads[m];
    const TieMapDims dm = tie_map_dims(md.n);
    uint32_t inv_min = 0u, mx = 0u;
    for (int64_t row = blockIdx.x; row < md.n; row += gridDim.x) {
      // the CTA's next row heads for L2 while this one is hashed (one
      // prefetch per 128-byte line)
      const int64_t next = row + gridDim.x;
      if (next < md.n)
        for (int64_t c = 32 * static_cast<int64_t>(threadIdx.x); c < md.n; c += 32 * TiePrep::kThreads)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(D + md.off + next * md.n + c));
      tie_map_row<TiePrep>(D + md.off, md.n, row, tmaps + md.tmap_off, dm, sm,
                            PrepVisit{Dp + pd.off_p + row * pd.pitch, &inv_min, &mx});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      inv_min = max(inv_min, __shfl_xor_sync(0xffffffffu, inv_min, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (inv_min) atomicMax(&scans[m].inv_min_pos_bits, inv_min);
      if (mx) atomicMax(&scans[m].max_bits, mx);
    }
  }
}

// Work-list cursor of a persistent CTA: `slot` (shared) holds the current
// item; thread 0 claims the next one as soon as an item starts, so the
// atomic round trip overlaps the work.
struct ItemCursor {
  int* counter;
  int* slot;
  int next;
  __device__ __forceinline__ int64_t first() {
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
  }
  __device__ __forceinline__ void claim_next() {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
  }
  __device__ __forceinline__ int64_t advance() {
    __syncthreads();  // every thread has read the slot and is done with the item's shared memory
    if (threadIdx.x == 0) *slot = next;
    __syncthreads();
    return *slot;
  }
};

// Pass 1's queue holds every 64 x 64 tile, largest matrices first.
// maps[2m] is matrix m's padded D, maps[2m + 1] its padded R.  Three CTAs
// per SM (80 registers, 48 KB ring each): short tiles leave gaps (claim,
// first TMA stage, epilogue) that a third CTA fills; measured 6% faster on
// the batched workload than two CTAs with 128 registers.
__global__ void __launch_bounds__(FG::NT, 3) batched_focus_kernel(const float* __restrict__ D, int32_t* __restrict__ U,
                                                               float* __restrict__ Rp,
                                                               const MatrixDesc* __restrict__ mats,
                                                               const PadDesc* __restrict__ pads,
                                                               const ScanResult* __restrict__ scans,
                                                               const CUtensorMap* __restrict__ maps,
                                                               const WorkItem* __restrict__ items, int64_t n_items,
                                                               int* counter) {
  extern __shared__ __align__(128) float smem[];
  __shared__ int slot;
  TmaRing<2, FG::BK> ring;
  ring.carve(smem);
  ItemCursor cur{counter, &slot, 0};
  for (int64_t it = cur.first(); it < n_items; it = cur.advance()) {
    cur.claim_next();
    const WorkItem w = items[it];
    const MatrixDesc md = mats[w.matrix];
    const PadDesc pd = pads[w.matrix];
    const float scale = focus_scale(scans[w.matrix].inv_min_pos_bits);
    const bool ok = w.kind == kItemDiagPair
                        ? focus_diag_pair_tma<FG>(maps + 2 * w.matrix, D + md.off, md.n, U + md.off, w.a, w.b, scale,
                                                  md.n % 4 == 0, ring, Rp + pd.off_p, pd.pitch)
                        : focus_tile_tma<FG>(maps + 2 * w.matrix, D + md.off, md.n, U + md.off, w.a, w.b, scale,
                                             md.n % 4 == 0, ring, Rp + pd.off_p, pd.pitch, false);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(&g_batched_faults, 1u);
      break;
    }
  }
}

// Pass 2's queue holds every tile, largest matrices first; the pairs inside
// the groups of four points that split diagonal tiles leave out come after,
// from batched_cohesion_group_kernel.
template <int MODE>
__global__ void __launch_bounds__(CG::NT, 2) batched_cohesion_kernel(const float* __restrict__ D,
                                                                     float* __restrict__ C,
                                                                     const MatrixDesc* __restrict__ mats,
                                                                     const ScanResult* __restrict__ scans,
                                                                     const uint32_t* __restrict__ tmaps,
                                                                     const CUtensorMap* __restrict__ maps,
                                                                     const WorkItem* __restrict__ items,
                                                                     int64_t n_items, int* counter) {
  extern __shared__ __align__(128) float smem[];
  __shared__ int slot;
  TmaRing<4, CG::BK> ring;
  uint32_t* tie_words = reinterpret_cast<uint32_t*>(ring.carve(smem));
  ItemCursor cur{counter, &slot, 0};
  for (int64_t it = cur.first(); it < n_items; it = cur.advance()) {
    cur.claim_next();
    const WorkItem w = items[it];
    const MatrixDesc md = mats[w.matrix];
    const float S = focus_scale(scans[w.matrix].inv_min_pos_bits);
    // One call site for every tile.  Pass 2 takes a pair item's diagonal
    // tiles one after the other, four warps each (the in-group pairs are the
    // group kernel's): on the two halves of one CTA, as pass 1 does, it
    // measured no faster, and the second tile function raised register spills.
    bool ok = true;
    const bool pair = w.kind == kItemDiagPair;
    const int nsub = pair && w.b >= 0 ? 2 : 1;
    for (int h = 0; h < nsub && ok; ++h) {
      const int bi = pair && h == 1 ? w.b : w.a;
      ok = cohesion_tile_tma<CG, MODE>(maps + 2 * w.matrix, maps + 2 * w.matrix + 1, D + md.off, md.n, C + md.off,
                                       tmaps + md.tmap_off, S, bi, pair ? bi : w.b, md.n % 4 == 0, ring, tie_words,
                                       pair);
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(&g_batched_faults, 1u);
      break;
    }
  }
}

// Pass 1's pairs inside each group of four points, which paired diagonal
// tiles leave out: one thread per group (focus_group), the listed matrices
// along blockIdx.y, groups along x.  Runs after the pass-1 tiles, before
// pass 2 reads R.
__global__ void __launch_bounds__(kGroupThreads) batched_focus_group_kernel(
    int32_t* __restrict__ U, const float* __restrict__ Dp, float* __restrict__ Rp,
    const MatrixDesc* __restrict__ mats, const PadDesc* __restrict__ pads, const ScanResult* __restrict__ scans,
    const int32_t* __restrict__ order, int count) {
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const int m = order[k];
    const MatrixDesc md = mats[m];
    const int64_t q = int64_t(blockIdx.x) * kGroupThreads + threadIdx.x;
    if (4 * q >= md.n) continue;
    const PadDesc pd = pads[m];
    focus_group(Dp + pd.off_p, pd.pitch, md.n, q, focus_scale(scans[m].inv_min_pos_bits), U + md.off,
                Rp + pd.off_p, pd.pitch);
  }
}

// Pass 2's pairs inside each group of four points, which split diagonal
// tiles leave out: one thread per group, the listed matrices along
// blockIdx.y (largest first), groups along x.  Reads the padded copies of D
// and R.
template <int MODE>
__global__ void __launch_bounds__(kGroupThreads, 3) batched_cohesion_group_kernel(
    float* __restrict__ C, const float* __restrict__ Dp, const float* __restrict__ Rp,
    const MatrixDesc* __restrict__ mats, const PadDesc* __restrict__ pads, const ScanResult* __restrict__ scans,
    const uint32_t* __restrict__ tmaps, const int32_t* __restrict__ order, int count) {
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const int m = order[k];
    const MatrixDesc md = mats[m];
    const int64_t q = int64_t(blockIdx.x) * kGroupThreads + threadIdx.x;
    if (4 * q >= md.n) continue;
    const PadDesc pd = pads[m];
    cohesion_group<MODE>(Dp + pd.off_p, Rp + pd.off_p, pd.pitch, md.n, q, focus_scale(scans[m].inv_min_pos_bits),
                         C + md.off, md.n % 4 == 0, tmaps + md.tmap_off);
  }
}

int resident_ctas(const void* fn, int threads, int smem) {
  int per = 1;
  if (smem_opt_in(fn, smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) per = 1;
  return sm_count() * per;
}

// ---------------------------------------------------------------------------
// plan cache

struct Plan {
  void* dev_mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;  // recorded after each replay: the next replay of this plan waits on it
  uint64_t last_use = 0;       // for least-recently-used eviction
  int device = 0;
};

// Plans kept at once; building one more frees the least recently used.
constexpr size_t kMaxPlans = 16;

struct PlanKey {
  std::vector<int64_t> words;
  bool operator==(const PlanKey& o) const { return words == o.words; }
};
struct PlanKeyHash {
  size_t operator()(const PlanKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t w : k.words) {
      h ^= static_cast<uint64_t>(w);
      h *= 1099511628211ull;
    }
    return static_cast<size_t>(h);
  }
};

std::mutex g_plan_mu;
std::unordered_map<PlanKey, Plan, PlanKeyHash>* g_plans = nullptr;
cudaStream_t g_capture_stream[64] = {};

// Waits for the plan's last replay, then frees everything it holds.
void destroy_plan(Plan& p) {
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p.device);
  if (p.done) {
    cudaEventSynchronize(p.done);
    cudaEventDestroy(p.done);
  }
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.graph) cudaGraphDestroy(p.graph);
  if (p.dev_mem) cudaFree(p.dev_mem);
  cudaSetDevice(prev);
  p = Plan{};
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

pald_status build_plan(int32_t count, const int64_t* ns, const int64_t* offs, const float* D, int32_t* U, float* C,
                       const pald_opts& o, int device, Plan* out) {
  // descriptors, padded layout and the tile list (shared by both passes)
  std::vector<MatrixDesc> mats(count);
  std::vector<PadDesc> pads(count);
  std::vector<int> order(count);
  int64_t tmap_words = 0, pad_elems = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t T = (ns[i] + kB - 1) / kB;
    const int32_t tiles = static_cast<int32_t>(T * (T + 1) / 2);
    mats[i] = MatrixDesc{offs[i], static_cast<int32_t>(ns[i]), tiles, tiles, 0, tmap_words};
    tmap_words += tie_map_words(ns[i]);
    const int64_t pitch = (ns[i] + 3) / 4 * 4;
    pads[i] = PadDesc{pad_elems, pitch};
    pad_elems += ns[i] * pitch;
    order[i] = i;
  }
  // longest-processing-time first: a tile costs ~ n (its streamed dimension)
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
  const bool ignore_ties = (o.flags & PALD_FLAG_IGNORE_TIES) != 0;
  // pass 1: every tile, then the tie-map rows (none when ties are ignored:
  // the zeroed maps then select the short form everywhere); pass 2: every
  // tile, with each matrix's group items after its tiles
  // Whether diagonal tiles split off their in-group pairs is chosen per
  // order from the schedule table (pald_schedule_bucket.batched_split).
  std::vector<WorkItem> items1, items2;
  std::vector<int32_t> group_order;  // matrices whose group pairs the group kernel computes
  int64_t group_max_n = 0;
  for (int i : order) {
    ScheduleBucket sb;
    schedule_for(ns[i], &sb);
    const int T = static_cast<int>((ns[i] + kB - 1) / kB);
    for (int bi = 0; bi < T; ++bi)
      for (int bj = bi; bj < T; ++bj) {
        if (bi == bj && sb.batched_split) {
          if (bi % 2 == 1) continue;  // taken with bi - 1
          const WorkItem w{i, bi, bi + 1 < T ? bi + 1 : -1, kItemDiagPair};
          items1.push_back(w);
          items2.push_back(w);
          continue;
        }
        const int32_t kind = sb.batched_split ? kItemTile : kItemTileWhole;
        items1.push_back(WorkItem{i, bi, bj, kind});
        items2.push_back(WorkItem{i, bi, bj, kind});
      }
    if (sb.batched_split) {
      group_order.push_back(i);
      group_max_n = std::max(group_max_n, ns[i]);
    }
  }
  const size_t o_mats = 0;
  const size_t o_pads = align_up(o_mats + sizeof(MatrixDesc) * count, 256);
  const size_t o_scans = align_up(o_pads + sizeof(PadDesc) * count, 256);
  const size_t o_order = align_up(o_scans + sizeof(ScanResult) * count, 256);
  const size_t o_items1 = align_up(o_order + sizeof(int32_t) * (group_order.size() + 1), 256);
  const size_t o_items2 = align_up(o_items1 + sizeof(WorkItem) * items1.size(), 256);
  const size_t o_counters = align_up(o_items2 + sizeof(WorkItem) * items2.size(), 256);
  const size_t o_tmaps = align_up(o_counters + 256, 256);
  const size_t o_maps = align_up(o_tmaps + sizeof(uint32_t) * static_cast<size_t>(tmap_words), 256);
  const size_t o_dpad = align_up(o_maps + sizeof(CUtensorMap) * 2 * static_cast<size_t>(count), 256);
  const size_t o_rpad = align_up(o_dpad + sizeof(float) * static_cast<size_t>(pad_elems), 256);
  const size_t total = o_rpad + sizeof(float) * static_cast<size_t>(pad_elems);

  Plan p;
  p.device = device;
  cudaError_t e = cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMalloc(&p.dev_mem, total);
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e);
  }
  char* base = static_cast<char*>(p.dev_mem);
  auto* d_mats = reinterpret_cast<MatrixDesc*>(base + o_mats);
  auto* d_pads = reinterpret_cast<PadDesc*>(base + o_pads);
  auto* d_scans = reinterpret_cast<ScanResult*>(base + o_scans);
  auto* d_order = reinterpret_cast<int32_t*>(base + o_order);
  auto* d_items1 = reinterpret_cast<WorkItem*>(base + o_items1);
  auto* d_items2 = reinterpret_cast<WorkItem*>(base + o_items2);
  auto* d_counters = reinterpret_cast<int*>(base + o_counters);
  auto* d_tmaps = reinterpret_cast<uint32_t*>(base + o_tmaps);
  auto* d_maps = reinterpret_cast<CUtensorMap*>(base + o_maps);
  auto* d_dpad = reinterpret_cast<float*>(base + o_dpad);
  auto* d_rpad = reinterpret_cast<float*>(base + o_rpad);
  // tensor maps of the padded copies (their addresses are fixed by the plan)
  std::vector<CUtensorMap> maps(2 * static_cast<size_t>(count));
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    e = encode_panel_map(&maps[2 * i], d_dpad + pads[i].off_p, ns[i], pads[i].pitch, FG::BK);
    if (e == cudaSuccess) e = encode_panel_map(&maps[2 * i + 1], d_rpad + pads[i].off_p, ns[i], pads[i].pitch, CG::BK);
  }
  if (e == cudaSuccess) e = cudaMemcpy(d_mats, mats.data(), sizeof(MatrixDesc) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_pads, pads.data(), sizeof(PadDesc) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !group_order.empty())
    e = cudaMemcpy(d_order, group_order.data(), sizeof(int32_t) * group_order.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(d_items1, items1.data(), sizeof(WorkItem) * items1.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(d_items2, items2.data(), sizeof(WorkItem) * items2.size(), cudaMemcpyHostToDevice);
  // the pad columns of the padded copies are read (by the pass-2 group
  // kernel) but never written: zero them once
  if (e == cudaSuccess) e = cudaMemset(d_dpad, 0, sizeof(float) * static_cast<size_t>(pad_elems));
  if (e == cudaSuccess) e = cudaMemset(d_rpad, 0, sizeof(float) * static_cast<size_t>(pad_elems));
  // the uploads above ran on the legacy stream, which need not order the
  // caller's (possibly non-blocking) stream: finish them first
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e);
  }

  cudaStream_t cs = g_capture_stream[device];
  if (!cs) {
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
      destroy_plan(p);
      return cuda_fail(e);
    }
    g_capture_stream[device] = cs;
  }
  const bool plain = o.accum_mode == PALD_ACCUM_PLAIN;
  const int fsmem = TmaRing<2, FG::BK>::BYTES + 128;
  const int csmem = TmaRing<4, CG::BK>::BYTES + 128 + 4 * kTieWordsBatched;
  const int gf = resident_ctas(reinterpret_cast<const void*>(batched_focus_kernel), FG::NT, fsmem);
  const void* cfn = plain ? reinterpret_cast<const void*>(batched_cohesion_kernel<PALD_ACCUM_PLAIN>)
                          : reinterpret_cast<const void*>(batched_cohesion_kernel<PALD_ACCUM_COMPENSATED>);
  const int gc = resident_ctas(cfn, CG::NT, csmem);
  if (gf == 0 || gc == 0) {
    destroy_plan(p);
    return cuda_fail(cudaErrorInvalidValue);
  }
  const int64_t n1 = static_cast<int64_t>(items1.size()), n2 = static_cast<int64_t>(items2.size());
  const int ng = static_cast<int>(group_order.size());

  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const unsigned gy = static_cast<unsigned>(std::min(count, kMaxGridY));
    const dim3 ggrid(static_cast<unsigned>((group_max_n + 4 * kGroupThreads - 1) / (4 * kGroupThreads)),
                     static_cast<unsigned>(std::min(std::max(ng, 1), kMaxGridY)));
    cudaMemsetAsync(d_scans, 0, sizeof(ScanResult) * count, cs);
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(int), cs);
    cudaMemsetAsync(d_tmaps, 0, sizeof(uint32_t) * static_cast<size_t>(tmap_words), cs);
    if (ignore_ties)  // empty maps: the short (strict) form everywhere
      batched_copy_kernel<<<dim3(kCopyBlocksPerMatrix, gy), kCopyThreads, 0, cs>>>(D, d_mats, d_pads, d_dpad,
                                                                                    d_scans, count);
    else
      batched_prep_kernel<<<dim3(kTieBlocksPerMatrix, gy), TiePrep::kThreads, 0, cs>>>(D, d_mats, d_pads, d_dpad,
                                                                                        d_scans, d_tmaps, count);
    batched_focus_kernel<<<gf, FG::NT, fsmem, cs>>>(D, U, d_rpad, d_mats, d_pads, d_scans, d_maps, d_items1, n1,
                                                    d_counters);
    if (ng > 0)
      batched_focus_group_kernel<<<ggrid, kGroupThreads, 0, cs>>>(U, d_dpad, d_rpad, d_mats, d_pads, d_scans,
                                                                  d_order, ng);
    if (plain) {
      batched_cohesion_kernel<PALD_ACCUM_PLAIN><<<gc, CG::NT, csmem, cs>>>(D, C, d_mats, d_scans, d_tmaps, d_maps,
                                                                          d_items2, n2, d_counters + 1);
      if (ng > 0)
        batched_cohesion_group_kernel<PALD_ACCUM_PLAIN><<<ggrid, kGroupThreads, 0, cs>>>(
            C, d_dpad, d_rpad, d_mats, d_pads, d_scans, d_tmaps, d_order, ng);
    } else {
      batched_cohesion_kernel<PALD_ACCUM_COMPENSATED><<<gc, CG::NT, csmem, cs>>>(
          D, C, d_mats, d_scans, d_tmaps, d_maps, d_items2, n2, d_counters + 1);
      if (ng > 0)
        batched_cohesion_group_kernel<PALD_ACCUM_COMPENSATED><<<ggrid, kGroupThreads, 0, cs>>>(
            C, d_dpad, d_rpad, d_mats, d_pads, d_scans, d_tmaps, d_order, ng);
    }
    cudaError_t launch_err = cudaGetLastError();
    e = cudaStreamEndCapture(cs, &p.graph);
    if (e == cudaSuccess && launch_err != cudaSuccess) e = launch_err;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p.exec, p.graph, 0);
  if (e != cudaSuccess) {
    destroy_plan(p);
    return cuda_fail(e);
  }
  *out = p;
  return PALD_OK;
}

}  // namespace

cudaError_t take_batched_faults(uint32_t* out, cudaStream_t s) {
  uint32_t zero = 0;
  cudaError_t e = cudaMemcpyFromSymbolAsync(out, g_batched_faults, sizeof(uint32_t), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *out != 0u)
    e = cudaMemcpyToSymbolAsync(g_batched_faults, &zero, sizeof(uint32_t), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace pald

using namespace pald;

extern "C" {

pald_status pald_validate(const float* D, int64_t n, pald_stream_t stream);

pald_status pald_batched(int32_t count, const int64_t* n_host, const int64_t* off_host, const float* D, int32_t* U,
                         float* C, const pald_opts* opts, pald_stream_t stream) {
  if (count < 1 || count > (1 << 20) || !n_host || !off_host || !D || !U || !C || !opts_ok(opts))
    return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  // orders, alignment and non-overlap
  std::vector<std::pair<int64_t, int64_t>> spans(count);
  for (int i = 0; i < count; ++i) {
    const int64_t n = n_host[i], off = off_host[i];
    if (n < 2 || n > kMaxBatchedN || off < 0 || (off % 4) != 0) return PALD_ERR_INVALID_ARG;
    spans[i] = {off, off + n * n};
  }
  std::sort(spans.begin(), spans.end());
  for (int i = 1; i < count; ++i)
    if (spans[i].first < spans[i - 1].second) return PALD_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(D) | reinterpret_cast<uintptr_t>(U) | reinterpret_cast<uintptr_t>(C)) % 16)
    return PALD_ERR_INVALID_ARG;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.validate) {
    for (int i = 0; i < count; ++i) {
      pald_status st = pald_validate(D + off_host[i], n_host[i], stream);
      if (st != PALD_OK) return st;
    }
  }
  if (o.accum_mode == PALD_ACCUM_FIXED) {
    // exact integer sums: the matrices go one after another through the
    // single-matrix path (the same bits as pald_focus + pald_cohesion)
    pald_opts o1 = o;
    o1.validate = 0;
    o1.schedule_id = -1;
    for (int i = 0; i < count; ++i) {
      pald_status st = pald_focus(D + off_host[i], n_host[i], U + off_host[i], &o1, stream);
      if (st == PALD_OK) st = pald_cohesion(D + off_host[i], U + off_host[i], n_host[i], C + off_host[i], &o1, stream);
      if (st != PALD_OK) return st;
    }
    return PALD_OK;
  }
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e);
  if (device < 0 || device >= 64) return PALD_ERR_UNSUPPORTED;

  PlanKey key;
  key.words.reserve(2 * static_cast<size_t>(count) + 8);
  key.words.push_back(device);
  key.words.push_back(count);
  key.words.push_back(static_cast<int64_t>(reinterpret_cast<uintptr_t>(D)));
  key.words.push_back(static_cast<int64_t>(reinterpret_cast<uintptr_t>(U)));
  key.words.push_back(static_cast<int64_t>(reinterpret_cast<uintptr_t>(C)));
  key.words.push_back(o.accum_mode);
  key.words.push_back(o.flags);
  key.words.push_back(static_cast<int64_t>(schedule_generation()));  // the plan follows the schedule table
  for (int i = 0; i < count; ++i) {
    key.words.push_back(n_host[i]);
    key.words.push_back(off_host[i]);
  }

  // The lock is held until the replay is queued, so pald_release or an
  // eviction on another thread cannot free the graph in between.
  std::lock_guard<std::mutex> lock(g_plan_mu);
  if (!g_plans) g_plans = new std::unordered_map<PlanKey, Plan, PlanKeyHash>();
  static uint64_t tick = 0;
  auto it = g_plans->find(key);
  if (it == g_plans->end()) {
    // the plan's graph reads D and writes U, C: order it after the caller's work
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
    if (g_plans->size() >= kMaxPlans) {  // free the least recently used plan
      auto lru = g_plans->begin();
      for (auto j = g_plans->begin(); j != g_plans->end(); ++j)
        if (j->second.last_use < lru->second.last_use) lru = j;
      destroy_plan(lru->second);
      g_plans->erase(lru);
    }
    Plan p;
    pald_status st = build_plan(count, n_host, off_host, D, U, C, o, device, &p);
    if (st != PALD_OK) return st;
    it = g_plans->emplace(std::move(key), p).first;
  }
  Plan& plan = it->second;
  plan.last_use = ++tick;
  // Every replay of a plan shares its scratch (work counters, padded copies,
  // tie maps): a replay on another stream first waits for the previous one.
  // Under stream capture the caller's graph orders its own nodes instead.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return cuda_fail(e);
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (!capturing && (e = cudaStreamWaitEvent(s, plan.done, 0)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaGraphLaunch(plan.exec, s)) != cudaSuccess) return cuda_fail(e);
  if (!capturing && (e = cudaEventRecord(plan.done, s)) != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}

void pald_release(void) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  if (!g_plans) return;
  for (auto& kv : *g_plans) destroy_plan(kv.second);
  g_plans->clear();
}

}  // extern "C"
