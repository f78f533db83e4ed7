// Batched PaLD: many independent matrices of uneven order in one persistent
// launch per pass.
//
// Host side: the orders and offsets are checked, every matrix is cut into
// upper-triangle tile pairs, and the tiles of all matrices are put in one
// work list ordered by cost (largest matrices first: a tile's cost is
// proportional to its matrix order, and longest-first keeps the tail short).
// The list, the per-matrix descriptors, scan results and tie maps live in one
// device allocation owned by a cached plan; the scan, tie-map, pass-1 and
// pass-2 launches (plus the resets) are captured once into a CUDA graph and
// replayed on later calls with the same arguments.
//
// Device side: each persistent CTA takes the next work item from a global
// atomic counter and runs the same tile code as the single-matrix kernels.
// There is no spin-wait anywhere: a CTA that finds the list exhausted exits.
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

using FG = FocusS0;     // 64 x 64 super-tiles, one CTA each
using CG = CohesionS0;  // 64 x 64 super-tiles, one CTA each
constexpr int kBF = FG::B;
constexpr int kBC = CG::B;
constexpr int kScanBlocksPerMatrix = 4;
constexpr int kTieBlocksPerMatrix = 8;
constexpr int kRecipBlocksPerMatrix = 8;
constexpr int kMaxGridY = 65535;  // matrices beyond it are strided over blockIdx.y

// Smallest positive and largest entry of every matrix: matrices along
// blockIdx.y, each matrix's entries strided over blockIdx.x.
__global__ void __launch_bounds__(256) batched_scan_kernel(const float* __restrict__ D,
                                                           const MatrixDesc* __restrict__ mats,
                                                           ScanResult* __restrict__ scans, int count) {
  for (int m = blockIdx.y; m < count; m += gridDim.y) {
    const MatrixDesc md = mats[m];
    const float* M = D + md.off;
    const int64_t elems = static_cast<int64_t>(md.n) * md.n;
    uint32_t inv_min = 0u, mx = 0u;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < elems;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const uint32_t b = __float_as_uint(__ldg(M + i));
      if (b < 0x7f800000u) {
        if (b != 0u) inv_min = max(inv_min, ~b);
        mx = max(mx, b);
      }
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

__device__ __forceinline__ int64_t next_item(int* counter, int* slot) {
  __syncthreads();  // every thread is done with the previous item's shared memory
  if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
  __syncthreads();
  return *slot;
}

__global__ void __launch_bounds__(FG::NT, 2) batched_focus_kernel(const float* __restrict__ D, int32_t* __restrict__ U,
                                                               const MatrixDesc* __restrict__ mats,
                                                               const ScanResult* __restrict__ scans,
                                                               const WorkItem* __restrict__ items, int64_t n_items,
                                                               int* counter) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int slot;
  for (;;) {
    const int64_t it = next_item(counter, &slot);
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const MatrixDesc md = mats[w.matrix];
    const float scale = focus_scale(scans[w.matrix].inv_min_pos_bits);
    focus_tile<FG>(D + md.off, md.n, U + md.off, w.bi, w.bj, w.slice, scale, smem);
  }
}

// R = 1/u for every matrix (zero diagonal): matrices along blockIdx.y.
__global__ void __launch_bounds__(256) batched_reciprocal_kernel(const int32_t* __restrict__ U, float* __restrict__ R,
                                                                 const MatrixDesc* __restrict__ mats, int count) {
  for (int m = blockIdx.y; m < count; m += gridDim.y) {
    const MatrixDesc md = mats[m];
    const bool vec = (md.n % 4) == 0;  // offsets are multiples of 4 elements
    for (int64_t row = blockIdx.x; row < md.n; row += gridDim.x)
      reciprocal_rows(U + md.off, R + md.off, md.n, row, vec);
  }
}

// Tie maps of every matrix (zeroed before): matrices along blockIdx.y, rows
// strided over blockIdx.x, one CTA per row at a time.
__global__ void __launch_bounds__(TieSmall::kThreads) batched_tie_kernel(const float* __restrict__ D,
                                                                         const MatrixDesc* __restrict__ mats,
                                                                         uint32_t* __restrict__ tmaps, int count) {
  __shared__ TieSmall::Smem sm;
  for (int m = blockIdx.y; m < count; m += gridDim.y) {
    const MatrixDesc md = mats[m];
    const TieMapDims dm = tie_map_dims(md.n);
    for (int64_t row = blockIdx.x; row < md.n; row += gridDim.x)
      tie_map_row<TieSmall>(D + md.off, md.n, row, tmaps + md.tmap_off, dm, sm);
  }
}

template <int MODE>
__global__ void __launch_bounds__(CG::NT, 2) batched_cohesion_kernel(const float* __restrict__ D,
                                                                     const float* __restrict__ R,
                                                                     float* __restrict__ C,
                                                                     const MatrixDesc* __restrict__ mats,
                                                                     const ScanResult* __restrict__ scans,
                                                                     const uint32_t* __restrict__ tmaps,
                                                                  const WorkItem* __restrict__ items,
                                                                  int64_t n_items, int* counter) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int slot;
  for (;;) {
    const int64_t it = next_item(counter, &slot);
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const MatrixDesc md = mats[w.matrix];
    const float S = focus_scale(scans[w.matrix].inv_min_pos_bits);
    cohesion_tile<CG, MODE>(D + md.off, R + md.off, md.n, C + md.off, tmaps + md.tmap_off, S, w.bi, w.bj, w.slice,
                            smem);
  }
}

int resident_ctas(const void* fn, int threads, int smem) {
  int per = 1;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) per = 1;
  return sm_count() * per;
}

// ---------------------------------------------------------------------------
// plan cache

struct Plan {
  void* dev_mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

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

void destroy_plan(Plan& p) {
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p.device);
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.graph) cudaGraphDestroy(p.graph);
  if (p.dev_mem) cudaFree(p.dev_mem);
  cudaSetDevice(prev);
  p = Plan{};
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

pald_status build_plan(int32_t count, const int64_t* ns, const int64_t* offs, const float* D, int32_t* U, float* C,
                       const pald_opts& o, int device, Plan* out) {
  // descriptors and tile lists
  std::vector<MatrixDesc> mats(count);
  std::vector<int> order(count);
  int64_t tmap_words = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t Tf = (ns[i] + kBF - 1) / kBF, Tc = (ns[i] + kBC - 1) / kBC;
    mats[i] = MatrixDesc{offs[i], static_cast<int32_t>(ns[i]), static_cast<int32_t>(Tf * (Tf + 1) / 2),
                         static_cast<int32_t>(Tc * (Tc + 1) / 2), 0, tmap_words};
    tmap_words += tie_map_words(ns[i]);
    order[i] = i;
  }
  // longest-processing-time first: a tile costs ~ n (its streamed dimension)
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ns[a] > ns[b]; });
  std::vector<WorkItem> fitems, citems;
  for (int i : order) {
    const int Tf = static_cast<int>((ns[i] + kBF - 1) / kBF), Tc = static_cast<int>((ns[i] + kBC - 1) / kBC);
    for (int bi = 0; bi < Tf; ++bi)
      for (int bj = bi; bj < Tf; ++bj)
        for (int h = 0; h < FG::H; ++h) fitems.push_back(WorkItem{i, bi, bj, h});
    for (int bi = 0; bi < Tc; ++bi)
      for (int bj = bi; bj < Tc; ++bj)
        for (int h = 0; h < CG::H; ++h) citems.push_back(WorkItem{i, bi, bj, h});
  }
  const size_t o_mats = 0;
  const size_t o_scans = align_up(o_mats + sizeof(MatrixDesc) * count, 256);
  const size_t o_fitems = align_up(o_scans + sizeof(ScanResult) * count, 256);
  const size_t o_citems = align_up(o_fitems + sizeof(WorkItem) * fitems.size(), 256);
  const size_t o_counters = align_up(o_citems + sizeof(WorkItem) * citems.size(), 256);
  int64_t r_elems = 0;  // R uses the same offsets as D, U and C
  for (int i = 0; i < count; ++i) r_elems = std::max<int64_t>(r_elems, offs[i] + ns[i] * ns[i]);
  const size_t o_tmaps = align_up(o_counters + 256, 256);
  const size_t o_recip = align_up(o_tmaps + sizeof(uint32_t) * static_cast<size_t>(tmap_words), 256);
  const size_t total = o_recip + sizeof(float) * static_cast<size_t>(r_elems);

  Plan p;
  p.device = device;
  cudaError_t e = cudaMalloc(&p.dev_mem, total);
  if (e != cudaSuccess) return cuda_fail(e);
  char* base = static_cast<char*>(p.dev_mem);
  auto* d_mats = reinterpret_cast<MatrixDesc*>(base + o_mats);
  auto* d_scans = reinterpret_cast<ScanResult*>(base + o_scans);
  auto* d_fitems = reinterpret_cast<WorkItem*>(base + o_fitems);
  auto* d_citems = reinterpret_cast<WorkItem*>(base + o_citems);
  auto* d_counters = reinterpret_cast<int*>(base + o_counters);
  auto* d_tmaps = reinterpret_cast<uint32_t*>(base + o_tmaps);
  auto* d_recip = reinterpret_cast<float*>(base + o_recip);
  e = cudaMemcpy(d_mats, mats.data(), sizeof(MatrixDesc) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_fitems, fitems.data(), sizeof(WorkItem) * fitems.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_citems, citems.data(), sizeof(WorkItem) * citems.size(), cudaMemcpyHostToDevice);
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
  const int fsmem = FocusSmem<FG>::FLOATS * static_cast<int>(sizeof(float));
  const int csmem = CohesionSmem<CG>::FLOATS * static_cast<int>(sizeof(float));
  const int gf = resident_ctas(reinterpret_cast<const void*>(batched_focus_kernel), FG::NT, fsmem);
  const void* cfn = plain ? reinterpret_cast<const void*>(batched_cohesion_kernel<PALD_ACCUM_PLAIN>)
                          : reinterpret_cast<const void*>(batched_cohesion_kernel<PALD_ACCUM_COMPENSATED>);
  const int gc = resident_ctas(cfn, CG::NT, csmem);
  if (gf == 0 || gc == 0) {
    destroy_plan(p);
    return cuda_fail(cudaErrorInvalidValue);
  }

  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const unsigned gy = static_cast<unsigned>(std::min(count, kMaxGridY));
    cudaMemsetAsync(d_scans, 0, sizeof(ScanResult) * count, cs);
    cudaMemsetAsync(d_counters, 0, 2 * sizeof(int), cs);
    cudaMemsetAsync(d_tmaps, 0, sizeof(uint32_t) * static_cast<size_t>(tmap_words), cs);
    batched_scan_kernel<<<dim3(kScanBlocksPerMatrix, gy), 256, 0, cs>>>(D, d_mats, d_scans, count);
    batched_tie_kernel<<<dim3(kTieBlocksPerMatrix, gy), TieSmall::kThreads, 0, cs>>>(D, d_mats, d_tmaps, count);
    batched_focus_kernel<<<gf, FG::NT, fsmem, cs>>>(D, U, d_mats, d_scans, d_fitems,
                                                static_cast<int64_t>(fitems.size()), d_counters);
    batched_reciprocal_kernel<<<dim3(kRecipBlocksPerMatrix, gy), 256, 0, cs>>>(U, d_recip, d_mats, count);
    if (plain)
      batched_cohesion_kernel<PALD_ACCUM_PLAIN><<<gc, CG::NT, csmem, cs>>>(
          D, d_recip, C, d_mats, d_scans, d_tmaps, d_citems, static_cast<int64_t>(citems.size()), d_counters + 1);
    else
      batched_cohesion_kernel<PALD_ACCUM_COMPENSATED><<<gc, CG::NT, csmem, cs>>>(
          D, d_recip, C, d_mats, d_scans, d_tmaps, d_citems, static_cast<int64_t>(citems.size()), d_counters + 1);
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
    if (n < 2 || n > 4096 || off < 0 || (off % 4) != 0) return PALD_ERR_INVALID_ARG;
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
  for (int i = 0; i < count; ++i) {
    key.words.push_back(n_host[i]);
    key.words.push_back(off_host[i]);
  }

  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    if (!g_plans) g_plans = new std::unordered_map<PlanKey, Plan, PlanKeyHash>();
    auto it = g_plans->find(key);
    if (it == g_plans->end()) {
      // the plan's graph reads D and writes U, C: order it after the caller's work
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e);
      Plan p;
      pald_status st = build_plan(count, n_host, off_host, D, U, C, o, device, &p);
      if (st != PALD_OK) return st;
      it = g_plans->emplace(std::move(key), p).first;
    }
    exec = it->second.exec;
  }
  e = cudaGraphLaunch(exec, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}

void pald_release(void) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  if (!g_plans) return;
  for (auto& kv : *g_plans) destroy_plan(kv.second);
  g_plans->clear();
}

}  // extern "C"
