// Tie map of one matrix (see tie_map_core.cuh): one CTA per row, strided
// over the rows, one CTA per SM (the hash table takes 147 KB of shared
// memory).  The batched path has its own smaller configuration.
#include "schedules.cuh"
#include "tie_map_core.cuh"

namespace pald {

namespace {

__global__ void __launch_bounds__(TieLarge::kThreads, 1)
    tie_map_kernel(const float* __restrict__ D, int64_t n, uint32_t* __restrict__ map, TieMapDims dm) {
  extern __shared__ __align__(16) unsigned char tie_smem[];
  auto& sm = *reinterpret_cast<TieLarge::Smem*>(tie_smem);
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) tie_map_row<TieLarge>(D, n, row, map, dm, sm);
}

}  // namespace

cudaError_t launch_tie_map(const float* D, int64_t n, uint32_t* map, cudaStream_t s) {
  const TieMapDims dm = tie_map_dims(n);
  cudaError_t e = cudaMemsetAsync(map, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  e = smem_opt_in(reinterpret_cast<const void*>(tie_map_kernel), static_cast<int>(sizeof(TieLarge::Smem)));
  if (e != cudaSuccess) return e;
  const int64_t cap = sm_count();
  const int64_t grid = n < cap ? n : cap;
  tie_map_kernel<<<static_cast<unsigned>(grid), TieLarge::kThreads, sizeof(TieLarge::Smem), s>>>(D, n, map, dm);
  return cudaGetLastError();
}

}  // namespace pald
