// After the two passes: local depths (the row sums of C, Sec. 2: the
// cohesion of x partitions its local depth, eq. (LD)) and the mask of
// strong ties for a given threshold (Sec. 2, Sec. 7).  Both are O(n^2)
// sweeps over C, bound by HBM.
#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

pald_status cuda_fail(cudaError_t e);

namespace {

constexpr int kDepthThreads = 256;

// Two-float running sum: (s, e) += v exactly up to the final rounding.
__device__ __forceinline__ void add_two(float& s, float& e, float v) {
  float t, r;
  two_sum(s, v, t, r);
  s = t;
  e = __fadd_rn(e, r);
}

// One CTA per row (strided): each thread sums a fixed strided subset of the
// row in two-float arithmetic, then the CTA combines the partials in a fixed
// tree order, so the result does not depend on timing.
__global__ void __launch_bounds__(kDepthThreads) local_depth_kernel(const float* __restrict__ C, int64_t n,
                                                                   float* __restrict__ L) {
  __shared__ float ss[kDepthThreads], se[kDepthThreads];
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
    const float* c = C + row * n;
    float s = 0.f, e = 0.f;
    for (int64_t k = threadIdx.x; k < n; k += kDepthThreads) add_two(s, e, __ldg(c + k));
    ss[threadIdx.x] = s;
    se[threadIdx.x] = e;
    __syncthreads();
    for (int w = kDepthThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        float a = ss[threadIdx.x], ae = se[threadIdx.x];
        add_two(a, ae, ss[threadIdx.x + w]);
        ae = __fadd_rn(ae, se[threadIdx.x + w]);
        ss[threadIdx.x] = a;
        se[threadIdx.x] = ae;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) L[row] = __fadd_rn(ss[0], se[0]);
    __syncthreads();  // ss/se are reused by the next row
  }
}

// The fused local depth's last step: L[x] = the sum over column blocks b
// (in order) of P[b * n + x], rounded once to FP32.  One thread per row;
// the threads of a warp read consecutive rows of one block.
__global__ void __launch_bounds__(kDepthThreads) depth_merge_kernel(const double* __restrict__ P, int64_t n,
                                                                   int64_t nb, float* __restrict__ L) {
  const int64_t x = static_cast<int64_t>(blockIdx.x) * kDepthThreads + threadIdx.x;
  if (x >= n) return;
  double s = 0.0;
  for (int64_t b = 0; b < nb; ++b) s += __ldg(P + b * n + x);
  L[x] = static_cast<float>(s);
}

__global__ void __launch_bounds__(256) strong_ties_kernel(const float* __restrict__ C, int64_t elems,
                                                          float threshold, uint8_t* __restrict__ T) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < elems;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    T[i] = __ldg(C + i) >= threshold ? 1u : 0u;
}

}  // namespace

cudaError_t launch_depth_merge(const double* P, int64_t n, float* L, cudaStream_t s) {
  const int64_t nb = (n + 63) / 64;
  depth_merge_kernel<<<static_cast<unsigned>((n + kDepthThreads - 1) / kDepthThreads), kDepthThreads, 0, s>>>(P, n, nb,
                                                                                                           L);
  return cudaGetLastError();
}

}  // namespace pald

using namespace pald;

extern "C" {

pald_status pald_local_depth(const float* C, int64_t n, float* L, pald_stream_t stream) {
  if (!C || !L || n < 2 || n > (int64_t(1) << 20)) return PALD_ERR_INVALID_ARG;
  const int64_t cap = int64_t(sm_count()) * 8;
  local_depth_kernel<<<static_cast<unsigned>(n < cap ? n : cap), kDepthThreads, 0,
                       reinterpret_cast<cudaStream_t>(stream)>>>(C, n, L);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

pald_status pald_strong_ties(const float* C, int64_t n, float threshold, uint8_t* T, pald_stream_t stream) {
  if (!C || !T || n < 2 || n > (int64_t(1) << 20) || !(threshold == threshold)) return PALD_ERR_INVALID_ARG;
  const int64_t elems = n * n;
  const int64_t blocks = (elems + 255) / 256, cap = int64_t(sm_count()) * 32;
  strong_ties_kernel<<<static_cast<unsigned>(blocks < cap ? blocks : cap), 256, 0,
                       reinterpret_cast<cudaStream_t>(stream)>>>(C, elems, threshold, T);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

}  // extern "C"
