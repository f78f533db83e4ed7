// pald_cohesion_noalloc: pass 2 without any device allocation.
//
// Some callers cannot let a library call cudaMalloc or cudaMallocAsync: an
// application whose device memory is already handed out by its own pool (an
// extra allocation would fail or fragment it), a latency-critical loop that
// cannot afford the implicit synchronisation an allocation may cause, or a
// program that allocates nothing after start-up by policy.  For them the R =
// 1/u scratch of pass 2 lives in a fixed array that is part of the library
// image: every GPU that loads the library holds it (16 MiB + 256 bytes)
// until the process exits, and matrices are limited to n <= 2048.
//
// The kernels are the ones pald_cohesion uses; only the scratch differs, and
// without room for a tie map every stage runs the long form of the inner
// loop (identical results, slower).
#include <mutex>

#include "pald_internal.cuh"

namespace pald {

pald_status cuda_fail(cudaError_t e);
bool opts_ok(const pald_opts* o);
pald_opts opts_or_default(const pald_opts* o);
pald_status status_from_scan(const ScanResult& r);

namespace {

constexpr int64_t kNoAllocMaxN = 2048;
constexpr size_t kNoAllocRFloats = static_cast<size_t>(kNoAllocMaxN) * kNoAllocMaxN;  // R, 16 MiB
constexpr size_t kNoAllocFloats = kNoAllocRFloats + 64;  // + one ScanResult (validation), padded

// The scratch: R first, the validation summary after it.  In host code this
// name is only a stand-in for the symbol, never a device address.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of the array, per device

// Device address of the array on the current device (looked up once).
pald_status scratch_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return PALD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    g_scratch_dev[dev] = p;
  }
  *out = static_cast<float*>(g_scratch_dev[dev]);
  return PALD_OK;
}

}  // namespace

}  // namespace pald

using namespace pald;

extern "C" pald_status pald_cohesion_noalloc(const float* D, const int32_t* U, int64_t n, float* C,
                                             const pald_opts* opts, pald_stream_t stream) {
  if (!D || !U || !C || n < 2 || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  if (opts && (opts->flags & PALD_FLAG_IGNORE_TIES)) return PALD_ERR_INVALID_ARG;  // needs a tie map
  if (opts && opts->accum_mode == PALD_ACCUM_FIXED) return PALD_ERR_INVALID_ARG;    // needs two weight arrays
  if (n > kNoAllocMaxN) return PALD_ERR_UNSUPPORTED;  // R would not fit the fixed array
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* R = nullptr;
  pald_status st = scratch_address(&R);
  if (st != PALD_OK) return st;
  // the scan summary (pass-1 scale, and validation when asked) sits after R;
  // launch_scan clears it before scanning
  auto* scan = reinterpret_cast<ScanResult*>(R + kNoAllocRFloats);
  cudaError_t e = launch_scan(D, n, scan, o.validate != 0, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (o.validate) {
    ScanResult host{};
    e = cudaMemcpyAsync(&host, scan, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((st = status_from_scan(host)) != PALD_OK) return st;
  }
  // R is written in full (every entry of the n x n block, inside
  // launch_cohesion) before it is read, so nothing left by an earlier call
  // leaks into this one.  No tie map (it would need scratch): every stage
  // takes the long form, which gives the same bits as pald_cohesion's mix of
  // forms.
  e = launch_cohesion(D, U, R, n, C, nullptr, scan, o.accum_mode, o.schedule_id, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}
