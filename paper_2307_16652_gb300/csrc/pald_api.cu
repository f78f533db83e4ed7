// extern "C" entry points of libpald (declared in include/pald.h).
//
// This file holds argument checking, scratch management, validation and
// dispatch; the arithmetic of both passes lives in the kernels.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "pald_internal.cuh"
#include "schedules.cuh"

namespace pald {

// Autotuned tables, generated at build time from tuned_schedules.json (the
// autotuner's output) into the build directory.
struct TunedTable {
  const char* gpu;  // cudaDeviceProp::name
  int sms;          // multiprocessor count
  int count;
  ScheduleBucket buckets[kMaxBuckets];
};
#include "tuned_schedules.inc"  // kTunedTables[], kTunedTableCount

thread_local int32_t g_last_cuda_error = 0;

pald_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = static_cast<int32_t>(e);
  return e == cudaErrorMemoryAllocation ? PALD_ERR_NO_MEMORY : PALD_ERR_CUDA;
}

bool opts_ok(const pald_opts* o) {
  if (!o) return true;
  if ((o->flags & ~PALD_FLAG_IGNORE_TIES) != 0) return false;
  if (o->accum_mode != PALD_ACCUM_COMPENSATED && o->accum_mode != PALD_ACCUM_PLAIN &&
      o->accum_mode != PALD_ACCUM_FIXED)
    return false;
  if (o->schedule_id < -1 || o->schedule_id >= kScheduleCount) return false;
  return true;
}

pald_opts opts_or_default(const pald_opts* o) {
  pald_opts d{0, PALD_ACCUM_COMPENSATED, -1, 0};
  return o ? *o : d;
}

constexpr int64_t kMaxN = int64_t(1) << 20;

// ---------------------------------------------------------------------------
// schedule tables, one per device

namespace {

constexpr int kMaxDevices = 64;

struct DeviceTable {
  bool init = false;
  int source = 0;  // 0 built-in defaults, 1 tuned table of this GPU, 2 set by the caller
  int count = 0;
  ScheduleBucket b[kMaxBuckets];
};

std::mutex g_sched_mu;
DeviceTable g_sched[kMaxDevices];
uint64_t g_sched_gen = 1;

bool bucket_ok(const ScheduleBucket& b) {
  return b.focus >= 0 && b.focus < kScheduleCount && b.cohesion >= 0 && b.cohesion < kScheduleCount &&
         (b.batched_split == 0 || b.batched_split == 1) && b.n_max >= 2;
}

bool table_ok(const ScheduleBucket* b, int count) {
  if (count < 1 || count > kMaxBuckets) return false;
  for (int i = 0; i < count; ++i)
    if (!bucket_ok(b[i]) || (i > 0 && b[i].n_max <= b[i - 1].n_max)) return false;
  return true;
}

// The built-in choice for this device: its tuned table, if one was built in.
void load_builtin(int dev, DeviceTable& t) {
  t = DeviceTable{};
  t.init = true;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return;
  for (int i = 0; i < kTunedTableCount; ++i) {
    const TunedTable& tt = kTunedTables[i];
    if (tt.sms == prop.multiProcessorCount && std::strcmp(tt.gpu, prop.name) == 0 &&
        table_ok(tt.buckets, tt.count)) {
      t.source = 1;
      t.count = tt.count;
      for (int k = 0; k < tt.count; ++k) t.b[k] = tt.buckets[k];
      return;
    }
  }
}

}  // namespace

int schedule_for(int64_t n, ScheduleBucket* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *out = builtin_schedule(n);
    return 0;
  }
  std::lock_guard<std::mutex> lock(g_sched_mu);
  DeviceTable& t = g_sched[dev];
  if (!t.init) load_builtin(dev, t);
  if (t.count == 0) {
    *out = builtin_schedule(n);
    return 0;
  }
  int k = 0;
  while (k + 1 < t.count && n > t.b[k].n_max) ++k;
  *out = t.b[k];
  return t.source;
}

uint64_t schedule_generation() {
  std::lock_guard<std::mutex> lock(g_sched_mu);
  return g_sched_gen;
}

cudaError_t smem_opt_in(const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> done;  // (kernel, device) -> bytes opted in
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(fn, dev);
  const auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

// Maps a scan result (already on the host) to a status.
pald_status status_from_scan(const ScanResult& r) {
  if (r.flags & kFlagAsymmetric) return PALD_ERR_NOT_SYMMETRIC;
  if (r.flags & kFlagBadDiagonal) return PALD_ERR_BAD_DIAGONAL;
  if (r.flags & (kFlagBadValue | kFlagRange)) return PALD_ERR_BAD_VALUE;
  if (r.inv_min_pos_bits != 0u) {
    uint32_t mn = ~r.inv_min_pos_bits, mx = r.max_bits;
    float fmn, fmx;
    std::memcpy(&fmn, &mn, 4);
    std::memcpy(&fmx, &mx, 4);
    if (static_cast<double>(fmx) >= std::ldexp(static_cast<double>(fmn), 100)) return PALD_ERR_BAD_VALUE;
  }
  return PALD_OK;
}

// Runs the scan (and validation when asked) into `scratch`; when validating,
// copies the result back and synchronises the stream.
pald_status scan_and_check(const float* D, int64_t n, ScanResult* scratch, bool validate, cudaStream_t s) {
  cudaError_t e = launch_scan(D, n, scratch, validate, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!validate) return PALD_OK;
  ScanResult host{};
  e = cudaMemcpyAsync(&host, scratch, sizeof host, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  return status_from_scan(host);
}

// Stream-ordered scratch that is released on every exit path.
struct Scratch {
  void* p = nullptr;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

// Pass 2 in fixed point (PALD_ACCUM_FIXED) on tiles [t0, t1) (t1 < 0: all):
// scan, tie map, the integer weight pieces, then the exact tiles.
pald_status cohesion_fixed(const float* D, const int32_t* U, int64_t n, float* C, const pald_opts& o, int64_t t0,
                           int64_t t1, cudaStream_t s) {
  const size_t fbytes = (fixed_scratch_bytes(D, n) + 255) / 256 * 256;
  const size_t tbytes = (static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t) + 255) / 256 * 256;
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(fbytes + tbytes + 256);
  if (e != cudaSuccess) return cuda_fail(e);
  auto* tmap = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch.p) + fbytes);
  auto* scan = reinterpret_cast<ScanResult*>(static_cast<char*>(scratch.p) + fbytes + tbytes);
  const pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if (o.flags & PALD_FLAG_IGNORE_TIES)
    e = cudaMemsetAsync(tmap, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  else
    e = launch_tie_map(D, n, tmap, s);
  if (e == cudaSuccess) e = launch_fixed_cohesion(D, U, n, C, tmap, scan, scratch.p, t0, t1, s);
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

}  // namespace pald

using namespace pald;

extern "C" {

pald_status pald_focus(const float* D, int64_t n, int32_t* U, const pald_opts* opts, pald_stream_t stream) {
  if (!D || !U || n < 2 || n > kMaxN || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(sizeof(ScanResult));
  if (e != cudaSuccess) return cuda_fail(e);
  auto* scan = static_cast<ScanResult*>(scratch.p);
  pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  e = launch_focus(D, n, U, scan, o.schedule_id, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}

pald_status pald_cohesion(const float* D, const int32_t* U, int64_t n, float* C, const pald_opts* opts,
                          pald_stream_t stream) {
  if (!D || !U || !C || n < 2 || n > kMaxN || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.accum_mode == PALD_ACCUM_FIXED) return cohesion_fixed(D, U, n, C, o, 0, -1, s);
  // scratch: R = 1/u (n x n FP32), the tie map, the scan summary
  const size_t rbytes = static_cast<size_t>(n) * static_cast<size_t>(n) * sizeof(float);
  const size_t tbytes = (static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t) + 255) / 256 * 256;
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(rbytes + tbytes + 256);
  if (e != cudaSuccess) return cuda_fail(e);
  float* R = static_cast<float*>(scratch.p);
  auto* tmap = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch.p) + rbytes);
  auto* scan = reinterpret_cast<ScanResult*>(static_cast<char*>(scratch.p) + rbytes + tbytes);
  pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if (o.flags & PALD_FLAG_IGNORE_TIES)  // an empty map: the short (strict) form everywhere
    e = cudaMemsetAsync(tmap, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  else
    e = launch_tie_map(D, n, tmap, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if ((e = launch_cohesion(D, U, R, n, C, tmap, scan, o.accum_mode, o.schedule_id, s)) != cudaSuccess)
    return cuda_fail(e);
  return PALD_OK;
}

pald_status pald_cohesion_depth(const float* D, const int32_t* U, int64_t n, float* C, float* L,
                                const pald_opts* opts, pald_stream_t stream) {
  if (!D || !U || !C || !L || n < 2 || n > kMaxN || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool fused = o.accum_mode != PALD_ACCUM_FIXED && (o.schedule_id < 0 || o.schedule_id == 7) &&
                     cohesion_depth_fused_ok(D, C, n);
  if (!fused) {  // the row sums from a separate pass over C
    const pald_status st = pald_cohesion(D, U, n, C, opts, stream);
    return st == PALD_OK ? pald_local_depth(C, n, L, stream) : st;
  }
  // scratch: R = 1/u, the tie map, the scan summary, the per-tile row sums
  const size_t rbytes = static_cast<size_t>(n) * static_cast<size_t>(n) * sizeof(float);
  const size_t tbytes = (static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t) + 255) / 256 * 256;
  const size_t pbytes = static_cast<size_t>((n + 63) / 64) * static_cast<size_t>(n) * sizeof(double);
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(rbytes + tbytes + pbytes + 256);
  if (e != cudaSuccess) return cuda_fail(e);
  char* base = static_cast<char*>(scratch.p);
  float* R = reinterpret_cast<float*>(base);
  auto* tmap = reinterpret_cast<uint32_t*>(base + rbytes);
  auto* P = reinterpret_cast<double*>(base + rbytes + tbytes);
  auto* scan = reinterpret_cast<ScanResult*>(base + rbytes + tbytes + pbytes);
  pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if (o.flags & PALD_FLAG_IGNORE_TIES)
    e = cudaMemsetAsync(tmap, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  else
    e = launch_tie_map(D, n, tmap, s);
  if (e == cudaSuccess) e = launch_cohesion_depth(D, U, R, n, C, tmap, scan, o.accum_mode, P, s);
  if (e == cudaSuccess) e = launch_depth_merge(P, n, L, s);
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

pald_status pald_validate(const float* D, int64_t n, pald_stream_t stream) {
  if (!D || n < 2 || n > kMaxN) return PALD_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(sizeof(ScanResult));
  if (e != cudaSuccess) return cuda_fail(e);
  return scan_and_check(D, n, static_cast<ScanResult*>(scratch.p), true, s);
}

pald_status pald_host(const float* D_host, int64_t n, int32_t* U_host, float* C_host, const pald_opts* opts) {
  if (!D_host || !U_host || !C_host || n < 2 || n > kMaxN || !opts_ok(opts)) return PALD_ERR_INVALID_ARG;
  const size_t bytes = static_cast<size_t>(n) * static_cast<size_t>(n) * 4u;
  // s runs the passes; s2 copies U back while pass 2 runs (pass 2 only reads U)
  cudaStream_t s = nullptr, s2 = nullptr;
  cudaEvent_t u_ready = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&u_ready, cudaEventDisableTiming);
  float* dD = nullptr;
  int32_t* dU = nullptr;
  float* dC = nullptr;
  pald_status st = PALD_OK;
  bool u_copy_issued = false;
  while (e == cudaSuccess) {
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&dD), bytes, s)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&dU), bytes, s)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&dC), bytes, s)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(dD, D_host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
    st = pald_focus(dD, n, dU, opts, reinterpret_cast<pald_stream_t>(s));
    if (st != PALD_OK) break;
    if ((e = cudaEventRecord(u_ready, s)) != cudaSuccess) break;
    if ((e = cudaStreamWaitEvent(s2, u_ready, 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(U_host, dU, bytes, cudaMemcpyDeviceToHost, s2)) != cudaSuccess) break;
    u_copy_issued = true;
    pald_opts o2 = opts_or_default(opts);
    o2.validate = 0;  // already checked by pass 1 when asked
    st = pald_cohesion(dD, dU, n, dC, &o2, reinterpret_cast<pald_stream_t>(s));
    if (st != PALD_OK) break;
    if ((e = cudaMemcpyAsync(C_host, dC, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    break;
  }
  // U's buffer is freed only after its copy: order the frees after s2
  cudaError_t e3 = cudaSuccess;
  if (u_copy_issued) {
    e3 = cudaEventRecord(u_ready, s2);
    if (e3 == cudaSuccess) e3 = cudaStreamWaitEvent(s, u_ready, 0);
  }
  if (dD) cudaFreeAsync(dD, s);
  if (dU) cudaFreeAsync(dU, s);
  if (dC) cudaFreeAsync(dC, s);
  cudaError_t e2 = s ? cudaStreamSynchronize(s) : cudaSuccess;
  if (s2) {
    cudaError_t e4 = cudaStreamSynchronize(s2);
    if (e2 == cudaSuccess) e2 = e4;
    cudaStreamDestroy(s2);
  }
  if (u_ready) cudaEventDestroy(u_ready);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (st != PALD_OK) return st;
  if (e3 != cudaSuccess) return cuda_fail(e3);
  if (e2 != cudaSuccess) return cuda_fail(e2);
  return PALD_OK;
}

int64_t pald_tie_map_words(int64_t n) { return (n < 2 || n > kMaxN) ? 0 : tie_map_words(n); }

pald_status pald_tie_map(const float* D, int64_t n, uint32_t* map, pald_stream_t stream) {
  if (!D || !map || n < 2 || n > kMaxN) return PALD_ERR_INVALID_ARG;
  cudaError_t e = launch_tie_map(D, n, map, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

pald_status pald_check_faults(pald_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t f1 = 0, f2 = 0, f3 = 0, f4 = 0, f5 = 0;
  cudaError_t e = take_focus_faults(&f1, s);
  if (e == cudaSuccess) e = take_cohesion_faults(&f2, s);
  if (e == cudaSuccess) e = take_batched_faults(&f3, s);
  if (e == cudaSuccess) e = take_pairwise_faults(&f4, s);
  if (e == cudaSuccess) e = take_fixed_faults(&f5, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return (f1 | f2 | f3 | f4 | f5) ? PALD_ERR_TIMEOUT : PALD_OK;
}

pald_status pald_test_bounded_wait(int64_t limit_ns, pald_stream_t stream) {
  if (limit_ns < 1000 || limit_ns > static_cast<int64_t>(kWaitLimitNs)) return PALD_ERR_INVALID_ARG;
  const cudaError_t e = launch_wait_selftest(static_cast<uint64_t>(limit_ns), reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

pald_status pald_set_schedule_table(const pald_schedule_bucket* buckets, int32_t count) {
  if (count < 0 || count > kMaxBuckets || (count > 0 && !buckets)) return PALD_ERR_INVALID_ARG;
  ScheduleBucket b[kMaxBuckets];
  for (int i = 0; i < count; ++i) {
    if (buckets[i].reserved != 0) return PALD_ERR_INVALID_ARG;
    b[i] = ScheduleBucket{buckets[i].n_max, buckets[i].focus, buckets[i].cohesion, buckets[i].batched_split};
  }
  if (count > 0 && !table_ok(b, count)) return PALD_ERR_INVALID_ARG;
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return PALD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_sched_mu);
  DeviceTable& t = g_sched[dev];
  if (count == 0) {
    load_builtin(dev, t);
  } else {
    t.init = true;
    t.source = 2;
    t.count = count;
    for (int i = 0; i < count; ++i) t.b[i] = b[i];
  }
  ++g_sched_gen;
  return PALD_OK;
}

pald_status pald_get_schedule(int64_t n, pald_schedule_bucket* out, int32_t* source) {
  if (!out || n < 2 || n > kMaxN) return PALD_ERR_INVALID_ARG;
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  ScheduleBucket b;
  const int src = schedule_for(n, &b);
  *out = pald_schedule_bucket{b.n_max, b.focus, b.cohesion, b.batched_split, 0};
  if (source) *source = src;
  return PALD_OK;
}

int32_t pald_schedule_count(void) { return kScheduleCount; }

const char* pald_schedule_name(int32_t id) {
  switch (id) {
    case 0: return "focus 64x64 tile, 4x4 pairs/thread, 16-deep stages | cohesion 64x64, 4x4, 16-deep";
    case 1: return "focus 32x32 tile, 4x4 pairs/thread | cohesion 32x32, 4x4 (small matrices)";
    case 2: return "focus 64x64 tile, 4x4, 32-deep stages | cohesion 64x32 slices, 4x2 pairs/thread, 16-deep";
    case 3: return "focus 128x64 slices, 8x4 pairs/thread | cohesion 64x64, 4x4, 32-deep stages";
    case 4: return "focus 64x32 slices, 4x4, 32-deep | cohesion 64x32 slices, 4x2, 32-deep";
    case 5: return "focus 64x64, 4x4, 64-deep stages unrolled 16 | cohesion 64x64, 4x4, 32-deep unrolled 4";
    case 6: return "focus 128x64 slices, 8x4, 32-deep | cohesion 64x64, 4x4, 64-deep unrolled 8";
    case 7:
      return "focus 64x64, 4x4, 32-deep, TMA-staged, 3 CTAs/SM | cohesion 64x64, 4x4, 32-deep, TMA-staged, "
             "2 CTAs/SM (both need n % 4 == 0, else the same tile with per-thread copies)";
    default: return nullptr;
  }
}

const char* pald_status_string(pald_status status) {
  switch (status) {
    case PALD_OK: return "ok";
    case PALD_ERR_INVALID_ARG: return "invalid argument";
    case PALD_ERR_NOT_SYMMETRIC: return "distance matrix is not exactly symmetric";
    case PALD_ERR_BAD_DIAGONAL: return "distance matrix diagonal is not +0.0";
    case PALD_ERR_BAD_VALUE: return "distance matrix has a NaN, infinite, negative, -0.0 or out-of-range entry";
    case PALD_ERR_CUDA: return "CUDA runtime error";
    case PALD_ERR_NO_MEMORY: return "out of device memory";
    case PALD_ERR_TIMEOUT: return "device-side wait timed out";
    case PALD_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

int32_t pald_last_cuda_error(void) { return g_last_cuda_error; }

int32_t pald_version(void) { return 100; }

}  // extern "C"
