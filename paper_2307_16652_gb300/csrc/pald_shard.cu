// Sharding one matrix over several GPUs (one process per GPU).
//
// The triplet blocks of the method are independent given D (Sec. 3.2, the
// blocked triplet algorithm), so both passes split over the 64 x 64
// upper-triangle super-tiles (bi <= bj) in the launch order of decode_tile:
// every rank takes one contiguous range of tiles.  Pass 1 on a range writes
// u for the tile's pairs and their mirror images; pass 2 needs all of u, so
// between the passes each rank packs its tiles of U, the ranks all-gather
// the packed buffers once (a plain collective of the caller's choice: no
// device-side waiting on other GPUs here), and every rank unpacks all of
// them.  Pass 2 on the same range then writes C[X, Z] and C[Z, X] of its
// tiles; C can be gathered the same way (both blocks of each tile).
//
// The pack layout: tile t of the range occupies 4096 words (block [X, Y],
// 64 rows of 64 words, zero outside the matrix), or 8192 with `both` (then
// block [Y, X] after it).
#include "cohesion_core.cuh"
#include "schedules.cuh"

namespace pald {

pald_status cuda_fail(cudaError_t e);
bool opts_ok(const pald_opts* o);
pald_opts opts_or_default(const pald_opts* o);
pald_status scan_and_check(const float* D, int64_t n, ScanResult* scratch, bool validate, cudaStream_t s);
pald_status cohesion_fixed(const float* D, const int32_t* U, int64_t n, float* C, const pald_opts& o, int64_t t0,
                           int64_t t1, cudaStream_t s);

namespace {

constexpr int64_t kMaxN = int64_t(1) << 20;
constexpr int kShardB = 64;
constexpr int kPackThreads = 256;

int64_t tiles_of(int64_t n) {
  const int64_t T = (n + kShardB - 1) / kShardB;
  return T * (T + 1) / 2;
}

bool range_ok(int64_t n, int64_t t0, int64_t t1) { return 0 <= t0 && t0 <= t1 && t1 <= tiles_of(n); }

// One CTA per tile of the range.  Block [X, Y] row by row (coalesced 64-word
// row segments); with `both` also block [Y, X].
__global__ void __launch_bounds__(kPackThreads) pack_tiles_kernel(const uint32_t* __restrict__ M, int64_t n,
                                                                  int64_t T, int64_t t0, int both,
                                                                  uint32_t* __restrict__ out) {
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0, T, 1, &bi, &bj, &slice);
  const int halves = both ? 2 : 1;
  uint32_t* dst = out + static_cast<int64_t>(blockIdx.x) * 4096 * halves;
  for (int h = 0; h < halves; ++h) {
    const int64_t r0 = int64_t(h == 0 ? bi : bj) * kShardB, c0 = int64_t(h == 0 ? bj : bi) * kShardB;
    for (int k = threadIdx.x; k < 4096; k += kPackThreads) {
      const int64_t r = r0 + k / 64, c = c0 + k % 64;
      dst[h * 4096 + k] = (r < n && c < n) ? __ldg(M + r * n + c) : 0u;
    }
  }
}

// The inverse: block [X, Y] back in place; without `both` its transpose goes
// to [Y, X] (a symmetric matrix such as U), through shared memory so that
// both writes are row segments.
__global__ void __launch_bounds__(kPackThreads) unpack_tiles_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                    int64_t T, int64_t t0, int both,
                                                                    uint32_t* __restrict__ M) {
  __shared__ uint32_t tile[64][65];
  int bi, bj, slice;
  decode_tile(blockIdx.x + t0, T, 1, &bi, &bj, &slice);
  const uint32_t* src = in + static_cast<int64_t>(blockIdx.x) * 4096 * (both ? 2 : 1);
  const int64_t X0 = int64_t(bi) * kShardB, Y0 = int64_t(bj) * kShardB;
  for (int k = threadIdx.x; k < 4096; k += kPackThreads) {
    const int i = k / 64, j = k % 64;
    const uint32_t v = src[k];
    tile[i][j] = v;
    if (X0 + i < n && Y0 + j < n) M[(X0 + i) * n + Y0 + j] = v;
  }
  if (both) {
    for (int k = threadIdx.x; k < 4096; k += kPackThreads) {
      const int i = k / 64, j = k % 64;
      if (Y0 + i < n && X0 + j < n) M[(Y0 + i) * n + X0 + j] = src[4096 + k];
    }
    return;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 4096; k += kPackThreads) {
    const int i = k / 64, j = k % 64;  // row Y0 + i, column X0 + j of the mirror
    if (Y0 + i < n && X0 + j < n) M[(Y0 + i) * n + X0 + j] = tile[j][i];
  }
}

// Stream-ordered scratch released on every exit path.
struct Scratch {
  void* p = nullptr;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, bytes, s); }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace

}  // namespace pald

using namespace pald;

extern "C" {

int64_t pald_shard_tiles(int64_t n) { return (n < 2 || n > kMaxN) ? 0 : tiles_of(n); }

pald_status pald_shard_range(int64_t n, int32_t rank, int32_t world, int64_t* t0, int64_t* t1) {
  if (n < 2 || n > kMaxN || world < 1 || rank < 0 || rank >= world || !t0 || !t1) return PALD_ERR_INVALID_ARG;
  const int64_t N = tiles_of(n);
  *t0 = N * rank / world;
  *t1 = N * (rank + 1) / world;
  return PALD_OK;
}

pald_status pald_focus_tiles(const float* D, int64_t n, int64_t t0, int64_t t1, int32_t* U, const pald_opts* opts,
                             pald_stream_t stream) {
  if (!D || !U || n < 2 || n > kMaxN || !opts_ok(opts) || !range_ok(n, t0, t1)) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(sizeof(ScanResult));
  if (e != cudaSuccess) return cuda_fail(e);
  auto* scan = static_cast<ScanResult*>(scratch.p);
  const pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if ((e = launch_focus_range(D, n, U, scan, t0, t1, s)) != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}

pald_status pald_cohesion_tiles(const float* D, const int32_t* U, int64_t n, int64_t t0, int64_t t1, float* C,
                                const pald_opts* opts, pald_stream_t stream) {
  if (!D || !U || !C || n < 2 || n > kMaxN || !opts_ok(opts) || !range_ok(n, t0, t1)) return PALD_ERR_INVALID_ARG;
  const pald_opts o = opts_or_default(opts);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.accum_mode == PALD_ACCUM_FIXED) return cohesion_fixed(D, U, n, C, o, t0, t1, s);
  const size_t rbytes = static_cast<size_t>(n) * static_cast<size_t>(n) * sizeof(float);
  const size_t tbytes = (static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t) + 255) / 256 * 256;
  Scratch scratch(s);
  cudaError_t e = scratch.alloc(rbytes + tbytes + 256);
  if (e != cudaSuccess) return cuda_fail(e);
  float* R = static_cast<float*>(scratch.p);
  auto* tmap = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch.p) + rbytes);
  auto* scan = reinterpret_cast<ScanResult*>(static_cast<char*>(scratch.p) + rbytes + tbytes);
  const pald_status st = scan_and_check(D, n, scan, o.validate != 0, s);
  if (st != PALD_OK) return st;
  if (o.flags & PALD_FLAG_IGNORE_TIES)
    e = cudaMemsetAsync(tmap, 0, static_cast<size_t>(tie_map_words(n)) * sizeof(uint32_t), s);
  else
    e = launch_tie_map(D, n, tmap, s);
  if (e == cudaSuccess) e = launch_cohesion_range(D, U, R, n, C, tmap, scan, o.accum_mode, t0, t1, s);
  if (e != cudaSuccess) return cuda_fail(e);
  return PALD_OK;
}

pald_status pald_pack_tiles(const void* M, int64_t n, int64_t t0, int64_t t1, int32_t both, void* packed,
                            pald_stream_t stream) {
  if (!M || !packed || n < 2 || n > kMaxN || (both != 0 && both != 1) || !range_ok(n, t0, t1))
    return PALD_ERR_INVALID_ARG;
  if (t1 == t0) return PALD_OK;
  const int64_t T = (n + kShardB - 1) / kShardB;
  pack_tiles_kernel<<<static_cast<unsigned>(t1 - t0), kPackThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      static_cast<const uint32_t*>(M), n, T, t0, both, static_cast<uint32_t*>(packed));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

pald_status pald_unpack_tiles(const void* packed, int64_t n, int64_t t0, int64_t t1, int32_t both, void* M,
                              pald_stream_t stream) {
  if (!M || !packed || n < 2 || n > kMaxN || (both != 0 && both != 1) || !range_ok(n, t0, t1))
    return PALD_ERR_INVALID_ARG;
  if (t1 == t0) return PALD_OK;
  const int64_t T = (n + kShardB - 1) / kShardB;
  unpack_tiles_kernel<<<static_cast<unsigned>(t1 - t0), kPackThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      static_cast<const uint32_t*>(packed), n, T, t0, both, static_cast<uint32_t*>(M));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PALD_OK : cuda_fail(e);
}

}  // extern "C"
