/*
 * pald.h - C ABI of libpald: the two O(n^3) triplet passes of partitioned
 * local depths (PaLD) on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: Devarakonda & Ballard, "Sequential and Shared-Memory Parallel
 * Algorithms for Partitioned Local Depths".  For an n x n distance matrix D:
 *
 *   pass 1  local focus sizes (Sec. 2 definition of the local focus):
 *           u_xy = #{ z : d_xz <= d_xy  or  d_yz <= d_xy },  every x, y;
 *   pass 2  cohesion (Sec. 2, eq. (cohesion) written out as eq. (fxz), with
 *           the half-credit tie split of Sec. 5):
 *           c_xz = 1/(n-1) * sum_{y != x} [z in U_xy] * w(d_zx, d_zy) / u_xy,
 *           w(p, q) = 1 if p < q, 1/2 if p == q, 0 if p > q.
 *
 * Conventions shared by every entry point
 *   - Matrices are dense, row-major, n x n, element (i, j) at index i*n + j,
 *     and live in device memory that the CALLER allocated and owns (unless an
 *     entry point says "host").  The library never frees caller memory.
 *   - Input contract for D (checked only when pald_opts.validate != 0 or by
 *     pald_validate): exactly symmetric bit for bit, +0.0 on the diagonal,
 *     every entry finite and >= +0.0 (no NaN, no negative value, no -0.0),
 *     every positive entry >= 2^-100, and (largest entry) / (smallest positive
 *     entry) < 2^100.  PaLD only compares distances, so a matrix outside the
 *     last two limits can be rescaled by a power of two without changing u or
 *     C.  Results for inputs that break the contract are unspecified.
 *   - Calls are asynchronous and ordered on `stream` (NULL = the legacy
 *     default stream), except that validation copies one small status word to
 *     the host and synchronises `stream`.
 *   - Scratch memory that a call needs is taken with cudaMallocAsync on
 *     `stream` and released on the same stream before the call returns
 *     (pald_cohesion_noalloc and pald_batched's cached plans are the
 *     exceptions, described with them).
 *   - Every function returns a status and never aborts, traps or prints.
 *     On any error the contents of the outputs are unspecified.
 */
#ifndef PALD_H
#define PALD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, so callers can pass a CUDA stream directly. */
typedef struct CUstream_st* pald_stream_t;

typedef enum pald_status {
  PALD_OK = 0,
  PALD_ERR_INVALID_ARG = 1,    /* null pointer, n < 2, bad count/offset, bad opts */
  PALD_ERR_NOT_SYMMETRIC = 2,  /* validation: d_ij and d_ji differ in some bit */
  PALD_ERR_BAD_DIAGONAL = 3,   /* validation: a diagonal entry is not +0.0 */
  PALD_ERR_BAD_VALUE = 4,      /* validation: NaN, inf, negative, -0.0, or out of range */
  PALD_ERR_CUDA = 5,           /* a CUDA runtime call failed (see pald_last_cuda_error) */
  PALD_ERR_NO_MEMORY = 6,      /* scratch allocation failed */
  PALD_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up (pald_check_faults) */
  PALD_ERR_UNSUPPORTED = 8     /* size beyond what this build handles */
} pald_status;

/* Accumulation of the cohesion sums (pass 2). */
enum {
  /* FP32 partial sums over 8 consecutive y, folded into an FP32 running sum
   * (biased so that Fast2Sum is error-free) whose exact error is carried into
   * the next partial; the final merge and the 1/(n-1) normalisation are
   * exact two-float arithmetic with one rounding to FP32 (the precision of an
   * FP64 merge) (default). */
  PALD_ACCUM_COMPENSATED = 0,
  /* one FP32 running sum per entry (precision baseline), normalised the same way */
  PALD_ACCUM_PLAIN = 1,
  /* exact fixed-point sums (deterministic whatever the order of the terms):
   * each 1/u_xy becomes the integer round(2^40 / u_xy), the half credits are
   * kept exact, the sum over y is an exact integer, and one FP64 scaling by
   * 2^-41 / (n-1) and one rounding give c_xz.  Relative error at most
   * max(u) / 2^41 (3e-8 at n = 65536).  Permuting the points permutes C bit
   * for bit.  Slower than the compensated mode (one CTA per SM, two weight
   * arrays of n x n floats as scratch); pald_batched runs it matrix by matrix
   * through the single-matrix path; pald_pairwise and pald_cohesion_noalloc
   * do not take it (INVALID_ARG). */
  PALD_ACCUM_FIXED = 2
};

/* Bits of pald_opts.flags. */
enum {
  /* Pass 2 credits z to x only when d_xz < min(d_xy, d_zy): no half credit,
   * no credit on a tie, as the paper's optimised codes do (Sec. 5).  INEXACT
   * unless no row of D holds the same value twice; it skips the tie map and
   * runs the short inner loop everywhere.  Pass 1 is unaffected (exact). */
  PALD_FLAG_IGNORE_TIES = 1
};

typedef struct pald_opts {
  int32_t validate;     /* nonzero: check the input contract before computing */
  int32_t accum_mode;   /* PALD_ACCUM_COMPENSATED, PALD_ACCUM_PLAIN or PALD_ACCUM_FIXED */
  int32_t schedule_id;  /* -1 = automatic tile schedule; >= 0 forces one (pald_schedule_name) */
  int32_t flags;        /* 0 (exact, the default) or PALD_FLAG_IGNORE_TIES; other bits must be 0 */
} pald_opts;          /* a NULL opts pointer means {0, PALD_ACCUM_COMPENSATED, -1, 0} */

/*
 * pald_focus - pass 1, local focus sizes (Sec. 2, the definition of U_xy;
 * computed pair by pair like the pairwise algorithm of Sec. 3.1, blocked over
 * x, y and z like Sec. 3.2).
 *   D  device, n x n FP32, the input contract above.
 *   n  order of the matrix, 2 <= n <= 2^20 (n*n elements addressable).
 *   U  device, n x n int32, written completely: U[x*n+y] = u_xy, including the
 *      diagonal u_xx = #{z : d_xz <= 0}.  U is symmetric.
 * Errors: INVALID_ARG (null pointer, n out of range, bad opts); validation
 * errors; CUDA; NO_MEMORY.
 */
pald_status pald_focus(const float* D, int64_t n, int32_t* U,
                       const pald_opts* opts, pald_stream_t stream);

/*
 * pald_cohesion - pass 2, the cohesion matrix (Sec. 2 eq. (cohesion) in the
 * form of eq. (fxz), ties split per Sec. 5, normalised by 1/(n-1)).
 *   D  device, n x n FP32 (the same matrix pald_focus saw).
 *   U  device, n x n int32 focus sizes as written by pald_focus (a saved U
 *      can be passed back to resume after pass 1); only u_xy for x != y is
 *      read.  Each such entry must be in [2, n].
 *   C  device, n x n FP32, written completely: C[x*n+z] = c_xz.
 * Errors: as pald_focus.
 */
pald_status pald_cohesion(const float* D, const int32_t* U, int64_t n, float* C,
                          const pald_opts* opts, pald_stream_t stream);

/*
 * pald_cohesion_depth - pass 2 with the local depths fused into its
 * epilogue (Sec. 2: the cohesion of x partitions its local depth, eq. (LD),
 * so l_x is the sum of row x of C).
 *   D, U, C, opts  as pald_cohesion; C receives the same bits.
 *   L  device, n FP32, written completely: L[x] = sum over z of c_xz, the
 *      sum of the stored FP32 entries of row x of C.
 * Each 64 x 64 tile sums, in a fixed order and in FP64, the entries it
 * stores into a per-tile partial (scratch of 8 * n * ceil(n / 64) bytes); a
 * last kernel adds each row's partials in block order and rounds once to
 * FP32.  The result does not depend on timing.  This needs the TMA layout
 * (n % 4 == 0, n >= 64, D and C 16-byte aligned), an automatic schedule or
 * schedule 7 and a floating-point accum_mode; otherwise L comes from
 * pald_local_depth on C after pald_cohesion (the same sum up to the last
 * rounding).
 * Errors: as pald_cohesion; INVALID_ARG also for a null L.
 */
pald_status pald_cohesion_depth(const float* D, const int32_t* U, int64_t n, float* C, float* L,
                                const pald_opts* opts, pald_stream_t stream);

/*
 * pald_batched - both passes for `count` independent matrices of uneven order
 * in one persistent launch per pass, replayed from a cached CUDA graph.
 *   count     number of matrices, 1 <= count <= 2^20.
 *   n_host    host array [count], orders n_i with 2 <= n_i <= 4096.
 *   off_host  host array [count], element offset of matrix i in D, U and C;
 *             each a multiple of 4 (16-byte aligned); the regions
 *             [off_i, off_i + n_i^2) must not overlap.
 *   D         device FP32, matrix i is n_i x n_i row-major at D + off_i.
 *   U         device int32, same layout as D; receives u for every matrix.
 *   C         device FP32, same layout as D; receives C for every matrix.
 * The first call for a given (count, n, off, D, U, C, opts) builds a work
 * plan and a CUDA graph (host work; it synchronises `stream` and then the
 * device, once its uploads are queued); later calls with the same arguments
 * only launch the graph.  A plan holds device memory of about twice the
 * packed D (row-padded copies of D and of R = 1/u, whose 16-byte row pitch
 * the TMA copies need) until pald_release() frees it.  At most 16 plans are
 * kept: building a 17th first frees the least recently used one (after its
 * last replay has finished).  The cache is keyed on the buffer addresses, so
 * callers should reuse their D, U and C buffers between calls.
 * Replays of one plan share its scratch; each replay waits (on the GPU) for
 * the previous replay of the same plan, whatever stream either was issued
 * on, so overlapping calls with the same arguments are safe.  Inside a
 * stream capture that wait is left out and the caller's graph must order
 * such calls.
 * Errors: INVALID_ARG (bad count, n_i, misaligned or overlapping offsets);
 * validation errors; CUDA; NO_MEMORY.
 */
pald_status pald_batched(int32_t count, const int64_t* n_host, const int64_t* off_host,
                         const float* D, int32_t* U, float* C,
                         const pald_opts* opts, pald_stream_t stream);

/*
 * pald_host - convenience call on HOST buffers: copies D to the device, runs
 * both passes, copies U and C back, and synchronises.  U's copy back runs on
 * a second stream while pass 2 computes.  Device buffers are allocated and
 * freed inside the call.  Pinned host memory makes the copies faster and
 * lets U's copy overlap pass 2, but is not required.
 *   D_host  host n x n FP32; U_host host n x n int32; C_host host n x n FP32.
 * Errors: as pald_focus and pald_cohesion.
 */
pald_status pald_host(const float* D_host, int64_t n, int32_t* U_host, float* C_host,
                      const pald_opts* opts);

/*
 * pald_pairwise - both passes for matrices too large to also hold u (the
 * pairwise algorithm of Sec. 3.1, Alg. 1, blocked by strips of rows): for
 * each strip of 256 rows x, the focus sizes u_xy of the strip's pairs (x, all
 * y) are counted and kept only as 1/u in a strip buffer (256 x n floats),
 * and the strip's rows of C are written from it.  Each pair's u is counted
 * once per orientation, so it does about twice the work of pald_focus +
 * pald_cohesion, but device memory holds only D, C and its scratch
 * (pald_pairwise_scratch_bytes(n): the strip buffer, the tie map and, when
 * n % 4 != 0, a row-padded copy of D) instead of D, U, C and an n x n R.
 * C is bit for bit the C of pald_focus + pald_cohesion.
 *   D  device, n x n FP32 (the input contract above), 16-byte aligned.
 *   C  device, n x n FP32, 16-byte aligned, written completely.
 *   opts  as pald_cohesion (validate, accum_mode, flags); schedule_id is ignored.
 * Scratch is taken with cudaMallocAsync on `stream`.
 * Errors: INVALID_ARG (null or misaligned pointer, n out of range, bad
 * opts); validation errors; CUDA; NO_MEMORY.
 */
pald_status pald_pairwise(const float* D, int64_t n, float* C, const pald_opts* opts, pald_stream_t stream);

/* Device scratch bytes pald_pairwise takes for order n (0 if out of range). */
int64_t pald_pairwise_scratch_bytes(int64_t n);

/*
 * pald_cohesion_noalloc - pass 2 for callers that must not allocate device
 * memory.  (The paper has no counterpart: this is a deployment variant.)
 * It computes exactly what pald_cohesion computes, with the same kernels,
 * but it never calls cudaMalloc, cudaMallocAsync, cudaFree or any other
 * allocating routine.  Its scratch (R = 1/u) is a fixed array built into the
 * library, 16 MiB + 256 bytes, which every GPU that loads the library holds
 * until the process exits.
 *   D, U, n, C, opts, stream  as pald_cohesion, with 2 <= n <= 2048;
 *   PALD_FLAG_IGNORE_TIES is not supported here (INVALID_ARG).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * begins.  Every call on a device shares the one array and overwrites it:
 * calls whose GPU work overlaps in time (different streams, or different host
 * threads on the same device) race on it and must be serialised by the
 * caller, for example by issuing them on one stream.
 * Errors: UNSUPPORTED for n > 2048 (the array is too small); otherwise as
 * pald_cohesion.
 */
pald_status pald_cohesion_noalloc(const float* D, const int32_t* U, int64_t n, float* C,
                                  const pald_opts* opts, pald_stream_t stream);

/*
 * Sharding one matrix over several GPUs, one process per GPU (Sec. 3.2: the
 * triplet blocks are independent given D).  The units are the 64 x 64
 * upper-triangle super-tiles (bi <= bj) of the matrix in a fixed order;
 * each rank takes a contiguous range [t0, t1) of them (pald_shard_range).
 * A run on N ranks:
 *   1. pald_focus_tiles on the rank's range (U needs no initialisation);
 *   2. pald_pack_tiles(U, ..., both = 0) of the range into a buffer of
 *      4096 words per tile; the caller all-gathers the ranks' buffers once
 *      (e.g. NCCL) and calls pald_unpack_tiles(..., both = 0) for every
 *      rank's range, which completes U (each tile also fills its mirror);
 *   3. pald_cohesion_tiles on the rank's range; to collect C, pack with
 *      both = 1 (8192 words per tile: blocks [X, Z] and [Z, X]), all-gather
 *      and unpack with both = 1.
 * Every tile gives the bits of the single-GPU passes, so the gathered U and
 * C equal pald_focus and pald_cohesion's bit for bit.
 */

/* Number of 64 x 64 upper-triangle super-tiles of order n: T(T+1)/2 with
 * T = ceil(n/64); 0 if n is out of range. */
int64_t pald_shard_tiles(int64_t n);

/* The balanced contiguous range of rank `rank` of `world`: tiles
 * [floor(N*rank/world), floor(N*(rank+1)/world)), N = pald_shard_tiles(n).
 * Errors: INVALID_ARG. */
pald_status pald_shard_range(int64_t n, int32_t rank, int32_t world, int64_t* t0, int64_t* t1);

/*
 * pald_focus_tiles - pass 1 (as pald_focus) on tiles [t0, t1) only: writes
 * u_xy and u_yx for every pair of those tiles into U (device, n x n int32);
 * other entries of U are left as they are.
 * Errors: as pald_focus; INVALID_ARG for a range outside [0, pald_shard_tiles(n)].
 */
pald_status pald_focus_tiles(const float* D, int64_t n, int64_t t0, int64_t t1, int32_t* U,
                             const pald_opts* opts, pald_stream_t stream);

/*
 * pald_cohesion_tiles - pass 2 (as pald_cohesion) on tiles [t0, t1) only:
 * U must be complete; writes C[X, Z] and C[Z, X] of those tiles.  It builds
 * R = 1/u and the tie map of the whole matrix (O(n^2)) in scratch it takes
 * with cudaMallocAsync.
 * Errors: as pald_cohesion; INVALID_ARG for a bad range.
 */
pald_status pald_cohesion_tiles(const float* D, const int32_t* U, int64_t n, int64_t t0, int64_t t1, float* C,
                                const pald_opts* opts, pald_stream_t stream);

/*
 * pald_pack_tiles / pald_unpack_tiles - copy tiles [t0, t1) of an n x n
 * matrix of 4-byte words (device) to or from a packed device buffer: tile k
 * of the range at word 4096*k (both = 0: block [X, Y], row by row, zeros
 * outside the matrix) or 8192*k (both = 1: block [X, Y], then block [Y, X]).
 * Unpacking with both = 0 also writes the transpose of each block to
 * [Y, X] (for the symmetric U).
 * Errors: INVALID_ARG (null pointer, n, both or range out of range); CUDA.
 */
pald_status pald_pack_tiles(const void* M, int64_t n, int64_t t0, int64_t t1, int32_t both, void* packed,
                            pald_stream_t stream);
pald_status pald_unpack_tiles(const void* packed, int64_t n, int64_t t0, int64_t t1, int32_t both, void* M,
                              pald_stream_t stream);

/*
 * pald_validate - check the input contract of D (see above) on the device.
 * Reads D twice (row-wise and transposed), copies one status word to the
 * host and synchronises `stream`.  Returns PALD_OK or the first violation
 * found in the order NOT_SYMMETRIC, BAD_DIAGONAL, BAD_VALUE.
 */
pald_status pald_validate(const float* D, int64_t n, pald_stream_t stream);

/*
 * pald_local_depth - local depths from a cohesion matrix: L[x] = sum over z
 * of c_xz, the local depth of x (Sec. 2: cohesion partitions local depth,
 * eq. (LD)).  Deterministic: a fixed per-row order in two-float arithmetic,
 * one rounding to FP32.
 *   C  device, n x n FP32 (as written by pald_cohesion).
 *   L  device, n FP32, written completely.
 * Errors: INVALID_ARG (null pointer, n out of range); CUDA.
 */
pald_status pald_local_depth(const float* C, int64_t n, float* L, pald_stream_t stream);

/*
 * pald_strong_ties - the strong-tie mask for a threshold: T[x*n+z] = 1 when
 * c_xz >= threshold, else 0 (Sec. 2: cohesion stronger than a random focus
 * point would give; Sec. 7 applies a universal threshold defined outside
 * this paper, so the caller supplies it).  The mask is directed (row x, the
 * cohesion of z to x); a symmetric tie graph is T AND T^T or T OR T^T.
 *   C  device, n x n FP32.  T  device, n x n uint8, written completely.
 * Errors: INVALID_ARG (null pointer, n out of range, NaN threshold); CUDA.
 */
pald_status pald_strong_ties(const float* C, int64_t n, float threshold, uint8_t* T, pald_stream_t stream);

/*
 * pald_tie_map - diagnostic: the tie map that pald_cohesion builds for D and
 * reads to pick, per tile and group of y, between its short inner loop
 * (valid when no one-sided tie d_xy == d_xz or d_zy == d_zx can occur) and
 * its long one.  The paper has no counterpart; both loops compute Sec. 2
 * eq. (fxz) with the Sec. 5 tie split and give identical bits.
 *   D    device, n x n FP32 (the input contract above).
 *   map  device uint32 array of pald_tie_map_words(n) words, overwritten.
 *        With groups of G = 8 y for n <= 65536 and G = 32 y beyond,
 *        nb = ceil(n/64) and wpp = ceil(ceil(n/G)/32): word
 *        (a*nb + b)*wpp + g/32, a <= b, holds bit g%32 set when some row r
 *        in block a or b (rows 64a.., 64b..) has equal entries at two
 *        columns p != q with q in the other block of the pair and p in
 *        y group g (columns G*g .. G*g+G-1); words nb*nb*wpp + a (a < nb) are
 *        nonzero when a row of block a had too many repeated values to list
 *        (the tile then runs the long loop throughout).
 * Errors: INVALID_ARG (null pointer, n out of range); CUDA.
 */
pald_status pald_tie_map(const float* D, int64_t n, uint32_t* map, pald_stream_t stream);

/* Words of the tie map for order n (0 if n is out of range). */
int64_t pald_tie_map_words(int64_t n);

/*
 * pald_check_faults - synchronises `stream`, then reports whether a kernel of
 * this library gave up a bounded device-side wait (a TMA copy that never
 * completed within 2 s) since the previous call on this device, and clears
 * that record.  Such a kernel stops early instead of hanging the GPU; the
 * outputs of the call it belonged to are then unspecified.
 * Returns PALD_OK, PALD_ERR_TIMEOUT, or PALD_ERR_CUDA.
 */
pald_status pald_check_faults(pald_stream_t stream);

/*
 * pald_test_bounded_wait - diagnostic for the bounded device-side waits (the
 * paper has no counterpart).  Launches on `stream` one CTA that runs the
 * TMA pipeline of the pass kernels with no copy ever issued, so its first
 * mbarrier wait gives up after `limit_ns` nanoseconds; the CTA then takes the
 * same give-up path as a pass kernel whose copy never completed and records
 * the fault word that pald_check_faults reports.  The kernel ends after about
 * three limits; nothing faults or hangs.  Afterwards pald_check_faults
 * returns PALD_ERR_TIMEOUT once (and clears the record).
 *   limit_ns  1000 <= limit_ns <= 2e9.
 * Errors: INVALID_ARG (limit out of range); CUDA.
 */
pald_status pald_test_bounded_wait(int64_t limit_ns, pald_stream_t stream);

/*
 * Schedule tables (block-size tuning of Sec. 5, done for GPU tiles).  A table
 * is a list of buckets sorted by n_max; a matrix of order n takes the first
 * bucket with n <= n_max (the last bucket for larger n).  The library is
 * built with the tables that the project's autotuner
 * (paper_2307_16652_gb300/autotune.py) measured, keyed by GPU name and SM
 * count; on a GPU without one it uses built-in defaults.  All schedules of a
 * pass give identical bits; only the speed differs.
 */
typedef struct pald_schedule_bucket {
  int64_t n_max;          /* largest order of the bucket */
  int32_t focus;          /* pald_focus schedule (0 .. pald_schedule_count()-1) */
  int32_t cohesion;       /* pald_cohesion schedule */
  int32_t batched_split;  /* pald_batched: 1 = a diagonal tile leaves the pairs inside each group of
                             four points to a separate work item (four warps instead of five on the
                             tile); 0 = the tile computes them itself */
  int32_t reserved;       /* must be 0 */
} pald_schedule_bucket;

/*
 * pald_set_schedule_table - replaces the table of the CURRENT device (for
 * example with one the caller tuned); count == 0 (buckets may be NULL)
 * restores the table the library was built with.  Later pald_batched calls
 * build new plans with it.
 *   buckets  host array [count], 1 <= count <= 16, n_max strictly increasing.
 * Errors: INVALID_ARG (bad count, order, schedule id, split flag); CUDA.
 */
pald_status pald_set_schedule_table(const pald_schedule_bucket* buckets, int32_t count);

/*
 * pald_get_schedule - the bucket that applies to order n on the current
 * device.  *source (may be NULL) receives 0 for the built-in defaults, 1 for
 * a tuned table built into the library, 2 for a table set by the caller.
 * Errors: INVALID_ARG (null out, n out of range); CUDA.
 */
pald_status pald_get_schedule(int64_t n, pald_schedule_bucket* out, int32_t* source);

/* Number of built-in tile schedules and the name of schedule `id` (static
 * string, or NULL if id is out of range).  Used by the autotuner. */
int32_t pald_schedule_count(void);
const char* pald_schedule_name(int32_t id);

/* Static, human-readable description of a status code. */
const char* pald_status_string(pald_status status);

/* The cudaError_t value behind the most recent PALD_ERR_CUDA on this thread. */
int32_t pald_last_cuda_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t pald_version(void);

/* Frees the cached batched plans and graphs of every device, after waiting
 * for each plan's last replay to finish. */
void pald_release(void);

#ifdef __cplusplus
}
#endif

#endif /* PALD_H */
