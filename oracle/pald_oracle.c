/*
 * PaLD oracle: a plain, slow, obviously correct CPU implementation of the
 * two quantities the partitioned-local-depth method computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the tests, the smoke check and the timed CPU
 * baseline of the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Definitions followed (Devarakonda & Ballard, "Sequential and Shared-Memory
 * Parallel Algorithms for Partitioned Local Depths"):
 *
 *   local focus (Sec. 2):   U_xy = { z : d_xz <= d_xy  or  d_yz <= d_xy },
 *                           u_xy = |U_xy|,  for every x, y (also x == y).
 *
 *   cohesion (Sec. 2, eq. (cohesion), with the tie rule of Sec. 5):
 *       c_xz = Pr[ Z = z and z supports x against Y ],
 *       Y uniform on S \ {x}, Z uniform on U_xY, so
 *       c_xz = sum_{y != x} 1/(n-1) * [z in U_xy] / u_xy * w(d_zx, d_zy),
 *       w(p, q) = 1 if p < q, 1/2 if p == q, 0 if p > q.
 *
 * Readings taken where the paper is loose (each listed in the design notes):
 *   - focus membership uses <= (Sec. 2 definition, eq. (fxz)); support uses
 *     strict < with half credit on equality (Sec. 5, tie splitting);
 *   - y ranges over S \ {x} (eq. (LD)), y == z included;
 *   - the diagonal c_xx is part of C (the z == x case of eq. (cohesion));
 *   - u_xx follows the definition literally: #{z : d_xz <= 0}.
 *
 * Arithmetic: every comparison is made on the FP32 inputs promoted exactly to
 * double; the sum over y runs in FP64 in increasing y; the 1/(n-1) factor is
 * applied in FP64 at the end.  There is no blocking, no symmetry shortcut and
 * no reordering.  Rows x are independent and are split over threads.
 *
 * PALD_ORACLE_MUTANT (compile-time, default 0) plants one deliberate mistake
 * so the tests can show that their pins catch it; the default build has none.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef PALD_ORACLE_MUTANT
#define PALD_ORACLE_MUTANT 0
#endif

/* Entry (x, y) of the row-major n x n matrix, promoted exactly to double. */
static inline double dist(const float* D, int64_t n, int64_t x, int64_t y) {
  return (double)D[x * n + y];
}

/* z in U_xy  (Sec. 2): d_xz <= d_xy or d_yz <= d_xy. */
static inline int in_focus(double dxy, double dxz, double dyz) {
#if PALD_ORACLE_MUTANT == 1
  return dxz < dxy || dyz < dxy;      /* mutant: strict inequality in the focus */
#elif PALD_ORACLE_MUTANT == 2
  (void)dyz;
  return dxz <= dxy;                  /* mutant: dropped second condition */
#else
  return dxz <= dxy || dyz <= dxy;
#endif
}

/* Support weight w(d_zx, d_zy): z is closer to x than to y, half on a tie. */
static inline double support(double dzx, double dzy) {
#if PALD_ORACLE_MUTANT == 3
  /* mutant: no tie split */
  return dzx < dzy ? 1.0 : 0.0;
#elif PALD_ORACLE_MUTANT == 4
  /* mutant: wrong direction */
  return dzx > dzy ? 1.0 : (dzx == dzy ? 0.5 : 0.0);
#else
  return dzx < dzy ? 1.0 : (dzx == dzy ? 0.5 : 0.0);
#endif
}

/* u_xy for one pair, straight from the definition. */
static int32_t focus_size(const float* D, int64_t n, int64_t x, int64_t y) {
  int64_t count = 0;
  const double dxy = dist(D, n, x, y);
#if PALD_ORACLE_MUTANT == 9
  for (int64_t z = 1; z < n; ++z)     /* mutant: drops z = 0 */
#else
  for (int64_t z = 0; z < n; ++z)
#endif
    count += in_focus(dxy, dist(D, n, x, z), dist(D, n, y, z));
  return (int32_t)count;
}

/* Row x of C given row x of u (u_x[y] = u_xy).
 * The y loop reads d_yz as entry (z, y): D is exactly symmetric (an input
 * requirement the tests check), and this keeps every inner-loop read
 * contiguous, which matters at n = 65536. */
static void cohesion_row(const float* D, int64_t n, int64_t x, const int32_t* u_x, double* c_x) {
  for (int64_t z = 0; z < n; ++z) {
    const double dxz = dist(D, n, x, z);
    const double dzx = dist(D, n, z, x);
    double sum = 0.0;
    for (int64_t y = 0; y < n; ++y) {
#if PALD_ORACLE_MUTANT == 5
      /* mutant: y == x not excluded */
#else
      if (y == x) continue;
#endif
      const double dxy = dist(D, n, x, y);
      const double dzy = dist(D, n, z, y);
      if (!in_focus(dxy, dxz, dzy)) continue;         /* z in U_xy, d_yz == d_zy */
#if PALD_ORACLE_MUTANT == 7
      sum += support(dzx, dxy) / (double)u_x[y];      /* mutant: d_xy for d_zy */
#elif PALD_ORACLE_MUTANT == 8
      sum += support(dzx, dzy) / (double)u_x[z];      /* mutant: u_xz for u_xy */
#else
      sum += support(dzx, dzy) / (double)u_x[y];
#endif
    }
#if PALD_ORACLE_MUTANT == 6
    c_x[z] = sum / (double)n;          /* mutant: wrong normalisation */
#else
    c_x[z] = sum / (double)(n - 1);
#endif
  }
}

/* ------------------------------------------------------------------------ */
/* threading: rows are handed out in a fixed round-robin, one writer per row */

typedef struct {
  const float* D;
  int64_t n;
  const int64_t* rows;   /* NULL: all rows 0..n-1 */
  int64_t nrows;
  int32_t* U;            /* nrows x n */
  double* C;             /* nrows x n or NULL */
  const int32_t* Uin;    /* full n x n u (cohesion-only mode) or NULL */
  int tid, nthreads;
} job_t;

static void* worker(void* arg) {
  job_t* j = (job_t*)arg;
  const int64_t n = j->n;
  for (int64_t i = j->tid; i < j->nrows; i += j->nthreads) {
    int64_t x = j->rows ? j->rows[i] : i;
    int32_t* u_x = j->U ? j->U + i * n : NULL;
    if (j->Uin) {
      cohesion_row(j->D, n, x, j->Uin + x * n, j->C + i * n);
      continue;
    }
    for (int64_t y = 0; y < n; ++y) u_x[y] = focus_size(j->D, n, x, y);
    if (j->C) cohesion_row(j->D, n, x, u_x, j->C + i * n);
  }
  return NULL;
}

static int run(job_t proto, int threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pthread_t th[256];
  job_t jobs[256];
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    jobs[t] = proto;
    jobs[t].tid = t;
    jobs[t].nthreads = threads;
    if (threads == 1) break;
    if (pthread_create(&th[t], NULL, worker, &jobs[t]) != 0) break;
    ++started;
  }
  if (threads == 1 || started == 0) {
    jobs[0].tid = 0;
    jobs[0].nthreads = 1;
    worker(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  if (started != threads) {
    /* finish the rows of threads that failed to start, on this thread */
    for (int t = started; t < threads; ++t) worker(&jobs[t]);
  }
  return 0;
}

/* u (n x n) and, if C != NULL, C (n x n, FP64) for the whole matrix. */
int pald_oracle(const float* D, int64_t n, int32_t* U, double* C, int threads) {
  if (!D || !U || n < 2) return 1;
  job_t j;
  memset(&j, 0, sizeof j);
  j.D = D; j.n = n; j.rows = NULL; j.nrows = n; j.U = U; j.C = C;
  return run(j, threads);
}

/* C (n x n, FP64) from a u the oracle computed itself (pald_oracle with
 * C == NULL); lets the tests time and check the two passes separately. */
int pald_oracle_cohesion(const float* D, const int32_t* U, int64_t n, double* C, int threads) {
  if (!D || !U || !C || n < 2) return 1;
  job_t j;
  memset(&j, 0, sizeof j);
  j.D = D; j.n = n; j.rows = NULL; j.nrows = n; j.C = C; j.Uin = U;
  return run(j, threads);
}

/* Selected rows only: Urows[i*n + y] = u_{rows[i], y},
 * Crows[i*n + z] = c_{rows[i], z}.  Cost O(k n^2). */
int pald_oracle_rows(const float* D, int64_t n, const int64_t* rows, int64_t k,
                     int32_t* Urows, double* Crows, int threads) {
  if (!D || !rows || !Urows || n < 2 || k < 0) return 1;
  for (int64_t i = 0; i < k; ++i)
    if (rows[i] < 0 || rows[i] >= n) return 1;
  job_t j;
  memset(&j, 0, sizeof j);
  j.D = D; j.n = n; j.rows = rows; j.nrows = k; j.U = Urows; j.C = Crows;
  return run(j, threads);
}

int pald_oracle_mutant(void) { return PALD_ORACLE_MUTANT; }
