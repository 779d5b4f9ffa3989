/*
 * ProHD oracle: a plain, slow, FP64 CPU restatement of what the ProHD hot path
 * computes (arxiv 2511.18207). TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the benchmark's CPU-baseline leg call it; the product path never
 * does. It shares no code, header, table or constant generator with the CUDA
 * library.
 *
 * Every loop is written in the order the definitions state; nothing is blocked,
 * fused or reordered. Build flags: -O2 -fno-fast-math -ffp-contract=off, so
 * each FP64 multiply and add is rounded on its own (no fused multiply-add).
 * OpenMP only splits independent outer iterations (rows, directions).
 *
 * Functions and the passages they follow:
 *   oracle_directed_hd      Eq. 1 (h(A,B) = max_a min_b ||a-b||_2), Methodology – Background and Notation
 *   oracle_centroid         Algorithm 1, centroid step
 *   oracle_centroid_axis    Algorithm 1, direction step (1e-9 fallback to e_1)
 *   oracle_union_covariance Algorithm 2, "principal components of [X;Y]"
 *   oracle_power_iteration  Algorithm 2, top-m components (power iteration with
 *                           Gram-Schmidt deflation; Methodology – Analysis names truncated SVD)
 *   oracle_project          Methodology – Background and Notation projection pi_u(p) = p^T u
 *   oracle_select           Algorithms 1-2 (bottom-k and top-k per direction and
 *                           per set, union, unique)
 *   oracle_hd_1d            Methodology – Theoretical Properties, 1D directed HD along u
 *   oracle_delta            Eq. 2, delta(u) = max_p ||p - (p^T u) u||
 *   oracle_splitmix64_unit  the counter-based generator for power-iteration
 *                           start vectors (SplitMix64, Steele/Lea/Flood 2014)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Exact Hausdorff distance by brute force (Eq. 1).                          */
/* ------------------------------------------------------------------------ */

/* Squared Euclidean distance by direct differences, summed over k = 0..D-1. */
static double sqdist64(const float* x, const float* y, int D) {
  double s = 0.0;
  for (int k = 0; k < D; ++k) {
    double d = (double)x[k] - (double)y[k];
    s = s + d * d;
  }
  return s;
}

/*
 * Directed HD h(X,Y) restricted to the outer rows [row_begin, row_end):
 *   for each x_i: NN distance min_j ||x_i - y_j|| (lowest j on ties),
 *   result: max over i (lowest i on ties).
 * rowmin_sq / rowarg (optional, length nX) receive each row's squared NN
 * distance and NN index for rows in the range.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_directed_hd(const float* X, int64_t nX, const float* Y, int64_t nY, int D,
                       int64_t row_begin, int64_t row_end, double* out_h,
                       int64_t* out_i, int64_t* out_j, double* rowmin_sq,
                       int64_t* rowarg) {
  if (!X || !Y || nX <= 0 || nY <= 0 || D <= 0) return -1;
  if (row_begin < 0) row_begin = 0;
  if (row_end > nX) row_end = nX;
  if (row_end <= row_begin) return -1;
  int64_t nr = row_end - row_begin;
  double* mins = (double*)malloc(sizeof(double) * (size_t)nr);
  int64_t* args = (int64_t*)malloc(sizeof(int64_t) * (size_t)nr);
  if (!mins || !args) { free(mins); free(args); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < nr; ++r) {
    const float* x = X + (size_t)(row_begin + r) * (size_t)D;
    double best = INFINITY;
    int64_t bj = -1;
    for (int64_t j = 0; j < nY; ++j) {
      double s = sqdist64(x, Y + (size_t)j * (size_t)D, D);
      if (s < best) { best = s; bj = j; }
    }
    mins[r] = best;
    args[r] = bj;
  }
  double h2 = -1.0;
  int64_t bi = -1, bj = -1;
  for (int64_t r = 0; r < nr; ++r) {
    if (mins[r] > h2) { h2 = mins[r]; bi = row_begin + r; bj = args[r]; }
    if (rowmin_sq) rowmin_sq[row_begin + r] = mins[r];
    if (rowarg) rowarg[row_begin + r] = args[r];
  }
  free(mins);
  free(args);
  if (out_h) *out_h = sqrt(h2);
  if (out_i) *out_i = bi;
  if (out_j) *out_j = bj;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Directions: centroids, centroid axis, union covariance, power iteration.   */
/* ------------------------------------------------------------------------ */

/* Mean of the n rows of X, accumulated in FP64 in row order (Algorithm 1). */
void oracle_centroid(const float* X, int64_t n, int D, double* out) {
  for (int k = 0; k < D; ++k) out[k] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < D; ++k) out[k] = out[k] + (double)X[(size_t)i * D + k];
  for (int k = 0; k < D; ++k) out[k] = out[k] / (double)n;
}

/* u = ybar - xbar, normalised; e_1 when ||u|| < 1e-9 (Algorithm 1). */
void oracle_centroid_axis(const double* xbar, const double* ybar, int D, double* u) {
  double s = 0.0;
  for (int k = 0; k < D; ++k) {
    u[k] = ybar[k] - xbar[k];
    s = s + u[k] * u[k];
  }
  double nrm = sqrt(s);
  if (nrm < 1e-9) {
    for (int k = 0; k < D; ++k) u[k] = 0.0;
    u[0] = 1.0;
  } else {
    for (int k = 0; k < D; ++k) u[k] = u[k] / nrm;
  }
}

/*
 * Covariance of the stacked set Z = [A; B] (Algorithm 2): two passes, first the
 * mean mu over all N = nA + nB rows, then C = (1/N) sum (z - mu)(z - mu)^T.
 * C is D x D row-major, FP64. Rows of C are independent, so OpenMP splits them.
 */
void oracle_union_covariance(const float* A, int64_t nA, const float* B, int64_t nB,
                             int D, double* mu, double* C) {
  int64_t N = nA + nB;
  for (int k = 0; k < D; ++k) mu[k] = 0.0;
  for (int64_t i = 0; i < nA; ++i)
    for (int k = 0; k < D; ++k) mu[k] = mu[k] + (double)A[(size_t)i * D + k];
  for (int64_t i = 0; i < nB; ++i)
    for (int k = 0; k < D; ++k) mu[k] = mu[k] + (double)B[(size_t)i * D + k];
  for (int k = 0; k < D; ++k) mu[k] = mu[k] / (double)N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int r = 0; r < D; ++r) {
    double* row = C + (size_t)r * D;
    for (int c = 0; c < D; ++c) row[c] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      const float* z = (i < nA) ? A + (size_t)i * D : B + (size_t)(i - nA) * D;
      double zr = (double)z[r] - mu[r];
      for (int c = 0; c < D; ++c) row[c] = row[c] + zr * ((double)z[c] - mu[c]);
    }
    for (int c = 0; c < D; ++c) row[c] = row[c] / (double)N;
  }
}

/* SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used counter-style. */
static uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/*
 * Start-vector component j of component l (l >= 1): counter c = l * 2^32 + j,
 * state = seed + (c + 1) * 0x9e3779b97f4a7c15, mixed, top 53 bits mapped to
 * [-1, 1). Exported so tests can pin it against the published constants.
 */
double oracle_splitmix64_unit(uint64_t seed, uint64_t l, uint64_t j) {
  uint64_t c = (l << 32) + j;
  uint64_t z = splitmix64_mix(seed + (c + 1ULL) * 0x9e3779b97f4a7c15ULL);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

static double dot64(const double* a, const double* b, int D) {
  double s = 0.0;
  for (int k = 0; k < D; ++k) s = s + a[k] * b[k];
  return s;
}

/* w <- w - sum_k (u_k . w) u_k over the previous components, applied twice. */
static void deflate(double* w, const double* U, int l, int D) {
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < l; ++k) {
      const double* u = U + (size_t)k * D;
      double c = dot64(u, w, D);
      for (int j = 0; j < D; ++j) w[j] = w[j] - c * u[j];
    }
}

/*
 * Top-m eigenvectors of the symmetric PSD matrix C by power iteration with
 * deflation (Algorithm 2's "top m principal components").
 * For component l = 1..m:
 *   v_0 = splitmix64 start vector, deflated against u_1..u_{l-1}, normalised;
 *   repeat: w = C v; deflate(w) (Gram-Schmidt twice); v_new = w / ||w||;
 *           stop when 1 - |<v_new, v>| < tol, or after maxit steps;
 *   lambda_l = v^T C v (Rayleigh quotient);
 *   sign: the entry of largest magnitude is made positive (lowest index wins
 *   ties), so the output does not depend on the start vector's sign.
 * If ||w|| == 0 the iteration stops with the current v and lambda = 0.
 * U is m x D row-major. Returns 0, or -1 on bad arguments / allocation.
 */
int oracle_power_iteration(const double* C, int D, int m, uint64_t seed, double tol,
                           int maxit, double* U, double* lam, int* iters) {
  if (!C || D <= 0 || m < 0 || m > D) return -1;
  double* v = (double*)malloc(sizeof(double) * D);
  double* w = (double*)malloc(sizeof(double) * D);
  if (!v || !w) { free(v); free(w); return -1; }
  for (int l = 1; l <= m; ++l) {
    double* u = U + (size_t)(l - 1) * D;
    for (int j = 0; j < D; ++j) v[j] = oracle_splitmix64_unit(seed, (uint64_t)l, (uint64_t)j);
    deflate(v, U, l - 1, D);
    double nv = sqrt(dot64(v, v, D));
    if (nv > 0.0)
      for (int j = 0; j < D; ++j) v[j] = v[j] / nv;
    int t = 0;
    for (t = 1; t <= maxit; ++t) {
      for (int r = 0; r < D; ++r) w[r] = dot64(C + (size_t)r * D, v, D);
      deflate(w, U, l - 1, D);
      double nw = sqrt(dot64(w, w, D));
      if (nw == 0.0) break;
      for (int j = 0; j < D; ++j) w[j] = w[j] / nw;
      double c = fabs(dot64(w, v, D));
      for (int j = 0; j < D; ++j) v[j] = w[j];
      if (1.0 - c < tol) break;
    }
    if (iters) iters[l - 1] = t > maxit ? maxit : t;
    /* Rayleigh quotient */
    for (int r = 0; r < D; ++r) w[r] = dot64(C + (size_t)r * D, v, D);
    double rq = dot64(v, w, D);
    /* sign canonicalisation */
    int jm = 0;
    for (int j = 1; j < D; ++j)
      if (fabs(v[j]) > fabs(v[jm])) jm = j;
    double sgn = v[jm] < 0.0 ? -1.0 : 1.0;
    for (int j = 0; j < D; ++j) u[j] = sgn * v[j];
    lam[l - 1] = rq;
  }
  free(v);
  free(w);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection and extreme selection (Algorithms 1-2).                        */
/* ------------------------------------------------------------------------ */

/* p_i = x_i^T u, summed sequentially over k = 0..D-1 in FP64, each product and
 * sum rounded separately (Methodology – Background and Notation projection). +0.0 is added last so that a
 * result of -0.0 compares and sorts as +0.0. */
void oracle_project(const float* X, int64_t n, int D, const double* u, double* p) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const float* x = X + (size_t)i * D;
    double s = 0.0;
    for (int k = 0; k < D; ++k) s = s + (double)x[k] * u[k];
    p[i] = s + 0.0;
  }
}

typedef struct { double p; int64_t i; } keyed_t;

/* ascending (p, index) */
static int cmp_asc(const void* a, const void* b) {
  const keyed_t* x = (const keyed_t*)a;
  const keyed_t* y = (const keyed_t*)b;
  if (x->p < y->p) return -1;
  if (x->p > y->p) return 1;
  return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* descending p, ascending index on ties */
static int cmp_desc(const void* a, const void* b) {
  const keyed_t* x = (const keyed_t*)a;
  const keyed_t* y = (const keyed_t*)b;
  if (x->p > y->p) return -1;
  if (x->p < y->p) return 1;
  return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* k = max(1, floor(alpha * n)) in FP64, clamped to n (Algorithms 1-2). */
int64_t oracle_k_of(double alpha, int64_t n) {
  double f = floor(alpha * (double)n);
  int64_t k = (int64_t)f;
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

/*
 * Marks mask[i] = 1 for every point of X that is among the k[d] smallest or the
 * k[d] largest projections onto dirs[d], for any d (Algorithms 1-2, union and
 * unique). Ordering is by full sort: bottom = first k of ascending (p, i); top
 * = first k of descending p with ascending i on ties. mask must be zeroed by
 * the caller or hold a previous union. Returns 0, or -1 on bad arguments.
 */
int oracle_select(const float* X, int64_t n, int D, const double* dirs, int nd,
                  const int64_t* k, uint8_t* mask) {
  if (!X || n <= 0 || D <= 0 || nd <= 0 || !mask) return -1;
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int d = 0; d < nd; ++d) {
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    keyed_t* kv = (keyed_t*)malloc(sizeof(keyed_t) * (size_t)n);
    if (!p || !kv) {
      free(p); free(kv);
#pragma omp atomic write
      rc = -1;
      continue;
    }
    const double* u = dirs + (size_t)d * D;
    for (int64_t i = 0; i < n; ++i) {
      const float* x = X + (size_t)i * D;
      double s = 0.0;
      for (int kk = 0; kk < D; ++kk) s = s + (double)x[kk] * u[kk];
      p[i] = s + 0.0;
    }
    int64_t kd = k[d] < n ? k[d] : n;
    for (int64_t i = 0; i < n; ++i) { kv[i].p = p[i]; kv[i].i = i; }
    qsort(kv, (size_t)n, sizeof(keyed_t), cmp_asc);
    for (int64_t r = 0; r < kd; ++r) mask[kv[r].i] = 1; /* benign race: all write 1 */
    for (int64_t i = 0; i < n; ++i) { kv[i].p = p[i]; kv[i].i = i; }
    qsort(kv, (size_t)n, sizeof(keyed_t), cmp_desc);
    for (int64_t r = 0; r < kd; ++r) mask[kv[r].i] = 1;
    free(p);
    free(kv);
  }
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics for the bounds of Methodology – Theoretical Properties.                                 */
/* ------------------------------------------------------------------------ */

/* 1D directed HD: max_i min_j |pX[i] - pY[j]|, by brute force. */
double oracle_hd_1d(const double* pX, int64_t nX, const double* pY, int64_t nY) {
  double h = 0.0;
  for (int64_t i = 0; i < nX; ++i) {
    double best = INFINITY;
    for (int64_t j = 0; j < nY; ++j) {
      double d = fabs(pX[i] - pY[j]);
      if (d < best) best = d;
    }
    if (best > h) h = best;
  }
  return h;
}

/* delta(u) over one set: max_i ||x_i - (x_i^T u) u|| (Eq. 2; take the max of
 * the two sets' values for A union B). u is assumed unit-length. */
double oracle_delta(const float* X, int64_t n, int D, const double* u) {
  double best = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const float* x = X + (size_t)i * D;
    double t = 0.0;
    for (int k = 0; k < D; ++k) t = t + (double)x[k] * u[k];
    double s = 0.0;
    for (int k = 0; k < D; ++k) {
      double r = (double)x[k] - t * u[k];
      s = s + r * r;
    }
    if (s > best) best = s;
  }
  return sqrt(best);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Raw SplitMix64 output for counter c: mix(seed + (c + 1) * golden gamma),
 * i.e. the (c+1)-th output of the sequential generator seeded with seed. */
uint64_t oracle_splitmix64_raw(uint64_t seed, uint64_t c) {
  return splitmix64_mix(seed + (c + 1ULL) * 0x9e3779b97f4a7c15ULL);
}
