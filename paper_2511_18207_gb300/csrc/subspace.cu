// Top-m principal components of the union covariance C (Algorithm 2 step 2)
// by block (subspace) iteration with Rayleigh-Ritz, for D <= 256 and m <= 24.
//
// The top-m eigenvectors of C are a plain definition; the oracle reaches them
// by deflated power iteration, one vector at a time, and this path reaches
// the same vectors with a block of b vectors iterated together: b = D when
// D <= 32 (the block spans the space, so the first Rayleigh-Ritz step is
// already the full eigendecomposition whatever the eigengaps), else
// b = min(max(2m, m + 8), 32):
//   V orthonormal (D x b); W = C V; H = V^T W; H = Y diag(theta) Y^T (Jacobi);
//   Ritz vectors X = V Y, residuals r_j = W y_j - theta_j x_j;
//   stop when ||r_j|| <= eps theta_1 for the m leading pairs, else
//   V = orth((W Y + sigma X) diag(1 / (theta + sigma))) by Cholesky-QR, twice;
//   also stop (at the cap, or earlier once the observed rate shows the cap
//   cannot be met: the stall test below) with the current Ritz vectors.
// The error of the leading m Ritz vectors falls like ((lambda_{b+1} + sigma) /
// (lambda_m + sigma))^t, against lambda_{l+1}/lambda_l per step for each
// vector of the power iteration. The shift sigma = theta_1 / 100 bounds the
// condition number of the scaled block (its Gram matrix is I plus the residual
// Gram over (theta + sigma)^2, so at most 1 + b 10^4), which keeps the FP32
// Cholesky-QR well conditioned; it slows the convergence factor only from
// lambda_{b+1}/lambda_m to (lambda_{b+1} + sigma)/(lambda_m + sigma).
// A residual bound eps = max(sqrt(2 tol), 2e-6) certifies each returned
// vector to within eps lambda_1 / gap_l in angle (the residual bound of the
// symmetric eigenproblem); FP32 arithmetic (Jacobi stopping at 4 units of
// rounding, C V to a few units) cannot certify much below 1e-6.
//
// One cluster of 8 CTAs runs the iteration: CTA r owns rows [r0, r1) of C
// (FP32, in shared memory) and of every D x b block, and holds a full copy of
// V. Each step exchanges three small b x b matrices (H, the two Cholesky-QR
// Gram matrices) and the new rows of V through distributed shared memory;
// every CTA sums the exchanged partials in the same order and repeats the
// small dense work (Jacobi, Cholesky), so all CTAs take the same decisions.
// C V accumulates 8-term FFMA blocks with error-free (TwoSum) addition of the
// blocks. The m Ritz vectors are then orthonormalised in FP64 (Cholesky-QR,
// twice), signed (largest |entry| positive, lowest index on ties) and their
// Rayleigh quotients taken with the FP64 C.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kSiCTAs = 8;
constexpr int kSiThreads = 512;
constexpr int kSiFinThreads = 256;
constexpr int kSiJacThreads = 256;  // the Jacobi rounds run on 8 warps (one warp alone is slower: the rounds are latency-bound)
constexpr int kSiMaxD = 256;
constexpr int kSiMaxB = 32;
constexpr int kSiStallWin = 8;     // steps per window of the stall test
constexpr int kSiStallStart = 16;  // no stall test before this step
constexpr int kSiRRWarm = 2;       // steps with a Rayleigh-Ritz step every time

// block size for D dimensions and m components (D <= 256, m <= 24)
__host__ __device__ inline int si_block(int D, int m) {
  const int want = 2 * m > m + 8 ? 2 * m : m + 8;
  return D <= kSiMaxB ? D : (want < kSiMaxB ? want : kSiMaxB);
}
constexpr int kSiMaxM = 24;
constexpr int kSiMaxRows = kSiMaxD / kSiCTAs;      // 32
constexpr int kSiLd = kSiMaxB + 1;                 // row stride of the small matrices
constexpr int kSiX = kSiMaxB * kSiMaxB + kSiMaxB;  // one exchange slot: b x b matrix + b values
constexpr int kSiVld = kSiMaxD + 4;                // row stride of V^T (floats): 128-bit aligned, staggered banks

// NC CTAs (a cluster when NC > 1) share the iteration; each holds ROWS rows
// of every D x b block (and, in a cluster, its rows of C), V^T with row
// stride VLD floats.
template <int NC, int ROWS, int VLD>
struct SiSmemT {
  float Vt[kSiMaxB * VLD];                 // basis, transposed: column j of V at Vt[j * VLD], zero padded
  float Cl[NC > 1 ? ROWS * kSiMaxD : 4];   // this CTA's rows of C (cluster only), row stride Dq, zero padded
  float Cst[NC > 1 ? 4 : 2 * 16 * ROWS];   // one CTA: C streamed in 16-row chunks, double-buffered
  float Vn[NC > 1 ? 4 : ROWS * kSiMaxB];   // one CTA: V row-major [k][j], columns past b zero
  float W[ROWS * kSiMaxB];           // C V, local rows
  float Vr[ROWS * kSiMaxB];          // Ritz vectors V Y, local rows
  float Wr[ROWS * kSiMaxB];          // W Y -> scaled block -> Q1 -> Q
  float part[kSiX];                  // this CTA's partial before an exchange
  float X[2][NC][kSiX];              // exchange slots, double-buffered
  float M[kSiMaxB * kSiLd];          // summed small matrix
  float Y[kSiMaxB * kSiLd];          // Jacobi eigenvectors (columns)
  float L[kSiMaxB * kSiLd];          // inverse Cholesky factor L^{-1} (lower)
  float Lf[kSiMaxB * kSiLd];         // Cholesky factor L (lower)
  float red[2 * kSiThreads / 32];    // block reductions
  float dinv[kSiMaxB];               // reciprocal Cholesky pivots
  float theta[kSiMaxB];              // Ritz values by rank (descending)
  float res[kSiMaxB];                // summed squared residuals
  float cs[kSiMaxB / 2][2];
  int pq[kSiMaxB / 2][2];
  int perm[kSiMaxB];                 // perm[rank] = column of Y
  uint32_t key[kSiMaxB];             // order keys of the Ritz values
};
using SiSmem = SiSmemT<kSiCTAs, kSiMaxRows, kSiVld>;

// 1/sqrt(x) for x > 0: the hardware estimate refined by one Newton step
// (relative error well below FP32 rounding, without the division and square
// root sequences of IEEE-exact arithmetic on the small matrices' critical paths).
PROHD_DEV float rsqrt_nr(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x * r, r, 1.5f);
}

// Error-free s + x accumulated into (s, c).
PROHD_DEV void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

// Barrier over the CTAs that share the iteration.
template <int NC>
PROHD_DEV void si_sync() {
  if constexpr (NC > 1)
    cluster_sync();
  else
    __syncthreads();
}

// Sends this CTA's part[0..n) into slot X[buf][rank] of every CTA of the cluster.
template <int NC, class SM>
PROHD_DEV void si_broadcast(SM& S, int buf, uint32_t rank, int n) {
  float* dst = &S.X[buf][rank][0];
  for (int e = threadIdx.x; e < n * NC; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    if constexpr (NC > 1)
      st_cluster_f32(map_to_cta(dst + i, (uint32_t)c), S.part[i]);
    else
      dst[i] = S.part[i];
  }
}

// out[i] = sum over CTAs (fixed order) of X[buf][*][off + i], i < n.
template <int NC, class SM>
PROHD_DEV float si_sum(const SM& S, int buf, int idx) {
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < NC; ++r) s += S.X[buf][r][idx];
  return s;
}

// Pair k of round `round` of a round-robin tournament of n (even) players.
PROHD_DEV void si_pair(int n, int round, int k, int& p, int& q) {
  if (k == 0) {
    p = n - 1;
    q = round;
  } else {
    p = (round + k) % (n - 1);
    q = (round - k + n - 1) % (n - 1);
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// Block-wide maxima of two non-negative values (every thread gets them).
PROHD_DEV void si_block_max2(float& a, float& b, float* red /*[2][kSiThreads/32]*/) {
  a = warp_max(a);
  b = warp_max(b);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w] = a;
    red[kSiThreads / 32 + w] = b;
  }
  __syncthreads();
  a = 0.f;
  b = 0.f;
#pragma unroll
  for (int i = 0; i < kSiThreads / 32; ++i) {
    a = fmaxf(a, red[i]);
    b = fmaxf(b, red[kSiThreads / 32 + i]);
  }
  __syncthreads();
}

// Cyclic Jacobi on the symmetric b x b matrix S.M, all threads: S.M <- Y^T M Y
// diagonal, Y orthogonal. The disjoint rotations J_k of one round of a
// round-robin tournament act on M as independent 2 x 2 block transforms
// B_{k1,k2} <- J_{k1}^T B_{k1,k2} J_{k2} (one thread per block) and on Y as
// column pairs, so a round is two barrier-separated steps. Sweeps stop once
// every off-diagonal entry is within 4 units of FP32 rounding of the largest
// diagonal entry (rotations below that only move noise); then each Ritz
// vector's own residual in H is at most sqrt(b) 2.4e-7 theta_1.
// Maxima of two non-negative values over the Jacobi threads (all get them).
// Barrier of the Jacobi threads: the warp itself, or named barrier 1.
PROHD_DEV void si_jac_sync() {
  if constexpr (kSiJacThreads == 32)
    __syncwarp();
  else
    named_bar_sync(1, kSiJacThreads);
}

PROHD_DEV void si_jac_max2(float& a, float& b, float* red /*[2][kSiJacThreads/32]*/) {
  a = warp_max(a);
  b = warp_max(b);
  if constexpr (kSiJacThreads > 32) {
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
      red[w] = a;
      red[kSiJacThreads / 32 + w] = b;
    }
    si_jac_sync();
    a = 0.f;
    b = 0.f;
#pragma unroll
    for (int i = 0; i < kSiJacThreads / 32; ++i) {
      a = fmaxf(a, red[i]);
      b = fmaxf(b, red[kSiJacThreads / 32 + i]);
    }
  }
  si_jac_sync();
}

template <class SM>
PROHD_DEV void si_jacobi(SM& S, int b) {
  // run by the first kSiJacThreads threads, synchronised by si_jac_sync
  const int tid = threadIdx.x;
  float* A = S.M;
  float* Y = S.Y;
  for (int e = tid; e < kSiMaxB * kSiMaxB; e += kSiJacThreads) {
    const int r = e >> 5, c = e & 31;
    if (r < b && c < b) Y[r * kSiLd + c] = r == c ? 1.f : 0.f;
  }
  const int n = b + (b & 1);  // players; index b is a dummy when b is odd
  const int np = n / 2;
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = tid; e < kSiMaxB * kSiMaxB; e += kSiJacThreads) {
      const int r = e >> 5, c = e & 31;
      if (r < b && c < b) {
        const float v = fabsf(A[r * kSiLd + c]);
        if (r != c) off = fmaxf(off, v);
        else dia = fmaxf(dia, v);
      }
    }
    si_jac_max2(off, dia, S.red);  // also orders the Y initialisation before use
    if (!(off > 2.4e-7f * dia)) break;
    const float skip = 6e-8f * dia;
    for (int round = 0; round < n - 1; ++round) {
      if (tid < np) {
        int p, q;
        si_pair(n, round, tid, p, q);
        float c = 1.f, s = 0.f;
        if (q < b) {
          const float apq = A[p * kSiLd + q];
          if (fabsf(apq) > skip) {
            // tan of the rotation angle; t only steers the rotation (any
            // nearby angle still annihilates A[p][q] to rounding), while
            // c = 1/sqrt(1 + t^2), s = t c keep c^2 + s^2 = 1 to rounding
            const float tau = __fdividef(A[q * kSiLd + q] - A[p * kSiLd + p], 2.f * apq);
            const float h = fmaf(tau, tau, 1.f);
            const float t = fabsf(tau) < 1e18f ? __fdividef(copysignf(1.f, tau), fabsf(tau) + h * rsqrt_nr(h))
                                               : __fdividef(0.5f, tau);
            c = rsqrt_nr(fmaf(t, t, 1.f));
            s = t * c;
          }
        }
        S.cs[tid][0] = c;
        S.cs[tid][1] = s;
        S.pq[tid][0] = p;
        S.pq[tid][1] = q;
      }
      si_jac_sync();
      // work items: 2 x 2 blocks (k1, k2) of M, then the column pairs of Y
      const int nblk = np * np;
      for (int w = tid; w < nblk + b * np; w += kSiJacThreads) {
        if (w < nblk) {
          const int k1 = w / np, k2 = w - k1 * np;
          const int p1 = S.pq[k1][0], q1 = S.pq[k1][1], p2 = S.pq[k2][0], q2 = S.pq[k2][1];
          const float c1 = S.cs[k1][0], s1 = S.cs[k1][1], c2 = S.cs[k2][0], s2 = S.cs[k2][1];
          const bool v1 = q1 < b, v2 = q2 < b;  // a pair with the dummy is the identity on p
          const float app = A[p1 * kSiLd + p2];
          const float apq = v2 ? A[p1 * kSiLd + q2] : 0.f;
          const float aqp = v1 ? A[q1 * kSiLd + p2] : 0.f;
          const float aqq = v1 && v2 ? A[q1 * kSiLd + q2] : 0.f;
          // rows: J1^T B
          const float rpp = c1 * app - s1 * aqp, rpq = c1 * apq - s1 * aqq;
          const float rqp = s1 * app + c1 * aqp, rqq = s1 * apq + c1 * aqq;
          // columns: (J1^T B) J2
          A[p1 * kSiLd + p2] = c2 * rpp - s2 * rpq;
          if (v2) A[p1 * kSiLd + q2] = s2 * rpp + c2 * rpq;
          if (v1) A[q1 * kSiLd + p2] = c2 * rqp - s2 * rqq;
          if (v1 && v2) A[q1 * kSiLd + q2] = s2 * rqp + c2 * rqq;
        } else {
          const int e = w - nblk, k = e / b, row = e - k * b;
          const int p = S.pq[k][0], q = S.pq[k][1];
          if (q < b) {
            const float c = S.cs[k][0], s = S.cs[k][1];
            const float yp = Y[row * kSiLd + p], yq = Y[row * kSiLd + q];
            Y[row * kSiLd + p] = c * yp - s * yq;
            Y[row * kSiLd + q] = s * yp + c * yq;
          }
        }
      }
      si_jac_sync();
    }
  }
  // Ritz values by rank: descending, lower column first on ties. Every key
  // is computed once into shared memory and all comparisons read those
  // integers, so the ranks are a permutation whatever the values (NaN too).
  if (tid < b) S.key[tid] = f32_key(A[tid * kSiLd + tid]);
  si_jac_sync();
  if (tid < b) {
    const uint32_t kj = S.key[tid];
    int rank = 0;
    for (int kk = 0; kk < b; ++kk) {
      const uint32_t v = S.key[kk];
      rank += (v > kj) || (v == kj && kk < tid);
    }
    S.perm[rank] = tid;
    S.theta[rank] = A[tid * kSiLd + tid];
  }
  si_jac_sync();
}

// Cholesky S.M = L L^T (warp 0, lane i computes row i of L into S.Lf), then
// S.L = L^{-1} (lane j forms column j by forward substitution). Rolled loops
// over shared memory keep the code small. A pivot that rounding drove to or
// below zero is replaced by a tiny positive one: the column is then noise,
// which a second pass normalises.
template <class SM>
PROHD_DEV void si_chol_inv(SM& S, int b, int lane) {
  const float floor_piv = 1e-30f + 1e-12f * fabsf(S.M[0]);
  float* Lf = S.Lf;
  float* dinv = S.dinv;  // 1 / L[j][j]
  const int row = lane < b ? lane : b - 1;  // lanes past b shadow the last row, their stores are masked
  // every lane runs the same instructions (stores are predicated), so the
  // warp never splits
  for (int j = 0; j < b; ++j) {
    float acc = S.M[row * kSiLd + j];
#pragma unroll 4
    for (int k = 0; k < j; ++k) acc = fmaf(-Lf[row * kSiLd + k], Lf[j * kSiLd + k], acc);
    const float piv = fmaxf(__shfl_sync(0xffffffffu, acc, j), floor_piv);
    const float r = rsqrt_nr(piv);
    if (lane == j) {
      Lf[j * kSiLd + j] = piv * r;
      dinv[j] = r;
    }
    if (lane > j && lane < b) Lf[lane * kSiLd + j] = acc * r;
    __syncwarp();
  }
  // column `lane` of L^{-1}: x_i = (delta_{i,lane} - sum_{k<i} L[i][k] x_k) / L[i][i];
  // x_k = 0 for k < lane, so the sums can start at 0 for every lane
  const int col = lane < b ? lane : b - 1;
  for (int i = 0; i < b; ++i) {
    float acc = i == col ? 1.f : 0.f;
#pragma unroll 4
    for (int k = 0; k < i; ++k) acc = fmaf(-Lf[i * kSiLd + k], S.L[k * kSiLd + col], acc);
    const float x = i >= col ? acc * dinv[i] : 0.f;
    if (lane < b) S.L[i * kSiLd + lane] = x;
    __syncwarp();
  }
}

// dst (local rows) = src L^{-T}: dst[i][j] = sum_{k <= j} src[i][k] Linv[j][k].
template <int ROWS, class SM>
PROHD_DEV void si_apply_linv(SM& S, const float* src, float* dst, int nr, int b) {
  (void)ROWS;
  for (int o = threadIdx.x; o < nr * b; o += kSiThreads) {
    const int i = o / b, j = o - i * b;
    float v = 0.f;
    for (int kk = 0; kk <= j; ++kk) v = fmaf(src[i * b + kk], S.L[j * kSiLd + kk], v);
    dst[i * b + j] = v;
  }
}

// part[j*b + k] = sum_i src[i][j] src[i][k] over local rows.
// With many local rows (one CTA holding all D rows) and b <= 16 the rows are
// split in four quarters summed by separate threads into `scratch`
// ([4][b * b]) and combined in a fixed order.
template <class SM>
PROHD_DEV void si_local_gram(SM& S, const float* src, int nr, int b, float* scratch) {
  if (scratch && b <= 16 && nr > 64) {
    const int bb = b * b, q4 = (nr + 3) >> 2;
    for (int t = threadIdx.x; t < 4 * bb; t += kSiThreads) {
      const int q = t / bb, e = t - q * bb, j = e / b, k = e - j * b;
      float s = 0.f;
      for (int i = q * q4; i < min(nr, (q + 1) * q4); ++i) s = fmaf(src[i * b + j], src[i * b + k], s);
      scratch[t] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < bb; e += kSiThreads)
      S.part[e] = (scratch[e] + scratch[bb + e]) + (scratch[2 * bb + e] + scratch[3 * bb + e]);
    return;
  }
  for (int e = threadIdx.x; e < kSiMaxB * kSiMaxB; e += kSiThreads) {
    const int j = e >> 5, k = e & 31;
    if (j < b && k < b) {
      float s = 0.f;
      for (int i = 0; i < nr; ++i) s = fmaf(src[i * b + j], src[i * b + k], s);
      S.part[j * b + k] = s;
    }
  }
}

// The exchange half of a Cholesky-QR pass over the local rows in `src`:
// local Gram, exchange (n_extra further values of part ride along), summed
// Gram into S.M and the extra values into S.res.
template <int NC, class SM>
PROHD_DEV void si_cholqr_pass(SM& S, const float* src, int nr, int b, uint32_t rank, int& xb, int n_extra) {
  // one CTA: the idle exchange buffer is scratch (no other CTA writes it)
  si_local_gram(S, src, nr, b, NC == 1 ? &S.X[xb ^ 1][0][0] : nullptr);
  __syncthreads();
  si_broadcast<NC>(S, xb, rank, b * b + n_extra);
  si_sync<NC>();
  for (int e = threadIdx.x; e < kSiMaxB * kSiMaxB; e += kSiThreads) {
    const int j = e >> 5, k = e & 31;
    if (j < b && k < b) S.M[j * kSiLd + k] = si_sum<NC>(S, xb, j * b + k);
  }
  for (int j = threadIdx.x; j < n_extra; j += kSiThreads) S.res[j] = si_sum<NC>(S, xb, b * b + j);
  xb ^= 1;
  __syncthreads();
}

// The iteration, run by NC CTAs (a cluster of 8 for one pair, or one CTA per
// pair of a batch, which reads C from global memory and needs D % 4 == 0).
template <int NC, int ROWS, int VLD>
PROHD_DEV void subspace_body(SiSmemT<NC, ROWS, VLD>& S, const float* __restrict__ C32, int D, int m, int b,
                             int maxit, float eps, float sigma_rel, uint64_t seed, double* __restrict__ Uout,
                             int* __restrict__ iters_out) {
  uint32_t rank = 0;
  if constexpr (NC > 1) rank = cluster_rank();
  const int rows_per = (D + NC - 1) / NC;
  const int r0 = min(D, (int)rank * rows_per), r1 = min(D, r0 + rows_per);
  const int nr = r1 - r0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int Dq = (D + 3) & ~3;  // C rows and V columns padded with zeros to a multiple of 4
  if constexpr (NC > 1)
    for (int e = tid; e < nr * Dq; e += kSiThreads) {
      const int i = e / Dq, k = e - i * Dq;
      S.Cl[e] = k < D ? C32[(size_t)(r0 + i) * D + k] : 0.f;
    }
  // start block: column j is the oracle's start vector of component j + 1
  for (int e = tid; e < b * Dq; e += kSiThreads) {
    const int j = e / Dq, i = e - j * Dq;
    S.Vt[j * VLD + i] = i < D ? (float)splitmix64_unit(seed, (uint64_t)(j + 1), (uint64_t)i) : 0.f;
  }
  if constexpr (NC == 1)
    for (int e = tid; e < ROWS * kSiMaxB; e += kSiThreads) S.Vn[e] = 0.f;
  __syncthreads();
  si_sync<NC>();

  int xb = 0;  // exchange buffer
  int t = 0;
  // largest relative residual max_j ||r_j|| / theta_1 at the last two window
  // boundaries (every thread holds the same values: they come from the
  // summed shared-memory residuals)
  float r_prev = 0.f, r_cur = 0.f;
  for (;; ++t) {
    if (t == 0) {
      // first pass only orthonormalises the start block
      for (int e = tid; e < nr * b; e += kSiThreads) {
        const int i = e / b, j = e - i * b;
        S.Wr[e] = S.Vt[j * VLD + r0 + i];
      }
      __syncthreads();
      si_cholqr_pass<NC>(S, S.Wr, nr, b, rank, xb, 0);
    } else {
      // ---- W = C V for the local rows: 8-term FFMA blocks in two independent
      // chains (128-bit loads of a row of C and of a column of V), TwoSum
      // across blocks
      auto cv_row = [&](const float* __restrict__ crow_f, int j) -> float {
        const float4* crow = reinterpret_cast<const float4*>(crow_f);
        const float4* vcol = reinterpret_cast<const float4*>(S.Vt + j * VLD);
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
        int k4 = 0;
        const int n4 = Dq >> 2;
        for (; k4 + 4 <= n4; k4 += 4) {
          const float4 a0 = crow[k4], a1 = crow[k4 + 1], a2 = crow[k4 + 2], a3 = crow[k4 + 3];
          const float4 v0 = vcol[k4], v1 = vcol[k4 + 1], v2 = vcol[k4 + 2], v3 = vcol[k4 + 3];
          float b0 = a0.x * v0.x, b1 = a2.x * v2.x;
          b0 = fmaf(a0.y, v0.y, b0);
          b1 = fmaf(a2.y, v2.y, b1);
          b0 = fmaf(a0.z, v0.z, b0);
          b1 = fmaf(a2.z, v2.z, b1);
          b0 = fmaf(a0.w, v0.w, b0);
          b1 = fmaf(a2.w, v2.w, b1);
          b0 = fmaf(a1.x, v1.x, b0);
          b1 = fmaf(a3.x, v3.x, b1);
          b0 = fmaf(a1.y, v1.y, b0);
          b1 = fmaf(a3.y, v3.y, b1);
          b0 = fmaf(a1.z, v1.z, b0);
          b1 = fmaf(a3.z, v3.z, b1);
          b0 = fmaf(a1.w, v1.w, b0);
          b1 = fmaf(a3.w, v3.w, b1);
          two_sum_acc(s0, c0, b0);
          two_sum_acc(s1, c1, b1);
        }
        float bt = 0.f;
        for (; k4 < n4; ++k4) {
          const float4 a = crow[k4], v = vcol[k4];
          bt = fmaf(a.x, v.x, bt);
          bt = fmaf(a.y, v.y, bt);
          bt = fmaf(a.z, v.z, bt);
          bt = fmaf(a.w, v.w, bt);
        }
        two_sum_acc(s0, c0, bt);
        two_sum_acc(s0, c0, s1);
        return s0 + (c0 + c1);
      };
      if constexpr (NC > 1) {
        for (int o = tid; o < nr * b; o += kSiThreads) {
          const int i = o / b, j = o - i * b;
          S.W[o] = cv_row(S.Cl + i * Dq, j);
        }
      } else if (b > 16) {
        // (b > 16, m > 8): one output per thread and step, C rows from L2
        for (int o = tid; o < nr * b; o += kSiThreads) {
          const int i = o / b, j = o - i * b;
          S.W[o] = cv_row(C32 + (size_t)i * D, j);
        }
      } else {
        // C streams from global memory (L2) through two 16-row shared
        // buffers by cp.async, the next chunk in flight while this one is
        // used. C is symmetric, so chunk c (rows 16c..16c+15) holds the k
        // terms 16c..16c+15 of every output W[i][j] = sum_k C[k][i] V[k][j].
        // A thread owns a 2 x 4 block (rows i0, i0 + 1; columns 4g..4g+3)
        // and per k loads one float2 of C and one float4 of V: eight FMAs
        // per 24 bytes of shared memory instead of one per 8. Each 8-term
        // FMA block is added to the output by TwoSum.
        const int n4 = Dq >> 2;
        const int nchunk = (D + 15) >> 4;
        auto issue = [&](int c) {
          float* dst = S.Cst + (c & 1) * 16 * ROWS;
          const int rows = min(16, D - c * 16);
          for (int e = tid; e < rows * n4; e += kSiThreads) {
            const int i = e / n4, k4 = e - i * n4;
            const uint32_t sa = smem_u32(dst + i * Dq + 4 * k4);
            const float* gp = C32 + (size_t)(c * 16 + i) * D + 4 * k4;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gp) : "memory");
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
        };
        const int gj = (b + 3) >> 2;
        const int ntask = (D >> 1) * gj;
        const bool act = tid < ntask;
        const int i0 = act ? 2 * (tid / gj) : 0, g = act ? tid % gj : 0;
        float sa[8], sc[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) sa[o] = sc[o] = 0.f;
        issue(0);
        for (int c = 0; c < nchunk; ++c) {
          if (c + 1 < nchunk) {
            issue(c + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
          } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
          }
          __syncthreads();
          const float* cb = S.Cst + (c & 1) * 16 * ROWS;
          const int kn = min(16, D - c * 16);
          if (act) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float pb[8];
#pragma unroll
              for (int o = 0; o < 8; ++o) pb[o] = 0.f;
              if (h * 8 < kn) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                  const int k = h * 8 + kk;
                  if (k >= kn) break;  // the last chunk may hold 4, 8 or 12 rows
                  const float2 cv = *reinterpret_cast<const float2*>(cb + k * Dq + i0);
                  const float4 v = *reinterpret_cast<const float4*>(S.Vn + (c * 16 + k) * kSiMaxB + 4 * g);
                  pb[0] = fmaf(cv.x, v.x, pb[0]);
                  pb[1] = fmaf(cv.x, v.y, pb[1]);
                  pb[2] = fmaf(cv.x, v.z, pb[2]);
                  pb[3] = fmaf(cv.x, v.w, pb[3]);
                  pb[4] = fmaf(cv.y, v.x, pb[4]);
                  pb[5] = fmaf(cv.y, v.y, pb[5]);
                  pb[6] = fmaf(cv.y, v.z, pb[6]);
                  pb[7] = fmaf(cv.y, v.w, pb[7]);
                }
#pragma unroll
                for (int o = 0; o < 8; ++o) two_sum_acc(sa[o], sc[o], pb[o]);
              }
            }
          }
          __syncthreads();  // the buffer is refilled two chunks later
        }
        if (act) {
#pragma unroll
          for (int o = 0; o < 8; ++o) {
            const int i = i0 + (o >> 2), j = 4 * g + (o & 3);
            if (j < b) S.W[i * b + j] = sa[o] + sc[o];
          }
        }
      }
      __syncthreads();
      // Plain steps: after kSiRRWarm steps, seven steps of every eight skip
      // the Rayleigh-Ritz part (H, Jacobi, Ritz vectors, residuals). The
      // block spans C^t V_0 either way, so the subspace converges at the same
      // rate per multiplication; the basis from the last Rayleigh-Ritz step
      // keeps its column order and Ritz values for the scaling, and the last
      // step before the cap, like every stop test (steps 8, 16, ...: each is
      // also a window boundary of the stall test), is a Rayleigh-Ritz step.
      static_assert(kSiStallWin % 8 == 0, "stall-test windows end on Rayleigh-Ritz steps");
      const bool plain = t > kSiRRWarm && (t & 7) && t < maxit;
      if (plain) {
        const float sigma_p = sigma_rel * fmaxf(S.theta[0], 0.f);
        for (int o = tid; o < nr * b; o += kSiThreads) {
          const int i = o / b, j = o - i * b;
          const float den = fmaxf(S.theta[j], 0.f) + sigma_p;
          const float w = S.W[i * b + j], v = S.Vt[j * VLD + r0 + i];
          S.Wr[i * b + j] = den > 1e-30f ? (w + sigma_p * v) / den : v;
        }
        __syncthreads();
        si_cholqr_pass<NC>(S, S.Wr, nr, b, rank, xb, 0);
      } else {
      // ---- H = V^T W (local rows), exchanged
      if (NC == 1 && b <= 16 && nr > 64) {
        // rows split in quarters (see si_local_gram), the idle exchange buffer as scratch
        float* scr = &S.X[xb ^ 1][0][0];
        const int bb = b * b, q4 = (nr + 3) >> 2;
        for (int t2 = tid; t2 < 4 * bb; t2 += kSiThreads) {
          const int q = t2 / bb, e = t2 - q * bb, j = e / b, k = e - j * b;
          float s = 0.f;
          for (int i = q * q4; i < min(nr, (q + 1) * q4); ++i) s = fmaf(S.Vt[j * VLD + r0 + i], S.W[i * b + k], s);
          scr[t2] = s;
        }
        __syncthreads();
        for (int e = tid; e < bb; e += kSiThreads) S.part[e] = (scr[e] + scr[bb + e]) + (scr[2 * bb + e] + scr[3 * bb + e]);
      } else {
        for (int e = tid; e < kSiMaxB * kSiMaxB; e += kSiThreads) {
          const int j = e >> 5, k = e & 31;
          if (j < b && k < b) {
            float s = 0.f;
            for (int i = 0; i < nr; ++i) s = fmaf(S.Vt[j * VLD + r0 + i], S.W[i * b + k], s);
            S.part[j * b + k] = s;
          }
        }
      }
      __syncthreads();
      si_broadcast<NC>(S, xb, rank, b * b);
      si_sync<NC>();
      for (int e = tid; e < kSiMaxB * kSiMaxB; e += kSiThreads) {
        const int j = e >> 5, k = e & 31;
        if (j < b && k < b) S.M[j * kSiLd + k] = 0.5f * (si_sum<NC>(S, xb, j * b + k) + si_sum<NC>(S, xb, k * b + j));
      }
      xb ^= 1;
      __syncthreads();
      // ---- Rayleigh-Ritz
      if (tid < kSiJacThreads) si_jacobi(S, b);
      __syncthreads();
      const float th0 = fmaxf(S.theta[0], 0.f);
      const float sigma = sigma_rel * th0;
      for (int o = tid; o < nr * b; o += kSiThreads) {
        const int i = o / b, j = o - i * b;
        const int col = min(max(S.perm[j], 0), b - 1);
        float v = 0.f, w = 0.f;
        for (int kk = 0; kk < b; ++kk) {
          const float y = S.Y[kk * kSiLd + col];
          v = fmaf(S.Vt[kk * VLD + r0 + i], y, v);
          w = fmaf(S.W[i * b + kk], y, w);
        }
        S.Vr[i * b + j] = v;
        S.Wr[i * b + j] = w;
      }
      __syncthreads();
      // residual partials of the m leading pairs, then the scaled block
      // (C x_j + sigma x_j) / (theta_j + sigma)
      if (NC == 1) {
        // one warp per component, lanes over rows
        for (int j = warp; j < b; j += kSiThreads / 32) {
          float s = 0.f;
          if (j < m)
            for (int i = lane; i < nr; i += 32) {
              const float r = fmaf(-S.theta[j], S.Vr[i * b + j], S.Wr[i * b + j]);
              s = fmaf(r, r, s);
            }
          s = warp_sum(s);
          if (lane == 0) S.part[b * b + j] = s;
        }
      } else {
        for (int j = tid; j < b; j += kSiThreads) {
          float s = 0.f;
          if (j < m)
            for (int i = 0; i < nr; ++i) {
              const float r = fmaf(-S.theta[j], S.Vr[i * b + j], S.Wr[i * b + j]);
              s = fmaf(r, r, s);
            }
          S.part[b * b + j] = s;
        }
      }
      __syncthreads();  // the residuals read Wr before it is scaled in place
      for (int o = tid; o < nr * b; o += kSiThreads) {
        const int i = o / b, j = o - i * b;
        const float den = fmaxf(S.theta[j], 0.f) + sigma;
        const float w = S.Wr[i * b + j], v = S.Vr[i * b + j];
        S.Wr[i * b + j] = den > 1e-30f ? (w + sigma * v) / den : v;
      }
      __syncthreads();
      // ---- first Cholesky-QR exchange, carrying the residuals
      si_cholqr_pass<NC>(S, S.Wr, nr, b, rank, xb, b);
      bool done = t >= maxit;
      const float lim = eps * fmaxf(S.theta[0], 0.f);
      bool conv = true, bad = !(lim == lim);
      float rmax = 0.f;
      for (int j = 0; j < m; ++j) {
        conv = conv && (sqrtf(S.res[j]) <= lim);
        bad = bad || !(S.res[j] == S.res[j]);
        rmax = fmaxf(rmax, sqrtf(S.res[j]));
      }
      // Stall: once past kSiStallStart steps, at every window boundary the
      // observed contraction of the largest residual over the last window
      // predicts the steps still needed to reach eps; when that does not fit
      // in the cap (or the residual no longer falls: the FP32 floor), stop
      // now with the current Ritz vectors rather than at the cap. Nearly
      // degenerate spectra (isotropic clouds, D > 32) converge at rates of
      // 0.99 per step or slower and would otherwise run to the cap.
      if (!conv && t % kSiStallWin == 0) {
        r_prev = r_cur;
        r_cur = S.theta[0] > 0.f ? rmax / S.theta[0] : 0.f;
        if (t >= kSiStallStart && r_prev > 0.f) {
          const float rate = r_cur / r_prev;
          if (!(rate < 1.f)) {
            done = true;
          } else {
            const float need = (float)kSiStallWin * logf(eps / r_cur) / logf(rate);
            done = done || (float)t + need > (float)maxit;
          }
        }
      }
      if (done || conv || bad) {  // NaN input: stop (the Gram pass flags it)
        for (int e = tid; e < nr * m; e += kSiThreads) {
          const int i = e / m, j = e - i * m;
          Uout[(size_t)j * D + r0 + i] = (double)S.Vr[i * b + j];
        }
        if (rank == 0 && tid == 0 && iters_out) *iters_out = t;
        break;
      }
      }  // Rayleigh-Ritz step
    }
    // ---- finish the first pass (Wr -> W). A second pass (W -> Wr) restores
    // orthogonality to FP32 rounding when the first one was not well
    // conditioned: the loss after one pass is about u kappa^2, and the
    // normalised Gram matrix I + E has kappa <= (1 + (b-1) e) / (1 - (b-1) e)
    // for off-diagonal correlations |E_jk| <= e: e <= 1e-2 gives kappa <= 1.36
    // at b = 16 (1.9 at b = 32), so one pass stays within about 2u (4u) of
    // orthogonality, and the next step's pass starts from there.
    float corr = 0.f, dummy = 0.f;
    for (int e = tid; e < kSiMaxB * kSiMaxB; e += kSiThreads) {
      const int j = e >> 5, k = e & 31;
      if (j < b && k < b && j != k) {
        const float den = sqrtf(S.M[j * kSiLd + j] * S.M[k * kSiLd + k]);
        corr = fmaxf(corr, den > 0.f ? fabsf(S.M[j * kSiLd + k]) / den : 1.f);
      }
    }
    si_block_max2(corr, dummy, S.red);
    const bool second = !(corr <= 1e-2f);
    if (warp == 0) si_chol_inv(S, b, lane);
    __syncthreads();
    si_apply_linv<ROWS>(S, S.Wr, S.W, nr, b);
    __syncthreads();
    const float* Q = S.W;
    if (second) {
      si_cholqr_pass<NC>(S, S.W, nr, b, rank, xb, 0);
      if (warp == 0) si_chol_inv(S, b, lane);
      __syncthreads();
      si_apply_linv<ROWS>(S, S.W, S.Wr, nr, b);
      __syncthreads();
      Q = S.Wr;
    }
    // ---- new rows of V to every CTA
    for (int e = tid; e < nr * b * NC; e += kSiThreads) {
      const int c = e / (nr * b), o = e - c * (nr * b);
      const int i = o / b, j = o - i * b;
      if constexpr (NC > 1)
        st_cluster_f32(map_to_cta(&S.Vt[j * VLD + r0 + i], (uint32_t)c), Q[o]);
      else {
        S.Vt[j * VLD + r0 + i] = Q[o];
        S.Vn[(r0 + i) * kSiMaxB + j] = Q[o];
      }
    }
    si_sync<NC>();
  }
  // every CTA leaves the loop in the same iteration; keep the cluster alive
  // until all remote accesses are done
  si_sync<NC>();
}

__global__ void __cluster_dims__(kSiCTAs, 1, 1) __launch_bounds__(kSiThreads, 1)
    subspace_kernel(const float* __restrict__ C32, int D, int m, int b, int maxit, float eps, float sigma_rel,
                    uint64_t seed, double* __restrict__ Uout, int* __restrict__ iters_out) {
  extern __shared__ __align__(16) uint8_t sism[];
  subspace_body<kSiCTAs, kSiMaxRows, kSiVld>(*reinterpret_cast<SiSmem*>(sism), C32, D, m, b, maxit, eps, sigma_rel,
                                             seed, Uout, iters_out);
}

// One CTA per pair of a batch; pairs of this launch's D class come from `list`.
template <int ROWS>
__global__ void __launch_bounds__(kSiThreads, 1)
    subspace1_batched_kernel(const BPair* __restrict__ P, const int* __restrict__ list, float eps, float sigma_rel,
                             uint64_t seed) {
  extern __shared__ __align__(16) uint8_t sism[];
  const BPair& q = P[list[blockIdx.x]];
  if (q.m < 1) return;
  const int b = si_block(q.D, q.m);
  subspace_body<1, ROWS, ROWS + 4>(*reinterpret_cast<SiSmemT<1, ROWS, ROWS + 4>*>(sism), q.C32, q.D, q.m, b,
                                   max(q.iters, 1), eps, sigma_rel, seed, q.U, q.iters_out);
}

// FP64 clean-up of the m Ritz vectors (one CTA of kSiFinThreads threads, D <=
// kSiFinThreads): Cholesky-QR applied twice in FP64, then the sign rule
// (largest |entry| positive, lowest index on ties). A pass forms the Gram
// matrix G = U^T U (each entry summed over kFinSplit row blocks, the blocks
// added in a fixed order), its Cholesky factor G = L L^T and U <- U L^-T.
// The Ritz vectors arrive orthonormal to FP32 rounding, so G = I + E with
// |E| ~ 1e-7: one pass leaves an orthogonality error of about u64 kappa(G)^2
// and the second removes what rounding of the first left. Q = U R^-1 with R
// upper triangular and a positive diagonal is the factorisation Gram-Schmidt
// computes, so the result is the same basis up to FP64 rounding, from a few
// block-wide steps instead of one reduction per vector and pass. A column
// whose pivot is not positive (a zero input vector) comes out zero.
constexpr int kFinSplit = 8;

size_t subspace_finalize_smem(int D, int m) {
  const size_t np = (size_t)m * (m + 1) / 2;
  return ((size_t)m * D + (size_t)2 * m * m + np * kFinSplit + m) * sizeof(double);
}

PROHD_DEV void subspace_finalize_body(const double* __restrict__ Uin, int D, int m, double* __restrict__ dirs,
                                      double* __restrict__ sm) {
  double* U = sm;                          // [m][D]: column k of the basis at U + k D
  double* G = U + (size_t)m * D;           // [m][m] Gram matrix, then L (lower)
  double* Li = G + m * m;                  // [m][m] L^-1 (lower)
  double* part = Li + m * m;               // [pairs][kFinSplit] partial sums
  double* dinv = part + (m * (m + 1) / 2) * kFinSplit;  // [m] 1 / L[j][j] (0: dropped column)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NW = kSiFinThreads / 32;
  for (int e = tid; e < m * D; e += kSiFinThreads) U[e] = Uin[e];
  __syncthreads();
  const int npair = m * (m + 1) / 2;
  const int rb = (D + kFinSplit - 1) / kFinSplit;
  for (int pass = 0; pass < 2; ++pass) {
    // partial sums of G[k][l] (k <= l) over row block s (rows s, s + 8, ...)
    for (int t = tid; t < npair * kFinSplit; t += kSiFinThreads) {
      const int pr = t / kFinSplit, s = t - pr * kFinSplit;
      int k = 0, rem = pr;  // pair index -> (k, l), k <= l, row-major over the upper triangle
      while (rem >= m - k) {
        rem -= m - k;
        ++k;
      }
      const int l = k + rem;
      const double* uk = U + (size_t)k * D;
      const double* ul = U + (size_t)l * D;
      double acc = 0.0;
      for (int i = 0; i < rb; ++i) {
        const int j = s + kFinSplit * i;
        if (j < D) acc = fma(uk[j], ul[j], acc);
      }
      part[t] = acc;
    }
    __syncthreads();
    for (int pr = tid; pr < npair; pr += kSiFinThreads) {
      int k = 0, rem = pr;
      while (rem >= m - k) {
        rem -= m - k;
        ++k;
      }
      const int l = k + rem;
      double g = 0.0;
#pragma unroll
      for (int s = 0; s < kFinSplit; ++s) g += part[pr * kFinSplit + s];
      G[k * m + l] = g;
      G[l * m + k] = g;
    }
    __syncthreads();
    // Cholesky (warp 0, lane i = row i; m <= 24 < 32), then column `lane` of L^-1
    if (warp == 0) {
      const int row = lane < m ? lane : m - 1;  // lanes past m shadow the last row, stores masked
      for (int j = 0; j < m; ++j) {
        double acc = G[row * m + j];
        for (int k = 0; k < j; ++k) acc = fma(-G[row * m + k], G[j * m + k], acc);
        const double piv = __shfl_sync(0xffffffffu, acc, j);
        const bool ok = piv > 0.0;
        const double r = ok ? 1.0 / sqrt(piv) : 0.0;
        __syncwarp();
        if (lane == j) {
          G[j * m + j] = ok ? piv * r : 0.0;
          dinv[j] = r;
        }
        if (lane > j && lane < m) G[lane * m + j] = acc * r;
        __syncwarp();
      }
      const int col = lane < m ? lane : m - 1;
      for (int i = 0; i < m; ++i) {
        double acc = i == col ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) acc = fma(-G[i * m + k], Li[k * m + col], acc);
        const double x = i >= col ? acc * dinv[i] : 0.0;
        __syncwarp();
        if (lane < m) Li[i * m + lane] = x;
        __syncwarp();
      }
    }
    __syncthreads();
    // U <- U L^-T, one row per thread: q[c] = sum_{k <= c} U[j][k] Li[c][k]
    for (int j = tid; j < D; j += kSiFinThreads) {
      double u[kSiMaxM];
#pragma unroll
      for (int k = 0; k < kSiMaxM; ++k) u[k] = k < m ? U[(size_t)k * D + j] : 0.0;
#pragma unroll
      for (int c = 0; c < kSiMaxM; ++c) {
        if (c < m) {
          double q = 0.0;
#pragma unroll
          for (int k = 0; k <= c; ++k) q = fma(u[k], Li[c * m + k], q);
          U[(size_t)c * D + j] = q;
        }
      }
    }
    __syncthreads();
  }
  // sign: one warp per vector
  for (int c = warp; c < m; c += NW) {
    const double* uc = U + (size_t)c * D;
    unsigned long long best = 0ull;
    int bi = D;
    for (int j = lane; j < D; j += 32) {  // ascending j: a tie keeps the lower index
      const unsigned long long mag = (unsigned long long)__double_as_longlong(fabs(uc[j]));
      if (bi == D || mag > best) {
        best = mag;
        bi = j;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const double sgn = uc[min(bi, D - 1)] < 0.0 ? -1.0 : 1.0;
    for (int j = lane; j < D; j += 32) dirs[(size_t)(c + 1) * D + j] = sgn * uc[j];
  }
}

// Rayleigh quotients lambda_l = u_l^T C u_l with the FP64 covariance: one warp
// per row i writes u_l[i] (C u_l)[i]; a second kernel sums the rows in order.
PROHD_DEV void rayleigh_rows_body(const double* __restrict__ C64, const double* __restrict__ dirs, int D, int m,
                                  double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= D) return;
  for (int l = 0; l < m; ++l) {
    const double* u = dirs + (size_t)(l + 1) * D;
    double s = 0.0;
    for (int k = lane; k < D; k += 32) s = fma(C64[(size_t)i * D + k], u[k], s);
    s = warp_sum(s);
    if (lane == 0) part[(size_t)l * D + i] = s * u[i];
  }
}

PROHD_DEV void rayleigh_sum_body(const double* __restrict__ part, int D, int m, double* __restrict__ eig) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = warp; l < m; l += blockDim.x >> 5) {
    double s = 0.0;
    for (int i = lane; i < D; i += 32) s += part[(size_t)l * D + i];
    s = warp_sum(s);
    if (lane == 0) eig[l] = s;
  }
}

__global__ void __launch_bounds__(kSiFinThreads)
    subspace_finalize_kernel(const double* __restrict__ Uin, int D, int m, double* __restrict__ dirs) {
  extern __shared__ double fin_sm[];
  subspace_finalize_body(Uin, D, m, dirs, fin_sm);
}
__global__ void rayleigh_rows_kernel(const double* __restrict__ C64, const double* __restrict__ dirs, int D, int m,
                                     double* __restrict__ part) {
  rayleigh_rows_body(C64, dirs, D, m, part);
}
__global__ void rayleigh_sum_kernel(const double* __restrict__ part, int D, int m, double* __restrict__ eig) {
  rayleigh_sum_body(part, D, m, eig);
}

// Batched forms: one block (finalize, sums) or one grid row (row partials) per pair.
__global__ void __launch_bounds__(kSiFinThreads) subspace_finalize_batched_kernel(const BPair* __restrict__ P) {
  extern __shared__ double fin_sm[];
  const BPair& q = P[blockIdx.x];
  if (q.m >= 1) subspace_finalize_body(q.U, q.D, q.m, q.dirs, fin_sm);
}
__global__ void rayleigh_rows_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  if (q.m >= 1) rayleigh_rows_body(q.C64, q.dirs, q.D, q.m, q.rpart);
}
__global__ void rayleigh_sum_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.x];
  if (q.m >= 1) rayleigh_sum_body(q.rpart, q.D, q.m, q.eig);
}

bool subspace_supported(int D, int m) { return D >= 1 && D <= kSiMaxD && m >= 1 && m <= kSiMaxM; }

size_t subspace_scratch_doubles(int D, int m) { return (size_t)2 * std::max(m, 1) * D + 8; }

cudaError_t subspace_run(prohd_ctx* ctx, const float* C32, const double* C64, int D, int m, int max_iters, double tol,
                         uint64_t seed, double* dirs, double* eig, double* scratch, cudaStream_t st) {
  (void)ctx;
  const int b = si_block(D, m);
  const float eps = (float)std::max(std::sqrt(2.0 * std::max(tol, 0.0)), 2e-6);
  double* Uout = scratch;
  double* part = scratch + (size_t)m * D;
  const size_t smem = sizeof(SiSmem);
  cudaError_t e = cudaFuncSetAttribute(subspace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  count_launch();
  subspace_kernel<<<kSiCTAs, kSiThreads, smem, st>>>(C32, D, m, b, std::max(max_iters, 1), eps, 0.01f, seed, Uout,
                                                     nullptr);
  if ((e = cudaGetLastError())) return e;
  const size_t fsm = subspace_finalize_smem(D, m);
  if ((e = cudaFuncSetAttribute(subspace_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm)))
    return e;
  count_launch();
  subspace_finalize_kernel<<<1, kSiFinThreads, fsm, st>>>(Uout, D, m, dirs);
  if (eig) {
    count_launch();
    rayleigh_rows_kernel<<<(D + 7) / 8, 256, 0, st>>>(C64, dirs, D, m, part);
    count_launch();
    rayleigh_sum_kernel<<<1, 256, 0, st>>>(part, D, m, eig);
  }
  return cudaGetLastError();
}

cudaError_t subspace_batched(const BPair* P, const int* const cls_pairs[3], const int ncls[3], int npairs, int Dmax,
                             int mmax, double tol, uint64_t seed, const cudaStream_t cls_st[3]) {
  (void)npairs;
  (void)Dmax;
  if (mmax < 1) return cudaSuccess;
  if (mmax > kSiMaxM || Dmax > kSiMaxD) return cudaErrorInvalidValue;
  const float eps = (float)std::max(std::sqrt(2.0 * std::max(tol, 0.0)), 2e-6);
  cudaError_t e;
  auto go = [&](auto kern, size_t smem, const int* list, int n, cudaStream_t s) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r) return r;
    count_launch();
    kern<<<n, kSiThreads, smem, s>>>(P, list, eps, 0.01f, seed);
    return cudaGetLastError();
  };
  // largest class first: its CTAs are the longest
  if ((e = go(subspace1_batched_kernel<256>, sizeof(SiSmemT<1, 256, 260>), cls_pairs[2], ncls[2], cls_st[2]))) return e;
  if ((e = go(subspace1_batched_kernel<128>, sizeof(SiSmemT<1, 128, 132>), cls_pairs[1], ncls[1], cls_st[1]))) return e;
  if ((e = go(subspace1_batched_kernel<64>, sizeof(SiSmemT<1, 64, 68>), cls_pairs[0], ncls[0], cls_st[0]))) return e;
  return cudaSuccess;
}

cudaError_t subspace_batched_finish(const BPair* P, int npairs, int Dmax, int mmax, cudaStream_t st) {
  if (mmax < 1) return cudaSuccess;
  const size_t fsm = subspace_finalize_smem(Dmax, mmax);
  cudaError_t e =
      cudaFuncSetAttribute(subspace_finalize_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  if (e) return e;
  count_launch();
  subspace_finalize_batched_kernel<<<npairs, kSiFinThreads, fsm, st>>>(P);
  count_launch();
  rayleigh_rows_batched_kernel<<<dim3((Dmax + 7) / 8, npairs), 256, 0, st>>>(P);
  count_launch();
  rayleigh_sum_batched_kernel<<<npairs, 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace prohd
