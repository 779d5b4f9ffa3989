// Top-m principal components of the union covariance C (Algorithm 2 step 2)
// by block (subspace) iteration with Rayleigh-Ritz, for D <= 256 and m <= 24.
//
// The top-m eigenvectors of C are a plain definition; the oracle reaches them
// by deflated power iteration, one vector at a time, and this path reaches
// the same vectors with a block of b = min(D, max(2m, m + 8), 32) vectors
// iterated together:
//   V orthonormal (D x b); W = C V; H = V^T W; H = Y diag(theta) Y^T (Jacobi);
//   Ritz vectors X = V Y, residuals r_j = W y_j - theta_j x_j;
//   stop when ||r_j|| <= eps theta_1 for the m leading pairs, else
//   V = orth((W Y + sigma X) diag(1 / (theta + sigma))) by Cholesky-QR, twice.
// The error of the leading m Ritz vectors falls like ((lambda_{b+1} + sigma) /
// (lambda_m + sigma))^t, against lambda_{l+1}/lambda_l per step for each
// vector of the power iteration. The shift sigma = theta_1 / 100 bounds the
// condition number of the scaled block (its Gram matrix is I plus the residual
// Gram over (theta + sigma)^2, so at most 1 + b 10^4), which keeps the FP32
// Cholesky-QR well conditioned; it slows the convergence factor only from
// lambda_{b+1}/lambda_m to (lambda_{b+1} + sigma)/(lambda_m + sigma).
// A residual bound eps = max(sqrt(2 tol), 1e-6) certifies each returned
// vector to within eps lambda_1 / gap_l in angle (the residual bound of the
// symmetric eigenproblem), FP32 arithmetic cannot certify much below 1e-6.
//
// One cluster of 8 CTAs runs the iteration: CTA r owns rows [r0, r1) of C
// (FP32, in shared memory) and of every D x b block, and holds a full copy of
// V. Each step exchanges three small b x b matrices (H, the two Cholesky-QR
// Gram matrices) and the new rows of V through distributed shared memory;
// every CTA sums the exchanged partials in the same order and repeats the
// small dense work (Jacobi, Cholesky), so all CTAs take the same decisions.
// C V accumulates 8-term FFMA blocks with error-free (TwoSum) addition of the
// blocks. The m Ritz vectors are then orthonormalised in FP64 (modified
// Gram-Schmidt, twice), normalised, signed (largest |entry| positive, lowest
// index on ties) and their Rayleigh quotients taken with the FP64 C.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kSiCTAs = 8;
constexpr int kSiThreads = 256;
constexpr int kSiMaxD = 256;
constexpr int kSiMaxB = 32;
constexpr int kSiMaxM = 24;
constexpr int kSiMaxRows = kSiMaxD / kSiCTAs;      // 32
constexpr int kSiLd = kSiMaxB + 1;                 // row stride of the small matrices
constexpr int kSiX = kSiMaxB * kSiMaxB + kSiMaxB;  // one exchange slot: b x b matrix + b values

struct SiSmem {
  float V[kSiMaxD * kSiMaxB];        // basis, all rows, row stride b
  float Cl[kSiMaxRows * kSiMaxD];    // this CTA's rows of C, row stride D
  float W[kSiMaxRows * kSiMaxB];     // C V, local rows
  float Vr[kSiMaxRows * kSiMaxB];    // Ritz vectors V Y, local rows
  float Wr[kSiMaxRows * kSiMaxB];    // W Y -> scaled block -> Q1 -> Q
  float part[kSiX];                  // this CTA's partial before an exchange
  float X[2][kSiCTAs][kSiX];         // exchange slots, double-buffered
  float M[kSiMaxB * kSiLd];          // summed small matrix
  float Y[kSiMaxB * kSiLd];          // Jacobi eigenvectors (columns)
  float L[kSiMaxB * kSiLd];          // Cholesky factor (lower)
  float theta[kSiMaxB];              // Ritz values by rank (descending)
  float res[kSiMaxB];                // summed squared residuals
  float cs[kSiMaxB / 2][2];
  int pq[kSiMaxB / 2][2];
  int perm[kSiMaxB];                 // perm[rank] = column of Y
  uint32_t key[kSiMaxB];             // order keys of the Ritz values
};

// Error-free s + x accumulated into (s, c).
PROHD_DEV void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float z = t - s;
  c += (s - (t - z)) + (x - z);
  s = t;
}

// Sends this CTA's part[0..n) into slot X[buf][rank] of every CTA of the cluster.
PROHD_DEV void si_broadcast(SiSmem& S, int buf, uint32_t rank, int n) {
  float* dst = &S.X[buf][rank][0];
  for (int e = threadIdx.x; e < n * kSiCTAs; e += blockDim.x) {
    const int c = e / n, i = e - c * n;
    st_cluster_f32(map_to_cta(dst + i, (uint32_t)c), S.part[i]);
  }
}

// out[i] = sum over CTAs (fixed order) of X[buf][*][off + i], i < n.
PROHD_DEV float si_sum(const SiSmem& S, int buf, int idx) {
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < kSiCTAs; ++r) s += S.X[buf][r][idx];
  return s;
}

// Cyclic Jacobi on the symmetric b x b matrix A (row stride kSiLd), one warp:
// A <- Y^T A Y diagonal, Y orthogonal. Disjoint rotations of one round of a
// round-robin tournament are applied together (rows, then columns).
PROHD_DEV void si_jacobi(SiSmem& S, int b, int lane) {
  float* A = S.M;
  float* Y = S.Y;
  for (int e = lane; e < b * b; e += 32) {
    const int r = e / b, c = e - r * b;
    Y[r * kSiLd + c] = r == c ? 1.f : 0.f;
  }
  __syncwarp();
  const int n = b + (b & 1);  // players; index b is a dummy when b is odd
  const int np = n / 2;
  for (int sweep = 0; sweep < 20; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = lane; e < b * b; e += 32) {
      const int r = e / b, c = e - r * b;
      const float v = A[r * kSiLd + c];
      if (r != c) off = fmaf(v, v, off);
      else dia = fmaf(v, v, dia);
    }
    off = __shfl_sync(0xffffffffu, warp_sum(off), 0);
    dia = __shfl_sync(0xffffffffu, warp_sum(dia), 0);
    if (!(off > 1e-14f * dia)) break;
    for (int round = 0; round < n - 1; ++round) {
      if (lane < np) {
        int p, q;
        if (lane == 0) {
          p = n - 1;
          q = round;
        } else {
          p = (round + lane) % (n - 1);
          q = (round - lane + n - 1) % (n - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        float c = 1.f, s = 0.f;
        if (q < b) {
          const float apq = A[p * kSiLd + q];
          if (apq != 0.f) {
            const float tau = (A[q * kSiLd + q] - A[p * kSiLd + p]) / (2.f * apq);
            const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
            c = 1.f / sqrtf(fmaf(t, t, 1.f));
            s = t * c;
          }
        }
        S.cs[lane][0] = c;
        S.cs[lane][1] = s;
        S.pq[lane][0] = p;
        S.pq[lane][1] = q;
      }
      __syncwarp();
      for (int e = lane; e < np * b; e += 32) {  // rows p, q
        const int k = e / b, col = e - k * b;
        const int p = S.pq[k][0], q = S.pq[k][1];
        if (q >= b) continue;
        const float c = S.cs[k][0], s = S.cs[k][1];
        const float ap = A[p * kSiLd + col], aq = A[q * kSiLd + col];
        A[p * kSiLd + col] = c * ap - s * aq;
        A[q * kSiLd + col] = s * ap + c * aq;
      }
      __syncwarp();
      for (int e = lane; e < np * b; e += 32) {  // columns p, q of A and of Y
        const int k = e / b, row = e - k * b;
        const int p = S.pq[k][0], q = S.pq[k][1];
        if (q >= b) continue;
        const float c = S.cs[k][0], s = S.cs[k][1];
        const float ap = A[row * kSiLd + p], aq = A[row * kSiLd + q];
        A[row * kSiLd + p] = c * ap - s * aq;
        A[row * kSiLd + q] = s * ap + c * aq;
        const float yp = Y[row * kSiLd + p], yq = Y[row * kSiLd + q];
        Y[row * kSiLd + p] = c * yp - s * yq;
        Y[row * kSiLd + q] = s * yp + c * yq;
      }
      __syncwarp();
    }
  }
  // Ritz values by rank: descending, lower column first on ties. Every key
  // is computed once into shared memory and all comparisons read those
  // integers, so the ranks are a permutation whatever the values (NaN too).
  if (lane < b) S.key[lane] = f32_key(A[lane * kSiLd + lane]);
  __syncwarp();
  if (lane < b) {
    const uint32_t kj = S.key[lane];
    int rank = 0;
    for (int k = 0; k < b; ++k) {
      const uint32_t kk = S.key[k];
      rank += (kk > kj) || (kk == kj && k < lane);
    }
    S.perm[rank] = lane;
    S.theta[rank] = A[lane * kSiLd + lane];
  }
  __syncwarp();
}

// Cholesky M = L L^T of the summed Gram matrix in S.M (one warp, lane = row).
// A pivot that rounding drove to or below zero is replaced by a tiny positive
// one: the corresponding column is then noise, which the second pass
// normalises.
PROHD_DEV void si_cholesky(SiSmem& S, int b, int lane) {
  const float floor_piv = 1e-30f + 1e-12f * fabsf(S.M[0]);
  for (int j = 0; j < b; ++j) {
    if (lane == j) {
      float d = S.M[j * kSiLd + j];
      for (int k = 0; k < j; ++k) d = fmaf(-S.L[j * kSiLd + k], S.L[j * kSiLd + k], d);
      S.L[j * kSiLd + j] = sqrtf(fmaxf(d, floor_piv));
    }
    __syncwarp();
    if (lane > j && lane < b) {
      float v = S.M[lane * kSiLd + j];
      for (int k = 0; k < j; ++k) v = fmaf(-S.L[lane * kSiLd + k], S.L[j * kSiLd + k], v);
      S.L[lane * kSiLd + j] = v / S.L[j * kSiLd + j];
    }
    __syncwarp();
  }
}

// Rows of Wr (local) <- rows of Wr L^{-T}: forward substitution per row.
PROHD_DEV void si_apply_rinv(SiSmem& S, int nr, int b) {
  const int i = threadIdx.x;
  if (i < nr) {
    float q[kSiMaxB];
#pragma unroll
    for (int j = 0; j < kSiMaxB; ++j) {
      if (j >= b) break;
      float v = S.Wr[i * b + j];
      for (int k = 0; k < j; ++k) v = fmaf(-S.L[j * kSiLd + k], q[k], v);
      q[j] = v / S.L[j * kSiLd + j];
    }
#pragma unroll
    for (int j = 0; j < kSiMaxB; ++j) {
      if (j >= b) break;
      S.Wr[i * b + j] = q[j];
    }
  }
}

// part[j*b + k] = sum_i Wr[i][j] Wr[i][k] over local rows.
PROHD_DEV void si_local_gram(SiSmem& S, int nr, int b) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int j = e / b, k = e - j * b;
    float s = 0.f;
    for (int i = 0; i < nr; ++i) s = fmaf(S.Wr[i * b + j], S.Wr[i * b + k], s);
    S.part[e] = s;
  }
}

__global__ void __cluster_dims__(kSiCTAs, 1, 1) __launch_bounds__(kSiThreads, 1)
    subspace_kernel(const float* __restrict__ C32, int D, int m, int b, int maxit, float eps, float sigma_rel,
                    uint64_t seed, double* __restrict__ Uout, int* __restrict__ iters_out) {
  extern __shared__ __align__(16) uint8_t sism[];
  SiSmem& S = *reinterpret_cast<SiSmem*>(sism);
  const uint32_t rank = cluster_rank();
  const int rows_per = (D + kSiCTAs - 1) / kSiCTAs;
  const int r0 = min(D, (int)rank * rows_per), r1 = min(D, r0 + rows_per);
  const int nr = r1 - r0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int e = tid; e < nr * D; e += kSiThreads) S.Cl[e] = C32[(size_t)r0 * D + e];
  // start block: column j is the oracle's start vector of component j + 1
  for (int e = tid; e < D * b; e += kSiThreads) {
    const int i = e / b, j = e - i * b;
    S.V[e] = (float)splitmix64_unit(seed, (uint64_t)(j + 1), (uint64_t)i);
  }
  __syncthreads();
  cluster_sync();

  int xb = 0;  // exchange buffer
  int t = 0;
  for (;; ++t) {
    float sigma = 0.f;
    if (t == 0) {
      // first pass only orthonormalises the start block
      for (int e = tid; e < nr * b; e += kSiThreads) S.Wr[e] = S.V[r0 * b + e];
      for (int j = tid; j < b; j += kSiThreads) S.part[b * b + j] = 0.f;
      __syncthreads();
    } else {
      // ---- W = C V for the local rows: 8-term FFMA blocks, TwoSum across blocks
      for (int o = tid; o < nr * b; o += kSiThreads) {
        const int i = o / b, j = o - i * b;
        const float* crow = S.Cl + i * D;
        float s = 0.f, c = 0.f;
        int k = 0;
        for (; k + 8 <= D; k += 8) {
          float blk = 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) blk = fmaf(crow[k + u], S.V[(k + u) * b + j], blk);
          two_sum_acc(s, c, blk);
        }
        float blk = 0.f;
        for (; k < D; ++k) blk = fmaf(crow[k], S.V[k * b + j], blk);
        two_sum_acc(s, c, blk);
        S.W[o] = s + c;
      }
      __syncthreads();
      // ---- H = V^T W (local rows), exchanged
      for (int e = tid; e < b * b; e += kSiThreads) {
        const int j = e / b, k = e - j * b;
        float s = 0.f;
        for (int i = 0; i < nr; ++i) s = fmaf(S.V[(r0 + i) * b + j], S.W[i * b + k], s);
        S.part[e] = s;
      }
      __syncthreads();
      si_broadcast(S, xb, rank, b * b);
      cluster_sync();
      for (int e = tid; e < b * b; e += kSiThreads) {
        const int j = e / b, k = e - j * b;
        S.M[j * kSiLd + k] = 0.5f * (si_sum(S, xb, j * b + k) + si_sum(S, xb, k * b + j));
      }
      xb ^= 1;
      __syncthreads();
      // ---- Rayleigh-Ritz
      if (warp == 0) si_jacobi(S, b, lane);
      __syncthreads();
      const float th0 = fmaxf(S.theta[0], 0.f);
      sigma = sigma_rel * th0;
      for (int o = tid; o < nr * b; o += kSiThreads) {
        const int i = o / b, j = o - i * b;
        const int col = min(max(S.perm[j], 0), b - 1);
        float v = 0.f, w = 0.f;
        for (int k = 0; k < b; ++k) {
          const float y = S.Y[k * kSiLd + col];
          v = fmaf(S.V[(r0 + i) * b + k], y, v);
          w = fmaf(S.W[i * b + k], y, w);
        }
        S.Vr[o] = v;
        S.Wr[o] = w;
      }
      __syncthreads();
      // residual partials of the m leading pairs, then the scaled block
      // (C x_j + sigma x_j) / (theta_j + sigma)
      for (int j = tid; j < b; j += kSiThreads) {
        float s = 0.f;
        if (j < m)
          for (int i = 0; i < nr; ++i) {
            const float r = fmaf(-S.theta[j], S.Vr[i * b + j], S.Wr[i * b + j]);
            s = fmaf(r, r, s);
          }
        S.part[b * b + j] = s;
      }
      __syncthreads();
      for (int o = tid; o < nr * b; o += kSiThreads) {
        const int j = o % b;
        const float den = fmaxf(S.theta[j], 0.f) + sigma;
        S.Wr[o] = den > 1e-30f ? (S.Wr[o] + sigma * S.Vr[o]) / den : S.Vr[o];
      }
      __syncthreads();
    }
    // ---- Cholesky-QR, first pass (its exchange also carries the residuals)
    si_local_gram(S, nr, b);
    __syncthreads();
    si_broadcast(S, xb, rank, b * b + b);
    cluster_sync();
    for (int e = tid; e < b * b; e += kSiThreads) {
      const int j = e / b, k = e - j * b;
      S.M[j * kSiLd + k] = si_sum(S, xb, e);
    }
    for (int j = tid; j < b; j += kSiThreads) S.res[j] = si_sum(S, xb, b * b + j);
    xb ^= 1;
    __syncthreads();
    if (t > 0) {
      bool done = t >= maxit;
      const float lim = eps * fmaxf(S.theta[0], 0.f);
      bool conv = true, bad = !(lim == lim);
      for (int j = 0; j < m; ++j) {
        conv = conv && (sqrtf(S.res[j]) <= lim);
        bad = bad || !(S.res[j] == S.res[j]);
      }
      done = done || conv || bad;  // NaN input: stop (the Gram pass flags it)
      if (done) {
        for (int e = tid; e < nr * m; e += kSiThreads) {
          const int i = e / m, j = e - i * m;
          Uout[(size_t)j * D + r0 + i] = (double)S.Vr[i * b + j];
        }
        if (rank == 0 && tid == 0 && iters_out) *iters_out = t;
        break;
      }
    }
    if (warp == 0) si_cholesky(S, b, lane);
    __syncthreads();
    si_apply_rinv(S, nr, b);
    __syncthreads();
    // ---- second pass
    si_local_gram(S, nr, b);
    __syncthreads();
    si_broadcast(S, xb, rank, b * b);
    cluster_sync();
    for (int e = tid; e < b * b; e += kSiThreads) {
      const int j = e / b, k = e - j * b;
      S.M[j * kSiLd + k] = si_sum(S, xb, e);
    }
    xb ^= 1;
    __syncthreads();
    if (warp == 0) si_cholesky(S, b, lane);
    __syncthreads();
    si_apply_rinv(S, nr, b);
    __syncthreads();
    // ---- new rows of V to every CTA
    for (int e = tid; e < nr * b * kSiCTAs; e += kSiThreads) {
      const int c = e / (nr * b), o = e - c * (nr * b);
      st_cluster_f32(map_to_cta(&S.V[r0 * b + o], (uint32_t)c), S.Wr[o]);
    }
    cluster_sync();
  }
  // every CTA leaves the loop in the same iteration; keep the cluster alive
  // until all remote accesses are done
  cluster_sync();
}

// FP64 clean-up of the m Ritz vectors (one CTA): modified Gram-Schmidt twice,
// normalisation, sign (largest |entry| positive, lowest index on ties).
__global__ void subspace_finalize_kernel(const double* __restrict__ Uin, int D, int m, double* __restrict__ dirs) {
  __shared__ double u[kSiMaxD];
  __shared__ double red[kSiThreads / 32];
  __shared__ unsigned long long s_best[kSiThreads / 32];
  __shared__ int s_idx;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto block_dot = [&](const double* a, const double* bvec) -> double {
    double s = 0.0;
    for (int j = tid; j < D; j += blockDim.x) s = fma(a[j], bvec[j], s);
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    double tsum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red[w];
    return tsum;
  };
  for (int l = 0; l < m; ++l) {
    for (int j = tid; j < D; j += blockDim.x) u[j] = Uin[(size_t)l * D + j];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < l; ++k) {
        const double* uk = dirs + (size_t)(k + 1) * D;
        const double d = block_dot(u, uk);
        for (int j = tid; j < D; j += blockDim.x) u[j] = fma(-d, uk[j], u[j]);
        __syncthreads();
      }
    const double nn = block_dot(u, u);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int j = tid; j < D; j += blockDim.x) u[j] *= inv;
    __syncthreads();
    // magnitudes are read back from shared memory in both passes, so the
    // maximum is always found again
    unsigned long long best = 0ull;
    for (int j = tid; j < D; j += blockDim.x) {
      const unsigned long long mag = (unsigned long long)__double_as_longlong(fabs(u[j]));
      best = mag > best ? mag : best;
    }
    best = warp_max_u64(best);
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long bb = 0ull;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bb = s_best[w] > bb ? s_best[w] : bb;
      s_best[0] = bb;
      s_idx = D;
    }
    __syncthreads();
    for (int j = tid; j < D; j += blockDim.x)
      if ((unsigned long long)__double_as_longlong(fabs(u[j])) == s_best[0]) atomicMin(&s_idx, j);
    __syncthreads();
    const double sgn = u[min(s_idx, D - 1)] < 0.0 ? -1.0 : 1.0;
    for (int j = tid; j < D; j += blockDim.x) dirs[(size_t)(l + 1) * D + j] = sgn * u[j];
    __syncthreads();
  }
}

// Rayleigh quotients lambda_l = u_l^T C u_l with the FP64 covariance: one warp
// per row i writes u_l[i] (C u_l)[i]; a second kernel sums the rows in order.
__global__ void rayleigh_rows_kernel(const double* __restrict__ C64, const double* __restrict__ dirs, int D, int m,
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

__global__ void rayleigh_sum_kernel(const double* __restrict__ part, int D, int m, double* __restrict__ eig) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = warp; l < m; l += blockDim.x >> 5) {
    double s = 0.0;
    for (int i = lane; i < D; i += 32) s += part[(size_t)l * D + i];
    s = warp_sum(s);
    if (lane == 0) eig[l] = s;
  }
}

bool subspace_supported(int D, int m) { return D >= 1 && D <= kSiMaxD && m >= 1 && m <= kSiMaxM; }

size_t subspace_scratch_doubles(int D, int m) { return (size_t)2 * std::max(m, 1) * D + 8; }

cudaError_t subspace_run(prohd_ctx* ctx, const float* C32, const double* C64, int D, int m, int max_iters, double tol,
                         uint64_t seed, double* dirs, double* eig, double* scratch, cudaStream_t st) {
  (void)ctx;
  const int b = std::min(D, std::min(kSiMaxB, std::max(2 * m, m + 8)));
  const float eps = (float)std::max(std::sqrt(2.0 * std::max(tol, 0.0)), 1e-6);
  double* Uout = scratch;
  double* part = scratch + (size_t)m * D;
  const size_t smem = sizeof(SiSmem);
  cudaError_t e = cudaFuncSetAttribute(subspace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  count_launch();
  subspace_kernel<<<kSiCTAs, kSiThreads, smem, st>>>(C32, D, m, b, std::max(max_iters, 1), eps, 0.01f, seed, Uout,
                                                     nullptr);
  if ((e = cudaGetLastError())) return e;
  count_launch();
  subspace_finalize_kernel<<<1, kSiThreads, 0, st>>>(Uout, D, m, dirs);
  if (eig) {
    count_launch();
    rayleigh_rows_kernel<<<(D + 7) / 8, 256, 0, st>>>(C64, dirs, D, m, part);
    count_launch();
    rayleigh_sum_kernel<<<1, 256, 0, st>>>(part, D, m, eig);
  }
  return cudaGetLastError();
}

}  // namespace prohd
