// Projection directions (Algorithm 1 step 2, Algorithm 2 step 2).
//  * centroid axis u0 = (ybar - xbar)/||ybar - xbar||, e_1 below 1e-9;
//  * union covariance C = (1/N) sum (z - mu)(z - mu)^T of Z = [A; B]:
//    one pass over the points computes the shifted Gram G = sum (z-s)(z-s)^T
//    and the per-set sums of z - s (s = mean of the first <= 4096 rows of A),
//    then C = G/N - (mu-s)(mu-s)^T. Tiles accumulate 32 rows in FP32 and 32
//    such partials in FP32 before every flush into FP64 (covariance
//    accumulation in FP64 across rows and blocks);
//  * top-m eigenvectors of C by power iteration with deflation, run by one
//    cluster of 8 CTAs that keeps an FP32 copy of C in distributed shared
//    memory. Each step: w = C v (FP32), Gram-Schmidt against the previous
//    components (FP32, twice), v = w/||w|| in FP64; the stop test
//    1 - |<v_t, v_{t-1}>| < tol is decided by CTA 0 and broadcast, so all CTAs
//    leave the loop together. A converged vector is re-orthogonalised against
//    the previous components in FP64 (twice), normalised, its Rayleigh
//    quotient taken with the FP64 C, and its largest-magnitude entry made
//    positive. Start vectors: SplitMix64 (Steele, Lea, Flood 2014) in the
//    same counter layout as the oracle's.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

// ---------------------------------------------------------------- pilot shift

// Column sums of rows [256 y, 256 y + 256) of the first min(n, cap) rows of
// X, FP64, into part[y][c]; grid (ceil(D/32), ceil(cap/256)). The sums are
// deterministic (fixed order) and spread over enough blocks to keep the read
// of a few MB off the critical path.
__global__ void colsum_part_kernel(const float* __restrict__ X, int64_t n, int cap, int D, double* __restrict__ part) {
  __shared__ double sh[8][33];
  const int cl = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cl;
  const int64_t rows = n < cap ? n : cap;
  const int64_t r0 = (int64_t)blockIdx.y * 256;
  double s = 0.0;
  if (c < D)
    for (int64_t i = r0 + rg; i < r0 + 256 && i < rows; i += 8) s += (double)X[i * D + c];
  sh[rg][cl] = s;
  __syncthreads();
  if (rg == 0 && c < D) {
    double t = 0.0;
    for (int g = 0; g < 8; ++g) t += sh[g][cl];
    part[(size_t)blockIdx.y * D + c] = t;
  }
}

// s32[c] = (sum over slices, in order) / min(n, cap).
__global__ void pilot_shift_kernel(const double* __restrict__ part, int nslices, int64_t n, int cap, int D,
                                   float* __restrict__ s32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  const int64_t rows = n < cap ? n : cap;
  double t = 0.0;
  for (int y = 0; y < nslices; ++y) t += part[(size_t)y * D + c];
  s32[c] = (float)(t / (double)rows);
}

// ---------------------------------------------------------------- Gram

constexpr int kGT = 128;   // output tile edge
constexpr int kGR = 32;    // rows per smem chunk
constexpr int kGStride = kGT + 4;
constexpr int kGFlush = 32;  // chunks per FP32 partial before the FP64 flush

struct GramSmem {
  float zi[kGR][kGStride];
  float zj[kGR][kGStride];
  double acc64[256][64 + 1];  // per-thread FP64 accumulators (odd stride: no bank conflicts)
};

// grid (ntiles_upper, nsplit). Thread (ty, tx): 4 ty x 8 tx per warp.
__global__ void __launch_bounds__(256, 1)
    gram_kernel(const float* __restrict__ A, int64_t nA, const float* __restrict__ B, int64_t nB, int D,
                const float* __restrict__ s32, double* __restrict__ Gpart, double* __restrict__ sumApart,
                double* __restrict__ sumBpart, int* __restrict__ status) {
  extern __shared__ __align__(16) uint8_t gsm[];
  GramSmem& S = *reinterpret_cast<GramSmem*>(gsm);
  const int nt = (D + kGT - 1) / kGT;
  // tile index -> (ti, tj), ti <= tj
  int t = blockIdx.x, ti = 0;
  while (t >= nt - ti) { t -= nt - ti; ++ti; }
  const int tj = ti + t;
  const bool diag = ti == tj;
  const int64_t N = nA + nB;
  const int64_t per = (N + gridDim.y - 1) / gridDim.y;
  const int64_t r_begin = blockIdx.y * per, r_end = min(N, r_begin + per);

  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int ty = (w & 3) * 4 + (l >> 3), tx = (w >> 2) * 8 + (l & 7);
  // loads: element e = tid + 256 q of the 32 x 128 chunk -> row e>>7, col e&127
  const int lc = tid & 127, lr0 = tid >> 7;  // this thread's column; rows lr0 + 2q
  const int ci = ti * kGT + lc, cj = tj * kGT + lc;
  const float si = ci < D ? s32[ci] : 0.f, sj = cj < D ? s32[cj] : 0.f;

  float acc[8][8], mid[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) mid[i][j] = 0.f;
  for (int i = 0; i < 64; ++i) S.acc64[tid][i] = 0.0;
  double csA = 0.0, csB = 0.0;
  bool bad = false;

  auto load_row = [&](int64_t r, float& vi, float& vj) {
    vi = 0.f;
    vj = 0.f;
    if (r < r_end) {
      const float* z = r < nA ? A + r * D : B + (r - nA) * D;
      if (ci < D) vi = z[ci];
      if (cj < D) vj = diag ? vi : z[cj];
    }
  };

  int chunk = 0;
  float pi[16], pj[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) load_row(r_begin + lr0 + 2 * q, pi[q], pj[q]);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGR) {
    __syncthreads();
    float csa = 0.f, csb = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int64_t r = r0 + lr0 + 2 * q;
      const bool valid = r < r_end;
      bad |= !isfinite(pi[q]) || !isfinite(pj[q]);
      const float zi = valid && ci < D ? pi[q] - si : 0.f;
      const float zj = valid && cj < D ? pj[q] - sj : 0.f;
      S.zi[lr0 + 2 * q][lc] = zi;
      S.zj[lr0 + 2 * q][lc] = zj;
      if (diag) {
        if (r < nA) csa += zi;
        else csb += zi;
      }
    }
    csA += (double)csa;
    csB += (double)csb;
    __syncthreads();
    // prefetch the next chunk while computing this one
#pragma unroll
    for (int q = 0; q < 16; ++q) load_row(r0 + kGR + lr0 + 2 * q, pi[q], pj[q]);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int r = 0; r < kGR; ++r) {
      float4 a0 = *reinterpret_cast<const float4*>(&S.zi[r][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&S.zi[r][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&S.zj[r][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&S.zj[r][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) mid[i][j] += acc[i][j];
    if (++chunk == kGFlush) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          S.acc64[tid][i * 8 + j] += (double)mid[i][j];
          mid[i][j] = 0.f;
        }
    }
  }
  // final flush and write-out
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) S.acc64[tid][i * 8 + j] += (double)mid[i][j];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = ti * kGT + ((i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gi >= D) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gj = tj * kGT + ((j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (gj < D && (!diag || gj >= gi)) Gpart[((size_t)blockIdx.y * D + gi) * D + gj] = S.acc64[tid][i * 8 + j];
    }
  }
  // column sums: the two loader threads of each column combine in a fixed order
  __shared__ double cs[2][2][kGT];
  if (diag) {
    cs[lr0][0][lc] = csA;
    cs[lr0][1][lc] = csB;
  }
  __syncthreads();
  if (diag && lr0 == 0 && ci < D) {
    sumApart[(size_t)blockIdx.y * D + ci] = cs[0][0][lc] + cs[1][0][lc];
    sumBpart[(size_t)blockIdx.y * D + ci] = cs[0][1][lc] + cs[1][1][lc];
  }
  if (__any_sync(0xffffffffu, bad) && l == 0) atomicMax(status, (int)PROHD_ENONFINITE);
}

// ---------------------------------------------------------------- finalise

// Block reduction of one double (fixed order: deterministic).
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = l < nw ? sh[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// Sums the per-split partials in split order (deterministic).
__global__ void reduce_parts_kernel(const double* __restrict__ Gpart, const double* __restrict__ sumApart,
                                    const double* __restrict__ sumBpart, int nsplit, int D, double* __restrict__ G,
                                    double* __restrict__ sumA, double* __restrict__ sumB) {
  const int64_t DD = (int64_t)D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < DD + 2 * D; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < DD) {
      const int i = (int)(e / D), j = (int)(e % D);
      if (j < i) continue;
      double s = 0.0;
      for (int p = 0; p < nsplit; ++p) s += Gpart[(size_t)p * DD + e];
      G[e] = s;
    } else {
      const int64_t c = e - DD;
      const double* src = c < D ? sumApart : sumBpart;
      const int cc = (int)(c < D ? c : c - D);
      double s = 0.0;
      for (int p = 0; p < nsplit; ++p) s += src[(size_t)p * D + cc];
      (c < D ? sumA : sumB)[cc] = s;
    }
  }
}

// dirs[0] = centroid axis; C64 = G/N - dmu dmu^T (full symmetric); C32 copy.
__device__ __forceinline__ void centroid_axis_body(const double* __restrict__ sumA, const double* __restrict__ sumB,
                                                   int64_t nA, int64_t nB, int D, double* __restrict__ dirs,
                                                   const float* __restrict__ s32 = nullptr,
                                                   float* __restrict__ center = nullptr, float* zero1 = nullptr) {
  __shared__ double sh[33];
  if (center) {
    // the union centroid: the shift plus the mean of the centred values
    const double invN = 1.0 / (double)(nA + nB);
    for (int c = threadIdx.x; c < D; c += blockDim.x) center[c] = (float)((double)s32[c] + (sumA[c] + sumB[c]) * invN);
  }
  if (zero1 && threadIdx.x == 0) *zero1 = 0.f;
  double part = 0.0;
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    double u = sumB[c] / (double)nB - sumA[c] / (double)nA;
    part += u * u;
  }
  const double nrm = sqrt(block_sum(part, sh));
  for (int c = threadIdx.x; c < D; c += blockDim.x) {
    double u = sumB[c] / (double)nB - sumA[c] / (double)nA;
    dirs[c] = nrm < 1e-9 ? (c == 0 ? 1.0 : 0.0) : u / nrm;
  }
}

__global__ void centroid_axis_kernel(const double* __restrict__ sumA, const double* __restrict__ sumB, int64_t nA,
                                     int64_t nB, int D, double* __restrict__ dirs, const float* __restrict__ s32,
                                     float* __restrict__ center, float* zero1) {
  centroid_axis_body(sumA, sumB, nA, nB, D, dirs, s32, center, zero1);
}

__device__ __forceinline__ void cov_finalize_body(const double* __restrict__ G, const double* __restrict__ sumA,
                                                  const double* __restrict__ sumB, int64_t nA, int64_t nB, int D,
                                                  double* __restrict__ C64, float* __restrict__ C32) {
  // one FP64 reciprocal, then products (FP64 division is slow on this GPU);
  // each product is within one rounding of the quotient
  const double invN = 1.0 / (double)(nA + nB);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)D * D;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / D), j = (int)(e % D);
    const int a = i < j ? i : j, b = i < j ? j : i;
    const double di = (__ldg(sumA + i) + __ldg(sumB + i)) * invN, dj = (__ldg(sumA + j) + __ldg(sumB + j)) * invN;
    const double c = __ldg(G + (size_t)a * D + b) * invN - di * dj;
    C64[e] = c;
    C32[e] = (float)c;
  }
}

__global__ void cov_finalize_kernel(const double* __restrict__ G, const double* __restrict__ sumA,
                                    const double* __restrict__ sumB, int64_t nA, int64_t nB, int D,
                                    double* __restrict__ C64, float* __restrict__ C32) {
  cov_finalize_body(G, sumA, sumB, nA, nB, D, C64, C32);
}

// ---------------------------------------------------------------- batched pairs

// Pilot shift of every pair: s = mean of the first <= 4096 rows of A. Any
// shift gives the same C in exact arithmetic; a nearby one keeps the
// centred values small, so FP32 column sums (combined in FP64) suffice.
// Grid (kPilotSlices, pairs): block y sums the 256-row slice x of pair y's
// first rows, thread (d, g) rows g, g + G, ... of column d; the slices'
// sums are then added in order.
constexpr int kPilotSlices = 16;
__global__ void pilot_batched_kernel(const BPair* __restrict__ P) {
  __shared__ double sh[256];
  const BPair& q = P[blockIdx.y];
  const int D = q.D;
  const int64_t rows = q.nA < 4096 ? q.nA : 4096;
  const int64_t r0 = (int64_t)blockIdx.x * 256, r1 = min(rows, r0 + 256);
  const int G = D < 256 ? 256 / D : 1;
  const int d = threadIdx.x % D, g = threadIdx.x / D;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (g < G && threadIdx.x < G * D) {
    int64_t r = r0 + g;
    for (; r + 3 * G < r1; r += 4 * G) {
      s0 += __ldg(q.A + r * D + d);
      s1 += __ldg(q.A + (r + G) * D + d);
      s2 += __ldg(q.A + (r + 2 * G) * D + d);
      s3 += __ldg(q.A + (r + 3 * G) * D + d);
    }
    for (; r < r1; r += G) s0 += __ldg(q.A + r * D + d);
  }
  sh[threadIdx.x] = ((double)s0 + (double)s1) + ((double)s2 + (double)s3);
  __syncthreads();
  if ((int)threadIdx.x < D) {
    double t = 0.0;
    for (int gg = 0; gg < G; ++gg) t += sh[gg * D + threadIdx.x];
    q.pilot_part[(size_t)blockIdx.x * D + threadIdx.x] = t;
  }
}

__global__ void pilot_finish_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.x];
  const int64_t rows = q.nA < 4096 ? q.nA : 4096;
  for (int d = threadIdx.x; d < q.D; d += blockDim.x) {
    double t = 0.0;
    for (int y = 0; y < kPilotSlices; ++y) t += q.pilot_part[(size_t)y * q.D + d];
    q.s32[d] = (float)(t / (double)rows);
  }
}

__global__ void centroid_axis_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.x];
  centroid_axis_body(q.sumA, q.sumB, q.nA, q.nB, q.D, q.dirs);
}

__global__ void cov_finalize_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  cov_finalize_body(q.G, q.sumA, q.sumB, q.nA, q.nB, q.D, q.C64, q.C32);
}

cudaError_t pilot_batched(const BPair* P, int npairs, cudaStream_t st) {
  count_launch(2);
  pilot_batched_kernel<<<dim3(kPilotSlices, npairs), 256, 0, st>>>(P);
  pilot_finish_batched_kernel<<<npairs, 256, 0, st>>>(P);
  return cudaGetLastError();
}

size_t pilot_part_doubles(int D) { return (size_t)kPilotSlices * D; }

cudaError_t covariance_batched(const BPair* P, int npairs, int Dmax, cudaStream_t st) {
  count_launch();
  centroid_axis_batched_kernel<<<npairs, 256, 0, st>>>(P);
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(32, ceil_div((int64_t)Dmax * Dmax, 1024)));
  count_launch();
  cov_finalize_batched_kernel<<<dim3(gx, npairs), 256, 0, st>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- power iteration

constexpr int kPiCTAs = 8;
constexpr int kPiThreads = 256;
constexpr int kPiMaxD = 1024;
constexpr int kPiMaxM = 64;

// Batched block sums of K values per thread (K <= KMAX), deterministic order.
template <int KMAX>
__device__ void block_sums(double (&v)[KMAX], int K, double* sh /*[8][KMAX]*/, double* out /*[KMAX]*/) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (k >= K) break;
    double x = warp_sum(v[k]);
    if (l == 0) sh[w * KMAX + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int ww = 0; ww < kPiThreads / 32; ++ww) s += sh[ww * KMAX + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Batched block sums of K FP32 values per thread (K <= KMAX), fixed order.
template <int KMAX>
__device__ void block_sums_f32(float (&v)[KMAX], int K, float* sh /*[8][KMAX]*/, float* out /*[KMAX]*/) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    if (k >= K) break;
    float x = warp_sum(v[k]);
    if (l == 0) sh[w * KMAX + k] = x;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    float s = 0.f;
    for (int ww = 0; ww < kPiThreads / 32; ++ww) s += sh[ww * KMAX + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

struct PiSmem {
  float w_recv[2][kPiMaxD];
  float v32[kPiMaxD];
  double v64[kPiMaxD];
  double red_sh[8 * 32];
  double red_out[32];
  float red_shf[8 * 32];
  float red_outf[32];
  double lam_part[kPiCTAs];
  int flag[2];
};

// Each CTA holds rows [r0, r1) of C (FP32) when they fit in shared memory;
// otherwise it reads them from C32 in global memory. U64 is a per-CTA scratch
// copy of the finished components: [kPiCTAs][m][D].
__global__ void __cluster_dims__(kPiCTAs, 1, 1) __launch_bounds__(kPiThreads, 1)
    power_iter_kernel(const double* __restrict__ C64, const float* __restrict__ C32, int D, int m, int maxit,
                      double tol, uint64_t seed, int c_in_smem, int u_in_smem, double* __restrict__ dirs,
                      double* __restrict__ eig,
                      double* __restrict__ U64all, float* __restrict__ U32all) {
  extern __shared__ __align__(16) uint8_t pism[];
  PiSmem& S = *reinterpret_cast<PiSmem*>(pism);
  float* Cs = reinterpret_cast<float*>(pism + sizeof(PiSmem));
  const uint32_t rank = cluster_rank();
  const int rows_per = (D + kPiCTAs - 1) / kPiCTAs;
  const int r0 = (int)rank * rows_per, r1 = min(D, r0 + rows_per);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* U64 = U64all + (size_t)rank * m * D;
  float* U32 = U32all + (size_t)rank * m * D;

  if (c_in_smem)
    for (int e = tid; e < (r1 - r0) * D; e += kPiThreads) Cs[e] = C32[(size_t)r0 * D + e];
  const float* Crow = c_in_smem ? Cs : C32 + (size_t)r0 * D;
  if (tid < 2) S.flag[tid] = 0;
  __syncthreads();
  cluster_sync();

  constexpr int KM = 12;  // values per batched block reduction (register-resident)
  double part[KM];
  const int rows_warp = (rows_per + kPiThreads / 32 - 1) / (kPiThreads / 32);
  // finished components in FP32 for the per-step Gram-Schmidt: shared memory when they fit
  float* Us = reinterpret_cast<float*>(pism + sizeof(PiSmem) + (c_in_smem ? (size_t)rows_per * D * sizeof(float) : 0));
  float* Uf = u_in_smem ? Us : U32;

  for (int l = 1; l <= m; ++l) {
    const int np = l - 1;  // previous components
    // ---- start vector, FP64 deflation (twice), normalisation
    for (int j = tid; j < D; j += kPiThreads) S.v64[j] = splitmix64_unit(seed, (uint64_t)l, (uint64_t)j);
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass)
      for (int k0 = 0; k0 < np; k0 += KM) {
        const int kk = min(KM, np - k0);
#pragma unroll
        for (int k = 0; k < KM; ++k) part[k] = 0.0;
        for (int j = tid; j < D; j += kPiThreads)
#pragma unroll
          for (int k = 0; k < KM; ++k)
            if (k < kk) part[k] += U64[(size_t)(k0 + k) * D + j] * S.v64[j];
        block_sums<KM>(part, kk, S.red_sh, S.red_out);
        for (int j = tid; j < D; j += kPiThreads) {
          double x = S.v64[j];
          for (int k = 0; k < kk; ++k) x -= S.red_out[k] * U64[(size_t)(k0 + k) * D + j];
          S.v64[j] = x;
        }
        __syncthreads();
      }
    {
      double nn = 0.0;
      for (int j = tid; j < D; j += kPiThreads) nn += S.v64[j] * S.v64[j];
#pragma unroll
      for (int k = 0; k < KM; ++k) part[k] = 0.0;
      part[0] = nn;
      block_sums<KM>(part, 1, S.red_sh, S.red_out);
      const double nv = sqrt(S.red_out[0]);
      for (int j = tid; j < D; j += kPiThreads) {
        if (nv > 0.0) S.v64[j] /= nv;
        S.v32[j] = (float)S.v64[j];
      }
      __syncthreads();
    }

    bool stop_local = false;  // CTA 0's decision, sent with the next step
    for (int t = 1; t <= maxit + 1; ++t) {
      const int buf = t & 1;
      // ---- w = C v for this CTA's rows, scattered to every CTA. Each warp
      // runs up to 4 rows (r0 + warp + 8 j) as independent compensated
      // (Ogita-Rump-Oishi Dot2) dot products: the FP32 result is as accurate
      // as twice-the-precision accumulation, so the iterate does not jitter
      // above the stop tolerance.
      for (int j0 = 0; j0 < rows_warp; j0 += 4) {
        float sum[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = lane; k < D; k += 32) {
          const float b = S.v32[k];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = r0 + warp + 8 * (j0 + u);
            if (r < r1) {
              const float a = Crow[(size_t)(r - r0) * D + k];
              const float pr = a * b;
              const float pe = fmaf(a, b, -pr);
              const float tt = sum[u] + pr;
              const float z = tt - sum[u];
              cmp[u] += (sum[u] - (tt - z)) + (pr - z) + pe;
              sum[u] = tt;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float sv = sum[u], cv = cmp[u];
          for (int o = 16; o > 0; o >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, sv, o), co = __shfl_xor_sync(0xffffffffu, cv, o);
            const float tt = sv + so;
            const float z = tt - sv;
            cv += co + (sv - (tt - z)) + (so - z);
            sv = tt;
          }
          const int r = r0 + warp + 8 * (j0 + u);
          if (r < r1 && lane < kPiCTAs) st_cluster_f32(map_to_cta(&S.w_recv[buf][r], lane), sv + cv);
        }
      }
      if (rank == 0 && tid < kPiCTAs) st_cluster_s32(map_to_cta(&S.flag[buf], tid), stop_local ? 1 : 0);
      cluster_sync();
      if (S.flag[buf] || t > maxit) break;  // v holds the result of the previous step
      float* w = S.w_recv[buf];
      // ---- Gram-Schmidt (FP32, twice) against the previous components. The
      // projections are small corrections and are reduced in FP32; the second
      // pass shares its reduction with ||w||^2 and <w, v_old>, which warp 0
      // sums in FP64 (FP64 arithmetic is scarce on this GPU, so only one warp
      // does it). With orthonormal u_k, ||w - sum d_k u_k||^2 = ||w||^2 -
      // sum d_k^2, and <u_k, v_old> vanishes to rounding.
      const bool merged = np <= KM;
      for (int pass = 0; pass < (merged ? 1 : 2); ++pass)
        for (int k0 = 0; k0 < np; k0 += KM) {
          const int kk = min(KM, np - k0);
          float pf[KM];
#pragma unroll
          for (int k = 0; k < KM; ++k) pf[k] = 0.f;
          for (int j = tid; j < D; j += kPiThreads)
#pragma unroll
            for (int k = 0; k < KM; ++k)
              if (k < kk) pf[k] = fmaf(Uf[(size_t)(k0 + k) * D + j], w[j], pf[k]);
          block_sums_f32<KM>(pf, kk, S.red_shf, S.red_outf);
          for (int j = tid; j < D; j += kPiThreads) {
            float x = w[j];
            for (int k = 0; k < kk; ++k) x -= S.red_outf[k] * Uf[(size_t)(k0 + k) * D + j];
            w[j] = x;
          }
          __syncthreads();
        }
      const int nq = merged ? np : 0;
      {
        float pf[KM];
#pragma unroll
        for (int k = 0; k < KM; ++k) pf[k] = 0.f;
        for (int j = tid; j < D; j += kPiThreads)
#pragma unroll
          for (int k = 0; k < KM; ++k)
            if (k < nq) pf[k] = fmaf(Uf[(size_t)k * D + j], w[j], pf[k]);
        if (warp == 0) {
          double nn = 0.0, dv = 0.0;
          for (int j = lane; j < D; j += 32) {
            const double x = (double)w[j];
            nn = fma(x, x, nn);
            dv = fma(x, S.v64[j], dv);
          }
          nn = warp_sum(nn);
          dv = warp_sum(dv);
          if (lane == 0) {
            S.red_out[0] = nn;
            S.red_out[1] = dv;
          }
        }
        block_sums_f32<KM>(pf, nq, S.red_shf, S.red_outf);  // its barriers also publish warp 0's sums
      }
      double nsq = S.red_out[0];
      for (int k = 0; k < nq; ++k) nsq -= (double)S.red_outf[k] * (double)S.red_outf[k];
      const double nw = sqrt(fmax(nsq, 0.0));
      const double cosv = nw > 0.0 ? fabs(S.red_out[1]) / nw : 1.0;
      // the second-pass correction is applied in FP64: an FP32 update would
      // move ||x|| away from nw by ~1e-8 and fake convergence at the next step
      if (nw > 0.0) {
        const double inv = 1.0 / nw;
        for (int j = tid; j < D; j += kPiThreads) {
          // the correction is ~1e-8 of w: FP32 suffices for it, the sum is FP64
          float corr = 0.f;
          for (int k = 0; k < nq; ++k) corr = fmaf(S.red_outf[k], Uf[(size_t)k * D + j], corr);
          S.v64[j] = ((double)w[j] - (double)corr) * inv;
          S.v32[j] = (float)S.v64[j];
        }
      }
      stop_local = (nw == 0.0) || (1.0 - cosv < tol);
      __syncthreads();
    }

    // ---- final FP64 deflation (twice) and normalisation
    for (int pass = 0; pass < 2; ++pass)
      for (int k0 = 0; k0 < np; k0 += KM) {
        const int kk = min(KM, np - k0);
#pragma unroll
        for (int k = 0; k < KM; ++k) part[k] = 0.0;
        for (int j = tid; j < D; j += kPiThreads)
#pragma unroll
          for (int k = 0; k < KM; ++k)
            if (k < kk) part[k] += U64[(size_t)(k0 + k) * D + j] * S.v64[j];
        block_sums<KM>(part, kk, S.red_sh, S.red_out);
        for (int j = tid; j < D; j += kPiThreads) {
          double x = S.v64[j];
          for (int k = 0; k < kk; ++k) x -= S.red_out[k] * U64[(size_t)(k0 + k) * D + j];
          S.v64[j] = x;
        }
        __syncthreads();
      }
    {
      double nn = 0.0;
      for (int j = tid; j < D; j += kPiThreads) nn += S.v64[j] * S.v64[j];
#pragma unroll
      for (int k = 0; k < KM; ++k) part[k] = 0.0;
      part[0] = nn;
      block_sums<KM>(part, 1, S.red_sh, S.red_out);
      const double nv = sqrt(S.red_out[0]);
      if (nv > 0.0)
        for (int j = tid; j < D; j += kPiThreads) S.v64[j] /= nv;
      __syncthreads();
    }
    // ---- sign: largest |entry| positive, lowest index on ties
    {
      // key: |v| bits (non-negative double) high, ~index low -> max picks lowest index
      unsigned long long best = 0ull;
      for (int j = tid; j < D; j += kPiThreads) {
        const unsigned long long mag = (unsigned long long)__double_as_longlong(fabs(S.v64[j]));
        // compare magnitudes exactly; pack index in a separate pass
        best = mag > best ? mag : best;
      }
      best = warp_max_u64(best);
      __shared__ unsigned long long s_best[8];
      __shared__ int s_idx;
      if (lane == 0) s_best[warp] = best;
      __syncthreads();
      if (tid == 0) {
        unsigned long long b = 0ull;
        for (int ww = 0; ww < kPiThreads / 32; ++ww) b = s_best[ww] > b ? s_best[ww] : b;
        s_best[0] = b;
        s_idx = D;
      }
      __syncthreads();
      for (int j = tid; j < D; j += kPiThreads)
        if ((unsigned long long)__double_as_longlong(fabs(S.v64[j])) == s_best[0]) atomicMin(&s_idx, j);
      __syncthreads();
      const double sgn = S.v64[min(s_idx, D - 1)] < 0.0 ? -1.0 : 1.0;
      for (int j = tid; j < D; j += kPiThreads) {
        const double x = sgn * S.v64[j];
        S.v64[j] = x;
        U64[(size_t)np * D + j] = x;
        Uf[(size_t)np * D + j] = (float)x;
        if (rank == 0) dirs[(size_t)l * D + j] = x;
      }
      __syncthreads();
    }
    // ---- Rayleigh quotient with the FP64 covariance, reduced over the cluster
    {
      double rq = 0.0;
      for (int r = r0 + warp; r < r1; r += kPiThreads / 32) {
        double s = 0.0;
        for (int c = lane; c < D; c += 32) s += C64[(size_t)r * D + c] * S.v64[c];
        s = warp_sum(s);
        rq += s * S.v64[r];
      }
      for (int k = 0; k < KM; ++k) part[k] = 0.0;
      part[0] = lane == 0 ? rq : 0.0;
      block_sums<KM>(part, 1, S.red_sh, S.red_out);
      if (tid == 0) st_cluster_f64(map_to_cta(&S.lam_part[rank], 0), S.red_out[0]);
      cluster_sync();
      if (rank == 0 && tid == 0 && eig) {
        double lam = 0.0;
        for (int c = 0; c < kPiCTAs; ++c) lam += S.lam_part[c];
        eig[l - 1] = lam;
      }
      cluster_sync();
    }
  }
}

// ---------------------------------------------------------------- host side

constexpr int kMaxSplit = 64;

struct DirBufs {
  float* s32 = nullptr;
  double* cpart = nullptr;  // pilot column sums per 256-row slice
  double *Gpart = nullptr, *sumApart = nullptr, *sumBpart = nullptr;
  double *G = nullptr, *sumA = nullptr, *sumB = nullptr, *C64 = nullptr;
  double* gc_scratch = nullptr;  // tensor-core Gram partials
  float* C32 = nullptr;
  double* U64 = nullptr;
  float* U32 = nullptr;
  double* si_scratch = nullptr;  // block-iteration outputs
};

static void dir_layout(Arena& ws, int D, int m, DirBufs& b, int gram_parts = 1) {
  b.s32 = ws.take<float>((size_t)D);
  b.cpart = ws.take<double>((size_t)16 * D);
  if (gram_tc_supported(D)) b.gc_scratch = ws.take<double>(gram_tc_scratch_doubles(D, kMaxSms, gram_parts));
  // CUDA-core Gram (D > 256, D % 4 != 0 or unaligned inputs)
  b.Gpart = ws.take<double>((size_t)kMaxSplit * D * D);
  b.sumApart = ws.take<double>((size_t)kMaxSplit * D);
  b.sumBpart = ws.take<double>((size_t)kMaxSplit * D);
  b.G = ws.take<double>((size_t)D * D);
  b.sumA = ws.take<double>((size_t)D);
  b.sumB = ws.take<double>((size_t)D);
  b.C64 = ws.take<double>((size_t)D * D);
  b.C32 = ws.take<float>((size_t)D * D);
  b.U64 = ws.take<double>((size_t)kPiCTAs * std::max(m, 1) * D);
  b.U32 = ws.take<float>((size_t)kPiCTAs * std::max(m, 1) * D);
  b.si_scratch = ws.take<double>(subspace_scratch_doubles(D, m));
}

void directions_layout(Arena& ws, int64_t nA, int64_t nB, int D, int m, int gram_parts) {
  (void)nA;
  (void)nB;
  DirBufs b;
  dir_layout(ws, D, m, b, gram_parts);
}

cudaError_t directions_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D, int m,
                           int max_iters, double tol, uint64_t seed, double* dirs, double* eig, int* status_dev,
                           Arena& ws, cudaStream_t st, int64_t timeout_ns, const InputFeed* feed, float* center32,
                           float* zero1) {
  DirBufs b;
  const int parts = feed ? feed->parts : 1;
  dir_layout(ws, D, m, b, parts);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  if (D > kPiMaxD || m > kPiMaxM) return cudaErrorInvalidValue;
  cudaError_t e;
  const int nsm = ctx->num_sms;
  const bool aligned = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
  const bool tc = gram_tc_supported(D) && aligned && ctx->num_sms <= kMaxSms && ctx->encode_tiled;
  if (feed && feed->ready) {
    // the pilot rows lie in A's first range when it holds 4096 rows; the
    // CUDA-core Gram reads everything at once
    const int wait_to = tc && nA / parts >= 4096 ? 1 : 2 * parts;
    for (int k = 0; k < wait_to; ++k)
      if ((e = cudaStreamWaitEvent(st, feed->ready[k], 0))) return e;
  }
  {
    // shift s = mean of the first <= 4096 rows of A (16 slices of 256 rows)
    const int nsl = (int)std::min<int64_t>(16, ceil_div(std::min<int64_t>(nA, 4096), 256));
    count_launch();
    colsum_part_kernel<<<dim3((D + 31) / 32, nsl), 256, 0, st>>>(A, nA, 4096, D, b.cpart);
    count_launch();
    pilot_shift_kernel<<<(D + 255) / 256, 256, 0, st>>>(b.cpart, nsl, nA, 4096, D, b.s32);
  }
  if (tc) {
    if ((e = gram_tc_run(ctx, A, nA, B, nB, D, b.s32, b.gc_scratch, b.G, b.sumA, b.sumB, status_dev,
                         timeout_ns > 0 ? timeout_ns : kDefaultTimeoutNs, st, feed)))
      return e;
  } else {
    const int nt = (D + kGT - 1) / kGT;
    const int ntiles = nt * (nt + 1) / 2;
    const int64_t N = nA + nB;
    // a whole number of blocks per SM wave
    int nsplit = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(nsm / ntiles, ceil_div(N, 4 * kGR)), kMaxSplit));
    cudaFuncSetAttribute(gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GramSmem));
    PhaseTimer pt_gram(ctx, PROHD_PH_GRAM, st);
    count_launch();
    gram_kernel<<<dim3(ntiles, nsplit), 256, sizeof(GramSmem), st>>>(A, nA, B, nB, D, b.s32, b.Gpart, b.sumApart,
                                                                    b.sumBpart, status_dev);
    pt_gram.stop();
    count_launch();
    reduce_parts_kernel<<<nsm, 256, 0, st>>>(b.Gpart, b.sumApart, b.sumBpart, nsplit, D, b.G, b.sumA, b.sumB);
    if ((e = cudaGetLastError())) return e;
  }
  count_launch();
  centroid_axis_kernel<<<1, 256, 0, st>>>(b.sumA, b.sumB, nA, nB, D, dirs, b.s32, center32, zero1);
  count_launch();
  cov_finalize_kernel<<<nsm, 256, 0, st>>>(b.G, b.sumA, b.sumB, nA, nB, D, b.C64, b.C32);
  if ((e = cudaGetLastError())) return e;
  if (m > 0 && subspace_supported(D, m)) {
    PhaseTimer pt_pow(ctx, PROHD_PH_POWER, st);
    if ((e = subspace_run(ctx, b.C32, b.C64, D, m, max_iters, tol, seed, dirs, eig, b.si_scratch, st))) return e;
  } else if (m > 0) {
    const int rows_per = (D + kPiCTAs - 1) / kPiCTAs;
    size_t cbytes = (size_t)rows_per * D * sizeof(float);
    int c_in_smem = sizeof(PiSmem) + cbytes <= (size_t)160 * 1024 ? 1 : 0;
    const size_t ubytes = (size_t)m * D * sizeof(float);
    int u_in_smem = sizeof(PiSmem) + (c_in_smem ? cbytes : 0) + ubytes <= (size_t)200 * 1024 ? 1 : 0;
    size_t smem = sizeof(PiSmem) + (c_in_smem ? cbytes : 0) + (u_in_smem ? ubytes : 0);
    cudaFuncSetAttribute(power_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    PhaseTimer pt_pow(ctx, PROHD_PH_POWER, st);
    count_launch();
    power_iter_kernel<<<kPiCTAs, kPiThreads, smem, st>>>(b.C64, b.C32, D, m, max_iters, tol, seed, c_in_smem,
                                                         u_in_smem, dirs, eig, b.U64, b.U32);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

// mean = s + (sum_A + sum_B) / N: the union mean from the shifted set sums.
__global__ void union_mean_kernel(const float* __restrict__ s32, const double* __restrict__ sumA,
                                  const double* __restrict__ sumB, int64_t N, int D, double* __restrict__ mean) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < D; d += gridDim.x * blockDim.x)
    mean[d] = (double)s32[d] + (sumA[d] + sumB[d]) / (double)N;
}

void covariance_layout(Arena& ws, int D) {
  DirBufs b;
  dir_layout(ws, D, 0, b);
  ws.take<double>((size_t)D);  // the centroid axis the directions pass writes
}

cudaError_t covariance_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D, double* C,
                           double* mean, int* status, Arena& ws, cudaStream_t st, int64_t timeout_ns) {
  Arena run = ws;
  DirBufs b;
  dir_layout(ws, D, 0, b);
  double* axis = ws.take<double>((size_t)D);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  cudaError_t e = directions_run(ctx, A, nA, B, nB, D, 0, 1, 0.0, 0, axis, nullptr, status, run, st, timeout_ns);
  if (e) return e;
  if ((e = cudaMemcpyAsync(C, b.C64, sizeof(double) * (size_t)D * D, cudaMemcpyDeviceToDevice, st))) return e;
  if (mean) {
    count_launch();
    union_mean_kernel<<<(D + 255) / 256, 256, 0, st>>>(b.s32, b.sumA, b.sumB, nA + nB, D, mean);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t directions_features(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                int max_iters, double tol, uint64_t seed, double* dirs, double* eig, float* feat,
                                int* status, Arena& ws, cudaStream_t st, int64_t timeout_ns) {
  Arena run = ws;
  cudaError_t e = directions_run(ctx, A, nA, B, nB, D, 8, max_iters, tol, seed, dirs, eig, status, run, st, timeout_ns);
  if (e) return e;
  DirBufs b;
  dir_layout(ws, D, 8, b);  // the buffers directions_run just filled
  return mlp_features(b.sumA, b.sumB, nA, nB, b.C64, dirs, eig, D, feat, st);
}

}  // namespace prohd
