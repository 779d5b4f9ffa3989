// Learned projection directions: a small network that proposes extra
// directions from cheap set statistics (the direction dictionary the paper
// names as future work, Conclusion and Future Work). It only ever adds directions to the
// centroid axis and the principal components, so plain ProHD stays the
// fallback and the reference for its error.
//
// Network (per pair, D = dimension):
//   x   = features [10 D]: centroid difference, the 8 leading components
//         scaled by sqrt(lambda), the per-dimension union variances, all
//         divided by s = sqrt(trace(C) / D) (variances by s^2)
//   h1  = relu(x W1 + b1)            W1 [10D x 256]
//   h2  = relu(h1 W2 + b2)           W2 [256 x 256]
//   z   = h2 W3 + b3                 W3 [256 x 4D], z = 4 vectors z_j of D
//   u_j = z_j / ||z_j||              (normalised inside the network)
// Loss against the unit witness direction w = (a* - b*)/||a* - b*|| of the
// exact Hausdorff distance: 1 - (1/tau) log sum_j exp(tau (u_j . w)^2),
// tau = 10 (a soft maximum of the squared alignments), averaged over a batch.
//
// Kernels: strided GEMMs (FP32 on CUDA cores, or BF16 operands on the
// tensor cores with mma.sync m16n8k16 and FP32 accumulation) with fused
// bias / ReLU / ReLU-mask epilogues, the normalise + loss head with its
// gradient, bias gradients, Adam on FP32 master weights, counter-based
// initialisation and the feature kernel.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kMlpH = 256;
constexpr int kMlpDirs = 4;
constexpr int kMlpPCs = 8;
constexpr float kMlpTau = 10.f;

MlpShape mlp_shape(int D) {
  MlpShape s;
  s.D = D;
  s.n_in = 10 * D;
  s.h = kMlpH;
  s.n_out = kMlpDirs * D;
  auto al = [](size_t x) { return (x + 63) / 64 * 64; };
  size_t o = 0;
  s.w1 = o;
  o += al((size_t)s.n_in * s.h);
  s.b1 = o;
  o += al(s.h);
  s.w2 = o;
  o += al((size_t)s.h * s.h);
  s.b2 = o;
  o += al(s.h);
  s.w3 = o;
  o += al((size_t)s.h * s.n_out);
  s.b3 = o;
  o += al(s.n_out);
  s.nparam = o;
  return s;
}

// ---------------------------------------------------------------- GEMM

// C[M x N] = op(A)[M x K] op(B)[K x N] with element (m, k) of A at
// A[m * sam + k * sak] and (k, n) of B at B[k * sbk + n * sbn]; epilogue:
enum { kEpiStore = 0, kEpiBias = 1, kEpiBiasRelu = 2, kEpiReluMask = 3 };
// kEpiStore:    C = acc
// kEpiBias:     C = acc + bias[n]
// kEpiBiasRelu: C = max(acc + bias[n], 0)
// kEpiReluMask: C = mask[m][n] > 0 ? acc : 0 (mask with row stride ldc)
constexpr int kGBM = 64, kGBN = 64, kGBK = 16;

__device__ __forceinline__ uint16_t bf16_bits_rn(float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  return *reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int EPI>
__device__ __forceinline__ void gemm_epilogue(float acc, int m, int n, int M, int N, float* C, int64_t ldc,
                                              const float* bias, const float* mask) {
  if (m >= M || n >= N) return;
  float v = acc;
  if (EPI == kEpiBias || EPI == kEpiBiasRelu) v += bias[n];
  if (EPI == kEpiBiasRelu) v = fmaxf(v, 0.f);
  if (EPI == kEpiReluMask) v = mask[(int64_t)m * ldc + n] > 0.f ? v : 0.f;
  C[(int64_t)m * ldc + n] = v;
}

// FP32 operands, 4 x 4 outputs per thread.
template <int EPI>
__global__ void __launch_bounds__(256)
    mlp_gemm_f32_kernel(int M, int N, int K, const float* __restrict__ A, int64_t sam, int64_t sak,
                        const float* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc,
                        const float* __restrict__ bias, const float* __restrict__ mask) {
  __shared__ float As[kGBK][kGBM + 4];
  __shared__ float Bs[kGBK][kGBN + 4];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGBK) {
    for (int e = tid; e < kGBM * kGBK; e += 256) {
      const int mm = e / kGBK, kk = e % kGBK;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : 0.f;
    }
    for (int e = tid; e < kGBK * kGBN; e += 256) {
      const int kk = e / kGBN, nn = e % kGBN;
      const int k = k0 + kk, n = n0 + nn;
      Bs[kk][nn] = (k < K && n < N) ? B[(int64_t)k * sbk + (int64_t)n * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) gemm_epilogue<EPI>(acc[i][j], m0 + ty * 4 + i, n0 + tx * 4 + j, M, N, C, ldc, bias, mask);
}

// BF16 operands (rounded to nearest), FP32 accumulation on the tensor cores:
// mma.sync m16n8k16; 8 warps tile the 64 x 64 block as 4 x 2 warp tiles of
// 16 x 32 (four n8 fragments each).
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(256)
    mlp_gemm_bf16_kernel(int M, int N, int K, const float* __restrict__ A, int64_t sam, int64_t sak,
                         const float* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t ldc,
                         const float* __restrict__ bias, const float* __restrict__ mask) {
  // A tile row-major [m][k], B tile n-major [n][k] (k contiguous: the pairs
  // of a fragment register are adjacent); rows padded by 8 halves
  __shared__ __align__(16) uint16_t As[kGBM][kGBK + 8];
  __shared__ __align__(16) uint16_t Bs[kGBN][kGBK + 8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * kGBM, n0 = blockIdx.x * kGBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGBK) {
    for (int e = tid; e < kGBM * kGBK; e += 256) {
      const int mm = e / kGBK, kk = e % kGBK;
      const int m = m0 + mm, k = k0 + kk;
      As[mm][kk] = bf16_bits_rn((m < M && k < K) ? A[(int64_t)m * sam + (int64_t)k * sak] : 0.f);
    }
    for (int e = tid; e < kGBK * kGBN; e += 256) {
      const int nn = e / kGBK, kk = e % kGBK;
      const int k = k0 + kk, n = n0 + nn;
      Bs[nn][kk] = bf16_bits_rn((k < K && n < N) ? B[(int64_t)k * sbk + (int64_t)n * sbn] : 0.f);
    }
    __syncthreads();
    uint32_t a[4];
    const int r0 = wm * 16 + g;
    a[0] = *reinterpret_cast<const uint32_t*>(&As[r0][2 * t]);
    a[1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][2 * t]);
    a[2] = *reinterpret_cast<const uint32_t*>(&As[r0][2 * t + 8]);
    a[3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][2 * t + 8]);
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int nn = wn * 32 + f * 8 + g;
      uint32_t b[2];
      b[0] = *reinterpret_cast<const uint32_t*>(&Bs[nn][2 * t]);
      b[1] = *reinterpret_cast<const uint32_t*>(&Bs[nn][2 * t + 8]);
      mma_bf16_16816(acc[f], a, b);
    }
    __syncthreads();
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int m = m0 + wm * 16 + g, n = n0 + wn * 32 + f * 8 + 2 * t;
    gemm_epilogue<EPI>(acc[f][0], m, n, M, N, C, ldc, bias, mask);
    gemm_epilogue<EPI>(acc[f][1], m, n + 1, M, N, C, ldc, bias, mask);
    gemm_epilogue<EPI>(acc[f][2], m + 8, n, M, N, C, ldc, bias, mask);
    gemm_epilogue<EPI>(acc[f][3], m + 8, n + 1, M, N, C, ldc, bias, mask);
  }
}

cudaError_t mlp_gemm(int prec, int epi, int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B,
                     int64_t sbk, int64_t sbn, float* C, int64_t ldc, const float* bias, const float* mask,
                     cudaStream_t st) {
  dim3 grid((unsigned)ceil_div(N, kGBN), (unsigned)ceil_div(M, kGBM));
  count_launch();
#define PROHD_GEMM_CASE(E)                                                                                      \
  case E:                                                                                                       \
    if (prec == PROHD_BF16)                                                                                     \
      mlp_gemm_bf16_kernel<E><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, mask);    \
    else                                                                                                        \
      mlp_gemm_f32_kernel<E><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, mask);     \
    break;
  switch (epi) {
    PROHD_GEMM_CASE(kEpiStore)
    PROHD_GEMM_CASE(kEpiBias)
    PROHD_GEMM_CASE(kEpiBiasRelu)
    PROHD_GEMM_CASE(kEpiReluMask)
    default:
      return cudaErrorInvalidValue;
  }
#undef PROHD_GEMM_CASE
  return cudaGetLastError();
}

// ---------------------------------------------------------------- head

// One block per sample: u_j = z_j / ||z_j||; with a label w, the loss
// 1 - (1/tau) log sum_j exp(tau c_j), c_j = (u_j . w)^2, and its gradient
// dz_j = (g_j - (u_j . g_j) u_j) / ||z_j||, g_j = -(p_j / B) 2 (u_j . w) w,
// p = softmax(tau c).
__global__ void __launch_bounds__(128)
    mlp_head_kernel(const float* __restrict__ Z, int D, const float* __restrict__ W, int nbatch, float* __restrict__ U,
                    float* __restrict__ dZ, float* __restrict__ loss) {
  __shared__ float red[kMlpDirs][4];
  __shared__ float s_nrm[kMlpDirs], s_dot[kMlpDirs], s_p[kMlpDirs];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float* z = Z + (int64_t)b * kMlpDirs * D;
  const float* w = W ? W + (int64_t)b * D : nullptr;
  // norms and alignments of the four raw vectors
  float nn[kMlpDirs], dw[kMlpDirs];
#pragma unroll
  for (int j = 0; j < kMlpDirs; ++j) {
    float a = 0.f, c = 0.f;
    for (int k = tid; k < D; k += blockDim.x) {
      const float v = z[j * D + k];
      a = fmaf(v, v, a);
      if (w) c = fmaf(v, w[k], c);
    }
    nn[j] = warp_sum(a);
    dw[j] = warp_sum(c);
  }
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < kMlpDirs; ++j) {
      red[j][warp] = nn[j];
    }
  __syncthreads();
  if (tid < kMlpDirs) s_nrm[tid] = sqrtf(fmaxf((red[tid][0] + red[tid][1]) + (red[tid][2] + red[tid][3]), 1e-30f));
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < kMlpDirs; ++j) red[j][warp] = dw[j];
  __syncthreads();
  if (tid < kMlpDirs) s_dot[tid] = ((red[tid][0] + red[tid][1]) + (red[tid][2] + red[tid][3])) / s_nrm[tid];  // u_j . w
  __syncthreads();
  for (int j = 0; j < kMlpDirs; ++j)
    for (int k = tid; k < D; k += blockDim.x) U[((int64_t)b * kMlpDirs + j) * D + k] = z[j * D + k] / s_nrm[j];
  if (!w) return;
  if (tid == 0) {
    float c[kMlpDirs], mx = -1e30f;
#pragma unroll
    for (int j = 0; j < kMlpDirs; ++j) {
      c[j] = s_dot[j] * s_dot[j];
      mx = fmaxf(mx, kMlpTau * c[j]);
    }
    float se = 0.f;
#pragma unroll
    for (int j = 0; j < kMlpDirs; ++j) se += expf(kMlpTau * c[j] - mx);
#pragma unroll
    for (int j = 0; j < kMlpDirs; ++j) s_p[j] = expf(kMlpTau * c[j] - mx) / se;
    loss[b] = 1.f - (mx + logf(se)) / kMlpTau;
  }
  __syncthreads();
  // g_j = coef_j w with coef_j = -(p_j / B) 2 (u_j . w); u_j . g_j = coef_j (u_j . w)
  for (int j = 0; j < kMlpDirs; ++j) {
    const float coef = -(s_p[j] / (float)nbatch) * 2.f * s_dot[j];
    const float ug = coef * s_dot[j];
    const float inv = 1.f / s_nrm[j];
    for (int k = tid; k < D; k += blockDim.x) {
      const float u = z[j * D + k] * inv;
      dZ[((int64_t)b * kMlpDirs + j) * D + k] = (coef * w[k] - ug * u) * inv;
    }
  }
}

// db[n] = sum_m dY[m][n] (fixed order), and the mean loss when asked.
__global__ void mlp_colsum_kernel(const float* __restrict__ dY, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dY[(int64_t)m * N + n];
  db[n] = s;
}

__global__ void mlp_loss_mean_kernel(const float* __restrict__ loss, int B, float* __restrict__ out) {
  __shared__ float sh[32];
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += loss[b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t / (float)B;
  }
}

// ---------------------------------------------------------------- Adam, init

// Adam with bias correction: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void mlp_adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                                float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Weights uniform on [-r, r], r = sqrt(6 / fan_in) (He-uniform for ReLU),
// from the counter-based SplitMix64 stream of layer l: element i draws
// splitmix64_unit(seed, 100 + l, i). Biases zero; Adam moments zero.
__global__ void mlp_init_kernel(float* __restrict__ state, MlpShape s, uint64_t seed) {
  const int64_t total = 3 * (int64_t)s.nparam;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (e < (int64_t)s.nparam) {
      int layer = -1;
      int64_t i = 0;
      int fan = 1;
      if (e >= (int64_t)s.w1 && e < (int64_t)s.w1 + (int64_t)s.n_in * s.h) {
        layer = 1; i = e - s.w1; fan = s.n_in;
      } else if (e >= (int64_t)s.w2 && e < (int64_t)s.w2 + (int64_t)s.h * s.h) {
        layer = 2; i = e - s.w2; fan = s.h;
      } else if (e >= (int64_t)s.w3 && e < (int64_t)s.w3 + (int64_t)s.h * s.n_out) {
        layer = 3; i = e - s.w3; fan = s.h;
      }
      if (layer > 0) v = (float)(sqrt(6.0 / (double)fan) * splitmix64_unit(seed, (uint64_t)(100 + layer), (uint64_t)i));
    }
    state[e] = v;
  }
}

// ---------------------------------------------------------------- features

// x = [dmu / s, sqrt(max(lambda_l, 0)) u_l / s (l = 1..8), diag(C) / s^2],
// s^2 = trace(C) / D, from the set sums (shifted by the same pilot, so it
// cancels), the covariance and the components.
__device__ double mlp_block_sum(double v, double* sh /*[33]*/) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = l < (int)(blockDim.x >> 5) ? sh[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

__global__ void mlp_features_kernel(const double* __restrict__ sumA, const double* __restrict__ sumB, int64_t nA,
                                    int64_t nB, const double* __restrict__ C64, const double* __restrict__ dirs,
                                    const double* __restrict__ eig, int D, float* __restrict__ feat) {
  __shared__ double sh[33];
  double tr = 0.0;
  for (int k = threadIdx.x; k < D; k += blockDim.x) tr += C64[(int64_t)k * D + k];
  tr = mlp_block_sum(tr, sh);
  const double s2 = tr > 0.0 ? tr / (double)D : 1.0;
  const double is = 1.0 / sqrt(s2), is2 = 1.0 / s2;
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    feat[k] = (float)((sumB[k] / (double)nB - sumA[k] / (double)nA) * is);
    for (int l = 0; l < kMlpPCs; ++l)
      feat[(int64_t)(1 + l) * D + k] = (float)(sqrt(fmax(eig[l], 0.0)) * dirs[(int64_t)(1 + l) * D + k] * is);
    feat[(int64_t)9 * D + k] = (float)(C64[(int64_t)k * D + k] * is2);
  }
}

cudaError_t mlp_features(const double* sumA, const double* sumB, int64_t nA, int64_t nB, const double* C64,
                         const double* dirs, const double* eig, int D, float* feat, cudaStream_t st) {
  count_launch();
  mlp_features_kernel<<<1, 256, 0, st>>>(sumA, sumB, nA, nB, C64, dirs, eig, D, feat);
  return cudaGetLastError();
}

// FP64 unit directions from the network's FP32 ones (renormalised in FP64).
__global__ void mlp_dirs64_kernel(const float* __restrict__ U, int D, double* __restrict__ out) {
  __shared__ double sh[33];
  const float* u = U + (int64_t)blockIdx.x * D;
  double a = 0.0;
  for (int k = threadIdx.x; k < D; k += blockDim.x) a += (double)u[k] * (double)u[k];
  a = mlp_block_sum(a, sh);
  const double inv = a > 0.0 ? 1.0 / sqrt(a) : 0.0;
  for (int k = threadIdx.x; k < D; k += blockDim.x) out[(int64_t)blockIdx.x * D + k] = (double)u[k] * inv;
}

cudaError_t mlp_dirs64(const float* U, int count, int D, double* out, cudaStream_t st) {
  count_launch();
  mlp_dirs64_kernel<<<count, 128, 0, st>>>(U, D, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- passes

// Activations of a batch of B samples inside the scratch buffer.
struct MlpActs {
  float *h1, *h2, *z, *u, *dz, *dh2, *dh1, *loss, *grad, *lmean;
};
static MlpActs acts(const MlpShape& s, int B, float* scratch) {
  MlpActs a;
  size_t o = 0;
  auto take = [&](size_t n) {
    float* p = scratch + o;
    o += (n + 63) / 64 * 64;
    return p;
  };
  a.h1 = take((size_t)B * s.h);
  a.h2 = take((size_t)B * s.h);
  a.z = take((size_t)B * s.n_out);
  a.u = take((size_t)B * s.n_out);
  a.dz = take((size_t)B * s.n_out);
  a.dh2 = take((size_t)B * s.h);
  a.dh1 = take((size_t)B * s.h);
  a.loss = take((size_t)B);
  a.grad = take(s.nparam);
  a.lmean = take(1);
  return a;
}

size_t mlp_scratch_floats(int D, int B) {
  const MlpShape s = mlp_shape(D);
  auto al = [](size_t n) { return (n + 63) / 64 * 64; };
  return al((size_t)B * s.h) * 4 + al((size_t)B * s.n_out) * 3 + al(B) + al(s.nparam) + 64;
}

cudaError_t mlp_forward(const MlpShape& s, const float* P, const float* X, int B, int prec, float* scratch,
                        const float* W, cudaStream_t st) {
  MlpActs a = acts(s, B, scratch);
  cudaError_t e;
  if ((e = mlp_gemm(prec, kEpiBiasRelu, B, s.h, s.n_in, X, s.n_in, 1, P + s.w1, s.h, 1, a.h1, s.h, P + s.b1, nullptr, st)))
    return e;
  if ((e = mlp_gemm(prec, kEpiBiasRelu, B, s.h, s.h, a.h1, s.h, 1, P + s.w2, s.h, 1, a.h2, s.h, P + s.b2, nullptr, st)))
    return e;
  if ((e = mlp_gemm(prec, kEpiBias, B, s.n_out, s.h, a.h2, s.h, 1, P + s.w3, s.n_out, 1, a.z, s.n_out, P + s.b3, nullptr,
                    st)))
    return e;
  count_launch();
  mlp_head_kernel<<<B, 128, 0, st>>>(a.z, s.D, W, B, a.u, a.dz, a.loss);
  if ((e = cudaGetLastError())) return e;
  if (W) {
    count_launch();
    mlp_loss_mean_kernel<<<1, 256, 0, st>>>(a.loss, B, a.lmean);
  }
  return cudaGetLastError();
}

// Gradient of the mean loss with respect to every parameter into the
// scratch's grad block (layout of the parameters).
cudaError_t mlp_backward(const MlpShape& s, const float* P, const float* X, int B, int prec, float* scratch,
                         cudaStream_t st) {
  MlpActs a = acts(s, B, scratch);
  float* G = a.grad;
  cudaError_t e;
  // layer 3: dW3 = h2^T dz, db3 = colsum(dz), dh2 = (dz W3^T) * [h2 > 0]
  if ((e = mlp_gemm(prec, kEpiStore, s.h, s.n_out, B, a.h2, 1, s.h, a.dz, s.n_out, 1, G + s.w3, s.n_out, nullptr,
                    nullptr, st)))
    return e;
  count_launch();
  mlp_colsum_kernel<<<(unsigned)ceil_div(s.n_out, 256), 256, 0, st>>>(a.dz, B, s.n_out, G + s.b3);
  if ((e = mlp_gemm(prec, kEpiReluMask, B, s.h, s.n_out, a.dz, s.n_out, 1, P + s.w3, 1, s.n_out, a.dh2, s.h, nullptr,
                    a.h2, st)))
    return e;
  // layer 2
  if ((e = mlp_gemm(prec, kEpiStore, s.h, s.h, B, a.h1, 1, s.h, a.dh2, s.h, 1, G + s.w2, s.h, nullptr, nullptr, st)))
    return e;
  count_launch();
  mlp_colsum_kernel<<<(unsigned)ceil_div(s.h, 256), 256, 0, st>>>(a.dh2, B, s.h, G + s.b2);
  if ((e = mlp_gemm(prec, kEpiReluMask, B, s.h, s.h, a.dh2, s.h, 1, P + s.w2, 1, s.h, a.dh1, s.h, nullptr, a.h1, st)))
    return e;
  // layer 1 (the input gradient is not needed)
  if ((e = mlp_gemm(prec, kEpiStore, s.n_in, s.h, B, X, 1, s.n_in, a.dh1, s.h, 1, G + s.w1, s.h, nullptr, nullptr, st)))
    return e;
  count_launch();
  mlp_colsum_kernel<<<(unsigned)ceil_div(s.h, 256), 256, 0, st>>>(a.dh1, B, s.h, G + s.b1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpShape& s, float* state, const float* grad, float lr, int64_t step, cudaStream_t st) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
  count_launch();
  mlp_adam_kernel<<<(unsigned)std::min<int64_t>(4096, ceil_div((int64_t)s.nparam, 256)), 256, 0, st>>>(
      state, state + s.nparam, state + 2 * s.nparam, grad, (int64_t)s.nparam, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_init(const MlpShape& s, float* state, uint64_t seed, cudaStream_t st) {
  count_launch();
  mlp_init_kernel<<<1024, 256, 0, st>>>(state, s, seed);
  return cudaGetLastError();
}

MlpActsView mlp_acts_view(int D, int B, float* scratch) {
  const MlpShape s = mlp_shape(D);
  MlpActs a = acts(s, B, scratch);
  MlpActsView v;
  v.u = a.u;
  v.loss = a.loss;
  v.lmean = a.lmean;
  v.grad = a.grad;
  return v;
}

}  // namespace prohd
