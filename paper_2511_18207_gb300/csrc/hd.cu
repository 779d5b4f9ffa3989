// Exact Hausdorff distance H(A,B) = max{h(A,B), h(B,A)},
// h(A,B) = max_a min_b ||a-b||_2 (Eq. 1), as one distance contraction per
// pair of sets with the row minimum (h(A,B)) and the column minimum (h(B,A))
// reduced in the same pass.
//
// Two paths:
//  * PROHD_FP32 - CUDA-core tiles of direct differences sum_k (a_k-b_k)^2;
//    every row/column minimum carries its argmin (packed 64-bit atomics).
//  * PROHD_FP16 / PROHD_BF16 - tcgen05 tensor-core tiles of
//    ||a||^2 + ||b||^2 - 2 a.b on rounded, centred, power-of-two-scaled
//    copies of the points, FP32 accumulation in TMEM, fused row-min and
//    column-min epilogue. A rigorous per-row margin (rounding of the copies,
//    of the FP32 accumulation and of the epilogue) turns each low-precision
//    minimum into an interval; every row (column) whose interval reaches the
//    largest lower bound is rescored with the FP32 direct-difference tiles,
//    so the result is the FP32 path's up to FP32 rounding.
// The witness pairs' distances are finally recomputed in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

// =====================================================================
// FP32 direct-difference tiles (exact path and rescoring)
// =====================================================================

constexpr int kSimtBM = 128, kSimtBN = 128, kSimtBK = 16;

__device__ __forceinline__ int64_t ceil_div_dev(int64_t x, int64_t m) { return (x + m - 1) / m; }
// Candidate lists up to this length are rescored by rescore_few_kernel; the
// tiled kernel takes longer lists (it would spend whole 128-row tiles on them).
constexpr int kFewRows = 64;

// Persistent tile loop over rows of X (optionally a list of row ids) against
// all rows of Y. WANT_ROW: rowbest[out_row] = min (d^2, j); WANT_COL:
// colbest[j] = min (d^2, row id). Packed values are (float bits << 32 | idx).
// Two k-stages of the operand tiles; the column-minimum scratch reuses them
// after the k-loop (a barrier separates the last reads from its writes).
template <bool WANT_COL>
union SimtSmem {
  struct {
    __align__(16) float As[2][kSimtBK][kSimtBM + 4];
    __align__(16) float Bs[2][kSimtBK][kSimtBN + 4];
  } t;
  unsigned long long s_col[WANT_COL ? 16 : 1][WANT_COL ? kSimtBN : 1];
};

// One 128 x 128 tile (row block rt, column block ct).
template <bool ROW_LIST, bool WANT_ROW, bool WANT_COL>
__device__ __forceinline__ void simt_tile(SimtSmem<WANT_COL>& sm, const float* __restrict__ X,
                                          const int32_t* __restrict__ rowlist, int64_t nrows,
                                          const float* __restrict__ Y, int64_t ncols, int D,
                                          unsigned long long* __restrict__ rowbest,
                                          unsigned long long* __restrict__ colbest, int64_t rt, int64_t ct) {
  auto& As = sm.t.As;
  auto& Bs = sm.t.Bs;
  auto& s_col = sm.s_col;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int lr = tid >> 1, koff = (tid & 1) * 8;
  {
    const int64_t xr = rt * kSimtBM + lr, yr = ct * kSimtBN + lr;
    const bool vx = xr < nrows, vy = yr < ncols;
    const int64_t srcx = vx ? (ROW_LIST ? (int64_t)rowlist[xr] : xr) : 0;
    const float* xrow = X + srcx * D;
    const float* yrow = Y + (vy ? yr : 0) * D;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    // double-buffered k-steps: the next step's global loads are in flight
    // (in registers) while this step's tiles are used; one barrier per step
    float xa[8], yb[8];
    auto load = [&](int k0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + koff + e;
        xa[e] = (vx && k < D) ? __ldg(xrow + k) : 0.f;
        yb[e] = (vy && k < D) ? __ldg(yrow + k) : 0.f;
      }
    };
    auto store = [&](int stg) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        As[stg][koff + e][lr] = xa[e];
        Bs[stg][koff + e][lr] = yb[e];
      }
    };
    load(0);
    __syncthreads();  // the previous tile's readers of stage 0 (and of the column scratch) are done
    store(0);
    __syncthreads();
    for (int k0 = 0, stg = 0; k0 < D; k0 += kSimtBK, stg ^= 1) {
      const bool more = k0 + kSimtBK < D;
      if (more) load(k0 + kSimtBK);
#pragma unroll
      for (int kk = 0; kk < kSimtBK; ++kk) {
        float4 a0 = *reinterpret_cast<const float4*>(&As[stg][kk][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4*>(&As[stg][kk][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4*>(&Bs[stg][kk][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4*>(&Bs[stg][kk][64 + tx * 4]);
        float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float d = a[i] - b[j];
            acc[i][j] = fmaf(d, d, acc[i][j]);
          }
      }
      if (more) store(stg ^ 1);
      __syncthreads();
    }

    if (WANT_ROW) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        unsigned long long best = ~0ull;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
          const int64_t gc = ct * kSimtBN + c;
          if (gc < ncols) {
            unsigned long long p = pack_min(acc[i][j], (uint32_t)gc);
            best = p < best ? p : best;
          }
        }
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
          unsigned long long w = __shfl_xor_sync(0xffffffffu, best, o);
          best = w < best ? w : best;
        }
        const int64_t gr = rt * kSimtBM + r;
        if (tx == 0 && gr < nrows && best != ~0ull) atomicMin(rowbest + gr, best);
      }
    }
    if (WANT_COL) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
        unsigned long long best = ~0ull;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
          const int64_t gr = rt * kSimtBM + r;
          if (gr < nrows) {
            const uint32_t id = ROW_LIST ? (uint32_t)rowlist[gr] : (uint32_t)gr;
            unsigned long long p = pack_min(acc[i][j], id);
            best = p < best ? p : best;
          }
        }
        s_col[ty][c] = best;
      }
      __syncthreads();
      if (tid < kSimtBN) {
        unsigned long long best = s_col[0][tid];
#pragma unroll
        for (int t = 1; t < 16; ++t) best = s_col[t][tid] < best ? s_col[t][tid] : best;
        const int64_t gc = ct * kSimtBN + tid;
        if (gc < ncols && best != ~0ull) atomicMin(colbest + gc, best);
      }
      __syncthreads();
    }
  }
}

template <bool ROW_LIST, bool WANT_ROW, bool WANT_COL>
__device__ __forceinline__ void simt_dist_body(const float* __restrict__ X, const int32_t* __restrict__ rowlist,
                                               const int64_t* __restrict__ nrows_dev, const float* __restrict__ Y,
                                               const int64_t* __restrict__ ncols_dev, int D,
                                               unsigned long long* __restrict__ rowbest,
                                               unsigned long long* __restrict__ colbest) {
  __shared__ SimtSmem<WANT_COL> sm;
  const int64_t nrows = *nrows_dev, ncols = *ncols_dev;
  if (ROW_LIST && nrows <= kFewRows) return;
  const int64_t nct = (ncols + kSimtBN - 1) / kSimtBN;
  const int64_t ntiles = ((nrows + kSimtBM - 1) / kSimtBM) * nct;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    simt_tile<ROW_LIST, WANT_ROW, WANT_COL>(sm, X, rowlist, nrows, Y, ncols, D, rowbest, colbest, tile / nct,
                                            tile % nct);
}

template <bool ROW_LIST, bool WANT_ROW, bool WANT_COL>
__global__ void __launch_bounds__(256, 1)
    simt_dist_kernel(const float* __restrict__ X, const int32_t* __restrict__ rowlist,
                     const int64_t* __restrict__ nrows_dev, const float* __restrict__ Y,
                     const int64_t* __restrict__ ncols_dev, int D, unsigned long long* __restrict__ rowbest,
                     unsigned long long* __restrict__ colbest) {
  simt_dist_body<ROW_LIST, WANT_ROW, WANT_COL>(X, rowlist, nrows_dev, Y, ncols_dev, D, rowbest, colbest);
}

// Rescoring of a short candidate list (at most kFewRows rows of X, given by
// rowlist) against every row of Y, D <= 256: the candidates sit in shared
// memory, each warp streams rows of Y (lane = dimension, coalesced) and forms
// the FP32 direct-difference squared distance to every candidate, keeping
// per candidate the minimum packed (d^2, j). rowbest is indexed by position
// in the list, as in the tiled kernel.
__device__ __forceinline__ void rescore_few_body(const float* __restrict__ X, const int32_t* __restrict__ rowlist,
                                                 const int64_t* __restrict__ nrows_dev, const float* __restrict__ Y,
                                                 const int64_t* __restrict__ ncols_dev, int D,
                                                 unsigned long long* __restrict__ rowbest) {
  extern __shared__ __align__(16) float few_sm[];
  const int64_t nrows = *nrows_dev, ncols = *ncols_dev;
  if (nrows <= 0 || nrows > kFewRows) return;
  const int nr = (int)nrows;
  const int Dp = (D + 31) & ~31;
  float* xs = few_sm;                                                           // [nr][Dp]
  unsigned long long* best = reinterpret_cast<unsigned long long*>(xs + (size_t)kFewRows * 256);  // [8][kFewRows]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < nr * Dp; e += blockDim.x) {
    const int r = e / Dp, k = e - r * Dp;
    xs[e] = k < D ? X[(int64_t)rowlist[r] * D + k] : 0.f;
  }
  for (int e = threadIdx.x; e < 8 * kFewRows; e += blockDim.x) best[e] = ~0ull;
  __syncthreads();
  const int T = Dp >> 5;  // dimensions per lane
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  // the next row's values are loaded while this row is scored
  float y[8], yn[8];
  auto load_row = [&](float (&dst)[8], int64_t jj) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = lane + 32 * t;
      dst[t] = (jj < ncols && t < T && k < D) ? __ldg(Y + jj * D + k) : 0.f;
    }
  };
  int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  load_row(y, j);
  for (; j < ncols; j += nw) {
    load_row(yn, j + nw);
    // four candidates at a time: their sums and butterflies interleave (each
    // candidate's own order of operations is unchanged); the last one to
    // three alone
    int r0 = 0;
    for (; r0 + 4 <= nr; r0 += 4) {
      float acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* xr = xs + (r0 + u) * Dp + lane;
        float a = 0.f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (t < T) {
            const float d = xr[32 * t] - y[t];
            a = fmaf(d, d, a);
          }
        }
        acc[u] = a;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned long long pk = pack_min(acc[u], (uint32_t)j);
          if (pk < best[warp * kFewRows + r0 + u]) best[warp * kFewRows + r0 + u] = pk;
        }
      }
    }
    for (int r = r0; r < nr; ++r) {
      const float* xr = xs + r * Dp + lane;
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (t < T) {
          const float d = xr[32 * t] - y[t];
          acc = fmaf(d, d, acc);
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        const unsigned long long pk = pack_min(acc, (uint32_t)j);
        if (pk < best[warp * kFewRows + r]) best[warp * kFewRows + r] = pk;
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) y[t] = yn[t];
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nr; r += blockDim.x) {
    unsigned long long b = ~0ull;
#pragma unroll
    for (int w = 0; w < 8; ++w) b = best[w * kFewRows + r] < b ? best[w * kFewRows + r] : b;
    if (b != ~0ull) atomicMin(rowbest + r, b);
  }
}

__global__ void __launch_bounds__(256)
    rescore_few_kernel(const float* __restrict__ X, const int32_t* __restrict__ rowlist,
                       const int64_t* __restrict__ nrows_dev, const float* __restrict__ Y,
                       const int64_t* __restrict__ ncols_dev, int D, unsigned long long* __restrict__ rowbest) {
  rescore_few_body(X, rowlist, nrows_dev, Y, ncols_dev, D, rowbest);
}

__global__ void fill_u64_kernel(unsigned long long* p, int64_t n, unsigned long long v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void fill_u32_kernel(unsigned* p, int64_t n, unsigned v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// =====================================================================
// Tensor-core path: centring shift, scale, rounded copies
// =====================================================================

// Shift s = mean of the first <= 2048 rows of A and of B (FP64 sums), a
// common origin that keeps ||a - s|| small; distances do not depend on it.
// Stage 1: column sums of 256-row slices, grid (ceil(D/32), 8, 2 sets);
// stage 2 sums the slices in order. Row counts are read on the device.
__device__ __forceinline__ void hd_colsum_body(const float* __restrict__ A, const int64_t* nA_dev,
                                               const float* __restrict__ B, const int64_t* nB_dev, int D,
                                               double* __restrict__ part /*[2][8][D]*/, int set) {
  // FP32 sums of at most 32 values per thread and 256 per block (the shift
  // only centres the rounded copies: any value is exact for the result)
  __shared__ float sh[8][33];
  const float* X = set ? B : A;
  const int64_t n = set ? *nB_dev : *nA_dev;
  const int64_t rows = n < 2048 ? n : 2048;
  const int cl = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cl;
  const int64_t r0 = (int64_t)blockIdx.y * 256;
  float s = 0.f;
  if (c < D)
    for (int64_t i = r0 + rg; i < r0 + 256 && i < rows; i += 8) s += X[i * D + c];
  sh[rg][cl] = s;
  __syncthreads();
  if (rg == 0 && c < D) {
    float t = 0.f;
    for (int g = 0; g < 8; ++g) t += sh[g][cl];
    part[((size_t)set * 8 + blockIdx.y) * D + c] = (double)t;
  }
}

__global__ void hd_colsum_kernel(const float* __restrict__ A, const int64_t* nA_dev, const float* __restrict__ B,
                                 const int64_t* nB_dev, int D, double* __restrict__ part /*[2][8][D]*/) {
  hd_colsum_body(A, nA_dev, B, nB_dev, D, part, blockIdx.z);
}

__device__ __forceinline__ void hd_shift_body(const double* __restrict__ part, const int64_t* nA_dev,
                                              const int64_t* nB_dev, int D, float* __restrict__ shift) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  const int64_t na = *nA_dev < 2048 ? *nA_dev : 2048, nb = *nB_dev < 2048 ? *nB_dev : 2048;
  double ta = 0.0, tb = 0.0;
  for (int y = 0; y < 8; ++y) {
    ta += part[(size_t)y * D + c];
    tb += part[(size_t)(8 + y) * D + c];
  }
  shift[c] = (float)(0.5 * (ta / (double)na + tb / (double)nb));
}

__global__ void hd_shift_kernel(const double* __restrict__ part, const int64_t* nA_dev, const int64_t* nB_dev, int D,
                                float* __restrict__ shift) {
  hd_shift_body(part, nA_dev, nB_dev, D, shift);
}

// max |x - s| over both sets (in FP32, the same values the copies use), and
// the non-finite input check.
__device__ __forceinline__ void hd_maxabs_body(const float* __restrict__ X, const int64_t* n_dev, int D,
                                               const float* __restrict__ shift, float* __restrict__ maxabs,
                                               int* status) {
  const int64_t n = *n_dev;
  const int lane = threadIdx.x & 31;
  const int64_t total = n * D;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  float m = 0.f;
  bool bad = false;
  if ((D & 3) == 0 && D <= 256 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    // a warp per row, lane l on columns 4l.. and 128 + 4l..; the shift stays
    // in registers and four rows' loads are in flight (columns past D read as
    // the shift itself, |x - s| = 0)
    const int c0 = 4 * lane, c1 = 128 + 4 * lane;
    const float4 s0 = c0 < D ? make_float4(shift[c0], shift[c0 + 1], shift[c0 + 2], shift[c0 + 3])
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 s1 = c1 < D ? make_float4(shift[c1], shift[c1 + 1], shift[c1 + 2], shift[c1 + 3])
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t warp = tid >> 5, nwarps = nth >> 5;
    auto acc = [&](const float4 v, const float4 sv) {
      bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x - sv.x), fabsf(v.y - sv.y)), fmaxf(fabsf(v.z - sv.z), fabsf(v.w - sv.w))));
    };
    for (int64_t r = warp; r < n; r += 4 * nwarps) {
      float4 v[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t rr = r + u * nwarps;
        v[u][0] = rr < n && c0 < D ? __ldg(reinterpret_cast<const float4*>(X + rr * D + c0)) : s0;
        v[u][1] = rr < n && c1 < D ? __ldg(reinterpret_cast<const float4*>(X + rr * D + c1)) : s1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc(v[u][0], s0);
        acc(v[u][1], s1);
      }
    }
  } else if ((D & 3) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    // element stream in 128-bit loads, independent of the row structure
    const float4* X4 = reinterpret_cast<const float4*>(X);
    const int D4 = D >> 2;
    for (int64_t e = tid; e < (total >> 2); e += nth) {
      const float4 v = __ldg(X4 + e);
      const int c = (int)(e % D4) * 4;
      bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x - shift[c]), fabsf(v.y - shift[c + 1])),
                         fmaxf(fabsf(v.z - shift[c + 2]), fabsf(v.w - shift[c + 3]))));
    }
  } else {
    for (int64_t e = tid; e < total; e += nth) {
      const float v = X[e];
      bad |= !isfinite(v);
      m = fmaxf(m, fabsf(v - shift[e % D]));
    }
  }
  m = warp_max(m);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(status, (int)PROHD_ENONFINITE);
  if (lane == 0) atomic_max_nonneg(maxabs, m);
}

__global__ void hd_maxabs_kernel(const float* __restrict__ X, const int64_t* n_dev, int D,
                                 const float* __restrict__ shift, float* __restrict__ maxabs, int* status) {
  hd_maxabs_body(X, n_dev, D, shift, maxabs, status);
}

// Scale exponent: max|x - s| * 2^sigma lies in [2^12, 2^13), so the rounded
// values stay below 2^13 and -2x below 2^14 (FP16 range 65504).
__device__ __forceinline__ int scale_exponent(float maxabs) {
  if (!(maxabs > 0.f)) return 0;
  int e;
  frexpf(maxabs, &e);  // maxabs = f 2^e, f in [0.5, 1)
  return max(-120, min(120, 13 - e));
}

template <int BF16>
struct TileT;
template <>
struct TileT<0> {
  using T = __half;
  static __device__ __forceinline__ T from(float x) { return __float2half_rn(x); }
  static __device__ __forceinline__ float to(T h) { return __half2float(h); }
};
template <>
struct TileT<1> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ T from(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ float to(T h) { return __bfloat162float(h); }
};

// Entry `lane` (0..7) of a row's TF32 norm operand: the squared norm split
// exactly into three TF32 parts (truncation to 10 explicit mantissa bits
// leaves 11 + 11 + 2 bits: exact) next to three ones, [h, m, l, 1, 1, 1, 0, 0]
// for A and [1, 1, 1, h, m, l, 0, 0] for B, so that one TF32 MMA of the two
// tiles writes ||h_a||^2 + ||h_b||^2 into every accumulator entry.
__device__ __forceinline__ float tf32_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }
__device__ __forceinline__ float norm_part(float n2, int side, int lane) {
  const float h = tf32_trunc(n2);
  const float r = n2 - h;
  const float m = tf32_trunc(r);
  const float l = tf32_trunc(r - m);
  const int k = side ? lane - 3 : lane;
  const float part = k == 0 ? h : (k == 1 ? m : l);
  if (lane >= 6) return 0.f;
  return (k >= 0 && k < 3) ? part : 1.f;
}

// One warp per row. Writes the rounded copy h = round((x - s) 2^sigma)
// (times `mult`: -2 for A, 1 for B) into Xt [n_pad, Dp], ||h||^2 (FP32) into
// norm2, and eps >= ||(x - s) - h 2^-sigma|| + rounding of x - s (original
// units) into eps. Padding rows: zeros, norm2 = 1e30, eps = 0.
template <int BF16>
__device__ __forceinline__ void hd_prep_body(const float* __restrict__ X, const int64_t* n_dev, int64_t n_pad, int D,
                                             int Dp, const float* __restrict__ shift, const float* __restrict__ maxabs,
                                             float mult, typename TileT<BF16>::T* __restrict__ Xt,
                                             float* __restrict__ norm2, float* __restrict__ eps,
                                             float* __restrict__ maxnorm, float* __restrict__ maxeps,
                                             float* __restrict__ nparts, int side) {
  using TT = TileT<BF16>;
  using T = typename TT::T;
  const int64_t n = *n_dev;
  const int sig = scale_exponent(*maxabs);
  const float scale = ldexpf(1.f, sig), inv = ldexpf(1.f, -sig);
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float wmaxn = 0.f, wmaxe = 0.f;
  // a lane's values of the next row are loaded while this row is converted
  // (Dp <= 256: at most 8 values per lane)
  if ((D & 3) == 0 && (Dp & 3) == 0 && Dp <= 256 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    // 128-bit loads (lane l: columns 4l.. and 128 + 4l..), two rows ahead in
    // flight, four rounded values stored as one 8-byte word; per element the
    // same arithmetic as the scalar form below
    const int cc[2] = {4 * lane, 128 + 4 * lane};
    float4 sv[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      sv[h] = cc[h] < D ? make_float4(shift[cc[h]], shift[cc[h] + 1], shift[cc[h] + 2], shift[cc[h] + 3])
                        : make_float4(0.f, 0.f, 0.f, 0.f);
    auto ld = [&](float4 (&d)[2], int64_t rr) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        d[h] = rr < n && cc[h] < D ? __ldg(reinterpret_cast<const float4*>(X + rr * D + cc[h]))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    float4 xa[2], xb[2], xc[2];
    ld(xa, warp);
    ld(xb, warp + nwarps);
    for (int64_t r = warp; r < n_pad; r += nwarps) {
      ld(xc, r + 2 * nwarps);
      T* out = Xt + r * Dp;
      if (r < n) {
        float sn = 0.f, se = 0.f, st = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = cc[h];
          if (c >= Dp) continue;
          __align__(8) T q4[4];
          const float xs[4] = {xa[h].x, xa[h].y, xa[h].z, xa[h].w};
          const float ss[4] = {sv[h].x, sv[h].y, sv[h].z, sv[h].w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float hv = 0.f;
            if (c < D) {  // D % 4 == 0: the four columns are all data or all padding
              const float t = xs[k] - ss[k];
              hv = TT::to(TT::from(t * scale));
              const float rr = t - hv * inv;
              sn = fmaf(hv, hv, sn);
              se = fmaf(rr, rr, se);
              st = fmaf(t, t, st);
            }
            q4[k] = TT::from(hv * mult);
          }
          *reinterpret_cast<uint2*>(out + c) = *reinterpret_cast<const uint2*>(q4);
        }
        sn = __shfl_sync(0xffffffffu, warp_sum(sn), 0);
        se = warp_sum(se);
        st = warp_sum(st);
        if (lane < 8) nparts[r * 8 + lane] = norm_part(sn, side, lane);
        if (lane == 0) {
          const float e = 1.001f * (sqrtf(se) + 5.9604645e-8f * sqrtf(st)) + 1e-30f;
          norm2[r] = sn;
          eps[r] = e;
          wmaxn = fmaxf(wmaxn, sqrtf(sn));
          wmaxe = fmaxf(wmaxe, e);
        }
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h)
          if (cc[h] < Dp) *reinterpret_cast<uint2*>(out + cc[h]) = make_uint2(0u, 0u);
        if (lane == 0) {
          norm2[r] = 1e30f;
          eps[r] = 0.f;
        }
        if (lane < 8) nparts[r * 8 + lane] = norm_part(1e30f, side, lane);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        xa[h] = xb[h];
        xb[h] = xc[h];
      }
    }
    if (lane == 0) {
      atomic_max_nonneg(maxnorm, wmaxn);
      atomic_max_nonneg(maxeps, wmaxe);
    }
    return;
  }
  float xv[8], xn[8];
  auto load_row = [&](float (&dst)[8], int64_t rr) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int c = lane + 32 * t;
      dst[t] = (rr < n && c < D) ? __ldg(X + rr * D + c) : 0.f;
    }
  };
  load_row(xv, warp);
  for (int64_t r = warp; r < n_pad; r += nwarps) {
    load_row(xn, r + nwarps);
    T* out = Xt + r * Dp;
    if (r < n) {
      float sn = 0.f, se = 0.f, st = 0.f;
#pragma unroll
      for (int tt = 0; tt < 8; ++tt) {
        const int c = lane + 32 * tt;
        if (c >= Dp) break;
        float hv = 0.f;
        if (c < D) {
          float t = xv[tt] - shift[c];
          T h = TT::from(t * scale);
          hv = TT::to(h);
          float rr = t - hv * inv;  // exact: t and hv*inv agree to the tile precision
          sn = fmaf(hv, hv, sn);
          se = fmaf(rr, rr, se);
          st = fmaf(t, t, st);
        }
        out[c] = TT::from(hv * mult);
      }
      sn = __shfl_sync(0xffffffffu, warp_sum(sn), 0);
      se = warp_sum(se);
      st = warp_sum(st);
      if (lane < 8) nparts[r * 8 + lane] = norm_part(sn, side, lane);
      if (lane == 0) {
        // ||(x-s)_exact - h/scale|| <= ||t - h/scale|| + 2^-24 ||t||; the FP32
        // sums of squares are inflated for their own rounding.
        float e = 1.001f * (sqrtf(se) + 5.9604645e-8f * sqrtf(st)) + 1e-30f;
        norm2[r] = sn;
        eps[r] = e;
        wmaxn = fmaxf(wmaxn, sqrtf(sn));
        wmaxe = fmaxf(wmaxe, e);
      }
    } else {
      for (int c = lane; c < Dp; c += 32) out[c] = TT::from(0.f);
      if (lane == 0) {
        norm2[r] = 1e30f;  // padding: far from everything, finite in TMEM
        eps[r] = 0.f;
      }
      if (lane < 8) nparts[r * 8 + lane] = norm_part(1e30f, side, lane);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) xv[t] = xn[t];
  }
  if (lane == 0) {
    atomic_max_nonneg(maxnorm, wmaxn);
    atomic_max_nonneg(maxeps, wmaxe);
  }
}

template <int BF16>
__global__ void hd_prep_kernel(const float* __restrict__ X, const int64_t* n_dev, int64_t n_pad, int D, int Dp,
                               const float* __restrict__ shift, const float* __restrict__ maxabs, float mult,
                               typename TileT<BF16>::T* __restrict__ Xt, float* __restrict__ norm2,
                               float* __restrict__ eps, float* __restrict__ maxnorm, float* __restrict__ maxeps,
                               float* __restrict__ nparts, int side) {
  hd_prep_body<BF16>(X, n_dev, n_pad, D, Dp, shift, maxabs, mult, Xt, norm2, eps, maxnorm, maxeps, nparts, side);
}

// =====================================================================
// tcgen05 contraction with fused row-min / column-min epilogue
// =====================================================================
//
// Tile: 128 rows of A x 256 rows of B, K = Dp (<= 256) in 64-element blocks.
// A CTA owns a 128-row block of A for a whole sweep over B (rows' minima stay
// in registers), with the A block resident in shared memory; B streams
// through a 4-stage TMA ring in 128B-swizzled 256x64 tiles. Accumulators are
// double-buffered in TMEM (2 x 256 columns) so the epilogue of tile t
// overlaps the MMAs of tile t+1.
// Warps: 0 = TMA producer, 1 = MMA issuer (and TMEM owner), 2..17 = epilogue
// (warp w reads TMEM lanes 32*(w%4) .. +31 and column quarter (w-2)/4; four
// warps per lane quarter hide the latency of the per-element work).
// Each tile starts with one TF32 MMA (K = 8) of two small operands holding
// exact TF32 splits of the squared norms, which writes ||h_a||^2 + ||h_b||^2
// into every accumulator entry; the FP16/BF16 MMAs then add (-2 h_a) . h_b,
// so the accumulator holds the squared distance d2 of every pair. Epilogue per
// element: the row minimum comes with the TMEM load (tcgen05.ld.red.min), the
// column minimum over 32 rows is redux.sync.min.f32; both are combined over
// the CTA in shared memory, then one global atomicMin per column per tile
// (clamped at 0 so unsigned order = float order). A TMEM buffer goes back to
// the MMA as soon as it has been read.

constexpr int kTcBM = 128, kTcBN = 256, kTcBK = 64, kTcStages = 4;
constexpr int kTcAKBytes = kTcBM * kTcBK * 2;   // 16 KB per A K-block
constexpr int kTcBStage = kTcBN * kTcBK * 2;    // 32 KB per B stage
constexpr int kTcNBBytes = kTcBN * 32;          // 8 KB: B norm operand of one tile (256 rows x 8 TF32)
constexpr int kTcNABytes = kTcBM * 32;          // 4 KB: A norm operand of one row block
constexpr int kTcEpiWarps = 16;  // four per TMEM lane quarter, 64 columns each
constexpr int kTcThreads = (2 + kTcEpiWarps) * 32;

struct TcSmem {
  uint64_t b_full[kTcStages], b_empty[kTcStages];
  uint64_t nb_full[2], nb_empty[2];
  uint64_t a_full, a_empty;
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
  float col[2][4][kTcBN];  // [tile parity][lane quarter][column]
  float rowx[3][kTcBM];     // other column groups' row minima at the end of a row block
};

// [B norm ring 2 x 8 KB][A norm 4 KB][A: KB x 16 KB][B ring][TcSmem]; the small
// 32-byte-swizzled norm tiles sit first, on 256-byte boundaries.
__host__ __device__ constexpr size_t tc_smem_bytes(int KB) {
  return 1024 /*alignment slack*/ + 2 * kTcNBBytes + kTcNABytes + (size_t)KB * kTcAKBytes +
         (size_t)kTcStages * kTcBStage + sizeof(TcSmem);
}

// One unit of contraction work: row block rb of A against the CB column
// tiles of B starting at tile cb0, with the pair's operand maps, depth KB and
// minima. seg: the row block's columns are split over several items, so its
// row minima are combined with atomicMin (the buffer starts at +inf) rather
// than stored. cols: column minima wanted (else only the row minima).
struct TcItem {
  const CUtensorMap *tmA, *tmB, *tmNA, *tmNB;
  int KB, CB, cb0, rb;
  bool seg;
  bool cols = true;
  float* rowmin;
  unsigned* colmin;
};

// The items of one pair: row blocks blockIdx.x, blockIdx.x + gridDim.x, ...
struct TcItemsOne {
  const CUtensorMap *tmA, *tmB, *tmNA, *tmNB;
  int KB, RB, CB;
  float* rowmin;
  unsigned* colmin;
  __device__ bool get(int k, TcItem& it) const {
    const int rb = (int)blockIdx.x + k * (int)gridDim.x;
    if (rb >= RB) return false;
    it.tmA = tmA; it.tmB = tmB; it.tmNA = tmNA; it.tmNB = tmNB;
    it.KB = KB; it.CB = CB; it.cb0 = 0; it.seg = false; it.rb = rb; it.rowmin = rowmin; it.colmin = colmin;
    return true;
  }
};

// The items of one pair with the columns cut into segments (a few rows
// against many columns): item g = blockIdx.x + k gridDim.x is segment g % NS
// of row block g / NS, the CBall column tiles cut into NS non-empty segments
// of at most CS tiles, so that every CTA gets about two items.
struct TcItemsSeg {
  const CUtensorMap *tmA, *tmB, *tmNA, *tmNB;
  int KB, RB, CBall, NS, CS;
  float* rowmin;
  unsigned* colmin;
  __device__ bool get(int k, TcItem& it) const {
    const int64_t g = (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
    if (g >= (int64_t)RB * NS) return false;
    const int rb = (int)(g / NS), sg = (int)(g - (int64_t)rb * NS);
    it.tmA = tmA; it.tmB = tmB; it.tmNA = tmNA; it.tmNB = tmNB;
    it.KB = KB; it.rb = rb; it.rowmin = rowmin; it.colmin = colmin;
    it.cb0 = sg * CS;
    it.CB = min(CS, CBall - it.cb0);
    it.seg = NS > 1;
    return it.CB > 0;
  }
};

// The items of a batch: item i is row block i - prefix[p] of pair order[p]
// (prefix over pairs of their row-block counts), CTAs taking items
// blockIdx.x, blockIdx.x + gridDim.x, ... in every role alike.
struct TcItemsBatch {
  const BPair* P;
  const int* order;
  const int64_t* prefix;
  const CUtensorMap* maps;
  int npairs;
  __device__ bool get(int k, TcItem& it) const {
    const int64_t i = (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
    if (i >= prefix[npairs]) return false;
    int lo = 0, hi = npairs;  // prefix[lo] <= i < prefix[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= i) lo = mid;
      else hi = mid;
    }
    const BPair& q = P[order[lo]];
    const CUtensorMap* m = maps + q.hd_map;
    it.tmA = m; it.tmB = m + 1; it.tmNA = m + 2; it.tmNB = m + 3;
    it.KB = q.Dp / kTcBK;
    it.CB = (int)((q.nsel[1] + kTcBN - 1) / kTcBN);
    it.cb0 = 0;
    it.seg = false;
    it.rb = (int)(i - prefix[lo]);
    it.rowmin = q.hd_rowmin;
    it.colmin = q.hd_colmin;
    it.cols = !q.rows_only;
    return true;
  }
};

template <int BF16, class Items>
__device__ __forceinline__ void hd_tc_body(const Items& items, int KBmax, int* __restrict__ status,
                                           uint64_t timeout_ns, const CUtensorMap* const* prefetch) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_align<1024>(smem_raw);
  uint8_t* sNB = base;                        // [2][8 KB]
  uint8_t* sNA = base + 2 * kTcNBBytes;       // 4 KB
  uint8_t* sA = sNA + kTcNABytes;             // 1024-aligned (20 KB from base)
  uint8_t* sB = sA + (size_t)KBmax * kTcAKBytes;
  TcSmem& S = *reinterpret_cast<TcSmem*>(sB + (size_t)kTcStages * kTcBStage);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &S.abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&S.b_full[s], 1);
      mbar_init(&S.b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.nb_full[b], 1);
      mbar_init(&S.nb_empty[b], 1);
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], kTcEpiWarps);
    }
    mbar_init(&S.a_full, 1);
    mbar_init(&S.a_empty, 1);
    mbar_init(&S.drain, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tc_alloc(&S.tmem_base, 512);
    tc_relinquish();
  }
  if (warp == 0 && lane == 0 && prefetch)
    for (int i = 0; i < 4; ++i) tma_prefetch_desc(prefetch[i]);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t st = 0, ph = 0, aph = 0;
      uint32_t armed = 0, armed_ph = 0;  // B stages with a load in flight, and its phase parity
      uint32_t tile = 0;                 // running tile count (B norm ring slot and parity)
      uint32_t nb_issued = 0;            // B norm loads issued
      bool ok = true;
      TcItem it;
      for (int k = 0; ok && items.get(k, it); ++k) {
        const int rb = it.rb, KB = it.KB, CB = it.CB;
        if (!mbar_wait_bounded(&S.a_empty, aph ^ 1, abort, timeout_ns)) { ok = false; break; }
        aph ^= 1;
        mbar_arrive_expect_tx(&S.a_full, (uint32_t)(KB * kTcAKBytes + kTcNABytes));
        tma_load_2d(sNA, it.tmNA, 0, rb * kTcBM, &S.a_full);
        for (int kb = 0; kb < KB; ++kb) tma_load_2d(sA + kb * kTcAKBytes, it.tmA, kb * kTcBK, rb * kTcBM, &S.a_full);
        for (int cb = 0; cb < CB && ok; ++cb, ++tile) {
          const uint32_t ns = tile & 1u, nph = (tile >> 1) & 1u;
          if (!mbar_wait_bounded(&S.nb_empty[ns], nph ^ 1, abort, timeout_ns)) { ok = false; break; }
          mbar_arrive_expect_tx(&S.nb_full[ns], (uint32_t)kTcNBBytes);
          tma_load_2d(sNB + ns * kTcNBBytes, it.tmNB, 0, (it.cb0 + cb) * kTcBN, &S.nb_full[ns]);
          ++nb_issued;
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait_bounded(&S.b_empty[st], ph ^ 1, abort, timeout_ns)) { ok = false; break; }
            mbar_arrive_expect_tx(&S.b_full[st], (uint32_t)kTcBStage);
            tma_load_2d(sB + st * kTcBStage, it.tmB, kb * kTcBK, (it.cb0 + cb) * kTcBN, &S.b_full[st]);
            armed |= 1u << st;
            armed_ph = (armed_ph & ~(1u << st)) | (ph << st);
            if (++st == kTcStages) { st = 0; ph ^= 1; }
          }
        }
      }
      if (!ok) {
        // error path: let copies already issued land before the CTA exits
        for (int s2 = 0; s2 < kTcStages; ++s2) {
          if (!(armed >> s2 & 1u)) continue;
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&S.b_full[s2], (armed_ph >> s2) & 1u) && global_timer_ns() - t0 < 2000000ull) {
          }
        }
        for (uint32_t t2 = nb_issued >= 2 ? nb_issued - 2 : 0; t2 < nb_issued; ++t2) {
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&S.nb_full[t2 & 1u], (t2 >> 1) & 1u) && global_timer_ns() - t0 < 2000000ull) {
          }
        }
        const uint64_t t0 = global_timer_ns();
        while (!mbar_try_wait(&S.a_full, aph ^ 1) && global_timer_ns() - t0 < 2000000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(BF16, kTcBM, kTcBN);
      constexpr uint32_t idesc_n = idesc_tf32(kTcBM, kTcBN);
      uint32_t st = 0, ph = 0, aph = 0;
      uint32_t tile = 0;
      bool ok = true;
      TcItem it;
      for (int k = 0; ok && items.get(k, it); ++k) {
        const int KB = it.KB, CB = it.CB;
        if (!mbar_wait_bounded(&S.a_full, aph, abort, timeout_ns)) { ok = false; break; }
        aph ^= 1;
        tc_fence_after();
        for (int cb = 0; cb < CB && ok; ++cb, ++tile) {
          const uint32_t ab = tile & 1u, use = tile >> 1;
          if (!mbar_wait_bounded(&S.acc_empty[ab], (use & 1u) ^ 1u, abort, timeout_ns)) { ok = false; break; }
          if (!mbar_wait_bounded(&S.nb_full[ab], use & 1u, abort, timeout_ns)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem + ab * (uint32_t)kTcBN;
          // accumulator = ||h_a||^2 + ||h_b||^2
          tc_mma_tf32(d_tmem, smem_desc_sw32(smem_u32(sNA)), smem_desc_sw32(smem_u32(sNB + ab * kTcNBBytes)), idesc_n,
                      0u);
          tc_commit(&S.nb_empty[ab]);
          for (int kb = 0; kb < KB; ++kb) {
            if (!mbar_wait_bounded(&S.b_full[st], ph, abort, timeout_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(sA + kb * kTcAKBytes);
            const uint32_t b_addr = smem_u32(sB + st * kTcBStage);
#pragma unroll
            for (int k = 0; k < kTcBK / 16; ++k)
              tc_mma_f16(d_tmem, smem_desc_sw128(a_addr + k * 32), smem_desc_sw128(b_addr + k * 32), idesc, 1u);
            tc_commit(&S.b_empty[st]);
            if (++st == kTcStages) { st = 0; ph ^= 1; }
          }
          if (!ok) break;
          tc_commit(&S.acc_full[ab]);
        }
        tc_commit(&S.a_empty);
      }
      // make sure every MMA issued by this thread has finished before exit
      tc_commit(&S.drain);
      uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&S.drain, 0) && global_timer_ns() - t0 < 1000000000ull) {
      }
    }
  } else {
    // ---------------- epilogue (warps 2..17) ----------------
    // Every epilogue warp runs the same tile loop and reaches every named
    // barrier even after an abort (then it only skips the work), so the
    // barriers cannot wait on a warp that left early.
    const int ew = warp - 2;             // 0..15
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int grp = ew >> 2;             // column group: four per lane quarter
    const int hcol = grp * (kTcBN / 4);  // first column of this warp's group
    const int et = threadIdx.x - 64;     // 0..511 (the first 256 also combine columns)
    bool ok = true;
    float rmin = __int_as_float(0x7f800000);
    TcItem it;
    int i = 0;  // running tile count: TMEM buffer and phase
    for (int k = 0; items.get(k, it); ++k)
    for (int cb = 0; cb < it.CB; ++cb, ++i) {
      const int CB = it.CB, rb = it.rb;
      float* rowmin = it.rowmin;
      unsigned* colmin = it.colmin;
      const int ab = i & 1;
      const uint32_t par = (uint32_t)(i >> 1) & 1u;
      int got = 0;
      if (ok && lane == 0) got = mbar_wait_bounded(&S.acc_full[ab], par, abort, timeout_ns) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      ok = ok && got;
      if (ok) {
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * kTcBN + hcol);
        float v[32];
#pragma unroll 1
        for (int ch = 0; ch < kTcBN / 4 / 32; ++ch) {
          __syncwarp();
          float vmin;
          tc_ld_red_min_32x32b_x32(taddr + ch * 32, v, vmin);
          tc_wait_ld();
          rmin = fminf(rmin, vmin);
          if (!it.cols) continue;
          float cm[32];
#pragma unroll
          for (int c = 0; c < 32; ++c) cm[c] = redux_min_f32(v[c]);
          if (lane == 0) {
            float4* dst = reinterpret_cast<float4*>(&S.col[ab][q][hcol + ch * 32]);
#pragma unroll
            for (int c = 0; c < 8; ++c)
              dst[c] = make_float4(cm[4 * c], cm[4 * c + 1], cm[4 * c + 2], cm[4 * c + 3]);
          }
        }
        // this buffer's TMEM is read: hand it back to the MMA
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.acc_empty[ab]);
      }
      named_bar_sync(1, 32 * kTcEpiWarps);
      if (ok && et < kTcBN && it.cols) {
        const int c = et;
        float m = fminf(fminf(S.col[ab][0][c], S.col[ab][1][c]), fminf(S.col[ab][2][c], S.col[ab][3][c]));
        m = fmaxf(m, 0.f);
        atomicMin(colmin + (int64_t)(it.cb0 + cb) * kTcBN + c, __float_as_uint(m));
      }
      if (cb == CB - 1) {
        // the four warps of a lane quarter saw a quarter of the columns each
        if (grp > 0) S.rowx[grp - 1][q * 32 + lane] = rmin;
        named_bar_sync(1, 32 * kTcEpiWarps);
        if (ok && grp == 0) {
          const float r =
              fminf(fminf(rmin, S.rowx[0][q * 32 + lane]), fminf(S.rowx[1][q * 32 + lane], S.rowx[2][q * 32 + lane]));
          float* dst = rowmin + (int64_t)rb * kTcBM + q * 32 + lane;
          // clamped at 0 so unsigned order = float order (the margins treat
          // a negative low-precision d2 as 0 anyway)
          if (it.seg) atomicMin(reinterpret_cast<unsigned*>(dst), __float_as_uint(fmaxf(r, 0.f)));
          else *dst = r;
        }
        rmin = __int_as_float(0x7f800000);
      }
    }
  }

  __syncthreads();
  if (threadIdx.x == 0 && S.abort) atomicMax(status, (int)PROHD_ETIMEOUT);
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tc_dealloc(tmem, 512);
  }
}

template <int BF16, bool SEG>
__global__ void __launch_bounds__(kTcThreads, 1)
    hd_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ CUtensorMap tmNA, const __grid_constant__ CUtensorMap tmNB,
                 const int64_t* __restrict__ nA_dev, const int64_t* __restrict__ nB_dev, int KB,
                 float* __restrict__ rowmin, unsigned* __restrict__ colmin, int* __restrict__ status,
                 uint64_t timeout_ns) {
  const int64_t nA = *nA_dev, nB = *nB_dev;
  const CUtensorMap* pf[4] = {&tmA, &tmB, &tmNA, &tmNB};
  if constexpr (!SEG) {
    TcItemsOne items;
    items.tmA = &tmA; items.tmB = &tmB; items.tmNA = &tmNA; items.tmNB = &tmNB;
    items.KB = KB;
    items.RB = (int)((nA + kTcBM - 1) / kTcBM);
    items.CB = (int)((nB + kTcBN - 1) / kTcBN);
    items.rowmin = rowmin;
    items.colmin = colmin;
    hd_tc_body<BF16>(items, KB, status, timeout_ns, pf);
  } else {
    TcItemsSeg items;
    items.tmA = &tmA; items.tmB = &tmB; items.tmNA = &tmNA; items.tmNB = &tmNB;
    items.KB = KB;
    items.RB = (int)((nA + kTcBM - 1) / kTcBM);
    items.CBall = (int)((nB + kTcBN - 1) / kTcBN);
    // fewer than two row blocks per CTA: cut the columns into segments so
    // that every CTA gets about two items (the row minima buffer starts at +inf)
    const int want = 2 * (int)gridDim.x;
    items.NS = items.RB >= want ? 1 : min(items.CBall, (want + items.RB - 1) / items.RB);
    items.NS = max(items.NS, 1);
    items.CS = (items.CBall + items.NS - 1) / items.NS;
    // no empty segment: an item list must not end before its last item
    items.NS = max(1, (items.CBall + items.CS - 1) / items.CS);
    items.rowmin = rowmin;
    items.colmin = colmin;
    hd_tc_body<BF16>(items, KB, status, timeout_ns, pf);
  }
}

// Batched: every pair's row blocks against its own column tiles, the maps in
// device memory; the smem layout holds the deepest pair (KBmax).
template <int BF16>
__global__ void __launch_bounds__(kTcThreads, 1)
    hd_tc_batched_kernel(const BPair* __restrict__ P, const int* __restrict__ order, const int64_t* __restrict__ prefix,
                         const CUtensorMap* __restrict__ maps, int npairs, int KBmax, int* __restrict__ status,
                         uint64_t timeout_ns) {
  TcItemsBatch items;
  items.P = P;
  items.order = order;
  items.prefix = prefix;
  items.maps = maps;
  items.npairs = npairs;
  hd_tc_body<BF16>(items, KBmax, status, timeout_ns, nullptr);
}

// =====================================================================
// Margins, candidates, finalisation
// =====================================================================

struct HdScalars {
  float maxabs;          // max |x - s|
  float maxnormA, maxnormB;  // max ||h|| (scaled units)
  float maxepsA, maxepsB;    // max eps (original units)
  float lowp_max;        // max over rows/cols of the low-precision d^2 (scaled)
  double LB[2];          // largest lower bound of a row / column NN distance
  int64_t ncandA, ncandB;
};

// Margin of a low-precision squared minimum r2 (scaled units) of a row whose
// own copy has norm na and the other set's copies norms <= nbmax:
// |d2_lowp - ||h_a - h_b||^2| <= c1 (||h_a|| + ||h_b||)^2 with
// c1 = (2 Dp + 2 D + 16) 2^-24 (products exact, FP32 accumulation of Dp terms
// with truncation allowed, norms summed over D terms, two epilogue roundings,
// times 2 for safety); and ||x_true - x_copy|| <= eps in original units.
__device__ __forceinline__ void row_interval(float r2, float norm2_self, float maxnorm_other, float eps_self,
                                             float maxeps_other, double c1, double inv, double& lo, double& hi) {
  double ns = sqrt((double)norm2_self);
  double dd = c1 * (ns + (double)maxnorm_other) * (ns + (double)maxnorm_other);
  double r = (double)r2;
  double e = (double)eps_self + (double)maxeps_other;
  hi = (inv * sqrt(fmax(r, 0.0) + dd) + e) * (1.0 + 1e-6) + 1e-300;
  lo = (inv * sqrt(fmax(r - dd, 0.0)) - e) * (1.0 - 1e-6);
}

__device__ __forceinline__ void hd_bounds_body(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                                               const float* __restrict__ epsA, const int64_t* nA_dev,
                                               const unsigned* __restrict__ colmin, const float* __restrict__ nB2,
                                               const float* __restrict__ epsB, const int64_t* nB_dev, double c1,
                                               HdScalars* __restrict__ sc) {
  const int64_t nA = *nA_dev, nB = *nB_dev;
  const double inv = ldexp(1.0, -scale_exponent(sc->maxabs));
  double lbA = 0.0, lbB = 0.0;
  float lp = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nA; i += stride) {
    double lo, hi;
    row_interval(rowmin[i], nA2[i], sc->maxnormB, epsA[i], sc->maxepsB, c1, inv, lo, hi);
    lbA = fmax(lbA, lo);
    lp = fmaxf(lp, rowmin[i]);
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nB; j += stride) {
    double lo, hi;
    float c = __uint_as_float(colmin[j]);
    row_interval(c, nB2[j], sc->maxnormA, epsB[j], sc->maxepsA, c1, inv, lo, hi);
    lbB = fmax(lbB, lo);
    lp = fmaxf(lp, c);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lbA = fmax(lbA, __shfl_xor_sync(0xffffffffu, lbA, o));
    lbB = fmax(lbB, __shfl_xor_sync(0xffffffffu, lbB, o));
  }
  lp = warp_max(lp);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&sc->LB[0], lbA);
    atomic_max_nonneg(&sc->LB[1], lbB);
    atomic_max_nonneg(&sc->lowp_max, lp);
  }
}

__global__ void hd_bounds_kernel(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                                 const float* __restrict__ epsA, const int64_t* nA_dev,
                                 const unsigned* __restrict__ colmin, const float* __restrict__ nB2,
                                 const float* __restrict__ epsB, const int64_t* nB_dev, double c1,
                                 HdScalars* __restrict__ sc) {
  hd_bounds_body(rowmin, nA2, epsA, nA_dev, colmin, nB2, epsB, nB_dev, c1, sc);
}

// Appends every row (column) whose upper bound reaches the largest lower
// bound to the candidate list.
__device__ __forceinline__ void hd_flag_body(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                                             const float* __restrict__ epsA, const int64_t* nA_dev,
                                             const unsigned* __restrict__ colmin, const float* __restrict__ nB2,
                                             const float* __restrict__ epsB, const int64_t* nB_dev, double c1,
                                             HdScalars* __restrict__ sc, int32_t* __restrict__ candA,
                                             int32_t* __restrict__ candB, int64_t* __restrict__ ncandA,
                                             int64_t* __restrict__ ncandB) {
  const int64_t nA = *nA_dev, nB = *nB_dev;
  const double inv = ldexp(1.0, -scale_exponent(sc->maxabs));
  const double LBa = sc->LB[0], LBb = sc->LB[1];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t start = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t endA = (nA + 31) / 32 * 32, endB = (nB + 31) / 32 * 32;
  for (int64_t i = start; i < endA; i += stride) {
    bool f = false;
    if (i < nA) {
      double lo, hi;
      row_interval(rowmin[i], nA2[i], sc->maxnormB, epsA[i], sc->maxepsB, c1, inv, lo, hi);
      f = hi >= LBa;
    }
    unsigned m = __ballot_sync(0xffffffffu, f);
    int64_t base = 0;
    if (lane == 0 && m) base = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(ncandA), (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) candA[base + __popc(m & ((1u << lane) - 1))] = (int32_t)i;
  }
  for (int64_t j = start; j < endB; j += stride) {
    bool f = false;
    if (j < nB) {
      double lo, hi;
      row_interval(__uint_as_float(colmin[j]), nB2[j], sc->maxnormA, epsB[j], sc->maxepsA, c1, inv, lo, hi);
      f = hi >= LBb;
    }
    unsigned m = __ballot_sync(0xffffffffu, f);
    int64_t base = 0;
    if (lane == 0 && m) base = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(ncandB), (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) candB[base + __popc(m & ((1u << lane) - 1))] = (int32_t)j;
  }
}

__global__ void hd_flag_kernel(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                               const float* __restrict__ epsA, const int64_t* nA_dev,
                               const unsigned* __restrict__ colmin, const float* __restrict__ nB2,
                               const float* __restrict__ epsB, const int64_t* nB_dev, double c1,
                               HdScalars* __restrict__ sc, int32_t* __restrict__ candA, int32_t* __restrict__ candB,
                               int64_t* __restrict__ ncandA, int64_t* __restrict__ ncandB) {
  hd_flag_body(rowmin, nA2, epsA, nA_dev, colmin, nB2, epsB, nB_dev, c1, sc, candA, candB, ncandA, ncandB);
}

// Block-wide argmax over (value, lowest id): key = float bits << 32 | ~id.
__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
  v = warp_max_u64(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0ull;
    v = warp_max_u64(v);
    if (l == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

__device__ double dist64(const float* a, const float* b, int D) {
  double s = 0.0;
  for (int k = threadIdx.x & 31; k < D; k += 32) {
    double d = (double)a[k] - (double)b[k];
    s = fma(d, d, s);
  }
  s = warp_sum(s);
  return sqrt(s);
}

// One block. best arrays hold packed (d^2, nn index) per entry; ids (or the
// identity) give the row number of each entry. Every index is validated
// before use: with non-finite input the candidate lists can be empty, and the
// result is then NaN with the device status set.
__device__ __forceinline__ void hd_finalize_body(
    const float* __restrict__ A, const int64_t* nA_dev, const float* __restrict__ B, const int64_t* nB_dev, int D,
    const unsigned long long* __restrict__ bestA, const int32_t* __restrict__ idsA, const int64_t* cntA_dev,
    const unsigned long long* __restrict__ bestB, const int32_t* __restrict__ idsB, const int64_t* cntB_dev,
    const int32_t* __restrict__ mapA, const int32_t* __restrict__ mapB, const HdScalars* sc, int* status,
    prohd_hd_result* out, bool rows_only = false) {
  __shared__ unsigned long long sh[32];
  __shared__ int64_t s_nn[2];
  __shared__ double s_d[2];
  const int64_t nA = *nA_dev, nB = *nB_dev;
  const int64_t cA = *cntA_dev, cB = *cntB_dev;
  if (threadIdx.x == 0) s_nn[0] = s_nn[1] = -1;
  unsigned long long ka = 0, kb = 0;
  for (int64_t c = threadIdx.x; c < cA; c += blockDim.x) {
    uint32_t id = idsA ? (uint32_t)idsA[c] : (uint32_t)c;
    unsigned long long k = ((bestA[c] >> 32) << 32) | (unsigned long long)(~id);
    ka = k > ka ? k : ka;
  }
  for (int64_t c = threadIdx.x; c < cB; c += blockDim.x) {
    uint32_t id = idsB ? (uint32_t)idsB[c] : (uint32_t)c;
    unsigned long long k = ((bestB[c] >> 32) << 32) | (unsigned long long)(~id);
    kb = k > kb ? k : kb;
  }
  ka = block_max_u64(ka, sh);
  kb = block_max_u64(kb, sh);
  const int64_t ia = (cA > 0) ? (int64_t)(~(uint32_t)(ka & 0xffffffffu)) : -1;
  const int64_t jb = (cB > 0) ? (int64_t)(~(uint32_t)(kb & 0xffffffffu)) : -1;
  for (int64_t c = threadIdx.x; c < cA; c += blockDim.x) {
    uint32_t id = idsA ? (uint32_t)idsA[c] : (uint32_t)c;
    if ((int64_t)id == ia && bestA[c] != ~0ull) s_nn[0] = packed_idx(bestA[c]);
  }
  for (int64_t c = threadIdx.x; c < cB; c += blockDim.x) {
    uint32_t id = idsB ? (uint32_t)idsB[c] : (uint32_t)c;
    if ((int64_t)id == jb && bestB[c] != ~0ull) s_nn[1] = packed_idx(bestB[c]);
  }
  __syncthreads();
  const int64_t ja = s_nn[0], ib = s_nn[1];
  const bool okA = ia >= 0 && ia < nA && ja >= 0 && ja < nB;
  const bool okB = jb >= 0 && jb < nB && ib >= 0 && ib < nA;
  if (threadIdx.x < 32) {
    double d = okA ? dist64(A + ia * D, B + ja * D, D) : __longlong_as_double(0x7ff8000000000000ll);
    if (threadIdx.x == 0) s_d[0] = d;
  } else if (threadIdx.x < 64) {
    double d = okB ? dist64(B + jb * D, A + ib * D, D) : __longlong_as_double(0x7ff8000000000000ll);
    if (threadIdx.x == 32) s_d[1] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    prohd_hd_result r;
    r.h_ab = s_d[0];
    r.h_ba = s_d[1];
    r.ab_a = okA ? (mapA ? mapA[ia] : ia) : -1;
    r.ab_b = okA ? (mapB ? mapB[ja] : ja) : -1;
    r.ba_b = okB ? (mapB ? mapB[jb] : jb) : -1;
    r.ba_a = okB ? (mapA ? mapA[ib] : ib) : -1;
    r.dir = (r.h_ab >= r.h_ba) ? 0 : 1;
    r.H = r.dir == 0 ? r.h_ab : r.h_ba;
    r.wit_a = r.dir == 0 ? r.ab_a : r.ba_a;
    r.wit_b = r.dir == 0 ? r.ab_b : r.ba_b;
    if (!(okA && (okB || rows_only)) && *status == PROHD_OK) *status = PROHD_ENONFINITE;
    r.status = *status;
    if (sc) {
      r.H_lowp = ldexp(sqrt(fmax((double)sc->lowp_max, 0.0)), -scale_exponent(sc->maxabs));
      r.n_rescored_a = cA;
      r.n_rescored_b = cB;
    } else {
      r.H_lowp = r.H;
      r.n_rescored_a = 0;
      r.n_rescored_b = 0;
    }
    *out = r;
  }
}

__global__ void hd_finalize_kernel(const float* __restrict__ A, const int64_t* nA_dev, const float* __restrict__ B,
                                   const int64_t* nB_dev, int D, const unsigned long long* __restrict__ bestA,
                                   const int32_t* __restrict__ idsA, const int64_t* cntA_dev,
                                   const unsigned long long* __restrict__ bestB, const int32_t* __restrict__ idsB,
                                   const int64_t* cntB_dev, const int32_t* __restrict__ mapA,
                                   const int32_t* __restrict__ mapB, const HdScalars* sc, int* status,
                                   prohd_hd_result* out) {
  hd_finalize_body(A, nA_dev, B, nB_dev, D, bestA, idsA, cntA_dev, bestB, idsB, cntB_dev, mapA, mapB, sc, status, out);
}

// ---------------------------------------------------------------- batched pairs

// Exact FP32 HD of every pair's candidate subsets (direct differences, the
// FP32 path) as one persistent launch over a work queue of 128 x 128 tiles:
// tile t belongs to the pair whose range [prefix[i], prefix[i+1]) holds it
// (pairs in the batch's order, largest first), and blocks take tiles from an
// atomic ticket. Then one finalize block per pair maps the witnesses to
// caller indices and recomputes their distances in FP64.
// mode 0: 128 x 128 tiles of the subset product; mode 1: 128-row blocks of A.
__global__ void hd_tile_scan_kernel(const BPair* __restrict__ P, const int* __restrict__ order, int npairs,
                                    int64_t* __restrict__ prefix, int mode) {
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int base = 0; base < npairs; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int64_t v = 0;
    if (i < npairs) {
      const BPair& q = P[order[i]];
      v = mode == 0 ? ceil_div_dev(q.nsel[0], kSimtBM) * ceil_div_dev(q.nsel[1], kSimtBN)
                    : ceil_div_dev(q.nsel[0], 128);
    }
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int64_t x = lane < nw ? wsum[lane] : 0;
      int64_t xi = x;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += t;
      }
      if (lane < nw) wsum[lane] = xi - x;
    }
    __syncthreads();
    if (i < npairs) prefix[i] = carry + wsum[w] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) prefix[npairs] = carry;
}

__global__ void __launch_bounds__(256, 1)
    simt_dist_queue_kernel(const BPair* __restrict__ P, const int* __restrict__ order, int npairs,
                           const int64_t* __restrict__ prefix, unsigned long long* __restrict__ ticket) {
  __shared__ SimtSmem<true> sm;
  __shared__ int64_t s_t;
  const int64_t total = prefix[npairs];
  for (;;) {
    if (threadIdx.x == 0) s_t = (int64_t)atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t t = s_t;
    __syncthreads();
    if (t >= total) break;
    int lo = 0, hi = npairs;  // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= t) lo = mid;
      else hi = mid;
    }
    const BPair& q = P[order[lo]];
    const int64_t nrows = q.nsel[0], ncols = q.nsel[1];
    const int64_t nct = ceil_div_dev(ncols, kSimtBN), local = t - prefix[lo];
    simt_tile<false, true, true>(sm, q.As, nullptr, nrows, q.Bs, ncols, q.D, q.bestA, q.bestB, local / nct,
                                 local % nct);
  }
}

__global__ void hd_finalize_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.x];
  hd_finalize_body(q.As, q.nsel + 0, q.Bs, q.nsel + 1, q.D, q.bestA, nullptr, q.nsel + 0, q.bestB, nullptr,
                   q.nsel + 1, q.idxA, q.idxB, nullptr, q.status, &q.out->hd);
}

// =====================================================================
// Host orchestration
// =====================================================================

struct HdBufs {
  int64_t nA_pad = 0, nB_pad = 0;
  int Dp = 0;
  // FP32 path and rescoring
  unsigned long long* bestA = nullptr;
  unsigned long long* bestB = nullptr;
  // tensor path
  void* At = nullptr;
  void* Bt = nullptr;
  float *nA2 = nullptr, *nB2 = nullptr, *epsA = nullptr, *epsB = nullptr, *shift = nullptr;
  double* spart = nullptr;  // shift column sums [2][8][D]
  float *nA8 = nullptr, *nB8 = nullptr;  // TF32 norm operands [n_pad][8]
  float* rowmin = nullptr;
  unsigned* colmin = nullptr;
  int32_t *candA = nullptr, *candB = nullptr;
  HdScalars* sc = nullptr;
};

bool tc_supported_dim(int D) { return D >= 1 && D <= 256; }

static void layout(Arena& ws, int64_t nA_max, int64_t nB_max, int D, int precision, HdBufs& b) {
  b.bestA = ws.take<unsigned long long>((size_t)nA_max);
  b.bestB = ws.take<unsigned long long>((size_t)nB_max);
  if (precision != PROHD_FP32) {
    b.nA_pad = round_up(nA_max, kTcBM);
    b.nB_pad = round_up(nB_max, kTcBN);
    b.Dp = (int)round_up(D, kTcBK);
    b.At = ws.take<uint16_t>((size_t)b.nA_pad * b.Dp, 1024);
    b.Bt = ws.take<uint16_t>((size_t)b.nB_pad * b.Dp, 1024);
    b.nA2 = ws.take<float>((size_t)b.nA_pad);
    b.nB2 = ws.take<float>((size_t)b.nB_pad);
    b.epsA = ws.take<float>((size_t)b.nA_pad);
    b.epsB = ws.take<float>((size_t)b.nB_pad);
    b.rowmin = ws.take<float>((size_t)b.nA_pad);
    b.colmin = ws.take<unsigned>((size_t)b.nB_pad);
    b.candA = ws.take<int32_t>((size_t)nA_max);
    b.candB = ws.take<int32_t>((size_t)nB_max);
    b.shift = ws.take<float>((size_t)D);
    b.spart = ws.take<double>((size_t)16 * D);
    b.nA8 = ws.take<float>((size_t)b.nA_pad * 8, 1024);
    b.nB8 = ws.take<float>((size_t)b.nB_pad * 8, 1024);
    b.sc = ws.take<HdScalars>(1);
  }
}

void hd_core_layout(Arena& ws, int64_t nA_max, int64_t nB_max, int D, int precision) {
  HdBufs b;
  layout(ws, nA_max, nB_max, D, precision, b);
}

template <typename K>
static int blocks_for(K kernel, int threads, size_t smem, int num_sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return std::max(1, per_sm) * num_sms;
}

static cudaError_t launch_simt(bool row_list, bool want_row, bool want_col, const float* X, const int32_t* rowlist,
                               const int64_t* nrows_dev, const float* Y, const int64_t* ncols_dev, int D,
                               unsigned long long* rowbest, unsigned long long* colbest, int num_sms, cudaStream_t st) {
  const int grid = num_sms;
  count_launch();
  if (!row_list && want_row && want_col)
    simt_dist_kernel<false, true, true><<<grid, 256, 0, st>>>(X, rowlist, nrows_dev, Y, ncols_dev, D, rowbest, colbest);
  else if (row_list && want_row && !want_col)
    simt_dist_kernel<true, true, false><<<grid, 256, 0, st>>>(X, rowlist, nrows_dev, Y, ncols_dev, D, rowbest, colbest);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// The scalars of a shared preparation that every contraction against it uses.
__global__ void hd_shared_scalars_kernel(const HdScalars* __restrict__ src, HdScalars* __restrict__ dst) {
  dst->maxabs = src->maxabs;
  dst->maxnormB = src->maxnormB;
  dst->maxepsB = src->maxepsB;
}

void hd_shared_layout(Arena& ws, int64_t nY_max, int D, int precision, HdShared& s) {
  s.pad = round_up(nY_max, kTcBN);
  s.Dp = (int)round_up(D, kTcBK);
  s.Yt = ws.take<uint16_t>((size_t)s.pad * s.Dp, 1024);
  s.n2 = ws.take<float>((size_t)s.pad);
  s.eps = ws.take<float>((size_t)s.pad);
  s.n8 = ws.take<float>((size_t)s.pad * 8, 1024);
  s.shift = ws.take<float>((size_t)D);
  s.spart = ws.take<double>((size_t)16 * D);
  s.sc = ws.take<HdScalars>(1);
  (void)precision;
}

cudaError_t hd_shared_prepare(prohd_ctx* ctx, const float* X, const int64_t* nX_dev, const float* Y,
                              const int64_t* nY_dev, int D, int precision, HdShared& s, int* status_dev,
                              cudaStream_t st) {
  if (precision == PROHD_FP32 || !tc_supported_dim(D)) return cudaErrorInvalidValue;
  const int nsm = ctx->num_sms;
  HdScalars* sc = static_cast<HdScalars*>(s.sc);
  PhaseTimer pt(ctx, PROHD_PH_HD_PREP, st);
  cudaMemsetAsync(sc, 0, sizeof(HdScalars), st);
  count_launch();
  hd_colsum_kernel<<<dim3((D + 31) / 32, 8, 2), 256, 0, st>>>(X, nX_dev, Y, nY_dev, D, s.spart);
  count_launch();
  hd_shift_kernel<<<(D + 255) / 256, 256, 0, st>>>(s.spart, nX_dev, nY_dev, D, s.shift);
  count_launch();
  hd_maxabs_kernel<<<nsm * 4, 256, 0, st>>>(X, nX_dev, D, s.shift, &sc->maxabs, status_dev);
  count_launch();
  hd_maxabs_kernel<<<nsm * 4, 256, 0, st>>>(Y, nY_dev, D, s.shift, &sc->maxabs, status_dev);
  count_launch();
  if (precision == PROHD_BF16)
    hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(Y, nY_dev, s.pad, D, s.Dp, s.shift, &sc->maxabs, 1.f,
                                              (__nv_bfloat16*)s.Yt, s.n2, s.eps, &sc->maxnormB, &sc->maxepsB, s.n8, 1);
  else
    hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(Y, nY_dev, s.pad, D, s.Dp, s.shift, &sc->maxabs, 1.f, (__half*)s.Yt,
                                              s.n2, s.eps, &sc->maxnormB, &sc->maxepsB, s.n8, 1);
  return cudaGetLastError();
}

// Rounded copies, norms and margins of A and B (one shift and scale for both,
// or B's from a shared preparation).
static cudaError_t tc_prep(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, const float* B,
                           const int64_t* nB_dev, int D, int precision, HdBufs& b, int* status_dev, cudaStream_t st,
                           const HdShared* shared, const HdCenter* center = nullptr) {
  const int nsm = ctx->num_sms;
  const int bf16 = precision == PROHD_BF16 ? 1 : 0;
  PhaseTimer pt_prep(ctx, PROHD_PH_HD_PREP, st);
  cudaMemsetAsync(b.sc, 0, sizeof(HdScalars), st);
  if (center && !shared) {
    // the centre and the bound were taken before (the rows were scanned for
    // non-finite values then): the copies only
    b.shift = const_cast<float*>(center->shift);
    cudaError_t e = cudaMemcpyAsync(&b.sc->maxabs, center->maxabs, sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e) return e;
    count_launch(2);
    if (bf16) {
      hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                                (__nv_bfloat16*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                                b.nA8, 0);
      hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(B, nB_dev, b.nB_pad, D, b.Dp, b.shift, &b.sc->maxabs, 1.f,
                                                (__nv_bfloat16*)b.Bt, b.nB2, b.epsB, &b.sc->maxnormB, &b.sc->maxepsB,
                                                b.nB8, 1);
    } else {
      hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                                (__half*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                                b.nA8, 0);
      hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(B, nB_dev, b.nB_pad, D, b.Dp, b.shift, &b.sc->maxabs, 1.f,
                                                (__half*)b.Bt, b.nB2, b.epsB, &b.sc->maxnormB, &b.sc->maxepsB,
                                                b.nB8, 1);
    }
    return cudaGetLastError();
  }
  if (shared) {
    // B was prepared once (hd_shared_prepare) with a shift and scale that
    // cover every row set A is drawn from: take its copy, norms, margins and
    // scalars, and prepare A alone with the same shift and scale
    b.shift = shared->shift;
    b.Bt = shared->Yt;
    b.nB2 = shared->n2;
    b.epsB = shared->eps;
    b.nB8 = shared->n8;
    count_launch();
    hd_shared_scalars_kernel<<<1, 1, 0, st>>>(static_cast<const HdScalars*>(shared->sc), b.sc);
    if (bf16) {
      count_launch();
      hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                                (__nv_bfloat16*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                                b.nA8, 0);
    } else {
      count_launch();
      hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                                (__half*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                                b.nA8, 0);
    }
    return cudaGetLastError();
  }
  count_launch();
  hd_colsum_kernel<<<dim3((D + 31) / 32, 8, 2), 256, 0, st>>>(A, nA_dev, B, nB_dev, D, b.spart);
  count_launch();
  hd_shift_kernel<<<(D + 255) / 256, 256, 0, st>>>(b.spart, nA_dev, nB_dev, D, b.shift);
  count_launch();
  hd_maxabs_kernel<<<nsm * 4, 256, 0, st>>>(A, nA_dev, D, b.shift, &b.sc->maxabs, status_dev);
  count_launch();
  hd_maxabs_kernel<<<nsm * 4, 256, 0, st>>>(B, nB_dev, D, b.shift, &b.sc->maxabs, status_dev);
  if (bf16) {
    count_launch();
    hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                              (__nv_bfloat16*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                              b.nA8, 0);
    count_launch();
    hd_prep_kernel<1><<<nsm * 4, 256, 0, st>>>(B, nB_dev, b.nB_pad, D, b.Dp, b.shift, &b.sc->maxabs, 1.f,
                                              (__nv_bfloat16*)b.Bt, b.nB2, b.epsB, &b.sc->maxnormB, &b.sc->maxepsB,
                                              b.nB8, 1);
  } else {
    count_launch();
    hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(A, nA_dev, b.nA_pad, D, b.Dp, b.shift, &b.sc->maxabs, -2.f,
                                              (__half*)b.At, b.nA2, b.epsA, &b.sc->maxnormA, &b.sc->maxepsA,
                                              b.nA8, 0);
    count_launch();
    hd_prep_kernel<0><<<nsm * 4, 256, 0, st>>>(B, nB_dev, b.nB_pad, D, b.Dp, b.shift, &b.sc->maxabs, 1.f,
                                              (__half*)b.Bt, b.nB2, b.epsB, &b.sc->maxnormB, &b.sc->maxepsB,
                                              b.nB8, 1);
  }
  return cudaGetLastError();
}

// The four tensor maps of a contraction: rounded copies (K-major, 128-byte
// swizzle) and the TF32 norm operands (rows of 8 values, 32-byte swizzle).
struct TcMaps {
  CUtensorMap A, B, NA, NB;
};
static bool tc_maps(prohd_ctx* ctx, int precision, const void* At, int64_t nA_pad, const float* nA8, const void* Bt,
                    int64_t nB_pad, const float* nB8, int Dp, TcMaps& m) {
  const CUtensorMapDataType dt =
      precision == PROHD_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return encode_2d(ctx, &m.A, dt, At, (uint64_t)Dp, (uint64_t)nA_pad, (uint64_t)Dp * 2, kTcBK, kTcBM,
                   CU_TENSOR_MAP_SWIZZLE_128B) &&
         encode_2d(ctx, &m.B, dt, Bt, (uint64_t)Dp, (uint64_t)nB_pad, (uint64_t)Dp * 2, kTcBK, kTcBN,
                   CU_TENSOR_MAP_SWIZZLE_128B) &&
         encode_2d(ctx, &m.NA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nA8, 8, (uint64_t)nA_pad, 32, 8, kTcBM,
                   CU_TENSOR_MAP_SWIZZLE_32B) &&
         encode_2d(ctx, &m.NB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, nB8, 8, (uint64_t)nB_pad, 32, 8, kTcBN,
                   CU_TENSOR_MAP_SWIZZLE_32B);
}

// One contraction of the rows [0, *nA_dev) of m.A against the rows
// [0, *nB_dev) of m.B into rowmin / colmin (both must hold +inf where the
// kernel combines with atomicMin: colmin always, rowmin when seg).
static cudaError_t tc_contract(prohd_ctx* ctx, const TcMaps& m, const int64_t* nA_dev, const int64_t* nB_dev, int Dp,
                               int precision, bool seg, float* rowmin, unsigned* colmin, int* status_dev,
                               int64_t timeout_ns, cudaStream_t st) {
  const int nsm = ctx->num_sms;
  const int KB = Dp / kTcBK;
  const size_t smem = tc_smem_bytes(KB);
  const int grid = nsm;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    kern<<<grid, kTcThreads, smem, st>>>(m.A, m.B, m.NA, m.NB, nA_dev, nB_dev, KB, rowmin, colmin, status_dev,
                                         (uint64_t)timeout_ns);
  };
  if (precision == PROHD_BF16) {
    if (seg) go(hd_tc_kernel<1, true>);
    else go(hd_tc_kernel<1, false>);
  } else {
    if (seg) go(hd_tc_kernel<0, true>);
    else go(hd_tc_kernel<0, false>);
  }
  return cudaGetLastError();
}

// the margin constant of row_interval: the norms enter the accumulator
// through a TF32 MMA of six positive exact parts (up to eight roundings of
// |d2|), hence 32 rather than 16
static double tc_c1(int Dp, int D) { return (2.0 * Dp + 2.0 * D + 32.0) * 5.9604644775390625e-8; }

// Rounded copies, norms and margins of A and B, then the tensor-core
// contraction into b.rowmin / b.colmin (squared low-precision minima, scaled
// units). c1 receives the margin constant of row_interval.
static cudaError_t tc_prep_contract(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, const float* B,
                                    const int64_t* nB_dev, int D, int precision, HdBufs& b, int* status_dev,
                                    int64_t timeout_ns, cudaStream_t st, double& c1, bool few_rows = false,
                                    const HdShared* shared = nullptr, const HdCenter* center = nullptr) {
  if (!tc_supported_dim(D)) return cudaErrorInvalidValue;
  const int nsm = ctx->num_sms;
  cudaError_t e = tc_prep(ctx, A, nA_dev, B, nB_dev, D, precision, b, status_dev, st, shared, center);
  if (e) return e;
  count_launch();
  fill_u32_kernel<<<nsm * 2, 256, 0, st>>>(b.colmin, b.nB_pad, 0x7f800000u);
  count_launch();
  fill_u32_kernel<<<nsm, 256, 0, st>>>(reinterpret_cast<unsigned*>(b.rowmin), b.nA_pad, 0x7f800000u);
  if ((e = cudaGetLastError())) return e;
  TcMaps m;
  if (!tc_maps(ctx, precision, b.At, b.nA_pad, b.nA8, b.Bt, b.nB_pad, b.nB8, b.Dp, m)) return cudaErrorInvalidValue;
  // few row blocks (by the bound, or as the caller expects from a device
  // count): one CTA per SM with the columns cut into segments
  const bool seg = few_rows || b.nA_pad / kTcBM < 2 * (int64_t)nsm;
  {
    PhaseTimer pt_tc(ctx, PROHD_PH_HD_CONTRACT, st);
    if ((e = tc_contract(ctx, m, nA_dev, nB_dev, b.Dp, precision, seg, b.rowmin, b.colmin, status_dev, timeout_ns,
                         st)))
      return e;
  }
  c1 = tc_c1(b.Dp, D);
  return cudaSuccess;
}

cudaError_t hd_core(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, int64_t nA_max, const float* B,
                    const int64_t* nB_dev, int64_t nB_max, int D, int precision, const int32_t* mapA,
                    const int32_t* mapB, prohd_hd_result* out, int* status_dev, Arena& ws, int64_t timeout_ns,
                    cudaStream_t st, bool few_rows, const HdShared* shared, const HdCenter* center) {
  HdBufs b;
  layout(ws, nA_max, nB_max, D, precision, b);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  const int nsm = ctx->num_sms;
  cudaError_t e;

  if (precision == PROHD_FP32) {
    count_launch();
    fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestA, nA_max, ~0ull);
    count_launch();
    fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestB, nB_max, ~0ull);
    {
      PhaseTimer pt(ctx, PROHD_PH_HD_CONTRACT, st);
      if ((e = launch_simt(false, true, true, A, nullptr, nA_dev, B, nB_dev, D, b.bestA, b.bestB, nsm, st))) return e;
    }
    PhaseTimer pt2(ctx, PROHD_PH_HD_RESCORE, st);
    count_launch();
    hd_finalize_kernel<<<1, 1024, 0, st>>>(A, nA_dev, B, nB_dev, D, b.bestA, nullptr, nA_dev, b.bestB, nullptr,
                                           nB_dev, mapA, mapB, nullptr, status_dev, out);
    return cudaGetLastError();
  }

  double c1 = 0.0;
  if ((e = tc_prep_contract(ctx, A, nA_dev, B, nB_dev, D, precision, b, status_dev, timeout_ns, st, c1, few_rows,
                            shared, center)))
    return e;
  PhaseTimer pt_rs(ctx, PROHD_PH_HD_RESCORE, st);
  count_launch();
  hd_bounds_kernel<<<nsm * 2, 256, 0, st>>>(b.rowmin, b.nA2, b.epsA, nA_dev, b.colmin, b.nB2, b.epsB, nB_dev, c1, b.sc);
  count_launch();
  hd_flag_kernel<<<nsm * 2, 256, 0, st>>>(b.rowmin, b.nA2, b.epsA, nA_dev, b.colmin, b.nB2, b.epsB, nB_dev, c1, b.sc,
                                          b.candA, b.candB, &b.sc->ncandA, &b.sc->ncandB);
  count_launch();
  fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestA, nA_max, ~0ull);
  count_launch();
  fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestB, nB_max, ~0ull);
  if ((e = cudaGetLastError())) return e;
  // rescore candidate rows of A against all of B, candidate rows of B against all of A:
  // short lists by rescore_few_kernel, longer ones by the tiled kernel (each
  // kernel leaves the other's case alone, the list length being on the device)
  {
    const size_t fsm = (size_t)kFewRows * 256 * sizeof(float) + (size_t)8 * kFewRows * sizeof(unsigned long long);
    cudaFuncSetAttribute(rescore_few_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    count_launch();
    rescore_few_kernel<<<nsm * 2, 256, fsm, st>>>(A, b.candA, &b.sc->ncandA, B, nB_dev, D, b.bestA);
    count_launch();
    rescore_few_kernel<<<nsm * 2, 256, fsm, st>>>(B, b.candB, &b.sc->ncandB, A, nA_dev, D, b.bestB);
  }
  if ((e = launch_simt(true, true, false, A, b.candA, &b.sc->ncandA, B, nB_dev, D, b.bestA, nullptr, nsm, st))) return e;
  if ((e = launch_simt(true, true, false, B, b.candB, &b.sc->ncandB, A, nA_dev, D, b.bestB, nullptr, nsm, st))) return e;
  count_launch();
  hd_finalize_kernel<<<1, 1024, 0, st>>>(A, nA_dev, B, nB_dev, D, b.bestA, b.candA, &b.sc->ncandA, b.bestB, b.candB,
                                         &b.sc->ncandB, mapA, mapB, b.sc, status_dev, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- subset distance with row pruning

// H(A, B) of two row sets by the same intervals, candidates and FP32
// rescoring as hd_core, with the rows that cannot attain either directed
// maximum left out of the full contractions. With the rounded copies made
// once (one shift and scale):
//  1. all rows of A against B's first P rows: row i's minimum over them gives
//     hiA[i], an upper bound of its NN distance over B (a minimum over fewer
//     columns is larger); the P columns' minima run over all of A, so their
//     intervals' lower ends bound h(B, A) from below: LB_B.
//  2. A's first P rows against all of B: LB_A from those rows likewise, and
//     hiB[j] for every row of B.
//  3. the rows of A with hiA >= LB_A (the hard rows) are where the maximum
//     lies: kSubSample of them, evenly spread over the list, against all of
//     B give a larger lower bound (the largest lower end among them), and
//     likewise for B; the rows whose upper end reaches the new bound form
//     the next list, sampled once more. Keep the rows of A whose hiA reaches
//     the last bound, and the rows of B likewise (and row 0 of each, so that
//     no list is empty); copy the kept rows' rounded copies, norms and
//     margins into compact buffers.
//  4. the kept rows of A against all of B (row minima), all of A against the
//     kept rows of B (column minima): the full intervals of the kept rows.
//  5. bounds, candidates, rescoring and the witnesses as in hd_core, the
//     candidates mapped back to row numbers of A and B.
// The result equals hd_core's: every lower bound used is a row's own lower
// end, so at most hd_core's largest lower bound LB; the row attaining LB has
// an upper end >= LB over all columns, so over the prefix too, and is kept,
// and the kept rows give the same LB; a row hd_core flags has an upper end
// >= LB and is kept; the largest low-precision minimum is a kept row's for
// the same reason. The kept rows thus give the same candidate lists,
// rescored the same way.
constexpr int64_t kSubPrefix = 2048;  // rows of each set in the pruning passes
constexpr int64_t kSubSample = 1024;  // hard rows per set per sample
constexpr int kSubRounds = 2;          // samples of the hard rows

struct HdPruneBufs {
  int64_t *nAp = nullptr, *nBp = nullptr, *nkA = nullptr, *nkB = nullptr, *nsA = nullptr, *nsB = nullptr;
  double* lb = nullptr;  // [2]: LB_A, LB_B
  float *hiA = nullptr, *hiB = nullptr;
  int32_t *kA = nullptr, *kB = nullptr;
  void *AtK = nullptr, *BtK = nullptr;
  float *nA2K = nullptr, *epsAK = nullptr, *nA8K = nullptr;
  float *nB2K = nullptr, *epsBK = nullptr, *nB8K = nullptr;
  float* rowx = nullptr;     // row minima of A's prefix; then those of the passes against B's listed rows (not used)
  unsigned* colK = nullptr;  // column minima of B's kept rows over all of A
};

static void prune_sub_layout(Arena& ws, int64_t nA_max, int64_t nB_max, const HdBufs& b, HdPruneBufs& q) {
  q.nAp = ws.take<int64_t>(1);
  q.nBp = ws.take<int64_t>(1);
  q.nkA = ws.take<int64_t>(1);
  q.nkB = ws.take<int64_t>(1);
  q.nsA = ws.take<int64_t>(1);
  q.nsB = ws.take<int64_t>(1);
  q.lb = ws.take<double>(2);
  q.hiA = ws.take<float>((size_t)nA_max);
  q.hiB = ws.take<float>((size_t)nB_max);
  q.kA = ws.take<int32_t>((size_t)nA_max);
  q.kB = ws.take<int32_t>((size_t)nB_max);
  q.AtK = ws.take<uint16_t>((size_t)b.nA_pad * b.Dp, 1024);
  q.BtK = ws.take<uint16_t>((size_t)b.nB_pad * b.Dp, 1024);
  q.nA2K = ws.take<float>((size_t)b.nA_pad);
  q.epsAK = ws.take<float>((size_t)b.nA_pad);
  q.nA8K = ws.take<float>((size_t)b.nA_pad * 8, 1024);
  q.nB2K = ws.take<float>((size_t)b.nB_pad);
  q.epsBK = ws.take<float>((size_t)b.nB_pad);
  q.nB8K = ws.take<float>((size_t)b.nB_pad * 8, 1024);
  q.rowx = ws.take<float>((size_t)b.nA_pad);
  q.colK = ws.take<unsigned>((size_t)b.nB_pad);
}

bool hd_subset_prunable(int64_t nA_max, int64_t nB_max, int D, int precision) {
  return precision != PROHD_FP32 && tc_supported_dim(D) && nA_max >= 4 * kSubPrefix && nB_max >= 4 * kSubPrefix;
}

void hd_core_pruned_layout(Arena& ws, int64_t nA_max, int64_t nB_max, int D, int precision) {
  HdBufs b;
  layout(ws, nA_max, nB_max, D, precision, b);
  if (hd_subset_prunable(nA_max, nB_max, D, precision)) {
    HdPruneBufs q;
    prune_sub_layout(ws, nA_max, nB_max, b, q);
  }
}

__global__ void prune_sub_init_kernel(const int64_t* __restrict__ nA, const int64_t* __restrict__ nB, int64_t P,
                                      int64_t* __restrict__ nAp, int64_t* __restrict__ nBp, double* __restrict__ lb,
                                      int64_t* __restrict__ nkA, int64_t* __restrict__ nkB) {
  *nAp = *nA < P ? *nA : P;
  *nBp = *nB < P ? *nB : P;
  lb[0] = 0.0;
  lb[1] = 0.0;
  *nkA = 0;
  *nkB = 0;
}

// After a pass of rows [0, nr) against a prefix of the columns, or of a
// prefix of the rows against all columns: hi[] of the side that saw a prefix,
// and the largest lower end of the side that saw everything (over its first
// nlb entries) into *lb. rows: which side saw the prefix (1: the rows).
__global__ void prune_sub_pass_kernel(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                                      const float* __restrict__ epsA, const int64_t* __restrict__ nrow_dev,
                                      const unsigned* __restrict__ colmin, const float* __restrict__ nB2,
                                      const float* __restrict__ epsB, const int64_t* __restrict__ ncol_dev,
                                      const HdScalars* __restrict__ sc, double c1, int rows_saw_prefix,
                                      float* __restrict__ hi_out, double* __restrict__ lb) {
  const int64_t nr = *nrow_dev, nc = *ncol_dev;
  const double inv = ldexp(1.0, -scale_exponent(sc->maxabs));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double best = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nr; i += stride) {
    double lo, hi;
    row_interval(rowmin[i], nA2[i], sc->maxnormB, epsA[i], sc->maxepsB, c1, inv, lo, hi);
    if (rows_saw_prefix) hi_out[i] = __double2float_ru(hi);
    else best = fmax(best, lo);
  }
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nc; j += stride) {
    double lo, hi;
    row_interval(__uint_as_float(colmin[j]), nB2[j], sc->maxnormA, epsB[j], sc->maxepsA, c1, inv, lo, hi);
    if (rows_saw_prefix) best = fmax(best, lo);
    else hi_out[j] = __double2float_ru(hi);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(lb, best);
}

// The pruning state of both sets (index 0: A, 1: B).
struct PruneSets {
  const float* hi[2];
  const int64_t* n[2];
  const double* lb;
  int32_t* kidx[2];
  int64_t* nk[2];
  // rounded copies, norms, margins and norm operands, and their compact copies
  const uint16_t* Xt[2];
  const float *n2[2], *eps[2], *n8[2];
  uint16_t* XtK[2];
  float *n2K[2], *epsK[2], *n8K[2];
  int64_t* ns[2];
  int Dp;
};

// grid (blocks, 2 sets): the rows i < n whose upper end reaches the set's
// lower bound (and row 0), appended to kidx in any order (*nk starts at 0;
// every later step is independent of the order of the list).
__global__ void prune_sub_keep_kernel(const PruneSets q) {
  const int set = blockIdx.y;
  const float* __restrict__ hi = q.hi[set];
  const int64_t n = *q.n[set];
  const double L = q.lb[set];
  int32_t* kidx = q.kidx[set];
  unsigned long long* nk = reinterpret_cast<unsigned long long*>(q.nk[set]);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t end = (n + 31) / 32 * 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < end; i += stride) {
    const bool f = i < n && (i == 0 || (double)hi[i] >= L);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    unsigned long long base = 0;
    if (lane == 0 && m) base = atomicAdd(nk, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) kidx[base + __popc(m & ((1u << lane) - 1))] = (int32_t)i;
  }
}

// grid (blocks, 2 sets): the rounded copies, norms, margins and norm operands
// of listed rows, packed in list order, one warp per row (Dp a multiple of
// 64: whole 16-byte moves). S > 0: S rows evenly spread over the list
// (row i of the output is list entry i nk / S; the count min(nk, S) goes to
// *ns); S = 0: the whole list. Every block also fills its share of the three
// minimum buffers of the next contraction with +inf.
__global__ void prune_sub_gather_kernel(const PruneSets q, int64_t S, unsigned* __restrict__ f0, int64_t n0,
                                        unsigned* __restrict__ f1, int64_t n1, unsigned* __restrict__ f2,
                                        int64_t n2) {
  const int set = blockIdx.y;
  const int64_t nk = *q.nk[set];
  const int64_t cnt = S > 0 ? (nk < S ? nk : S) : nk;
  const int32_t* __restrict__ kidx = q.kidx[set];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int Dp = q.Dp;
  const int row16 = Dp / 8;  // 16-byte words per row
  if (S > 0 && blockIdx.x == 0 && threadIdx.x == 0) *q.ns[set] = cnt;
  for (int64_t c = warp; c < cnt; c += nw) {
    const int64_t r = kidx[(S > 0 && nk > S) ? (c * nk) / S : c];
    const uint4* src = reinterpret_cast<const uint4*>(q.Xt[set] + r * Dp);
    uint4* dst = reinterpret_cast<uint4*>(q.XtK[set] + c * Dp);
    for (int k = lane; k < row16; k += 32) dst[k] = src[k];
    if (lane < 8) q.n8K[set][c * 8 + lane] = q.n8[set][r * 8 + lane];
    if (lane == 0) {
      q.n2K[set][c] = q.n2[set][r];
      q.epsK[set][c] = q.eps[set][r];
    }
  }
  const int64_t tid = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t all = (int64_t)gridDim.x * gridDim.y * blockDim.x;
  for (int64_t i = tid; i < n0; i += all) f0[i] = 0x7f800000u;
  for (int64_t i = tid; i < n1; i += all) f1[i] = 0x7f800000u;
  for (int64_t i = tid; i < n2; i += all) f2[i] = 0x7f800000u;
}

// grid (blocks, 2 sets): the largest lower end over the sampled rows' full
// minima (set 0: row minima of A's sample; set 1: column minima of B's) into
// lb[set]; block (0, 0) also clears the kept-row counts for the next list.
__global__ void prune_sub_lb_kernel(const PruneSets q, const float* __restrict__ rowmin,
                                    const unsigned* __restrict__ colK, const HdScalars* __restrict__ sc, double c1,
                                    double* __restrict__ lb) {
  const int set = blockIdx.y;
  const int64_t n = *q.ns[set];
  const double inv = ldexp(1.0, -scale_exponent(sc->maxabs));
  const float maxnorm_other = set ? sc->maxnormA : sc->maxnormB;
  const float maxeps_other = set ? sc->maxepsA : sc->maxepsB;
  double best = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const float m = set ? __uint_as_float(colK[i]) : rowmin[i];
    double lo, hi;
    row_interval(m, q.n2K[set][i], maxnorm_other, q.epsK[set][i], maxeps_other, c1, inv, lo, hi);
    best = fmax(best, lo);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(lb + set, best);
  if (blockIdx.x == 0 && set == 0 && threadIdx.x == 0) {
    *q.nk[0] = 0;
    *q.nk[1] = 0;
  }
}

// candidate positions in the kept lists -> row numbers
__global__ void prune_sub_remap_kernel(int32_t* __restrict__ candA, const int64_t* __restrict__ ncA,
                                       const int32_t* __restrict__ kA, int32_t* __restrict__ candB,
                                       const int64_t* __restrict__ ncB, const int32_t* __restrict__ kB) {
  const int64_t na = *ncA, nb = *ncB;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < na; c += stride) candA[c] = kA[candA[c]];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nb; c += stride) candB[c] = kB[candB[c]];
}

cudaError_t hd_core_pruned(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, int64_t nA_max, const float* B,
                           const int64_t* nB_dev, int64_t nB_max, int D, int precision, const int32_t* mapA,
                           const int32_t* mapB, prohd_hd_result* out, int* status_dev, Arena& ws, int64_t timeout_ns,
                           cudaStream_t st, const HdCenter* center) {
  if (!hd_subset_prunable(nA_max, nB_max, D, precision)) return cudaErrorInvalidValue;
  HdBufs b;
  layout(ws, nA_max, nB_max, D, precision, b);
  HdPruneBufs q;
  prune_sub_layout(ws, nA_max, nB_max, b, q);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  const int nsm = ctx->num_sms;
  cudaError_t e = tc_prep(ctx, A, nA_dev, B, nB_dev, D, precision, b, status_dev, st, nullptr, center);
  if (e) return e;
  const double c1 = tc_c1(b.Dp, D);
  TcMaps full, keptA, keptB;
  if (!tc_maps(ctx, precision, b.At, b.nA_pad, b.nA8, b.Bt, b.nB_pad, b.nB8, b.Dp, full) ||
      !tc_maps(ctx, precision, q.AtK, b.nA_pad, q.nA8K, b.Bt, b.nB_pad, b.nB8, b.Dp, keptA) ||
      !tc_maps(ctx, precision, b.At, b.nA_pad, b.nA8, q.BtK, b.nB_pad, q.nB8K, b.Dp, keptB))
    return cudaErrorInvalidValue;
  PruneSets ps;
  ps.hi[0] = q.hiA;
  ps.hi[1] = q.hiB;
  ps.n[0] = nA_dev;
  ps.n[1] = nB_dev;
  ps.lb = q.lb;
  ps.kidx[0] = q.kA;
  ps.kidx[1] = q.kB;
  ps.nk[0] = q.nkA;
  ps.nk[1] = q.nkB;
  ps.Xt[0] = static_cast<const uint16_t*>(b.At);
  ps.Xt[1] = static_cast<const uint16_t*>(b.Bt);
  ps.n2[0] = b.nA2;
  ps.n2[1] = b.nB2;
  ps.eps[0] = b.epsA;
  ps.eps[1] = b.epsB;
  ps.n8[0] = b.nA8;
  ps.n8[1] = b.nB8;
  ps.XtK[0] = static_cast<uint16_t*>(q.AtK);
  ps.XtK[1] = static_cast<uint16_t*>(q.BtK);
  ps.n2K[0] = q.nA2K;
  ps.n2K[1] = q.nB2K;
  ps.epsK[0] = q.epsAK;
  ps.epsK[1] = q.epsBK;
  ps.n8K[0] = q.nA8K;
  ps.n8K[1] = q.nB8K;
  ps.ns[0] = q.nsA;
  ps.ns[1] = q.nsB;
  ps.Dp = b.Dp;
  unsigned* rowmin_u = reinterpret_cast<unsigned*>(b.rowmin);
  {
    PhaseTimer pt(ctx, PROHD_PH_HD_CONTRACT, st);
    count_launch();
    prune_sub_init_kernel<<<1, 1, 0, st>>>(nA_dev, nB_dev, kSubPrefix, q.nAp, q.nBp, q.lb, q.nkA, q.nkB);
    // 1. all of A against B's prefix
    count_launch();
    fill_u32_kernel<<<nsm * 2, 256, 0, st>>>(b.colmin, b.nB_pad, 0x7f800000u);
    if ((e = cudaGetLastError())) return e;
    if ((e = tc_contract(ctx, full, nA_dev, q.nBp, b.Dp, precision, false, b.rowmin, b.colmin, status_dev, timeout_ns,
                         st)))
      return e;
    count_launch();
    prune_sub_pass_kernel<<<nsm * 2, 256, 0, st>>>(b.rowmin, b.nA2, b.epsA, nA_dev, b.colmin, b.nB2, b.epsB, q.nBp,
                                                    b.sc, c1, 1, q.hiA, q.lb + 1);
    // 2. A's prefix against all of B (its own minimum buffers, filled here)
    count_launch();
    fill_u32_kernel<<<nsm * 2, 256, 0, st>>>(q.colK, b.nB_pad, 0x7f800000u);
    count_launch();
    fill_u32_kernel<<<nsm, 256, 0, st>>>(reinterpret_cast<unsigned*>(q.rowx), b.nA_pad, 0x7f800000u);
    if ((e = cudaGetLastError())) return e;
    if ((e = tc_contract(ctx, full, q.nAp, nB_dev, b.Dp, precision, true, q.rowx, q.colK, status_dev, timeout_ns,
                         st)))
      return e;
    count_launch();
    prune_sub_pass_kernel<<<nsm * 2, 256, 0, st>>>(q.rowx, b.nA2, b.epsA, q.nAp, q.colK, b.nB2, b.epsB, nB_dev, b.sc,
                                                    c1, 0, q.hiB, q.lb);
    // 3. the hard rows; a sample of them against everything raises the
    // bounds, twice (the second sample is drawn from the rows the first
    // bound left, which lie closer to the maximum)
    count_launch();
    prune_sub_keep_kernel<<<dim3(nsm, 2), 256, 0, st>>>(ps);
    for (int round = 0; round < kSubRounds; ++round) {
      count_launch();
      prune_sub_gather_kernel<<<dim3(nsm * 2, 2), 256, 0, st>>>(ps, kSubSample, rowmin_u, b.nA_pad, b.colmin,
                                                                 b.nB_pad, q.colK, b.nB_pad);
      if ((e = cudaGetLastError())) return e;
      if ((e = tc_contract(ctx, keptA, q.nsA, nB_dev, b.Dp, precision, true, b.rowmin, b.colmin, status_dev,
                           timeout_ns, st)))
        return e;
      if ((e = tc_contract(ctx, keptB, nA_dev, q.nsB, b.Dp, precision, false, q.rowx, q.colK, status_dev, timeout_ns,
                           st)))
        return e;
      count_launch();
      prune_sub_lb_kernel<<<dim3(nsm / 2, 2), 256, 0, st>>>(ps, b.rowmin, q.colK, b.sc, c1, q.lb);
      count_launch();
      prune_sub_keep_kernel<<<dim3(nsm, 2), 256, 0, st>>>(ps);
    }
    // 4. the kept rows: A's against all of B (row minima; the column minima
    // are not used), all of A against B's (column minima)
    count_launch();
    prune_sub_gather_kernel<<<dim3(nsm * 2, 2), 256, 0, st>>>(ps, 0, rowmin_u, b.nA_pad, b.colmin, b.nB_pad, q.colK,
                                                               b.nB_pad);
    if ((e = cudaGetLastError())) return e;
    if ((e = tc_contract(ctx, keptA, q.nkA, nB_dev, b.Dp, precision, true, b.rowmin, b.colmin, status_dev, timeout_ns,
                         st)))
      return e;
    if ((e = tc_contract(ctx, keptB, nA_dev, q.nkB, b.Dp, precision, false, q.rowx, q.colK, status_dev, timeout_ns,
                         st)))
      return e;
  }
  // 5. as hd_core, on the kept rows
  PhaseTimer pt_rs(ctx, PROHD_PH_HD_RESCORE, st);
  count_launch();
  hd_bounds_kernel<<<nsm * 2, 256, 0, st>>>(b.rowmin, q.nA2K, q.epsAK, q.nkA, q.colK, q.nB2K, q.epsBK, q.nkB, c1,
                                            b.sc);
  count_launch();
  hd_flag_kernel<<<nsm * 2, 256, 0, st>>>(b.rowmin, q.nA2K, q.epsAK, q.nkA, q.colK, q.nB2K, q.epsBK, q.nkB, c1, b.sc,
                                          b.candA, b.candB, &b.sc->ncandA, &b.sc->ncandB);
  count_launch();
  prune_sub_remap_kernel<<<nsm, 256, 0, st>>>(b.candA, &b.sc->ncandA, q.kA, b.candB, &b.sc->ncandB, q.kB);
  count_launch();
  fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestA, nA_max, ~0ull);
  count_launch();
  fill_u64_kernel<<<nsm * 4, 256, 0, st>>>(b.bestB, nB_max, ~0ull);
  if ((e = cudaGetLastError())) return e;
  {
    const size_t fsm = (size_t)kFewRows * 256 * sizeof(float) + (size_t)8 * kFewRows * sizeof(unsigned long long);
    cudaFuncSetAttribute(rescore_few_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    count_launch();
    rescore_few_kernel<<<nsm * 2, 256, fsm, st>>>(A, b.candA, &b.sc->ncandA, B, nB_dev, D, b.bestA);
    count_launch();
    rescore_few_kernel<<<nsm * 2, 256, fsm, st>>>(B, b.candB, &b.sc->ncandB, A, nA_dev, D, b.bestB);
  }
  if ((e = launch_simt(true, true, false, A, b.candA, &b.sc->ncandA, B, nB_dev, D, b.bestA, nullptr, nsm, st))) return e;
  if ((e = launch_simt(true, true, false, B, b.candB, &b.sc->ncandB, A, nA_dev, D, b.bestB, nullptr, nsm, st))) return e;
  count_launch();
  hd_finalize_kernel<<<1, 1024, 0, st>>>(A, nA_dev, B, nB_dev, D, b.bestA, b.candA, &b.sc->ncandA, b.bestB, b.candB,
                                         &b.sc->ncandB, mapA, mapB, b.sc, status_dev, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- row pruning

// hi[i] = the upper end of row i's interval: a certified upper bound (in
// original units, rounded up to FP32) of row i's NN distance over the columns
// the contraction saw, so of its NN distance over all columns.
__global__ void hd_row_upper_kernel(const float* __restrict__ rowmin, const float* __restrict__ nA2,
                                    const float* __restrict__ epsA, const int64_t* __restrict__ nA_dev,
                                    const HdScalars* __restrict__ sc, double c1, float* __restrict__ hi_out) {
  const int64_t n = *nA_dev;
  const double inv = ldexp(1.0, -scale_exponent(sc->maxabs));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    double lo, hi;
    row_interval(rowmin[i], nA2[i], sc->maxnormB, epsA[i], sc->maxepsB, c1, inv, lo, hi);
    hi_out[i] = __double2float_ru(hi);
  }
}

cudaError_t hd_prefix_upper(prohd_ctx* ctx, const float* X, const int64_t* nX_dev, int64_t nX_max, const float* Y,
                            const int64_t* nYp_dev, int64_t nYp_max, int D, int precision, float* hi, int* status_dev,
                            Arena& ws, int64_t timeout_ns, cudaStream_t st, const HdShared* shared) {
  if (precision == PROHD_FP32) return cudaErrorInvalidValue;
  HdBufs b;
  layout(ws, nX_max, nYp_max, D, precision, b);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  double c1 = 0.0;
  cudaError_t e =
      tc_prep_contract(ctx, X, nX_dev, Y, nYp_dev, D, precision, b, status_dev, timeout_ns, st, c1, false, shared);
  if (e) return e;
  count_launch();
  hd_row_upper_kernel<<<ctx->num_sms * 2, 256, 0, st>>>(b.rowmin, b.nA2, b.epsA, nX_dev, b.sc, c1, hi);
  return cudaGetLastError();
}

void hd_prefix_layout(Arena& ws, int64_t nX_max, int64_t nYp_max, int D, int precision) {
  HdBufs b;
  layout(ws, nX_max, nYp_max, D, precision, b);
}

cudaError_t hd_simt_batched(const BPair* P, const int* order, int npairs, int64_t* prefix, unsigned long long* ticket,
                            int num_sms, cudaStream_t st) {
  count_launch();
  hd_tile_scan_kernel<<<1, 1024, 0, st>>>(P, order, npairs, prefix, 0);
  cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st);
  count_launch();
  simt_dist_queue_kernel<<<num_sms * 2, 256, 0, st>>>(P, order, npairs, prefix, ticket);
  count_launch();
  hd_finalize_batched_kernel<<<npairs, 1024, 0, st>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched tensor-core subset distance

size_t hd_scalars_bytes() { return sizeof(HdScalars); }
size_t hd_tc_row_block() { return kTcBM; }

// The single-pair kernels of the tensor path, one grid row (y or z) per
// (pair, set) or per pair, the pair's buffers from its descriptor.
__global__ void hd_colsum_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.z >> 1];
  if ((int)blockIdx.x * 32 >= q.D) return;
  hd_colsum_body(q.As, q.nsel + 0, q.Bs, q.nsel + 1, q.D, q.hd_spart, blockIdx.z & 1);
}
__global__ void hd_shift_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  hd_shift_body(q.hd_spart, q.nsel + 0, q.nsel + 1, q.D, q.hd_shift);
}
__global__ void hd_maxabs_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y >> 1];
  const int set = blockIdx.y & 1;
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  hd_maxabs_body(set ? q.Bs : q.As, q.nsel + set, q.D, q.hd_shift, &sc->maxabs, q.status);
}
template <int BF16>
__global__ void hd_prep_batched_kernel(const BPair* __restrict__ P) {
  using T = typename TileT<BF16>::T;
  const BPair& q = P[blockIdx.y >> 1];
  const int set = blockIdx.y & 1;
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  if (set == 0)
    hd_prep_body<BF16>(q.As, q.nsel + 0, q.hd_nA_pad, q.D, q.Dp, q.hd_shift, &sc->maxabs, -2.f,
                       static_cast<T*>(q.hd_At), q.hd_nA2, q.hd_epsA, &sc->maxnormA, &sc->maxepsA, q.hd_nA8, 0);
  else
    hd_prep_body<BF16>(q.Bs, q.nsel + 1, q.hd_nB_pad, q.D, q.Dp, q.hd_shift, &sc->maxabs, 1.f,
                       static_cast<T*>(q.hd_Bt), q.hd_nB2, q.hd_epsB, &sc->maxnormB, &sc->maxepsB, q.hd_nB8, 1);
}
__device__ __forceinline__ double hd_c1(const BPair& q) {
  return (2.0 * q.Dp + 2.0 * q.D + 32.0) * 5.9604644775390625e-8;
}
// Column count the margin passes visit: none when only the rows' distance is wanted.
__device__ const int64_t kNoColumns = 0;
__global__ void hd_bounds_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  hd_bounds_body(q.hd_rowmin, q.hd_nA2, q.hd_epsA, q.nsel + 0, q.hd_colmin, q.hd_nB2, q.hd_epsB,
                 q.rows_only ? &kNoColumns : q.nsel + 1, hd_c1(q), static_cast<HdScalars*>(q.hd_sc));
}
__global__ void hd_flag_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  hd_flag_body(q.hd_rowmin, q.hd_nA2, q.hd_epsA, q.nsel + 0, q.hd_colmin, q.hd_nB2, q.hd_epsB,
               q.rows_only ? &kNoColumns : q.nsel + 1, hd_c1(q), sc, q.hd_candA, q.hd_candB, &sc->ncandA,
               &sc->ncandB);
}
// Candidate rows of A against all of B (set 0) and of B against all of A (set 1).
__global__ void __launch_bounds__(256) rescore_few_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y >> 1];
  const int set = blockIdx.y & 1;
  if (set == 1 && q.rows_only) return;
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  if (set == 0)
    rescore_few_body(q.As, q.hd_candA, &sc->ncandA, q.Bs, q.nsel + 1, q.D, q.bestA);
  else
    rescore_few_body(q.Bs, q.hd_candB, &sc->ncandB, q.As, q.nsel + 0, q.D, q.bestB);
}
__global__ void __launch_bounds__(256, 1) rescore_list_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y >> 1];
  const int set = blockIdx.y & 1;
  if (set == 1 && q.rows_only) return;
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  if (set == 0)
    simt_dist_body<true, true, false>(q.As, q.hd_candA, &sc->ncandA, q.Bs, q.nsel + 1, q.D, q.bestA, nullptr);
  else
    simt_dist_body<true, true, false>(q.Bs, q.hd_candB, &sc->ncandB, q.As, q.nsel + 0, q.D, q.bestB, nullptr);
}
__global__ void hd_finalize_tc_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.x];
  HdScalars* sc = static_cast<HdScalars*>(q.hd_sc);
  hd_finalize_body(q.As, q.nsel + 0, q.Bs, q.nsel + 1, q.D, q.bestA, q.hd_candA, &sc->ncandA, q.bestB, q.hd_candB,
                   &sc->ncandB, q.idxA, q.idxB, sc, q.status, &q.out->hd, q.rows_only != 0);
}

cudaError_t hd_tc_batched(const BPair* P, const int* order, int npairs, int64_t* prefix, const CUtensorMap* maps,
                          int Dmax, int bf16, int* batch_status, int num_sms, int64_t timeout_ns, cudaStream_t st,
                          int bx) {
  const int Dp_max = (int)round_up(Dmax, kTcBK), KBmax = Dp_max / kTcBK;
  cudaError_t e;
  count_launch(5);
  hd_colsum_batched_kernel<<<dim3((Dmax + 31) / 32, 8, 2 * npairs), 256, 0, st>>>(P);
  hd_shift_batched_kernel<<<dim3((Dmax + 255) / 256, npairs), 256, 0, st>>>(P);
  hd_maxabs_batched_kernel<<<dim3(bx, 2 * npairs), 256, 0, st>>>(P);
  if (bf16)
    hd_prep_batched_kernel<1><<<dim3(bx, 2 * npairs), 256, 0, st>>>(P);
  else
    hd_prep_batched_kernel<0><<<dim3(bx, 2 * npairs), 256, 0, st>>>(P);
  hd_tile_scan_kernel<<<1, 1024, 0, st>>>(P, order, npairs, prefix, 1);
  if ((e = cudaGetLastError())) return e;
  const size_t smem = tc_smem_bytes(KBmax);
  if (bf16) {
    cudaFuncSetAttribute(hd_tc_batched_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    hd_tc_batched_kernel<1><<<num_sms, kTcThreads, smem, st>>>(P, order, prefix, maps, npairs, KBmax, batch_status,
                                                               (uint64_t)timeout_ns);
  } else {
    cudaFuncSetAttribute(hd_tc_batched_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    hd_tc_batched_kernel<0><<<num_sms, kTcThreads, smem, st>>>(P, order, prefix, maps, npairs, KBmax, batch_status,
                                                               (uint64_t)timeout_ns);
  }
  if ((e = cudaGetLastError())) return e;
  const size_t fsm = (size_t)kFewRows * 256 * sizeof(float) + (size_t)8 * kFewRows * sizeof(unsigned long long);
  cudaFuncSetAttribute(rescore_few_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  count_launch(5);
  hd_bounds_batched_kernel<<<dim3(4, npairs), 256, 0, st>>>(P);
  hd_flag_batched_kernel<<<dim3(4, npairs), 256, 0, st>>>(P);
  rescore_few_batched_kernel<<<dim3(8, 2 * npairs), 256, fsm, st>>>(P);
  rescore_list_batched_kernel<<<dim3(8, 2 * npairs), 256, 0, st>>>(P);
  hd_finalize_tc_batched_kernel<<<npairs, 1024, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t fill_u32_region(unsigned* p, int64_t n, unsigned v, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  fill_u32_kernel<<<num_sms * 2, 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

}  // namespace prohd
