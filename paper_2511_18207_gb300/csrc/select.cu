// Extreme selection (Algorithms 1-2): for every direction u_d and each set,
// keep the k smallest and the k largest projections x_i^T u_d, then take the
// union over directions (Algorithm 3) as sorted unique indices.
//
// The order is the one of the FP64 projection summed sequentially over
// k = 0..D-1 with separately rounded products and sums, ties broken by the
// lower index at both ends. The GPU reaches it exactly without computing FP64
// projections for every point:
//  1. FP32 projections q (one HBM pass over the points, all directions at
//     once; both sets in one TMA-fed launch, cp.async-staged tiles for the
//     batched path and for more than 17 directions) and E = (D+8) 2^-24 max||x|| ||u|| (1.01)^2, a
//     bound on |q - p64| for every point.
//  2. The exact k-th smallest FP32 key T over order-preserving uint32 keys.
//     One pair: the projection pass also counts every key's top byte, one
//     pass counts the next 11 bits of the keys inside the byte holding rank
//     k; the 19-bit prefix found gives a value range [L, H] that contains T,
//     so q < L - 2E is certainly selected and q > H + 2E certainly not; one
//     pass over the keys marks the former and lists the rest of
//     [L - 2E, H + 2E] as candidates (a few hundred points), and the last
//     bits of T are found among the candidates alone. Batches: a 4-pass radix select over all keys of all
//     (pair, set, direction, side) problems at once.
//  3. q < T - 2E: certainly among the k smallest; q > T + 2E: certainly not;
//     the band in between is ranked by FP64 projections recomputed exactly as
//     the sequential definition (__dmul_rn / __dadd_rn), ties by index.
//  The largest side is the same on reversed keys.
#include <limits.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kProjRows = 256;   // rows per tile (2 per thread)
constexpr int kProjThreads = 128;
constexpr int kProjK = 32;       // dims per stage
constexpr int kProjStride = 36;  // padded row stride (floats): conflict-free 16-B reads

// ---------------------------------------------------------------- projection

// q[d*n + i] = fl32(x_i . u_d); rownorm max into *maxnorm; non-finite check.
// Requires D % 4 == 0 and a 16-byte aligned base (cp.async 16 B).
// Tiles t0, t0 + tstride, ... below t1 of the set.
// hist0 (may be null): [nd][256] counts of the top byte of f32_key(q) per
// direction, accumulated in shared memory and added once per block.
template <int ND>
__device__ __forceinline__ void proj_body(const float* __restrict__ X, int64_t n, int D,
                                          const double* __restrict__ dirs, int nd, float* __restrict__ q,
                                          float* __restrict__ maxnorm, int* __restrict__ status, int64_t t0,
                                          int64_t t1, int64_t tstride, unsigned* __restrict__ hist0) {
  extern __shared__ __align__(16) float psm[];
  const int Dq = (D + kProjK - 1) / kProjK * kProjK;
  float* us = psm;                               // [ND][Dq]
  float* xs = psm + (size_t)ND * Dq;             // [2][kProjRows][kProjStride]
  unsigned* hs = reinterpret_cast<unsigned*>(xs + (size_t)2 * kProjRows * kProjStride);  // [ND][256]
  for (int i = threadIdx.x; i < ND * Dq; i += blockDim.x) {
    int d = i / Dq, k = i % Dq;
    us[i] = (d < nd && k < D) ? (float)dirs[(size_t)d * D + k] : 0.f;
  }
  if (hist0)
    for (int i = threadIdx.x; i < ND * 256; i += blockDim.x) hs[i] = 0u;
  const int t = threadIdx.x;
  const int nchunks = Dq / kProjK;
  float wmax = 0.f;
  bool bad = false;

  // issue the cp.async copies of chunk c of tile `tile` into buffer `buf`
  auto issue = [&](int64_t tile, int c, int buf) {
    float* dst = xs + (size_t)buf * kProjRows * kProjStride;
    // 256 rows x 8 float4 = 2048 copies, 16 per thread
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      int idx = t + e * kProjThreads;
      int r = idx >> 3, f = idx & 7;
      int64_t gr = tile * kProjRows + r;
      int k = c * kProjK + f * 4;
      float* sp = dst + r * kProjStride + f * 4;
      uint32_t sa = smem_u32(sp);
      if (gr < n && k < D) {
        const float* gp = X + gr * D + k;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gp) : "memory");
      } else {
        *reinterpret_cast<float4*>(sp) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  __syncthreads();
  for (int64_t tile = t0; tile < t1; tile += tstride) {
    float acc0[ND], acc1[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) acc0[d] = acc1[d] = 0.f;
    float n0 = 0.f, n1 = 0.f;
    issue(tile, 0, 0);
    for (int c = 0; c < nchunks; ++c) {
      if (c + 1 < nchunks) {
        issue(tile, c + 1, (c + 1) & 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      __syncthreads();
      const float* xb = xs + (size_t)(c & 1) * kProjRows * kProjStride;
      const float* x0p = xb + t * kProjStride;
      const float* x1p = xb + (t + kProjThreads) * kProjStride;
#pragma unroll
      for (int f = 0; f < kProjK / 4; ++f) {
        float4 a = *reinterpret_cast<const float4*>(x0p + 4 * f);
        float4 b = *reinterpret_cast<const float4*>(x1p + 4 * f);
        n0 = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, n0))));
        n1 = fmaf(b.x, b.x, fmaf(b.y, b.y, fmaf(b.z, b.z, fmaf(b.w, b.w, n1))));
        const float* up = us + c * kProjK + 4 * f;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          float4 u = *reinterpret_cast<const float4*>(up + (size_t)d * Dq);
          acc0[d] = fmaf(a.w, u.w, fmaf(a.z, u.z, fmaf(a.y, u.y, fmaf(a.x, u.x, acc0[d]))));
          acc1[d] = fmaf(b.w, u.w, fmaf(b.z, u.z, fmaf(b.y, u.y, fmaf(b.x, u.x, acc1[d]))));
        }
      }
      __syncthreads();
    }
    const int64_t r0 = tile * kProjRows + t, r1 = r0 + kProjThreads;
    if (r0 < n) {
#pragma unroll
      for (int d = 0; d < ND; ++d)
        if (d < nd) {
          q[(size_t)d * n + r0] = acc0[d];
          if (hist0) atomicAdd(&hs[d * 256 + (f32_key(acc0[d]) >> 24)], 1u);
        }
      bad |= !isfinite(n0);
      wmax = fmaxf(wmax, sqrtf(n0));
    }
    if (r1 < n) {
#pragma unroll
      for (int d = 0; d < ND; ++d)
        if (d < nd) {
          q[(size_t)d * n + r1] = acc1[d];
          if (hist0) atomicAdd(&hs[d * 256 + (f32_key(acc1[d]) >> 24)], 1u);
        }
      bad |= !isfinite(n1);
      wmax = fmaxf(wmax, sqrtf(n1));
    }
  }
  if (hist0) {
    __syncthreads();
    for (int i = threadIdx.x; i < nd * 256; i += blockDim.x)
      if (hs[i]) atomicAdd(hist0 + i, hs[i]);
  }
  wmax = warp_max(wmax);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(maxnorm, wmax);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicMax(status, (int)PROHD_ENONFINITE);
}

template <int ND>
__global__ void __launch_bounds__(kProjThreads)
    proj_kernel(const float* __restrict__ X, int64_t n, int D, const double* __restrict__ dirs, int nd,
                float* __restrict__ q, float* __restrict__ maxnorm, int* __restrict__ status,
                unsigned* __restrict__ hist0) {
  proj_body<ND>(X, n, D, dirs, nd, q, maxnorm, status, blockIdx.x, (n + kProjRows - 1) / kProjRows, gridDim.x,
                hist0);
}

// Batched: one item (a row range of one set of one pair) per block.
template <int ND>
__global__ void __launch_bounds__(kProjThreads)
    proj_items_kernel(const BPair* __restrict__ P, const ProjItem* __restrict__ items) {
  const ProjItem it = items[blockIdx.x];
  const BPair& q = P[it.pair];
  const int64_t n = it.set ? q.nB : q.nA;
  proj_body<ND>(it.set ? q.B : q.A, n, q.D, q.dirs, q.nd, it.set ? q.qB : q.qA, q.maxnorm + it.set, q.status,
                it.r0 / kProjRows, (it.r1 + kProjRows - 1) / kProjRows, 1, nullptr);
}

// ---------------------------------------------------------------- TMA projection of a pair

// One persistent launch projects both sets: tiles of kPtRows rows, A's tiles
// first, then B's. A producer warp streams each tile through a ring of
// `stages` shared-memory stages, 32 dimensions (128 bytes) of every row per
// stage, by TMA with the 128-byte swizzle (chunk j of row r lands at
// position j ^ (r & 7) of the row, so the row-per-thread reads of a quarter
// warp hit eight different bank groups); rows past n and dimensions past D
// arrive as zeros. Each of the kPtThreads consumer threads owns kPtRpt rows
// (r, r + kPtThreads, ...) and sums the products of dimension pairs with
// packed FP32 FMAs (even and odd dimensions in the two halves, added at the
// end). Any summation order stays within the bound E of the header (the
// rounding error of a D-term dot product in FP32 is at most D 2^-24 sum
// |x_k u_k| for every order of the terms).
constexpr int kPtThreads = 256;                  // consumer threads
constexpr int kPtRpt = 2;                        // rows per consumer thread
constexpr int kPtRows = kPtThreads * kPtRpt;     // rows per tile
constexpr int kPtBox = 256;                      // rows per TMA box
constexpr uint32_t kPtStageBytes = kPtRows * 128;
constexpr int kPtMaxStages = 4;

struct ProjPairArgs {
  int64_t nA, nB, tilesA, tiles;
  int D, Dq, nd, nchunks, stages;
  const double* dirs;
  float *qA, *qB;
  float* maxnorm;      // [2]
  int* status;
  unsigned* hist;      // [2][nd][256] top-byte counts, or null
  int64_t timeout_ns;
};

__device__ __forceinline__ uint64_t pk_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float pk_sum(uint64_t v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return a + b;
}

template <int ND>
__global__ void __launch_bounds__(kPtThreads + 32, 1)
    proj_pair_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const ProjPairArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_align<1024>(smem_raw);
  const int S = p.stages;
  float* us = reinterpret_cast<float*>(base + (size_t)S * kPtStageBytes);  // [ND][Dq]
  unsigned* hs = reinterpret_cast<unsigned*>(us + (size_t)ND * p.Dq);      // [2][ND][256]
  uint64_t* full = reinterpret_cast<uint64_t*>(hs + 2 * ND * 256);
  uint64_t* empty = full + kPtMaxStages;
  volatile int* abort = reinterpret_cast<int*>(empty + kPtMaxStages);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

  for (int i = t; i < ND * p.Dq; i += blockDim.x) {
    const int d = i / p.Dq, k = i % p.Dq;
    us[i] = (d < p.nd && k < p.D) ? (float)p.dirs[(size_t)d * p.D + k] : 0.f;
  }
  if (p.hist)
    for (int i = t; i < 2 * ND * 256; i += blockDim.x) hs[i] = 0u;
  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kPtThreads / 32);
    }
    *abort = 0;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == kPtThreads / 32) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      uint32_t g = 0;  // stage uses issued
      for (int64_t tile = blockIdx.x; tile < p.tiles && !*abort; tile += gridDim.x) {
        const bool setB = tile >= p.tilesA;
        const CUtensorMap* m = setB ? &tmB : &tmA;
        const int y0 = (int)((setB ? tile - p.tilesA : tile) * kPtRows);
        for (int c = 0; c < p.nchunks; ++c) {
          const int s = (int)(g % (uint32_t)S);
          if (!mbar_wait_bounded(&empty[s], ((g / (uint32_t)S) & 1u) ^ 1u, abort, (uint64_t)p.timeout_ns)) break;
          mbar_arrive_expect_tx(&full[s], kPtStageBytes);
          uint8_t* dst = base + (size_t)s * kPtStageBytes;
#pragma unroll
          for (int b = 0; b < kPtRows / kPtBox; ++b) tma_load_2d(dst + b * kPtBox * 128, m, c * 32, y0 + b * kPtBox, &full[s]);
          ++g;
        }
      }
      if (*abort) {
        // error path: the copies already issued land before the CTA exits
        for (uint32_t h = g >= (uint32_t)S ? g - (uint32_t)S : 0u; h < g; ++h) {
          const uint64_t t0 = global_timer_ns();
          while (!mbar_try_wait(&full[h % (uint32_t)S], (h / (uint32_t)S) & 1u) && global_timer_ns() - t0 < 2000000ull) {
          }
        }
      }
    }
  } else {
    // ---------------- consumers ----------------
    float wmax0 = 0.f, wmax1 = 0.f;  // per set
    bool bad0 = false, bad1 = false;
    uint32_t g = 0;
    for (int64_t tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
      const int setB = tile >= p.tilesA ? 1 : 0;
      const int64_t r0 = (setB ? tile - p.tilesA : tile) * kPtRows;
      uint64_t acc[kPtRpt][ND], nrm[kPtRpt];
#pragma unroll
      for (int j = 0; j < kPtRpt; ++j) {
        nrm[j] = 0ull;
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[j][d] = 0ull;
      }
      bool ok = true;
      for (int c = 0; c < p.nchunks; ++c, ++g) {
        const int s = (int)(g % (uint32_t)S);
        ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (g / (uint32_t)S) & 1u, abort, (uint64_t)p.timeout_ns));
        if (!ok) break;
        const float* xb = reinterpret_cast<const float*>(base + (size_t)s * kPtStageBytes);
        const float* uc = us + c * 32;
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          ulonglong2 xv[kPtRpt];
#pragma unroll
          for (int j = 0; j < kPtRpt; ++j) {
            const int row = t + j * kPtThreads;
            xv[j] = *reinterpret_cast<const ulonglong2*>(xb + row * 32 + ((f ^ (row & 7)) << 2));
            nrm[j] = pk_fma(xv[j].y, xv[j].y, pk_fma(xv[j].x, xv[j].x, nrm[j]));
          }
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(uc + (size_t)d * p.Dq + 4 * f);
#pragma unroll
            for (int j = 0; j < kPtRpt; ++j) acc[j][d] = pk_fma(xv[j].y, u.y, pk_fma(xv[j].x, u.x, acc[j][d]));
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      if (!ok) break;
      const int64_t n = setB ? p.nB : p.nA;
      float* q = setB ? p.qB : p.qA;
#pragma unroll
      for (int j = 0; j < kPtRpt; ++j) {
        const int64_t r = r0 + t + j * kPtThreads;
        if (r < n) {
#pragma unroll
          for (int d = 0; d < ND; ++d)
            if (d < p.nd) {
              const float v = pk_sum(acc[j][d]);
              q[(size_t)d * n + r] = v;
              if (p.hist) atomicAdd(&hs[(setB * ND + d) * 256 + (f32_key(v) >> 24)], 1u);
            }
          const float nn = pk_sum(nrm[j]);
          if (setB) {
            bad1 |= !isfinite(nn);
            wmax1 = fmaxf(wmax1, sqrtf(nn));
          } else {
            bad0 |= !isfinite(nn);
            wmax0 = fmaxf(wmax0, sqrtf(nn));
          }
        }
      }
    }
    wmax0 = warp_max(wmax0);
    wmax1 = warp_max(wmax1);
    if (lane == 0) {
      atomic_max_nonneg(p.maxnorm + 0, wmax0);
      atomic_max_nonneg(p.maxnorm + 1, wmax1);
    }
    if (__any_sync(0xffffffffu, bad0 || bad1) && lane == 0) atomicMax(p.status, (int)PROHD_ENONFINITE);
  }
  __syncthreads();
  if (p.hist)
    for (int i = t; i < 2 * ND * 256; i += blockDim.x) {
      const int s = i / (ND * 256), d = (i / 256) % ND;
      if (d < p.nd && hs[i]) atomicAdd(p.hist + ((size_t)s * p.nd + d) * 256 + (i & 255), hs[i]);
    }
  if (t == 0 && *abort) atomicMax(p.status, (int)PROHD_ETIMEOUT);
}

// Fallback for D % 4 != 0 or unaligned bases: warp per row, lanes over dims.
__global__ void proj_simple_kernel(const float* __restrict__ X, int64_t n, int D, const double* __restrict__ dirs,
                                   int nd, float* __restrict__ q, float* __restrict__ maxnorm, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float wmax = 0.f;
  bool bad = false;
  for (int64_t r = warp; r < n; r += nw) {
    const float* x = X + r * D;
    float nn = 0.f;
    for (int k = lane; k < D; k += 32) nn = fmaf(x[k], x[k], nn);
    nn = warp_sum(nn);
    for (int d = 0; d < nd; ++d) {
      float s = 0.f;
      for (int k = lane; k < D; k += 32) s = fmaf(x[k], (float)dirs[(size_t)d * D + k], s);
      s = warp_sum(s);
      if (lane == 0) q[(size_t)d * n + r] = s;
    }
    bad |= !isfinite(nn);
    wmax = fmaxf(wmax, sqrtf(nn));
  }
  wmax = warp_max(wmax);
  if (lane == 0) atomic_max_nonneg(maxnorm, wmax);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(status, (int)PROHD_ENONFINITE);
}

// ---------------------------------------------------------------- radix select

// Per problem p = set * nd + d and side s (0 = smallest, 1 = largest):
struct SelProb {
  uint32_t prefix[2];   // key bits fixed so far
  int64_t rank[2];      // remaining 0-based rank inside the current prefix
  int64_t k;            // k of this (set, direction)
  double E;             // |q - p64| bound for this (set, direction)
  int64_t cin[2];       // points certainly selected on each side
  int64_t nband[2];     // band sizes (candidate counts between extraction and candidate selection)
  // one-pass extraction (single pair): side 0 selects v < t_in[0] and lists
  // the rest of v <= c_lim[0]; side 1 selects v > t_in[1] and lists the rest
  // of v >= c_lim[1]
  float t_in[2], c_lim[2];
  // the problem's data: FP32 keys q[0..n), points X [n][D], direction u,
  // selection mask, band lists and their FP64 keys (one per side)
  const float* q;
  int64_t n;
  const float* X;
  const double* u;
  uint8_t* mask;
  const float* maxnorm;  // max ||x|| of the set
  int D;
  int32_t* band[2];
  uint64_t* bkey[2];
};

constexpr int kMaxDirs = 64;
struct KList {
  int64_t k[2 * kMaxDirs];  // k of (set, direction) p = set * nd + d, passed by value
};

// Starting state of a problem whose data fields are set: ranks of the k-th
// smallest and largest keys, and the bound E.
__device__ __forceinline__ void sel_reset(SelProb& s, int64_t k) {
  const int64_t n = s.n;
  k = k < 1 ? 1 : (k > n ? n : k);
  double un = 0.0;
  for (int j = 0; j < s.D; ++j) un += s.u[j] * s.u[j];
  un = sqrt(un);
  s.prefix[0] = s.prefix[1] = 0;
  s.rank[0] = k - 1;
  s.rank[1] = n - k;
  s.k = k;
  s.E = ((double)s.D + 8.0) * 5.9604644775390625e-8 * 1.0201 * (double)(*s.maxnorm) * un + 1e-300;
  s.cin[0] = s.cin[1] = 0;
  s.nband[0] = s.nband[1] = 0;
}

// Batched: the data fields were written when the batch was planned; k comes
// from the problem's alpha (alpha_c on the centroid axis, alpha_p on the
// components) and the set size.
__global__ void sel_reset_batched_kernel(SelProb* __restrict__ P, int nprob, const double* __restrict__ alpha_of) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  SelProb& s = P[p];
  const double kk = floor(alpha_of[p] * (double)s.n);
  sel_reset(s, kk < 1.0 ? 1 : (int64_t)kk);
}

// grid (chunks, 2*nd). hist: [2*nd][2][256]
__global__ void radix_hist_kernel(const SelProb* __restrict__ P, int pass, unsigned* __restrict__ hist, int pbase) {
  __shared__ unsigned h[2][256];
  const int p = pbase + blockIdx.y;
  const int64_t n = P[p].n;
  const float* q = P[p].q;
  for (int i = threadIdx.x; i < 512; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const int shift = 24 - 8 * pass;
  const uint32_t himask = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
  const uint32_t p0 = P[p].prefix[0], p1 = P[p].prefix[1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // eight independent loads in flight per thread
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < n; base += 8 * stride) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * stride;
      v[u] = i < n ? __ldg(q + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (base + u * stride >= n) break;
      const uint32_t key = f32_key(v[u]);
      const uint32_t bin = (key >> shift) & 255u;
      if (((key ^ p0) & himask) == 0) atomicAdd(&h[0][bin], 1u);
      if (((key ^ p1) & himask) == 0) atomicAdd(&h[1][bin], 1u);
    }
  }
  __syncthreads();
  unsigned* g = hist + (size_t)p * 512;
  for (int i = threadIdx.x; i < 512; i += blockDim.x) {
    unsigned v = (&h[0][0])[i];
    if (v) atomicAdd(g + i, v);
  }
}

// One warp per (problem, side): pick the bin holding the target rank.
__global__ void radix_pick_kernel(SelProb* __restrict__ P, int nprob, int pass, unsigned* __restrict__ hist,
                                  int pbase) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nprob * 2) return;
  const int p = pbase + (w >> 1), side = w & 1;
  unsigned* h = hist + (size_t)p * 512 + side * 256;
  int64_t r = P[p].rank[side];
  // each lane owns 8 consecutive bins
  unsigned c[8];
  unsigned tot = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j] = h[lane * 8 + j];
    tot += c[j];
  }
  unsigned incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned excl = incl - tot;
  const bool mine = (int64_t)excl <= r && r < (int64_t)incl;
  const unsigned who = __ballot_sync(0xffffffffu, mine);
  if (who) {
    const int src = __ffs(who) - 1;
    if (lane == src) {
      int64_t rr = r - (int64_t)excl;
      int bin = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (rr < (int64_t)c[j]) { bin = lane * 8 + j; break; }
        rr -= c[j];
      }
      const int shift = 24 - 8 * pass;
      P[p].prefix[side] |= (uint32_t)bin << shift;
      P[p].rank[side] = rr;
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 8; ++j) h[lane * 8 + j] = 0;
}

// ---------------------------------------------------------------- band pass

// Float thresholds equivalent to comparing the double of a float with x:
// for every float v, (double)v < x <=> v < f32_up(x), (double)v <= x <=>
// v <= f32_down(x), and likewise for > and >= (NaN stays NaN, so every
// comparison with it stays false). FP64 comparisons per point would cost
// more than the whole pass on this GPU.
__device__ __forceinline__ float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, __int_as_float(0x7f800000));
  return f;
}
__device__ __forceinline__ float f32_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, __int_as_float(0xff800000));
  return f;
}

// ---------------------------------------------------------------- one pair: one pass over the keys

// Value of a key, with the keys that decode to NaN (bins beyond the finite
// range) mapped to -inf / +inf so that thresholds built from them select
// nothing as certain and list everything else as candidates.
__device__ __forceinline__ float key_value_lo(uint32_t k) {
  const float v = key_f32(k);
  return v == v ? v : __int_as_float(0xff800000);
}
__device__ __forceinline__ float key_value_hi(uint32_t k) {
  const float v = key_f32(k);
  return v == v ? v : __int_as_float(0x7f800000);
}

// Index of the bin holding rank r among n bins counted in ascending order
// (side 0) or descending order (side 1), and the rank left inside it; one
// block of 256 threads, bins in shared memory, the scan in the fixed order of
// thread indices. Writes *bin and *left from the thread that owns the bin.
template <int NB>
__device__ __forceinline__ void block_pick(const unsigned* __restrict__ h, int64_t r, int side, int* bin,
                                           int64_t* left) {
  constexpr int PER = NB / 256;
  __shared__ unsigned long long s_part[256];
  const int t = threadIdx.x;
  // thread t owns PER consecutive bins of the side's order
  unsigned long long own = 0;
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int o = t * PER + j;
    own += h[side ? NB - 1 - o : o];
  }
  s_part[t] = own;
  __syncthreads();
  // inclusive scan (Hillis-Steele) over 256 partial counts
  for (int off = 1; off < 256; off <<= 1) {
    const unsigned long long v = t >= off ? s_part[t - off] : 0ull;
    __syncthreads();
    s_part[t] += v;
    __syncthreads();
  }
  const unsigned long long incl = s_part[t], excl = incl - own;
  if ((int64_t)excl <= r && r < (int64_t)incl) {
    int64_t x = r - (int64_t)excl;
    for (int j = 0; j < PER; ++j) {
      const int o = t * PER + j;
      const int b = side ? NB - 1 - o : o;
      if (x < (int64_t)h[b]) {
        *bin = b;
        *left = x;
        break;
      }
      x -= h[b];
    }
  }
  __syncthreads();
}

// One block per (set, direction) problem: its data, k, the bound E, and
// from the top-byte histogram of its keys the byte of each side's k-th key
// (prefix[side] = byte << 24) and the rank left inside that byte (counted
// from the low end for side 0, from the high end for side 1).
__global__ void __launch_bounds__(256)
    sel_init_pick_kernel(SelProb* __restrict__ P, int nd, const KList kl, const float* __restrict__ A,
                         const float* __restrict__ qA, int64_t nA, uint8_t* __restrict__ maskA,
                         const float* __restrict__ B, const float* __restrict__ qB, int64_t nB,
                         uint8_t* __restrict__ maskB, int D, const double* __restrict__ dirs,
                         const float* __restrict__ maxnorm, int32_t* __restrict__ band,
                         uint64_t* __restrict__ bandkey, int64_t cap, const unsigned* __restrict__ hist0) {
  __shared__ unsigned h[256];
  __shared__ int s_bin[2];
  __shared__ int64_t s_left[2];
  const int p = blockIdx.x;
  const int set = p / nd, d = p % nd;
  const int64_t n = set ? nB : nA;
  int64_t k = kl.k[p];
  k = k < 1 ? 1 : (k > n ? n : k);
  h[threadIdx.x] = hist0[(size_t)p * 256 + threadIdx.x];
  if (threadIdx.x < 2) {
    s_bin[threadIdx.x] = threadIdx.x ? 0 : 255;
    s_left[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int side = 0; side < 2; ++side) block_pick<256>(h, k - 1, side, &s_bin[side], &s_left[side]);
  // ||u||^2 in parallel (the serial FP64 sum in sel_reset is a long chain of
  // dependent additions); any order gives a valid bound E
  __shared__ double s_un[256];
  double un = 0.0;
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    const double x = dirs[(size_t)d * D + j];
    un += x * x;
  }
  s_un[threadIdx.x] = un;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_un[threadIdx.x] += s_un[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  SelProb s;
  s.n = n;
  s.q = (set ? qB : qA) + (size_t)d * s.n;
  s.X = set ? B : A;
  s.u = dirs + (size_t)d * D;
  s.mask = set ? maskB : maskA;
  s.maxnorm = maxnorm + set;
  s.D = D;
  for (int side = 0; side < 2; ++side) {
    s.band[side] = band + ((size_t)p * 2 + side) * cap;
    s.bkey[side] = bandkey + ((size_t)p * 2 + side) * cap;
  }
  s.prefix[0] = s.prefix[1] = 0;
  s.k = k;
  s.E = ((double)D + 8.0) * 5.9604644775390625e-8 * 1.0201 * (double)(*s.maxnorm) * sqrt(s_un[0]) + 1e-300;
  s.cin[0] = s.cin[1] = 0;
  s.nband[0] = s.nband[1] = 0;
  for (int side = 0; side < 2; ++side) {
    s.prefix[side] = (uint32_t)s_bin[side] << 24;
    s.rank[side] = s_left[side];
  }
  P[p] = s;
}

constexpr int kHist1Bins = 2048;  // bits 23..13 of the key
constexpr int kHist1Blocks = 32;  // blocks per problem (each writes its own histogram pair)

// The keys of one problem as a 16-byte aligned float4 body and scalar ends:
// `head` keys before the first aligned one, nv float4s, then the rest.
struct KeySpan {
  int64_t head, nv;
};
__device__ __forceinline__ KeySpan key_span(const float* q, int64_t n) {
  KeySpan k;
  k.head = ((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15) >> 2;
  if (k.head > n) k.head = n;
  k.nv = (n - k.head) >> 2;
  return k;
}

// Second digit: histograms of bits 23..13 of the keys whose top byte is
// each side's byte. grid (kHist1Blocks, 2*nd); out [2*nd][blocks][2][2048].
__global__ void __launch_bounds__(512) hist1_kernel(const SelProb* __restrict__ P, unsigned* __restrict__ out) {
  __shared__ unsigned h[2][kHist1Bins];
  const SelProb& S = P[blockIdx.y];
  for (int i = threadIdx.x; i < 2 * kHist1Bins; i += blockDim.x) (&h[0][0])[i] = 0u;
  __syncthreads();
  const int64_t n = S.n;
  const uint32_t b0 = S.prefix[0] >> 24, b1 = S.prefix[1] >> 24;
  const float* q = S.q;
  auto count = [&](float v) {
    const uint32_t k = f32_key(v);
    const uint32_t top = k >> 24, dig = (k >> 13) & (kHist1Bins - 1);
    if (top == b0) atomicAdd(&h[0][dig], 1u);
    if (top == b1) atomicAdd(&h[1][dig], 1u);
  };
  const KeySpan ks = key_span(q, n);
  const float4* q4 = reinterpret_cast<const float4*>(q + ks.head);
  const int64_t c0 = ks.nv * blockIdx.x / gridDim.x, c1 = ks.nv * (blockIdx.x + 1) / gridDim.x;
  // eight independent 16-byte loads in flight per thread
  for (int64_t base = c0; base < c1; base += 8 * (int64_t)blockDim.x) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * (int64_t)blockDim.x + threadIdx.x;
      v[u] = i < c1 ? __ldg(q4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * (int64_t)blockDim.x + threadIdx.x;
      if (i >= c1) continue;
      count(v[u].x);
      count(v[u].y);
      count(v[u].z);
      count(v[u].w);
    }
  }
  if (blockIdx.x == 0)
    for (int64_t i = threadIdx.x; i < ks.head; i += blockDim.x) count(__ldg(q + i));
  if (blockIdx.x == gridDim.x - 1)
    for (int64_t i = ks.head + 4 * ks.nv + threadIdx.x; i < n; i += blockDim.x) count(__ldg(q + i));
  __syncthreads();
  unsigned* o = out + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 2 * kHist1Bins;
  for (int i = threadIdx.x; i < 2 * kHist1Bins; i += blockDim.x) o[i] = (&h[0][0])[i];
}

// One block per (problem, side): the 11-bit digit holding the side's rank
// inside its byte, then the thresholds of the extraction pass. With [L, H]
// the values of the 19-bit key prefix, the k-th smallest key T lies in
// [L, H]: v < L - 2E is certainly among the k smallest (it is below
// T - 2E), v > H + 2E certainly not (above T + 2E), and [L - 2E, H + 2E]
// holds every point the band can need. The largest side mirrors this.
__global__ void __launch_bounds__(256) pick1_kernel(SelProb* __restrict__ P, const unsigned* __restrict__ hist1) {
  __shared__ unsigned h[kHist1Bins];
  __shared__ int s_dig;
  __shared__ int64_t s_left;
  const int p = blockIdx.x >> 1, side = blockIdx.x & 1;
  SelProb& S = P[p];
  for (int i = threadIdx.x; i < kHist1Bins; i += blockDim.x) {
    unsigned t = 0;
    for (int b = 0; b < kHist1Blocks; ++b) t += hist1[(((size_t)p * kHist1Blocks + b) * 2 + side) * kHist1Bins + i];
    h[i] = t;
  }
  if (threadIdx.x == 0) {
    s_dig = side ? 0 : kHist1Bins - 1;
    s_left = 0;
  }
  __syncthreads();
  block_pick<kHist1Bins>(h, S.rank[side], side, &s_dig, &s_left);
  if (threadIdx.x != 0) return;
  const int dig = s_dig;
  const uint32_t pre = S.prefix[side] | ((uint32_t)dig << 13);
  const double L = (double)key_value_lo(pre), H = (double)key_value_hi(pre | 0x1fffu);
  const double E2 = 2.0 * S.E;
  if (side == 0) {
    S.t_in[0] = f32_up(L - E2);     // v < t_in  <=>  (double)v < L - 2E
    S.c_lim[0] = f32_down(H + E2);  // v <= c_lim <=> (double)v <= H + 2E
  } else {
    S.t_in[1] = f32_down(H + E2);   // v > t_in  <=>  (double)v > H + 2E
    S.c_lim[1] = f32_up(L - E2);    // v >= c_lim <=> (double)v >= L - 2E
  }
  S.nband[side] = 0;
  S.cin[side] = 0;
}

// One pass over the keys of every problem: certain members are marked and
// counted, candidates listed per side as (index, key) in the band buffers
// (side 1 stores the reversed key, so both sides look for a smallest key).
// grid (chunks, 2*nd). The keys are read as float4s (and the few keys before
// the first 16-byte boundary and after the last one as scalars).
__global__ void extract_kernel(SelProb* __restrict__ P) {
  SelProb& S = P[blockIdx.y];
  const int64_t n = S.n;
  const float* q = S.q;
  uint8_t* mask = S.mask;
  const float t0 = S.t_in[0], c0 = S.c_lim[0], t1 = S.t_in[1], c1 = S.c_lim[1];
  int32_t* b0 = S.band[0];
  int32_t* b1 = S.band[1];
  uint64_t* k0 = S.bkey[0];
  uint64_t* k1 = S.bkey[1];
  const int lane = threadIdx.x & 31;
  unsigned long long in0c = 0, in1c = 0;
  // classify one key; returns the candidate bits (1: side 0, 2: side 1)
  auto classify = [&](float v, int64_t i) -> unsigned {
    const bool in0 = v < t0, in1 = v > t1;
    if (in0 || in1) mask[i] = 1;
    in0c += in0;
    in1c += in1;
    return ((!in0 && v <= c0) ? 1u : 0u) | ((!in1 && v >= c1) ? 2u : 0u);
  };
  // append the warp's candidates of one slot (every lane of the warp calls it)
  auto append = [&](unsigned cd, float v, int64_t i) {
    const unsigned m0 = __ballot_sync(0xffffffffu, cd & 1u), m1 = __ballot_sync(0xffffffffu, cd & 2u);
    if (!(m0 | m1)) return;
    unsigned long long base0 = 0, base1 = 0;
    if (lane == 0 && m0)
      base0 = atomicAdd(reinterpret_cast<unsigned long long*>(&S.nband[0]), (unsigned long long)__popc(m0));
    if (lane == 0 && m1)
      base1 = atomicAdd(reinterpret_cast<unsigned long long*>(&S.nband[1]), (unsigned long long)__popc(m1));
    base0 = __shfl_sync(0xffffffffu, base0, 0);
    base1 = __shfl_sync(0xffffffffu, base1, 0);
    const unsigned below = (1u << lane) - 1;
    const uint32_t key = f32_key(v);
    if (cd & 1u) {
      const unsigned long long o = base0 + __popc(m0 & below);
      b0[o] = (int32_t)i;
      k0[o] = key;
    }
    if (cd & 2u) {
      const unsigned long long o = base1 + __popc(m1 & below);
      b1[o] = (int32_t)i;
      k1[o] = ~key;
    }
  };
  const KeySpan ks = key_span(q, n);
  const float4* q4 = reinterpret_cast<const float4*>(q + ks.head);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t end = (ks.nv + 31) / 32 * 32;  // whole warps step together
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < end; base += 4 * stride) {
    // four independent 16-byte loads in flight, classified before any warp-wide step
    float4 vv[4];
    uint32_t cand = 0;  // 2 bits per key: slot u, component e at bit 2 (4u + e)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = base + u * stride;
      vv[u] = j < ks.nv ? __ldg(q4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = base + u * stride;
      if (j >= ks.nv) continue;
      const int64_t i = ks.head + 4 * j;
      cand |= classify(vv[u].x, i) << (2 * (4 * u + 0));
      cand |= classify(vv[u].y, i + 1) << (2 * (4 * u + 1));
      cand |= classify(vv[u].z, i + 2) << (2 * (4 * u + 2));
      cand |= classify(vv[u].w, i + 3) << (2 * (4 * u + 3));
    }
    // candidates are rare: the append path runs only where a lane has one
    if (!__any_sync(0xffffffffu, cand != 0)) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = base + u * stride;
      if (j - lane >= end) break;  // the whole warp is past the end
      const int64_t i = ks.head + 4 * j;
      append((cand >> (2 * (4 * u + 0))) & 3u, vv[u].x, i);
      append((cand >> (2 * (4 * u + 1))) & 3u, vv[u].y, i + 1);
      append((cand >> (2 * (4 * u + 2))) & 3u, vv[u].z, i + 2);
      append((cand >> (2 * (4 * u + 3))) & 3u, vv[u].w, i + 3);
    }
  }
  // the scalar ends (at most 3 keys each), by the first warp of block 0
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    const int64_t tail0 = ks.head + 4 * ks.nv;
    const int64_t i = lane < ks.head ? lane : tail0 + (lane - 4);
    const bool mine = lane < ks.head || (lane >= 4 && lane < 8 && i < n);
    const float v = mine ? __ldg(q + i) : 0.f;
    const unsigned cd = mine ? classify(v, i) : 0u;
    append(cd, v, i);
  }
  in0c = warp_sum(in0c);
  in1c = warp_sum(in1c);
  if (lane == 0) {
    if (in0c) atomicAdd(reinterpret_cast<unsigned long long*>(&S.cin[0]), in0c);
    if (in1c) atomicAdd(reinterpret_cast<unsigned long long*>(&S.cin[1]), in1c);
  }
}

constexpr int kCandThreads = 512;
constexpr int kCandBins = 2048;

// One block per (problem, side): the exact k-th key T among the candidates
// (radix select over the 32-bit stored keys: 11 + 11 + 10 bits), then every
// candidate below T - 2E is marked certain and those within [T - 2E, T + 2E]
// are compacted, in order and in place, into the front of the band list.
__global__ void __launch_bounds__(kCandThreads) cand_select_kernel(SelProb* __restrict__ P) {
  __shared__ unsigned hist[kCandBins];
  __shared__ unsigned wsum[kCandThreads / 32];
  __shared__ int64_t s_rank;
  __shared__ uint32_t s_prefix;
  __shared__ int s_ok;
  __shared__ unsigned long long s_cert, s_band;
  const int p = blockIdx.x >> 1, side = blockIdx.x & 1;
  SelProb& S = P[p];
  const int64_t nc = S.nband[side];
  const int64_t r = S.k - 1 - S.cin[side];
  int32_t* lst = S.band[side];
  const uint64_t* keys = S.bkey[side];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_rank = r;
    s_prefix = 0;
    s_ok = (nc > 0 && r >= 0 && r < nc) ? 1 : 0;
    s_cert = 0;
    s_band = 0;
  }
  __syncthreads();
  if (!s_ok) {
    // no candidate holds rank k (only with non-finite keys, which the
    // projection reports): nothing more is selected on this side
    if (tid == 0) S.nband[side] = 0;
    return;
  }
  for (int pass = 0; pass < 3; ++pass) {
    const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    const int width = pass == 2 ? 10 : 11;
    const uint32_t dmask = (1u << width) - 1u;
    const uint32_t him = pass == 0 ? 0u : (0xffffffffu << (shift + width));
    for (int i = tid; i < kCandBins; i += kCandThreads) hist[i] = 0;
    __syncthreads();
    const uint32_t pre = s_prefix;
    for (int64_t i = tid; i < nc; i += kCandThreads) {
      const uint32_t k = (uint32_t)__ldg(keys + i);
      if (((k ^ pre) & him) == 0) atomicAdd(&hist[(k >> shift) & dmask], 1u);
    }
    __syncthreads();
    if (w == 0) {
      // lane l owns bins 64 l .. 64 l + 63
      unsigned tot = 0;
      for (int j = 0; j < 64; ++j) tot += hist[lane * 64 + j];
      unsigned incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const unsigned excl = incl - tot;
      const int64_t rr = s_rank;
      const bool mine = (int64_t)excl <= rr && rr < (int64_t)incl;
      if (mine) {
        int64_t x = rr - (int64_t)excl;
        int bin = lane * 64 + 63;
        for (int j = 0; j < 64; ++j) {
          const unsigned c = hist[lane * 64 + j];
          if (x < (int64_t)c) {
            bin = lane * 64 + j;
            break;
          }
          x -= c;
        }
        s_prefix = pre | ((uint32_t)bin << shift);
        s_rank = x;
      }
    }
    __syncthreads();
  }
  const uint32_t kstar = s_prefix;
  const double T = (double)key_f32(side ? ~kstar : kstar);
  const double E2 = 2.0 * S.E;
  // side 0: certain v < T - 2E, band v <= T + 2E; side 1: certain v > T + 2E,
  // band v >= T - 2E (as float thresholds)
  const float f_in = side ? f32_down(T + E2) : f32_up(T - E2);
  const float f_band = side ? f32_up(T - E2) : f32_down(T + E2);
  uint8_t* mask = S.mask;
  unsigned long long cert = 0;
  for (int64_t base = 0; base < nc; base += kCandThreads) {
    const int64_t i = base + tid;
    bool inb = false;
    int32_t id = 0;
    if (i < nc) {
      const uint32_t k = (uint32_t)__ldg(keys + i);
      const float v = key_f32(side ? ~k : k);
      id = lst[i];
      const bool in = side ? v > f_in : v < f_in;
      inb = !in && (side ? v >= f_band : v <= f_band);
      if (in) {
        mask[id] = 1;
        ++cert;
      }
    }
    // ordered block-wide compaction of the band members
    const unsigned m = __ballot_sync(0xffffffffu, inb);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int j = 0; j < kCandThreads / 32; ++j) {
      const unsigned c = wsum[j];
      before += j < w ? c : 0u;
      total += c;
    }
    const unsigned long long o = s_band + before + __popc(m & ((1u << lane) - 1));
    __syncthreads();  // every read of this chunk is done before any write
    if (inb) lst[o] = id;
    if (tid == 0) s_band += total;
    __syncthreads();
  }
  cert = warp_sum(cert);
  if (lane == 0 && cert) atomicAdd(&s_cert, cert);
  __syncthreads();
  if (tid == 0) {
    S.cin[side] += (int64_t)s_cert;
    S.nband[side] = (int64_t)s_band;
  }
}

// Marks certain members, counts them, and lists band members per side.
// band lists: [2*nd][2][cap] int32
__global__ void band_kernel(SelProb* __restrict__ P, int pbase) {
  const int p = pbase + blockIdx.y;
  const int64_t n = P[p].n;
  const float* q = P[p].q;
  uint8_t* mask = P[p].mask;
  const double E2 = 2.0 * P[p].E;
  const double Tlo = (double)key_f32(P[p].prefix[0]), Thi = (double)key_f32(P[p].prefix[1]);
  // q < lo_in, q <= lo_band, q > hi_in, q >= hi_band in double, as float comparisons
  const float f_lo_in = f32_up(Tlo - E2), f_lo_band = f32_down(Tlo + E2);
  const float f_hi_in = f32_down(Thi + E2), f_hi_band = f32_up(Thi - E2);
  int32_t* b0 = P[p].band[0];
  int32_t* b1 = P[p].band[1];
  const int lane = threadIdx.x & 31;
  unsigned long long c0 = 0, c1 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t end = (n + 31) / 32 * 32;
  // eight independent loads in flight, classified before any warp-wide step
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; base < end; base += 8 * stride) {
    float vv[8];
    unsigned bd = 0;  // bit u: band member of side 0; bit 8 + u: of side 1
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * stride;
      vv[u] = i < n ? __ldg(q + i) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * stride;
      if (i >= n) continue;
      const float v = vv[u];
      const bool in0 = v < f_lo_in, in1 = v > f_hi_in;
      if (in0 || in1) mask[i] = 1;
      c0 += in0;
      c1 += in1;
      bd |= ((!in0 && v <= f_lo_band) ? 1u : 0u) << u;
      bd |= ((!in1 && v >= f_hi_band) ? 1u : 0u) << (8 + u);
    }
    // band members are rare: the append path runs only where a lane has one
    if (!__any_sync(0xffffffffu, bd != 0)) continue;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t i = base + u * stride;
      if (i - lane >= end) break;  // the whole warp is past the end
      const bool bd0 = (bd >> u) & 1u, bd1 = (bd >> (8 + u)) & 1u;
      const unsigned m0 = __ballot_sync(0xffffffffu, bd0), m1 = __ballot_sync(0xffffffffu, bd1);
      if (!(m0 | m1)) continue;
      unsigned long long base0 = 0, base1 = 0;
      if (lane == 0 && m0)
        base0 = atomicAdd(reinterpret_cast<unsigned long long*>(&P[p].nband[0]), (unsigned long long)__popc(m0));
      if (lane == 0 && m1)
        base1 = atomicAdd(reinterpret_cast<unsigned long long*>(&P[p].nband[1]), (unsigned long long)__popc(m1));
      base0 = __shfl_sync(0xffffffffu, base0, 0);
      base1 = __shfl_sync(0xffffffffu, base1, 0);
      const unsigned below = (1u << lane) - 1;
      if (bd0) b0[base0 + __popc(m0 & below)] = (int32_t)i;
      if (bd1) b1[base1 + __popc(m1 & below)] = (int32_t)i;
    }
  }
  c0 = warp_sum(c0);
  c1 = warp_sum(c1);
  if (lane == 0) {
    if (c0) atomicAdd(reinterpret_cast<unsigned long long*>(&P[p].cin[0]), c0);
    if (c1) atomicAdd(reinterpret_cast<unsigned long long*>(&P[p].cin[1]), c1);
  }
}

// FP64 projection exactly as the sequential definition.
// FP64 keys of every band member, one thread per member and many blocks:
// the sequential FP64 sum is a chain of dependent additions whose latency is
// long on this GPU, so as many chains as possible run side by side (a warp
// per member, with one lane summing, was seven times slower).
// grid (chunks, 4 * nd): y = problem * 2 + side.
__global__ void band_keys_kernel(const SelProb* __restrict__ P) {
  const int p = blockIdx.y >> 1, side = blockIdx.y & 1;
  const float* X = P[p].X;
  const int D = P[p].D;
  const int64_t b = P[p].nband[side];
  const int64_t r = P[p].k - P[p].cin[side];
  if (b == 0 || r <= 0) return;
  __shared__ double us[1024];
  const double* u = P[p].u;
  const bool u_sm = D <= 1024;
  if (u_sm)
    for (int k = threadIdx.x; k < D; k += blockDim.x) us[k] = u[k];
  __syncthreads();
  const double* uu = u_sm ? us : u;
  const int32_t* lst = P[p].band[side];
  uint64_t* keys = P[p].bkey[side];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    const float* x = X + (int64_t)__ldg(lst + i) * D;
    int k = 0;
    for (; k + 8 <= D; k += 8) {
      float xv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) xv[j] = __ldg(x + k + j);
#pragma unroll
      for (int j = 0; j < 8; ++j) s = __dadd_rn(s, __dmul_rn((double)xv[j], uu[k + j]));
    }
    for (; k < D; ++k) s = __dadd_rn(s, __dmul_rn((double)__ldg(x + k), uu[k]));
    const uint64_t kk = f64_key(s);
    keys[i] = side ? ~kk : kk;
  }
}

constexpr int kBandSmem = 2048;

// One block per (problem, side): rank band members by (FP64 key, index) and
// mark the r = k - cin smallest. Small bands are ranked in shared memory by
// counting; large bands use a radix select over the 96-bit (key, index).
__global__ void __launch_bounds__(512)
    band_resolve_kernel(const SelProb* __restrict__ P) {
  __shared__ uint64_t sk[kBandSmem];
  __shared__ int32_t si[kBandSmem];
  __shared__ unsigned hist[256];
  __shared__ int64_t s_rank;
  __shared__ uint64_t s_prefix;
  const int p = blockIdx.x >> 1, side = blockIdx.x & 1;
  uint8_t* mask = P[p].mask;
  const int64_t b = P[p].nband[side];
  const int64_t r = P[p].k - P[p].cin[side];
  if (b == 0 || r <= 0) return;
  const int32_t* lst = P[p].band[side];
  const uint64_t* keys = P[p].bkey[side];
  if (b <= kBandSmem) {
    // bitonic sort of (key, index) pairs, padded with the largest pair up
    // to a power of two; then the first r are the selected ones
    int P2 = 1;
    while (P2 < b) P2 <<= 1;
    for (int i = threadIdx.x; i < P2; i += blockDim.x) {
      si[i] = i < b ? __ldg(lst + i) : INT_MAX;
      sk[i] = i < b ? __ldg(keys + i) : ~0ull;
    }
    __syncthreads();
    for (int size = 2; size <= P2; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = threadIdx.x; t < (P2 >> 1); t += blockDim.x) {
          const int i = 2 * t - (t & (stride - 1)), j = i + stride;
          const bool up = (i & size) == 0;
          const uint64_t ka = sk[i], kb = sk[j];
          const int32_t ia = si[i], ib = si[j];
          const bool gt = ka > kb || (ka == kb && ia > ib);
          if (gt == up) {
            sk[i] = kb;
            sk[j] = ka;
            si[i] = ib;
            si[j] = ia;
          }
        }
        __syncthreads();
      }
    for (int64_t i = threadIdx.x; i < r && i < b; i += blockDim.x) mask[si[i]] = 1;
    return;
  }

  // large band: radix select of the r-th smallest (key, idx) over the global keys
  if (threadIdx.x == 0) {
    s_rank = r - 1;
    s_prefix = 0;
  }
  __syncthreads();
  // 8 passes over the 64-bit key
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    const uint64_t him = pass == 0 ? 0ull : (~0ull << (64 - 8 * pass));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint64_t pre = s_prefix;
    for (int64_t i = threadIdx.x; i < b; i += blockDim.x) {
      uint64_t k = __ldg(keys + i);
      if (((k ^ pre) & him) == 0) atomicAdd(&hist[(k >> shift) & 255], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t rr = s_rank;
      int bin = 0;
      for (; bin < 256; ++bin) {
        if (rr < (int64_t)hist[bin]) break;
        rr -= hist[bin];
      }
      s_prefix = pre | ((uint64_t)bin << shift);
      s_rank = rr;
    }
    __syncthreads();
  }
  const uint64_t kstar = s_prefix;
  // among key == kstar, the (s_rank)-th smallest index: 4 passes over idx
  __shared__ uint32_t s_ipre;
  if (threadIdx.x == 0) s_ipre = 0;
  __syncthreads();
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t him = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const uint32_t pre = s_ipre;
    for (int64_t i = threadIdx.x; i < b; i += blockDim.x) {
      if (__ldg(keys + i) != kstar) continue;
      uint32_t id = (uint32_t)__ldg(lst + i);
      if (((id ^ pre) & him) == 0) atomicAdd(&hist[(id >> shift) & 255], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t rr = s_rank;
      int bin = 0;
      for (; bin < 256; ++bin) {
        if (rr < (int64_t)hist[bin]) break;
        rr -= hist[bin];
      }
      s_ipre = pre | ((uint32_t)bin << shift);
      s_rank = rr;
    }
    __syncthreads();
  }
  const uint32_t istar = s_ipre;
  for (int64_t i = threadIdx.x; i < b; i += blockDim.x) {
    const uint64_t k = __ldg(keys + i);
    const uint32_t id = (uint32_t)__ldg(lst + i);
    if (k < kstar || (k == kstar && id <= istar)) mask[id] = 1;
  }
}

// ---------------------------------------------------------------- compaction

constexpr int kCompactItems = 4096;  // mask bytes per block

__device__ __forceinline__ void compact_count_body(const uint8_t* __restrict__ mask, int64_t n,
                                                   unsigned* __restrict__ counts) {
  const int64_t base = (int64_t)blockIdx.x * kCompactItems;
  unsigned c = 0;
  for (int i = threadIdx.x; i < kCompactItems; i += blockDim.x) {
    int64_t g = base + i;
    c += (g < n && __ldg(mask + g)) ? 1u : 0u;
  }
  c = warp_sum(c);
  __shared__ unsigned s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    counts[blockIdx.x] = t;
  }
}

__global__ void compact_count_kernel(const uint8_t* __restrict__ mask, int64_t n, unsigned* __restrict__ counts) {
  compact_count_body(mask, n, counts);
}

// single block: exclusive scan of counts -> offsets; total -> *nsel
__device__ __forceinline__ void compact_scan_body(const unsigned* __restrict__ counts, int64_t nblocks,
                                                  int64_t* __restrict__ offsets, int64_t* __restrict__ nsel) {
  __shared__ int64_t carry;
  __shared__ int64_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t base = 0; base < nblocks; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nblocks ? (int64_t)counts[i] : 0;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int64_t s = lane < nw ? wsum[lane] : 0;
      int64_t si = s;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += t;
      }
      if (lane < nw) wsum[lane] = si - s;
    }
    __syncthreads();
    if (i < nblocks) offsets[i] = carry + wsum[w] + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += wsum[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *nsel = carry;
}

__global__ void compact_scan_kernel(const unsigned* __restrict__ counts, int64_t nblocks, int64_t* __restrict__ offsets,
                                    int64_t* __restrict__ nsel) {
  compact_scan_body(counts, nblocks, offsets, nsel);
}

__device__ __forceinline__ void compact_write_body(const uint8_t* __restrict__ mask, int64_t n,
                                                   const int64_t* __restrict__ offsets, int32_t* __restrict__ idx) {
  // blockDim = 1024; each thread handles 4 consecutive bytes
  __shared__ unsigned wsum[32];
  const int64_t base = (int64_t)blockIdx.x * kCompactItems + threadIdx.x * 4;
  unsigned f[4], c = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int64_t g = base + j;
    f[j] = (g < n && __ldg(mask + g)) ? 1u : 0u;
    c += f[j];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned s = wsum[lane], si = s;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    wsum[lane] = si - s;
  }
  __syncthreads();
  int64_t pos = offsets[blockIdx.x] + wsum[w] + incl - c;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (f[j]) idx[pos++] = (int32_t)(base + j);
}

__global__ void compact_write_kernel(const uint8_t* __restrict__ mask, int64_t n, const int64_t* __restrict__ offsets,
                                     int32_t* __restrict__ idx) {
  compact_write_body(mask, n, offsets, idx);
}

__device__ __forceinline__ void gather_rows_body(const float* __restrict__ X, int D, const int32_t* __restrict__ idx,
                                                 const int64_t* __restrict__ n_dev, float* __restrict__ out) {
  const int64_t n = *n_dev;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (D % 4) == 0 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (vec) {
    // 16-byte moves, four rows' loads in flight per warp
    const int D4 = D >> 2;
    const float4* X4 = reinterpret_cast<const float4*>(X);
    float4* out4 = reinterpret_cast<float4*>(out);
    for (int64_t r0 = warp * 4; r0 < n; r0 += nw * 4) {
      int64_t src[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) src[u] = r0 + u < n ? (int64_t)__ldg(idx + r0 + u) * D4 : -1;
      for (int k = lane; k < D4; k += 32) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (src[u] >= 0) v[u] = __ldg(X4 + src[u] + k);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (src[u] >= 0) out4[(r0 + u) * D4 + k] = v[u];
      }
    }
    return;
  }
  for (int64_t r = warp; r < n; r += nw) {
    const float* src = X + (int64_t)__ldg(idx + r) * D;
    float* dst = out + r * D;
    for (int k = lane; k < D; k += 32) dst[k] = __ldg(src + k);
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int D, const int32_t* __restrict__ idx,
                                   const int64_t* __restrict__ n_dev, float* __restrict__ out) {
  gather_rows_body(X, D, idx, n_dev, out);
}

// The gather with max |x - center| over the moved values (FP32, the values
// the rounded copies are made from) and the non-finite check, four rows in
// flight per warp as above.
__global__ void gather_rows_center_kernel(const float* __restrict__ X, int D, const int32_t* __restrict__ idx,
                                          const int64_t* __restrict__ n_dev, float* __restrict__ out,
                                          const float* __restrict__ center, float* __restrict__ maxabs,
                                          int* __restrict__ status) {
  const int64_t n = *n_dev;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float m = 0.f;
  bool bad = false;
  const bool vec = (D % 4) == 0 &&
                   ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(out) |
                     reinterpret_cast<uintptr_t>(center)) & 15) == 0;
  if (vec) {
    const int D4 = D >> 2;
    const float4* X4 = reinterpret_cast<const float4*>(X);
    const float4* C4 = reinterpret_cast<const float4*>(center);
    float4* out4 = reinterpret_cast<float4*>(out);
    for (int64_t r0 = warp * 4; r0 < n; r0 += nw * 4) {
      int64_t src[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) src[u] = r0 + u < n ? (int64_t)__ldg(idx + r0 + u) * D4 : -1;
      for (int k = lane; k < D4; k += 32) {
        const float4 c = __ldg(C4 + k);
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (src[u] >= 0) v[u] = __ldg(X4 + src[u] + k);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (src[u] >= 0) {
            out4[(r0 + u) * D4 + k] = v[u];
            bad |= !isfinite(v[u].x) || !isfinite(v[u].y) || !isfinite(v[u].z) || !isfinite(v[u].w);
            m = fmaxf(m, fmaxf(fmaxf(fabsf(v[u].x - c.x), fabsf(v[u].y - c.y)),
                               fmaxf(fabsf(v[u].z - c.z), fabsf(v[u].w - c.w))));
          }
      }
    }
  } else {
    for (int64_t r = warp; r < n; r += nw) {
      const float* src = X + (int64_t)__ldg(idx + r) * D;
      float* dst = out + r * D;
      for (int k = lane; k < D; k += 32) {
        const float v = __ldg(src + k);
        dst[k] = v;
        bad |= !isfinite(v);
        m = fmaxf(m, fabsf(v - center[k]));
      }
    }
  }
  m = warp_max(m);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(status, (int)PROHD_ENONFINITE);
  if (lane == 0) atomic_max_nonneg(maxabs, m);
}

// Batched compaction and gather: segment blockIdx.y = 2 * pair + set.
struct SegView {
  const uint8_t* mask;
  int64_t n;
  unsigned* counts;
  int64_t* offsets;
  int nblk;
  int32_t* idx;
  int64_t* nsel;
  const float* X;
  float* sub;
};
__device__ __forceinline__ SegView seg_view(const BPair& q, int set) {
  SegView v;
  v.mask = set ? q.maskB : q.maskA;
  v.n = set ? q.nB : q.nA;
  v.counts = q.counts + (set ? q.nblkA : 0);
  v.offsets = q.offsets + (set ? q.nblkA : 0);
  v.nblk = set ? q.nblkB : q.nblkA;
  v.idx = set ? q.idxB : q.idxA;
  v.nsel = q.nsel + set;
  v.X = set ? q.B : q.A;
  v.sub = set ? q.Bs : q.As;
  return v;
}
__global__ void compact_count_batched_kernel(const BPair* __restrict__ P) {
  const SegView v = seg_view(P[blockIdx.y >> 1], blockIdx.y & 1);
  if ((int)blockIdx.x < v.nblk) compact_count_body(v.mask, v.n, v.counts);
}
__global__ void compact_scan_batched_kernel(const BPair* __restrict__ P) {
  const SegView v = seg_view(P[blockIdx.x >> 1], blockIdx.x & 1);
  compact_scan_body(v.counts, v.nblk, v.offsets, v.nsel);
}
__global__ void compact_write_batched_kernel(const BPair* __restrict__ P) {
  const SegView v = seg_view(P[blockIdx.y >> 1], blockIdx.y & 1);
  if ((int)blockIdx.x < v.nblk) compact_write_body(v.mask, v.n, v.offsets, v.idx);
}
__global__ void gather_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y >> 1];
  const SegView v = seg_view(q, blockIdx.y & 1);
  gather_rows_body(v.X, q.D, v.idx, v.nsel, v.sub);
}

// ---------------------------------------------------------------- host side

struct SelBufs {
  float *qA = nullptr, *qB = nullptr;
  float* maxnorm = nullptr;  // [2]
  SelProb* P = nullptr;
  unsigned* hist = nullptr;
  unsigned* hist1 = nullptr;  // second-digit histograms (one pair)
  int32_t* band = nullptr;
  uint64_t* bandkey = nullptr;
  uint8_t *maskA = nullptr, *maskB = nullptr;
  unsigned* counts = nullptr;
  int64_t* offsets = nullptr;
  int64_t cap = 0;
};

static void sel_layout(Arena& ws, int64_t nA, int64_t nB, int D, int nd, SelBufs& b) {
  (void)D;
  b.cap = std::max(nA, nB);
  b.qA = ws.take<float>((size_t)nd * nA);
  b.qB = ws.take<float>((size_t)nd * nB);
  b.maxnorm = ws.take<float>(2);
  b.P = ws.take<SelProb>((size_t)2 * nd);
  b.hist = ws.take<unsigned>((size_t)2 * nd * 512);
  b.hist1 = ws.take<unsigned>((size_t)2 * nd * kHist1Blocks * 2 * kHist1Bins);
  b.band = ws.take<int32_t>((size_t)2 * nd * 2 * b.cap);
  b.bandkey = ws.take<uint64_t>((size_t)2 * nd * 2 * b.cap);
  b.maskA = ws.take<uint8_t>((size_t)nA);
  b.maskB = ws.take<uint8_t>((size_t)nB);
  const int64_t nblk = ceil_div(std::max(nA, nB), kCompactItems);
  b.counts = ws.take<unsigned>((size_t)nblk);
  b.offsets = ws.take<int64_t>((size_t)nblk);
}

void select_layout(Arena& ws, int64_t nA, int64_t nB, int D, int ndirs) {
  SelBufs b;
  sel_layout(ws, nA, nB, D, ndirs, b);
}

// hist0[d][b]: keys of direction d whose top byte is b, one 256-bin
// histogram per direction (fallback path for the CUDA-core projection).
__global__ void top_byte_hist_kernel(const float* __restrict__ q, int64_t n, unsigned* __restrict__ hist0) {
  __shared__ unsigned h[256];
  const int d = blockIdx.y;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const float* qd = q + (size_t)d * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[f32_key(__ldg(qd + i)) >> 24], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(hist0 + (size_t)d * 256 + i, h[i]);
}

static cudaError_t launch_proj(const float* X, int64_t n, int D, const double* dirs, int nd, float* q, float* maxnorm,
                               int* status, int num_sms, cudaStream_t st, unsigned* hist0) {
  const bool fast = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && nd <= 32;
  if (!fast) {
    count_launch();
    proj_simple_kernel<<<num_sms * 8, 256, 0, st>>>(X, n, D, dirs, nd, q, maxnorm, status);
    if (hist0) {
      const unsigned chunks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256 * 16), 4 * num_sms));
      count_launch();
      top_byte_hist_kernel<<<dim3(chunks, nd), 256, 0, st>>>(q, n, hist0);
    }
    return cudaGetLastError();
  }
  const int Dq = (int)round_up(D, kProjK);
  auto go = [&](auto kern, int ND) -> cudaError_t {
    size_t smem = (size_t)ND * Dq * 4 + (size_t)2 * kProjRows * kProjStride * 4 + (size_t)ND * 256 * 4;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kProjThreads, smem);
    int64_t ntiles = ceil_div(n, kProjRows);
    int grid = (int)std::min<int64_t>(ntiles, (int64_t)std::max(1, per_sm) * num_sms);
    count_launch();
    kern<<<grid, kProjThreads, smem, st>>>(X, n, D, dirs, nd, q, maxnorm, status, hist0);
    return cudaGetLastError();
  };
  if (nd <= 3) return go(proj_kernel<3>, 3);
  if (nd <= 5) return go(proj_kernel<5>, 5);
  if (nd <= 9) return go(proj_kernel<9>, 9);
  if (nd <= 13) return go(proj_kernel<13>, 13);
  if (nd <= 17) return go(proj_kernel<17>, 17);
  if (nd <= 24) return go(proj_kernel<24>, 24);
  return go(proj_kernel<32>, 32);
}

// Both sets' projections in one TMA-fed launch; returns false (nothing
// launched) where it does not apply: D % 4 != 0, a base that is not 16-byte
// aligned, more than 17 directions, fewer than two stages fitting in shared
// memory, or no tensor-map encoder. More than 17 directions go to the
// two-launch path (the per-thread accumulators would spill).
static bool launch_proj_pair(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                             const double* dirs, int nd, float* qA, float* qB, float* maxnorm, int* status,
                             unsigned* hist, int64_t timeout_ns, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (D % 4 != 0 || nd > 17 || ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) != 0)
    return false;
  const int ND = nd <= 3 ? 3 : nd <= 5 ? 5 : nd <= 9 ? 9 : nd <= 13 ? 13 : 17;
  const int Dq = (int)round_up(D, 32);
  const size_t fixed = 1024 + (size_t)ND * Dq * 4 + (size_t)2 * ND * 256 * 4 + 2 * kPtMaxStages * 8 + 16;
  const size_t cap = 227 * 1024;
  if (fixed + 2 * (size_t)kPtStageBytes > cap) return false;
  const int stages = (int)std::min<size_t>(kPtMaxStages, (cap - fixed) / kPtStageBytes);
  CUtensorMap tA, tB;
  if (!encode_2d(ctx, &tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)D, (uint64_t)nA, (uint64_t)D * 4, 32, kPtBox,
                 CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_2d(ctx, &tB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B, (uint64_t)D, (uint64_t)nB, (uint64_t)D * 4, 32, kPtBox,
                 CU_TENSOR_MAP_SWIZZLE_128B))
    return false;
  ProjPairArgs a;
  a.nA = nA;
  a.nB = nB;
  a.tilesA = ceil_div(nA, kPtRows);
  a.tiles = a.tilesA + ceil_div(nB, kPtRows);
  a.D = D;
  a.Dq = Dq;
  a.nd = nd;
  a.nchunks = Dq / 32;
  a.stages = stages;
  a.dirs = dirs;
  a.qA = qA;
  a.qB = qB;
  a.maxnorm = maxnorm;
  a.status = status;
  a.hist = hist;
  a.timeout_ns = timeout_ns > 0 ? timeout_ns : kDefaultTimeoutNs;
  const size_t smem = fixed + (size_t)stages * kPtStageBytes;
  const int grid = (int)std::min<int64_t>(a.tiles, ctx->num_sms);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    kern<<<grid, kPtThreads + 32, smem, st>>>(tA, tB, a);
    *err = cudaGetLastError();
  };
  switch (ND) {
    case 3: go(proj_pair_tma_kernel<3>); break;
    case 5: go(proj_pair_tma_kernel<5>); break;
    case 9: go(proj_pair_tma_kernel<9>); break;
    case 13: go(proj_pair_tma_kernel<13>); break;
    default: go(proj_pair_tma_kernel<17>); break;
  }
  return true;
}

int64_t compact_blocks(int64_t n) { return ceil_div(n, kCompactItems); }

cudaError_t mask_to_indices(const uint8_t* mask, int64_t n, int32_t* idx, int64_t* nsel, unsigned* counts,
                            int64_t* offsets, cudaStream_t st) {
  const int64_t nblk = ceil_div(n, kCompactItems);
  count_launch();
  compact_count_kernel<<<(unsigned)nblk, 256, 0, st>>>(mask, n, counts);
  count_launch();
  compact_scan_kernel<<<1, 1024, 0, st>>>(counts, nblk, offsets, nsel);
  count_launch();
  compact_write_kernel<<<(unsigned)nblk, 1024, 0, st>>>(mask, n, offsets, idx);
  return cudaGetLastError();
}

cudaError_t select_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                       const double* dirs, int nd, const int64_t* kA, const int64_t* kB, int32_t* idxA,
                       int64_t* nselA, int32_t* idxB, int64_t* nselB, int* status_dev, Arena& ws, cudaStream_t st,
                       int64_t timeout_ns) {
  SelBufs b;
  sel_layout(ws, nA, nB, D, nd, b);
  if (ws.overflow()) return cudaErrorMemoryAllocation;
  const int nsm = ctx->num_sms;
  cudaError_t e;
  if (nd > kMaxDirs) return cudaErrorInvalidValue;
  KList kl;
  for (int d = 0; d < nd; ++d) {
    kl.k[d] = kA[d];
    kl.k[nd + d] = kB[d];
  }
  cudaMemsetAsync(b.maxnorm, 0, 2 * sizeof(float), st);
  cudaMemsetAsync(b.hist, 0, sizeof(unsigned) * 2 * nd * 256, st);
  cudaMemsetAsync(b.maskA, 0, (size_t)nA, st);
  cudaMemsetAsync(b.maskB, 0, (size_t)nB, st);
  {
    PhaseTimer pt(ctx, PROHD_PH_PROJECT, st);
    if (launch_proj_pair(ctx, A, nA, B, nB, D, dirs, nd, b.qA, b.qB, b.maxnorm, status_dev, b.hist, timeout_ns, st,
                         &e)) {
      if (e) return e;
    } else {
      if ((e = launch_proj(A, nA, D, dirs, nd, b.qA, b.maxnorm + 0, status_dev, nsm, st, b.hist))) return e;
      if ((e = launch_proj(B, nB, D, dirs, nd, b.qB, b.maxnorm + 1, status_dev, nsm, st, b.hist + (size_t)nd * 256)))
        return e;
    }
  }
  PhaseTimer pt_sel(ctx, PROHD_PH_SELECT, st);
  count_launch();
  sel_init_pick_kernel<<<2 * nd, 256, 0, st>>>(b.P, nd, kl, A, b.qA, nA, b.maskA, B, b.qB, nB, b.maskB, D, dirs,
                                               b.maxnorm, b.band, b.bandkey, b.cap, b.hist);
  count_launch();
  hist1_kernel<<<dim3(kHist1Blocks, 2 * nd), 512, 0, st>>>(b.P, b.hist1);
  count_launch();
  pick1_kernel<<<4 * nd, 256, 0, st>>>(b.P, b.hist1);
  {
    // one wave: 4 blocks of 256 threads per SM (the register limit) over all 2 nd problems
    const int64_t nmax = std::max(nA, nB);
    const unsigned chunks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nmax, 256 * 8), (nsm * 4) / (2 * nd)));
    count_launch();
    extract_kernel<<<dim3(chunks, 2 * nd), 256, 0, st>>>(b.P);
  }
  count_launch();
  cand_select_kernel<<<4 * nd, kCandThreads, 0, st>>>(b.P);
  // one warp per block: a large band's FP64 chains spread over many SMs
  // (each SM's FP64 units are few)
  count_launch();
  band_keys_kernel<<<dim3(64, 4 * nd), 32, 0, st>>>(b.P);
  count_launch();
  band_resolve_kernel<<<4 * nd, 512, 0, st>>>(b.P);
  if ((e = cudaGetLastError())) return e;
  if ((e = mask_to_indices(b.maskA, nA, idxA, nselA, b.counts, b.offsets, st))) return e;
  if ((e = mask_to_indices(b.maskB, nB, idxB, nselB, b.counts, b.offsets, st))) return e;
  return cudaGetLastError();
}

cudaError_t gather_rows(const float* X, int D, const int32_t* idx, const int64_t* n_dev, int64_t n_max, float* out,
                        int num_sms, cudaStream_t st) {
  (void)n_max;
  count_launch();
  gather_rows_kernel<<<num_sms * 8, 256, 0, st>>>(X, D, idx, n_dev, out);
  return cudaGetLastError();
}

cudaError_t gather_rows_center(const float* X, int D, const int32_t* idx, const int64_t* n_dev, int64_t n_max,
                               float* out, const float* center, float* maxabs, int* status, int num_sms,
                               cudaStream_t st) {
  (void)n_max;
  count_launch();
  gather_rows_center_kernel<<<num_sms * 8, 256, 0, st>>>(X, D, idx, n_dev, out, center, maxabs, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched pairs

size_t sel_prob_bytes() { return sizeof(SelProb); }

void sel_prob_fill(void* dst, const float* q, int64_t n, const float* X, const double* u, uint8_t* mask,
                   const float* maxnorm, int D, int32_t* band0, int32_t* band1, uint64_t* key0, uint64_t* key1) {
  SelProb s;
  memset(&s, 0, sizeof s);
  s.q = q;
  s.n = n;
  s.X = X;
  s.u = u;
  s.mask = mask;
  s.maxnorm = maxnorm;
  s.D = D;
  s.band[0] = band0;
  s.band[1] = band1;
  s.bkey[0] = key0;
  s.bkey[1] = key1;
  memcpy(dst, &s, sizeof s);
}

cudaError_t proj_batched(const BPair* P, const ProjItem* items, int nitems, int ndmax, int* batch_status,
                         cudaStream_t st) {
  (void)batch_status;
  if (nitems == 0) return cudaSuccess;
  const int Dq = 256;  // smem sized for the largest D of a batch (D <= 256)
  auto go = [&](auto kern, int ND) -> cudaError_t {
    const size_t smem = (size_t)ND * Dq * 4 + (size_t)2 * kProjRows * kProjStride * 4;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r) return r;
    count_launch();
    kern<<<nitems, kProjThreads, smem, st>>>(P, items);
    return cudaGetLastError();
  };
  if (ndmax <= 3) return go(proj_items_kernel<3>, 3);
  if (ndmax <= 5) return go(proj_items_kernel<5>, 5);
  if (ndmax <= 9) return go(proj_items_kernel<9>, 9);
  if (ndmax <= 13) return go(proj_items_kernel<13>, 13);
  if (ndmax <= 17) return go(proj_items_kernel<17>, 17);
  if (ndmax <= 24) return go(proj_items_kernel<24>, 24);
  return go(proj_items_kernel<32>, 32);
}

// Radix select and band resolution of every (pair, set, direction) problem
// of the batch at once. `chunk` keys per block of the histogram and band
// passes (the grid's x extent covers the largest set).
cudaError_t select_batched(SelProb* probs, int nprob, const double* alpha_of, unsigned* hist, int64_t nmax, int chunk,
                           cudaStream_t st) {
  if (nprob > 32767) return cudaErrorInvalidValue;
  cudaMemsetAsync(hist, 0, sizeof(unsigned) * (size_t)nprob * 512, st);
  count_launch();
  sel_reset_batched_kernel<<<(nprob + 127) / 128, 128, 0, st>>>(probs, nprob, alpha_of);
  const unsigned chunks = (unsigned)std::max<int64_t>(1, ceil_div(nmax, std::max(chunk, 256)));
  dim3 g(chunks, nprob);
  for (int pass = 0; pass < 4; ++pass) {
    count_launch();
    radix_hist_kernel<<<g, 256, 0, st>>>(probs, pass, hist, 0);
    count_launch();
    radix_pick_kernel<<<(2 * nprob * 32 + 127) / 128, 128, 0, st>>>(probs, nprob, pass, hist, 0);
  }
  count_launch();
  band_kernel<<<g, 256, 0, st>>>(probs, 0);
  count_launch();
  band_keys_kernel<<<dim3(1, 2 * nprob), 256, 0, st>>>(probs);
  count_launch();
  band_resolve_kernel<<<2 * nprob, 512, 0, st>>>(probs);
  return cudaGetLastError();
}

cudaError_t compact_gather_batched(const BPair* P, int npairs, int nblk_max, int64_t nmax, cudaStream_t st) {
  (void)nmax;
  count_launch();
  compact_count_batched_kernel<<<dim3(nblk_max, 2 * npairs), 256, 0, st>>>(P);
  count_launch();
  compact_scan_batched_kernel<<<2 * npairs, 1024, 0, st>>>(P);
  count_launch();
  compact_write_batched_kernel<<<dim3(nblk_max, 2 * npairs), 1024, 0, st>>>(P);
  count_launch();
  gather_batched_kernel<<<dim3(16, 2 * npairs), 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace prohd
