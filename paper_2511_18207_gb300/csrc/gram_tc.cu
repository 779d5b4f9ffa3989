// Union Gram G = sum_z (z - s)(z - s)^T and per-set sums of z - s on tcgen05
// tensor cores (Algorithm 2 step 2: principal components of [A; B] need the
// union covariance), for D <= 256.
//
// Each FP32 centred value z is split exactly into three BF16 parts
// z = h + m + l (h = bf16(z), m = bf16(z - h), l = bf16(z - h - m); the
// residual is below 2^-25 |z|), and G is accumulated from the six products
// hh^T + hm^T + mh^T + hl^T + lh^T + mm^T, whose sum differs from zz^T by
// about 2^-24 |z_i z_j| per point. The tensor core accumulates 512 points in
// FP32 in TMEM; each 512-point partial is then added into a per-CTA FP64
// accumulator in global memory (covariance accumulation in FP64 across rows
// and CTAs), and a final kernel sums the CTAs in a fixed order.
//
// The input is row-major [points, D], i.e. the Gram's M/N index (the
// dimension) is the contiguous one. Converter warps therefore transpose while
// they split: they read 8 points x (32 lanes x T dims) with coalesced loads
// and write each dimension's 8 consecutive points as one 16-byte chunk of a
// K-major, 128B-swizzled BF16 tile [dims x 64 points] (the layout the
// distance contraction also feeds to tcgen05.mma).
//
// Work split: CTAs of type 0 own output rows 0..127 against all Dp columns,
// type 1 (when Dp > 128) rows 128..Dp-1 against columns 128..Dp-1; each type
// covers all points, with CTA counts in proportion to their work per point.
// Warps: 0..7 converters, 8 MMA issuer (and TMEM owner), 9..12 epilogue.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kGcPts = 64;          // points per chunk (one 128-byte K row of BF16)
constexpr int kGcConv = 8;          // converter warps, 8 points each
constexpr int kGcEpi = 4;
constexpr int kGcThreads = (kGcConv + 1 + kGcEpi) * 32;
constexpr int kGcFlush = 8;         // chunks per FP32 accumulation in TMEM (512 points)
constexpr int kGcMaxRows = 256;

// Kahan-compensated s += (z + e) with compensation c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float z, float e) {
  const float y = (z - c) + e;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

struct GcSmem {
  uint64_t full[2], empty[2], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_base;
  int abort;
};

__host__ __device__ constexpr size_t gc_tile_bytes(int rows) { return (size_t)rows * 128; }
__host__ __device__ constexpr size_t gc_smem_bytes(int rows) {
  return 1024 + 2 * 3 * gc_tile_bytes(rows) + sizeof(GcSmem);
}

struct GcParams {
  const float* A;
  const float* B;
  int64_t nA, nB;
  int D, Dp;
  const float* s32;   // pilot shift [D]
  int nc0;            // CTAs of type 0 (the rest are type 1)
  int rows0, rows1;   // tile rows loaded by each type (>= 128)
  int N0, N1;         // output columns of each type
  double* gacc;       // [gridDim][256 x 128] FP64 partials, element (col, row) at col*128 + row
  double* sums;       // [nc0][kGcConv][2][Dp] FP64 per-warp set sums of z - s
  int* status;
  uint64_t timeout_ns;
};

// 13 warps: one SMSP holds 4 of them, so 16384 / (4 x 32) = 128 registers per thread at most.
__global__ void __maxnreg__(128) gram_tc_kernel(const GcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const bool type0 = (int)blockIdx.x < p.nc0;
  const int rows = type0 ? p.rows0 : p.rows1;     // tile rows (dims loaded, zero padded)
  const int N = type0 ? p.N0 : p.N1;
  const int dim0 = type0 ? 0 : 128;               // first dimension loaded
  const size_t tb = gc_tile_bytes(rows);
  uint8_t* tiles = base;                           // [2][3][rows x 128 B]
  GcSmem& S = *reinterpret_cast<GcSmem*>(base + 2 * 3 * tb);
  volatile int* abort = &S.abort;

  const int64_t Ntot = p.nA + p.nB;
  const int nct = type0 ? p.nc0 : (int)gridDim.x - p.nc0;
  const int ci = type0 ? (int)blockIdx.x : (int)blockIdx.x - p.nc0;
  const int64_t p0 = Ntot * ci / nct, p1 = Ntot * (ci + 1) / nct;
  const int nchunks = (int)((p1 - p0 + kGcPts - 1) / kGcPts);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.full[s], kGcConv);
      mbar_init(&S.empty[s], 1);
      mbar_init(&S.acc_full[s], 1);
      mbar_init(&S.acc_empty[s], kGcEpi);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == kGcConv) {
    tc_alloc(&S.tmem_base, 512);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp < kGcConv) {
    // ---------------- converters: load, centre, split, transpose ----------------
    const int T = rows / 32;  // dims per lane: dim = dim0 + lane + 32 t
    float sA[8], cA[8], sB[8], cB[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) sA[t] = cA[t] = sB[t] = cB[t] = 0.f;
    float shift[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int d = dim0 + lane + 32 * t;
      shift[t] = (t < T && d < p.D) ? p.s32[d] : 0.f;
    }
    bool bad = false;
    uint32_t ph = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int s = c & 1;
      int got = 1;
      if (lane == 0) got = mbar_wait_bounded(&S.empty[s], ph ^ 1, abort, p.timeout_ns) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (!got) break;
      const int64_t pt0 = p0 + (int64_t)c * kGcPts + warp * 8;
      const float* zrow[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int64_t pt = pt0 + i;
        zrow[i] = nullptr;
        if (pt < p1) zrow[i] = pt < p.nA ? p.A + pt * p.D : p.B + (pt - p.nA) * p.D;
      }
      uint8_t* tH = tiles + (size_t)(s * 3 + 0) * tb;
      uint8_t* tM = tiles + (size_t)(s * 3 + 1) * tb;
      uint8_t* tL = tiles + (size_t)(s * 3 + 2) * tb;
      // two halves of at most 4 dims per lane keep the staging in registers
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (half * 4 >= T) break;
        float x[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = half * 4 + u;
            const int d = dim0 + lane + 32 * t;
            x[i][u] = (zrow[i] && t < T && d < p.D) ? __ldg(zrow[i] + d) : 0.f;
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = half * 4 + u;
          if (t >= T) break;
          const int d = dim0 + lane + 32 * t;
          const bool vd = d < p.D;
          uint32_t hv[4], mv[4], lv[4];
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            float h2[2], m2[2], l2[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int64_t pt = pt0 + i + j;
              const bool v = vd && pt < p1;
              const float xv = x[i + j][u];
              const float z = v ? xv - shift[t] : 0.f;
              bad |= v && !isfinite(xv);
              const __nv_bfloat16 h = __float2bfloat16_rn(z);
              const float r1 = z - __bfloat162float(h);
              const __nv_bfloat16 m = __float2bfloat16_rn(r1);
              const float r2 = r1 - __bfloat162float(m);
              h2[j] = __bfloat162float(h);
              m2[j] = __bfloat162float(m);
              l2[j] = r2;
              if (type0 && v) {
                // exact error of the centring (two-sum), folded into Kahan sums of z + e
                const float bb = z - xv;
                const float e = (xv - (z - bb)) + (-shift[t] - bb);
                if (pt < p.nA) kahan_add(sA[t], cA[t], z, e);
                else kahan_add(sB[t], cB[t], z, e);
              }
            }
            __nv_bfloat162 hh = __floats2bfloat162_rn(h2[0], h2[1]);
            __nv_bfloat162 mm = __floats2bfloat162_rn(m2[0], m2[1]);
            __nv_bfloat162 ll = __floats2bfloat162_rn(l2[0], l2[1]);
            hv[i / 2] = *reinterpret_cast<uint32_t*>(&hh);
            mv[i / 2] = *reinterpret_cast<uint32_t*>(&mm);
            lv[i / 2] = *reinterpret_cast<uint32_t*>(&ll);
          }
          const int row = lane + 32 * t;
          const size_t off = (size_t)row * 128 + (size_t)((warp ^ (row & 7)) * 16);
          *reinterpret_cast<uint4*>(tH + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<uint4*>(tM + off) = make_uint4(mv[0], mv[1], mv[2], mv[3]);
          *reinterpret_cast<uint4*>(tL + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.full[s]);
      if (s == 1) ph ^= 1;
    }
    if (type0) {
      double* out = p.sums + ((size_t)blockIdx.x * kGcConv + warp) * 2 * p.Dp;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int d = lane + 32 * t;
        if (t < T && d < p.Dp) {
          out[d] = (double)sA[t] - (double)cA[t];
          out[p.Dp + d] = (double)sB[t] - (double)cB[t];
        }
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(p.status, (int)PROHD_ENONFINITE);
  } else if (warp == kGcConv) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(1, 128, N);
      // products (A part, B part): hh, hm, mh, hl, lh, mm
      const int pa[6] = {0, 0, 1, 0, 2, 1};
      const int pb[6] = {0, 1, 0, 2, 0, 1};
      uint32_t ph = 0, ab = 0, aph = 0;
      bool ok = true;
      int in_acc = 0;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int s = c & 1;
        if (in_acc == 0) {
          if (!mbar_wait_bounded(&S.acc_empty[ab], aph ^ 1, abort, p.timeout_ns)) { ok = false; break; }
          tc_fence_after();
        }
        if (!mbar_wait_bounded(&S.full[s], ph, abort, p.timeout_ns)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem + ab * 256;
        const uint32_t t0 = smem_u32(tiles + (size_t)(s * 3) * tb);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint32_t a_addr = t0 + (uint32_t)(pa[q] * tb);
          const uint32_t b_addr = t0 + (uint32_t)(pb[q] * tb);
#pragma unroll
          for (int k = 0; k < kGcPts / 16; ++k)
            tc_mma_f16(d_tmem, smem_desc_sw128(a_addr + k * 32), smem_desc_sw128(b_addr + k * 32), idesc,
                       (in_acc | q | k) != 0);
        }
        tc_commit(&S.empty[s]);
        if (s == 1) ph ^= 1;
        if (++in_acc == kGcFlush || c == nchunks - 1) {
          tc_commit(&S.acc_full[ab]);
          in_acc = 0;
          ab ^= 1;
          if (ab == 0) aph ^= 1;
        }
      }
      tc_commit(&S.drain);
      const uint64_t t0 = global_timer_ns();
      while (!mbar_try_wait(&S.drain, 0) && global_timer_ns() - t0 < 1000000000ull) {
      }
    }
  } else {
    // ---------------- epilogue: FP32 TMEM partials -> FP64 accumulators ----------------
    const int q = warp & 3;
    const int row = q * 32 + lane;  // output row within this type's 128 rows
    double* g = p.gacc + (size_t)blockIdx.x * (256 * 128);
    const int nflush = (nchunks + kGcFlush - 1) / kGcFlush;
    uint32_t ab = 0, aph = 0;
    bool ok = true;
    for (int f = 0; f < nflush; ++f) {
      int got = 0;
      if (ok && lane == 0) got = mbar_wait_bounded(&S.acc_full[ab], aph, abort, p.timeout_ns) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      ok = ok && got;
      if (!ok) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + ab * 256;
      for (int cc = 0; cc < N / 32; ++cc) {
        float v[32];
        __syncwarp();
        tc_ld_32x32b_x32(taddr + cc * 32, v);
        tc_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          double* dst = g + (size_t)(cc * 32 + c) * 128 + row;
          *dst = (f == 0 ? 0.0 : *dst) + (double)v[c];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.acc_empty[ab]);
      ab ^= 1;
      if (ab == 0) aph ^= 1;
    }
    if (nflush == 0)
      for (int col = 0; col < N; ++col) g[(size_t)col * 128 + row] = 0.0;
  }

  __syncthreads();
  if (threadIdx.x == 0 && S.abort) atomicMax(p.status, (int)PROHD_ETIMEOUT);
  if (warp == kGcConv) {
    __syncwarp();
    tc_fence_after();
    tc_dealloc(tmem, 512);
  }
}

// G (upper triangle, FP64, row-major D x D) and the set sums, summed over the
// CTAs of each type in a fixed order.
__global__ void gram_tc_reduce_kernel(const GcParams p, int ncta, double* __restrict__ G, double* __restrict__ sumA,
                                      double* __restrict__ sumB) {
  const int D = p.D;
  const int64_t DD = (int64_t)D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < DD + 2 * D;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < DD) {
      const int i = (int)(e / D), j = (int)(e % D);
      if (j < i) continue;
      int c0, c1, row, col;
      if (i < 128) {
        c0 = 0; c1 = p.nc0; row = i; col = j;
      } else {
        c0 = p.nc0; c1 = ncta; row = i - 128; col = j - 128;
      }
      double s = 0.0;
      for (int c = c0; c < c1; ++c) s += p.gacc[(size_t)c * (256 * 128) + (size_t)col * 128 + row];
      G[e] = s;
    } else {
      const int64_t k = e - DD;
      const int set = k < D ? 0 : 1;
      const int d = (int)(set ? k - D : k);
      double s = 0.0;
      for (int c = 0; c < p.nc0; ++c)
        for (int w = 0; w < kGcConv; ++w) s += p.sums[((size_t)c * kGcConv + w) * 2 * p.Dp + (size_t)set * p.Dp + d];
      (set ? sumB : sumA)[d] = s;
    }
  }
}

bool gram_tc_supported(int D) { return D >= 1 && D <= kGcMaxRows; }

size_t gram_tc_scratch_doubles(int D, int num_sms) {
  const int Dp = (int)round_up(D, 64);
  return (size_t)num_sms * 256 * 128 + (size_t)num_sms * kGcConv * 2 * Dp;
}

cudaError_t gram_tc_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                        const float* s32, double* scratch, double* G, double* sumA, double* sumB, int* status,
                        int64_t timeout_ns, cudaStream_t st) {
  const int nsm = ctx->num_sms;
  GcParams p;
  p.A = A;
  p.B = B;
  p.nA = nA;
  p.nB = nB;
  p.D = D;
  p.Dp = (int)round_up(D, 64);
  p.s32 = s32;
  p.N0 = p.Dp;
  p.rows0 = std::max(128, p.Dp);
  p.N1 = p.Dp > 128 ? p.Dp - 128 : 0;
  p.rows1 = 128;
  if (p.N1 > 0) {
    // CTA counts in proportion to work per point (output columns)
    p.nc0 = (int)std::lround((double)nsm * p.N0 / (double)(p.N0 + p.N1));
    p.nc0 = std::min(std::max(p.nc0, 1), nsm - 1);
  } else {
    p.nc0 = nsm;
  }
  p.gacc = scratch;
  p.sums = scratch + (size_t)nsm * 256 * 128;
  p.status = status;
  p.timeout_ns = (uint64_t)timeout_ns;
  const size_t smem = gc_smem_bytes(p.rows0);
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  const int grid = p.N1 > 0 ? nsm : p.nc0;
  {
    PhaseTimer pt(ctx, PROHD_PH_GRAM, st);
    count_launch();
    gram_tc_kernel<<<grid, kGcThreads, smem, st>>>(p);
    if ((e = cudaGetLastError())) return e;
  }
  count_launch();
  gram_tc_reduce_kernel<<<nsm, 256, 0, st>>>(p, grid, G, sumA, sumB);
  return cudaGetLastError();
}

}  // namespace prohd
