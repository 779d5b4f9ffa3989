// Union Gram G = sum_z (z - s)(z - s)^T and per-set sums of z - s on tcgen05
// tensor cores (Algorithm 2 step 2: principal components of [A; B] need the
// union covariance), for D <= 256 with D % 4 == 0.
//
// Each FP32 centred value z is split exactly into three BF16 parts
// z = h + m + l (h = bf16(z), m = bf16(z - h), l = bf16(z - h - m); the
// residual is below 2^-25 |z|), and G is accumulated from the six products
// hh^T + hm^T + mh^T + hl^T + lh^T + mm^T, whose sum differs from zz^T by
// about 2^-24 |z_i z_j| per point. The tensor core accumulates 512 points in
// FP32 in TMEM; each 512-point partial is then added into a per-CTA
// Kahan-compensated FP32 accumulator in global memory, and a final kernel
// sums the CTAs in FP64 in a fixed order.
//
// Pipeline per CTA: a TMA warp streams FP32 tiles [64 points x rows dims]
// through a two-stage ring (dims past D arrive as zeros); eight converter
// warps read them from shared memory, centre, split and transpose them into
// one K-major, 128B-swizzled BF16 stage [dims x 64 points] x {h, m, l} (the
// operand layout of the distance contraction); one thread issues the MMAs
// slice by slice (16 points per slice, two converter warps per slice), and
// each slice is handed back to its converters as soon as its MMAs complete,
// so the conversion of the next chunk overlaps the MMAs of this one; four
// epilogue warps move finished 512-point partials from TMEM into the
// compensated accumulators.
//
// Work split: CTAs of type 0 own output rows 0..127 against all Dp columns,
// type 1 (when Dp > 128) rows 128..Dp-1 against columns 128..Dp-1; each type
// covers all points, with CTA counts in proportion to their work per point,
// and every CTA's points lie in one set (A or B).
// Warps: 0..7 converters, 8 MMA issuer (and TMEM owner), 9..12 epilogue,
// 13 TMA producer.
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kGcPts = 64;          // points per chunk (one 128-byte K row of BF16)
constexpr int kGcConv = 8;          // converter warps, 8 points each
constexpr int kGcEpi = 4;
constexpr int kGcMmaWarp = kGcConv;
constexpr int kGcTmaWarp = kGcConv + 1 + kGcEpi;
constexpr int kGcThreads = (kGcTmaWarp + 1) * 32;
constexpr int kGcFlush = 8;         // chunks per FP32 accumulation in TMEM (512 points)
constexpr int kGcMaxRows = 256;

// Packed round-to-nearest conversion of two FP32 values to BF16x2 (a in the
// low half, b in the high half), and the FP32 values of the halves.
__device__ __forceinline__ uint32_t bf16x2_rn(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Kahan-compensated s += x with compensation c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

constexpr int kGcSlices = kGcPts / 16;  // K-steps of one chunk

struct GcSmem {
  uint64_t ffull[2], fempty[2], sfull[kGcSlices], sempty[kGcSlices], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_base;
  int abort;
  int next;  // work item taken by this CTA (batched launches)
};

__host__ __device__ constexpr size_t gc_tile_bytes(int rows) { return (size_t)rows * 128; }
__host__ __device__ constexpr size_t gc_stage_bytes(int rows) { return (size_t)kGcPts * rows * 4; }
__host__ __device__ constexpr size_t gc_smem_bytes(int rows) {
  return 1024 + 3 * gc_tile_bytes(rows) + 2 * gc_stage_bytes(rows) + sizeof(GcSmem);
}

struct GcParams {
  int64_t nA, nB;
  int D, Dp;
  const float* s32;   // pilot shift [D]
  int nc0;            // CTAs of type 0 (the rest are type 1)
  int ncA0, ncA1;     // CTAs of each type that read set A (the rest read B)
  int rows0, rows1;   // tile rows (dims) of each type, 128, 192 or 256; also the FP32 box width
  int N0, N1;         // output columns of each type
  float2* gacc;       // [gridDim][256 x 128] Kahan (sum, compensation) partials, element (col, row) at col*128 + row
  double* sums;       // [gridDim][kGcConv][2][Dp] FP64 per-warp set sums of z - s
  int* status;
  uint64_t timeout_ns;
  // batched launches: CTAs take items from the table through an atomic
  // ticket; nullptr for one pair (CTA i is item i of the static split above)
  const GcItem* items;
  int nitems;
  int* ticket;
};

// Splits two FP32 values exactly enough into BF16 triples (see the file
// comment) and returns the packed pairs (point i in the low half).
__device__ __forceinline__ void gc_split_pair(float z0, float z1, uint32_t& h, uint32_t& m, uint32_t& l) {
  // one packed BF16x2 conversion per split level, unpacked to FP32 by
  // shifts (a BF16 is the top half of an FP32)
  h = bf16x2_rn(z0, z1);
  const float r0 = z0 - bf16_lo(h), r1 = z1 - bf16_hi(h);
  m = bf16x2_rn(r0, r1);
  l = bf16x2_rn(r0 - bf16_lo(m), r1 - bf16_hi(m));
}

// One converter warp's share of a chunk: 8 points x 32T dims from the FP32
// stage (row stride 32T floats) into the three BF16 tiles. `st` points at
// this warp's first point and this lane's dimension, `dst` at this lane's
// 16-byte slot in row `lane` of the h tile (rows lane + 32 t sit 4096 t
// bytes further). Only the first `nv` points are real when !FULL; the rest
// contribute zeros. Dimensions past D were zero-filled by the copy and have
// a zero shift.
template <int T, bool FULL>
__device__ __forceinline__ void gc_convert(const float* __restrict__ st, uint8_t* __restrict__ dst,
                                           const float (&shift)[8], float (&ss)[8], float (&sc)[8], int nv) {
  constexpr int BW = 32 * T;
  constexpr int TB = 4096 * T;  // bytes of one BF16 tile (32T rows x 128 B)
#pragma unroll
  for (int t = 0; t < T; ++t) {
    float z[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float x = st[i * BW + 32 * t];
      z[i] = (FULL || i < nv) ? x - shift[t] : 0.f;
    }
    kahan_add(ss[t], sc[t], ((z[0] + z[1]) + (z[2] + z[3])) + ((z[4] + z[5]) + (z[6] + z[7])));
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) gc_split_pair(z[2 * i], z[2 * i + 1], h[i], m[i], l[i]);
    uint8_t* o = dst + t * 4096;
    *reinterpret_cast<uint4*>(o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(o + TB) = make_uint4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<uint4*>(o + 2 * TB) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// All chunks of one converter warp (slice `warp / 2` of every chunk).
template <int T>
__device__ __forceinline__ bool gc_converter(GcSmem& S, const float* stage, uint8_t* tiles, int warp, int lane,
                                             int nchunks, uint32_t g0, int64_t p0, int64_t p1,
                                             const float (&shift)[8], float (&ss)[8], float (&sc)[8],
                                             uint64_t timeout_ns) {
  constexpr int BW = 32 * T;
  volatile int* abort = &S.abort;
  const int s = warp >> 1;
  const float* st0 = stage + (size_t)(warp * 8) * BW + lane;
  uint8_t* dst = tiles + lane * 128 + ((warp ^ (lane & 7)) * 16);
  for (int c = 0; c < nchunks; ++c) {
    const uint32_t g = g0 + (uint32_t)c;  // ring position over all of this CTA's chunks
    const int f = g & 1;
    int got = 1;
    if (lane == 0) {
      got = mbar_wait_bounded(&S.sempty[s], (g & 1u) ^ 1u, abort, timeout_ns) &&
            mbar_wait_bounded(&S.ffull[f], (g >> 1) & 1u, abort, timeout_ns);
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) return false;
    const float* st = st0 + (size_t)f * kGcPts * BW;
    const int64_t left = p1 - (p0 + (int64_t)c * kGcPts + warp * 8);
    if (left >= 8)
      gc_convert<T, true>(st, dst, shift, ss, sc, 8);
    else
      gc_convert<T, false>(st, dst, shift, ss, sc, left > 0 ? (int)left : 0);
    fence_proxy_async();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&S.fempty[f]);
      mbar_arrive(&S.sfull[s]);
    }
  }
  return true;
}

// 14 warps: one SMSP holds 4 of them, so 16384 / (4 x 32) = 128 registers per thread at most.
__global__ void __maxnreg__(128)
    gram_tc_kernel(const GcParams p, const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmB0,
                   const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmB1) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_align<1024>(smem_raw);
  const bool batched = p.items != nullptr;
  const bool btype0 = (int)blockIdx.x < p.nc0;
  // shared-memory layout for the largest tile this CTA can meet
  const int lrows = batched ? kGcMaxRows : (btype0 ? p.rows0 : p.rows1);
  const size_t ltb = gc_tile_bytes(lrows);
  uint8_t* tiles = base;                                    // [3][rows x 128 B]
  float* stage = reinterpret_cast<float*>(base + 3 * ltb);  // [2][64][rows]
  GcSmem& S = *reinterpret_cast<GcSmem*>(base + 3 * ltb + 2 * gc_stage_bytes(lrows));
  volatile int* abort = &S.abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S.ffull[s], 1);
      mbar_init(&S.fempty[s], kGcConv);
      mbar_init(&S.acc_full[s], 1);
      mbar_init(&S.acc_empty[s], kGcEpi);
    }
    for (int s = 0; s < kGcSlices; ++s) {
      mbar_init(&S.sfull[s], kGcConv / kGcSlices);
      mbar_init(&S.sempty[s], 1);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == kGcMmaWarp) {
    tc_alloc(&S.tmem_base, 512);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  // Ring positions run on over all items of this CTA, so every barrier's
  // phase parity follows from one chunk counter (g0 + c) and one flush
  // counter per consumer.
  uint32_t g0 = 0, armed = 0;
  uint32_t ab = 0, aph = 0;  // TMEM accumulator ring (MMA issuer and epilogue keep their own copies)

  for (int iter = 0;; ++iter) {
    GcItem w;
    if (!batched) {
      if (iter > 0) break;
      // this CTA's set and point range in the static split of one pair
      const int ci = btype0 ? (int)blockIdx.x : (int)blockIdx.x - p.nc0;
      const int nct = btype0 ? p.nc0 : (int)gridDim.x - p.nc0;
      const int ncA = btype0 ? p.ncA0 : p.ncA1;
      const bool setA = ci < ncA;
      const int64_t n = setA ? p.nA : p.nB;
      const int cj = setA ? ci : ci - ncA, ncj = setA ? ncA : nct - ncA;
      w.tm = btype0 ? (setA ? &tmA0 : &tmB0) : (setA ? &tmA1 : &tmB1);
      w.s32 = p.s32;
      w.gacc = p.gacc + (size_t)blockIdx.x * (256 * 128);
      w.sums = p.sums + (size_t)blockIdx.x * kGcConv * 2 * p.Dp;
      w.status = p.status;
      w.p0 = n * cj / ncj;
      w.p1 = n * (cj + 1) / ncj;
      w.D = p.D;
      w.Dp = p.Dp;
      w.type = btype0 ? 0 : 1;
      w.setA = setA ? 1 : 0;
    } else {
      if (threadIdx.x == 0) S.next = atomicAdd(p.ticket, 1);
      __syncthreads();
      const int it = S.next;
      if (it >= p.nitems) break;
      w = p.items[it];
    }
    const bool type0 = w.type == 0;
    const int rows = type0 ? max(128, w.Dp) : 128;  // tile rows (dims loaded, zero padded) = FP32 box width
    const int N = type0 ? w.Dp : w.Dp - 128;
    const int dim0 = type0 ? 0 : 128;                // first dimension loaded
    const size_t tb = gc_tile_bytes(rows);
    const int64_t p0 = w.p0, p1 = w.p1;
    const int nchunks = (int)((p1 - p0 + kGcPts - 1) / kGcPts);
    const bool setA = w.setA != 0;

    if (warp == kGcTmaWarp) {
      // ---------------- TMA producer: FP32 point tiles into the 2-stage ring ----------------
      if (lane == 0) {
        tma_prefetch_desc(w.tm);
        const uint32_t bytes = (uint32_t)gc_stage_bytes(rows);
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t g = g0 + (uint32_t)c;
          const int f = g & 1;
          if (!mbar_wait_bounded(&S.fempty[f], ((g >> 1) & 1u) ^ 1u, abort, p.timeout_ns)) break;
          mbar_arrive_expect_tx(&S.ffull[f], bytes);
          tma_load_2d(stage + (size_t)f * kGcPts * rows, w.tm, dim0, (int)(p0 + (int64_t)c * kGcPts), &S.ffull[f]);
          armed = g + 1;
        }
        if (*abort) {
          // error path: let the copies already issued land before the CTA exits
          for (uint32_t g = armed >= 2 ? armed - 2 : 0; g < armed; ++g) {
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(&S.ffull[g & 1], (g >> 1) & 1u) && global_timer_ns() - t0 < 2000000ull) {
            }
          }
        }
      }
    } else if (warp < kGcConv) {
      // ---------------- converters: centre, split, transpose ----------------
      const int T = rows / 32;  // dims per lane: dim = dim0 + lane + 32 t
      float ss[8], sc[8], shift[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        ss[t] = sc[t] = 0.f;
        const int d = dim0 + lane + 32 * t;
        shift[t] = (t < T && d < w.D) ? w.s32[d] : 0.f;
      }
      if (T == 8)
        gc_converter<8>(S, stage, tiles, warp, lane, nchunks, g0, p0, p1, shift, ss, sc, p.timeout_ns);
      else if (T == 6)
        gc_converter<6>(S, stage, tiles, warp, lane, nchunks, g0, p0, p1, shift, ss, sc, p.timeout_ns);
      else
        gc_converter<4>(S, stage, tiles, warp, lane, nchunks, g0, p0, p1, shift, ss, sc, p.timeout_ns);
      // A non-finite coordinate makes its dimension's running sum non-finite
      // (so does an FP32 overflow of the sum, which would also ruin G).
      bool bad = false;
      double* out = w.sums + (size_t)warp * 2 * w.Dp;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int d = dim0 + lane + 32 * t;
        if (t < T) bad |= !isfinite(ss[t]) || !isfinite(sc[t]);
        if (t < T && d < w.Dp) {
          const double v = type0 ? (double)ss[t] - (double)sc[t] : 0.0;
          out[(setA ? 0 : w.Dp) + d] = v;
          out[(setA ? w.Dp : 0) + d] = 0.0;
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(w.status, (int)PROHD_ENONFINITE);
    } else if (warp == kGcMmaWarp) {
      // ---------------- MMA issuer ----------------
      if (lane == 0) {
        const uint32_t idesc = idesc_f16(1, 128, N);
        // products (A part, B part): hh, hm, mh, hl, lh, mm
        const int pa[6] = {0, 0, 1, 0, 2, 1};
        const int pb[6] = {0, 1, 0, 2, 0, 1};
        int in_acc = 0;
        const uint32_t t0 = smem_u32(tiles);
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t g = g0 + (uint32_t)c;
          if (in_acc == 0) {
            if (!mbar_wait_bounded(&S.acc_empty[ab], aph ^ 1, abort, p.timeout_ns)) break;
            tc_fence_after();
          }
          const uint32_t d_tmem = tmem + ab * 256;
          bool ok = true;
#pragma unroll
          for (int k = 0; k < kGcSlices; ++k) {
            if (!mbar_wait_bounded(&S.sfull[k], g & 1u, abort, p.timeout_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < 6; ++q)
              tc_mma_f16(d_tmem, smem_desc_sw128(t0 + (uint32_t)(pa[q] * tb) + k * 32),
                         smem_desc_sw128(t0 + (uint32_t)(pb[q] * tb) + k * 32), idesc, (in_acc | q | k) != 0);
            tc_commit(&S.sempty[k]);  // slice k may be overwritten once these MMAs complete
          }
          if (!ok) break;
          if (++in_acc == kGcFlush || c == nchunks - 1) {
            tc_commit(&S.acc_full[ab]);
            in_acc = 0;
            ab ^= 1;
            if (ab == 0) aph ^= 1;
          }
        }
      }
    } else {
      // ---------------- epilogue: FP32 TMEM partials -> compensated accumulators ----------------
      const int q = warp & 3;
      const int row = q * 32 + lane;  // output row within this type's 128 rows
      float2* gsl = w.gacc;
      const int nflush = (nchunks + kGcFlush - 1) / kGcFlush;
      bool ok = true;
      for (int fl = 0; fl < nflush; ++fl) {
        int got = 0;
        if (ok && lane == 0) got = mbar_wait_bounded(&S.acc_full[ab], aph, abort, p.timeout_ns) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        ok = ok && got;
        if (!ok) break;
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + ab * 256;
        for (int cc = 0; cc < N / 32; ++cc) {
          // running sums are Kahan-compensated FP32 pairs (sum, compensation):
          // as accurate as FP64 accumulation of the 512-point partials, and
          // FP64 arithmetic is scarce here. Loads are issued before any add.
          float2 acc[32];
          float2* col0 = gsl + (size_t)(cc * 32) * 128 + row;
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[c] = fl == 0 ? make_float2(0.f, 0.f) : __ldcg(col0 + (size_t)c * 128);
          float v[32];
          __syncwarp();
          tc_ld_32x32b_x32(taddr + cc * 32, v);
          tc_wait_ld();
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            kahan_add(acc[c].x, acc[c].y, v[c]);
            __stcg(col0 + (size_t)c * 128, acc[c]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.acc_empty[ab]);
        ab ^= 1;
        if (ab == 0) aph ^= 1;
      }
      if (nflush == 0)
        for (int col = 0; col < N; ++col) gsl[(size_t)col * 128 + row] = make_float2(0.f, 0.f);
    }
    // the item is finished by every role: the rings are idle, so the next
    // item may change the tile geometry
    __syncthreads();
    g0 += (uint32_t)nchunks;
    if (*abort) break;
  }

  if (warp == kGcMmaWarp && lane == 0) {
    tc_commit(&S.drain);
    const uint64_t t0d = global_timer_ns();
    while (!mbar_try_wait(&S.drain, 0) && global_timer_ns() - t0d < 1000000000ull) {
    }
  }
  __syncthreads();
  // a batched launch reports a timeout batch-wide: items this CTA never ran belong to other pairs
  if (threadIdx.x == 0 && S.abort) atomicMax(p.status, (int)PROHD_ETIMEOUT);
  if (warp == kGcMmaWarp) {
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
      // consecutive threads take consecutive rows i of one column j, so the
      // partials (stored column-major per CTA) are read coalesced
      const int j = (int)(e / D), i = (int)(e % D);
      if (j < i) continue;
      int c0, c1, row, col;
      if (i < 128) {
        c0 = 0; c1 = p.nc0; row = i; col = j;
      } else {
        c0 = p.nc0; c1 = ncta; row = i - 128; col = j - 128;
      }
      // four interleaved partial sums (loads in flight), combined in a fixed order
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      int c = c0;
      for (; c + 4 <= c1; c += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 v = p.gacc[(size_t)(c + u) * (256 * 128) + (size_t)col * 128 + row];
          s4[u] += (double)v.x - (double)v.y;
        }
      }
      for (; c < c1; ++c) {
        const float2 v = p.gacc[(size_t)c * (256 * 128) + (size_t)col * 128 + row];
        s4[0] += (double)v.x - (double)v.y;
      }
      G[(int64_t)i * D + j] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    } else {
      const int64_t k = e - DD;
      const int set = k < D ? 0 : 1;
      const int d = (int)(set ? k - D : k);
      // one partial sum per converter warp slot (independent loads), combined in order
      double sw[kGcConv];
#pragma unroll
      for (int w = 0; w < kGcConv; ++w) sw[w] = 0.0;
      for (int c = 0; c < p.nc0; ++c)
#pragma unroll
        for (int w = 0; w < kGcConv; ++w) sw[w] += p.sums[((size_t)c * kGcConv + w) * 2 * p.Dp + (size_t)set * p.Dp + d];
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kGcConv; ++w) s += sw[w];
      (set ? sumB : sumA)[d] = s;
    }
  }
}

bool gram_tc_supported(int D) { return D >= 4 && D <= kGcMaxRows && D % 4 == 0; }

size_t gram_tc_scratch_doubles(int D, int num_sms) {
  const int Dp = (int)round_up(D, 64);
  return (size_t)num_sms * 256 * 128 + (size_t)num_sms * kGcConv * 2 * Dp;
}

cudaError_t gram_tc_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                        const float* s32, double* scratch, double* G, double* sumA, double* sumB, int* status,
                        int64_t timeout_ns, cudaStream_t st) {
  const int nsm = ctx->num_sms;
  GcParams p;
  p.nA = nA;
  p.nB = nB;
  p.D = D;
  p.Dp = (int)round_up(D, 64);
  p.s32 = s32;
  p.N0 = p.Dp;
  p.rows0 = std::max(128, p.Dp);
  p.N1 = p.Dp > 128 ? p.Dp - 128 : 0;
  p.rows1 = 128;
  const int grid = nsm;
  if (p.N1 > 0) {
    // CTA counts in proportion to each type's time per point: a fixed part
    // (handshakes, flushes) plus parts proportional to the output columns
    // (MMA operand reads) and to the tile rows (copy, conversion), with
    // weights fitted to measured per-chunk times at D = 256.
    const double w0 = 20.0 + 0.07 * (p.N0 + p.rows0), w1 = 20.0 + 0.07 * (p.N1 + p.rows1);
    p.nc0 = (int)std::lround((double)nsm * w0 / (w0 + w1));
    p.nc0 = std::min(std::max(p.nc0, 2), nsm - 2);
  } else {
    p.nc0 = nsm;
  }
  auto split = [&](int nct) {
    int a = (int)std::lround((double)nct * (double)nA / (double)(nA + nB));
    return std::min(std::max(a, 1), nct - 1);
  };
  p.ncA0 = split(p.nc0);
  p.ncA1 = p.N1 > 0 ? split(grid - p.nc0) : 0;
  p.gacc = reinterpret_cast<float2*>(scratch);
  p.sums = scratch + (size_t)nsm * 256 * 128;
  p.status = status;
  p.timeout_ns = (uint64_t)timeout_ns;
  p.items = nullptr;
  p.nitems = 0;
  p.ticket = nullptr;
  CUtensorMap tA0, tB0, tA1, tB1;
  const uint64_t rowb = (uint64_t)D * 4;
  if (!encode_2d(ctx, &tA0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)D, (uint64_t)nA, rowb, p.rows0, kGcPts,
                 CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_2d(ctx, &tB0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B, (uint64_t)D, (uint64_t)nB, rowb, p.rows0, kGcPts,
                 CU_TENSOR_MAP_SWIZZLE_NONE))
    return cudaErrorInvalidValue;
  tA1 = tA0;
  tB1 = tB0;
  if (p.N1 > 0 &&
      (!encode_2d(ctx, &tA1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)D, (uint64_t)nA, rowb, p.rows1, kGcPts,
                  CU_TENSOR_MAP_SWIZZLE_NONE) ||
       !encode_2d(ctx, &tB1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B, (uint64_t)D, (uint64_t)nB, rowb, p.rows1, kGcPts,
                  CU_TENSOR_MAP_SWIZZLE_NONE)))
    return cudaErrorInvalidValue;
  const size_t smem = std::max(gc_smem_bytes(p.rows0), gc_smem_bytes(p.rows1));
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  {
    PhaseTimer pt(ctx, PROHD_PH_GRAM, st);
    count_launch();
    gram_tc_kernel<<<grid, kGcThreads, smem, st>>>(p, tA0, tB0, tA1, tB1);
    if ((e = cudaGetLastError())) return e;
  }
  count_launch();
  gram_tc_reduce_kernel<<<nsm, 256, 0, st>>>(p, grid, G, sumA, sumB);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched pairs

// G and the set sums of every pair of a batch from its items' partials
// (type-0 items for rows 0..127 and the sums, type-1 items for the rest),
// in the fixed order of the pair's item list. grid (chunks, pairs).
__global__ void gram_tc_reduce_batched_kernel(const BPair* __restrict__ P, const GcItem* __restrict__ items,
                                              const int* __restrict__ ids) {
  const BPair& q = P[blockIdx.y];
  const int D = q.D, Dp = q.Dp;
  const int64_t DD = (int64_t)D * D;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < DD + 2 * D;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < DD) {
      const int j = (int)(e / D), i = (int)(e % D);
      if (j < i) continue;
      int l0, l1, row, col;
      if (i < 128) {
        l0 = q.gi0; l1 = q.gi0 + q.gn0; row = i; col = j;
      } else {
        l0 = q.gi1; l1 = q.gi1 + q.gn1; row = i - 128; col = j - 128;
      }
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      int l = l0;
      for (; l + 4 <= l1; l += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 v = __ldg(items[ids[l + u]].gacc + (size_t)col * 128 + row);
          s4[u] += (double)v.x - (double)v.y;
        }
      }
      for (; l < l1; ++l) {
        const float2 v = __ldg(items[ids[l]].gacc + (size_t)col * 128 + row);
        s4[0] += (double)v.x - (double)v.y;
      }
      q.G[(int64_t)i * D + j] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    } else {
      const int64_t k = e - DD;
      const int set = k < D ? 0 : 1;
      const int d = (int)(set ? k - D : k);
      double sw[kGcConv];
#pragma unroll
      for (int w = 0; w < kGcConv; ++w) sw[w] = 0.0;
      for (int l = q.gi0; l < q.gi0 + q.gn0; ++l) {
        const double* sm = items[ids[l]].sums;
#pragma unroll
        for (int w = 0; w < kGcConv; ++w) sw[w] += __ldg(sm + (size_t)w * 2 * Dp + (size_t)set * Dp + d);
      }
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kGcConv; ++w) s += sw[w];
      (set ? q.sumB : q.sumA)[d] = s;
    }
  }
}

size_t gram_tc_smem_batched() { return gc_smem_bytes(kGcMaxRows); }

cudaError_t gram_tc_batched(const GcItem* items, int nitems, int* ticket, int* batch_status, int grid,
                            int64_t timeout_ns, cudaStream_t st) {
  GcParams p{};
  p.items = items;
  p.nitems = nitems;
  p.ticket = ticket;
  p.status = batch_status;
  p.timeout_ns = (uint64_t)timeout_ns;
  p.nc0 = grid;  // unused in batched launches
  const size_t smem = gc_smem_bytes(kGcMaxRows);
  cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  // the tensor maps live in the item table; the kernel's own map parameters are unused
  CUtensorMap none;
  memset(&none, 0, sizeof none);
  count_launch();
  gram_tc_kernel<<<grid, kGcThreads, smem, st>>>(p, none, none, none, none);
  return cudaGetLastError();
}

cudaError_t gram_reduce_batched(const BPair* P, int npairs, const GcItem* items, const int* ids, int Dmax,
                                cudaStream_t st) {
  const int64_t work = (int64_t)Dmax * Dmax + 2 * Dmax;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(16, ceil_div(work, 256 * 4)));
  count_launch();
  gram_tc_reduce_batched_kernel<<<dim3(gx, npairs), 256, 0, st>>>(P, items, ids);
  return cudaGetLastError();
}

}  // namespace prohd
