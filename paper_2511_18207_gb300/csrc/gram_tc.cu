// Union Gram G = sum_z (z - s)(z - s)^T and per-set sums of z - s on tcgen05
// tensor cores (Algorithm 2 step 2: principal components of [A; B] need the
// union covariance), for D <= 256 with D % 4 == 0.
//
// Arithmetic. Each FP32 centred value z is split into two BF16 parts,
// z = h + m + r with h = bf16(z), m = bf16(z - h) and |r| <= 2^-16 |z|. The
// tensor cores accumulate X = sum h h^T + 2 sum m h^T in FP32, and
// (X + X^T) / 2 = sum (h h^T + h m^T + m h^T) is zz^T up to the terms m m^T
// and h r^T + r h^T, each at most 2^-16 |z_i z_j| per point. The rounding
// residuals m and r have zero mean, so these terms cancel in the sum over
// points except on the diagonal, where m_i^2 is always positive; the
// converters therefore add sum (z_i^2 - h_i^2 - 2 h_i m_i) to G_ii, computed
// per point in FP32 with one rounding. The tensor core adds 512 points (64
// MMAs) into a TMEM accumulator; two accumulators (the two halves of TMEM)
// alternate between such intervals, and each finished one is added in FP32
// into a running sum that lives in the CTA's output slot (stored by the first
// interval, then added at the L2 by bulk reduce-add copies, in interval
// order), so the MMAs never wait for the running sum. Two final kernels sum
// the CTAs' slots in FP64 in a fixed order and symmetrise.
//
// Work split. Two CTAs of a cluster work as a pair on one tile of 64 points
// per step (cta_group::2, M = 256): for D > 128 each CTA stages and converts
// its own 128 dimensions of the same points (CTA r: dimensions 128r ..
// 128r + 127), and the pair's two MMAs per 16-point slice produce the whole
// 256 x 256 product, rows 128r.. in CTA r's tensor memory. Every point is
// read from HBM once, and each CTA's tensor core reads its own A half and
// half of B. For D <= 128 the two CTAs convert different points (CTA r the
// r-th 64-point half of a 128-point step) in the same layout; the product's
// diagonal blocks hold each CTA's own Gram, and the off-diagonal blocks (one
// CTA's points against the other's) are computed and ignored.
//
// Pipeline per CTA: a TMA warp streams FP32 tiles [64 points x 128 dims]
// through a three-stage ring (dimensions past D arrive as zeros); sixteen
// converter warps centre, split and transpose them into K-major,
// 128B-swizzled BF16 tile pairs {h, 2m} [128 dims x 64 points] (the operand
// layout of the distance contraction; three pairs used in turn, so that a
// pair's round trip (conversion, the signal to the even CTA, the MMAs, the
// commit back) overlaps the next two steps: measured at 2M points, 2 pairs
// x 4 TMA stages 1.07 ms, 3 x 3 0.92 ms, 4 x 2 1.01 ms) and signal the even CTA's MMA
// thread; that thread issues the step's eight MMAs (two per 16-point slice)
// and hands the tile pair back to both CTAs' converters when they complete;
// four epilogue warps per CTA drain each 512-point accumulator into the
// running sum while the MMAs fill the other one. The converters work on point pairs with two-wide FP32
// arithmetic (f32x2), which halves their instruction count: conversion, not
// HBM or the tensor pipe, bounded the step rate. The odd CTA's converters and epilogue signal the even
// CTA's barriers with remote mbarrier arrives after fence.proxy.async (a
// release at cluster scope costs a memory barrier per arrive, which stalled
// every step).
// Warps: 0..15 converters, 16 MMA issuer (even CTA) and TMEM owner, 17..20
// epilogue, 21 TMA producer.
#include <cuda_bf16.h>
#include <limits.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace prohd {

constexpr int kGcPts = 64;          // points per tile (one 128-byte K row of BF16)
constexpr int kGcRows = 128;        // dimensions per CTA
constexpr int kGcConv = 16;         // converter warps: 8 points x 64 dimensions each
constexpr int kGcPg = kGcPts / 8;   // 8-point groups of a tile (one 16-byte unit of a BF16 row)
constexpr int kGcEpi = 4;
constexpr int kGcMmaWarp = kGcConv;
constexpr int kGcTmaWarp = kGcConv + 1 + kGcEpi;
constexpr int kGcThreads = (kGcTmaWarp + 1) * 32;
constexpr int kGcStages = 3;        // FP32 staging ring
constexpr int kGcBufs = 3;          // operand tile pairs: conversion runs up to two steps ahead of the MMAs
constexpr int kGcFlush = 8;         // steps per TMEM accumulation (512 points per CTA row)
constexpr int kGcSlices = kGcPts / 16;
constexpr uint32_t kGcTileBytes = kGcRows * 128;             // one BF16 operand tile
constexpr uint32_t kGcStageBytes = kGcPts * kGcRows * 4;     // one FP32 stage
constexpr int kGcSlotFloats = 2 * 256 * kGcRows;             // per pair: [rank][col][row] partial products
constexpr int kGcSumsDoubles = 2 * kGcPg * 2 * kGcRows;      // per pair: [rank][point group][z | corr][dim]

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

struct GcSmem {
  uint64_t ffull[kGcStages], fempty[kGcStages];
  uint64_t sfull[kGcBufs];   // even CTA: tile pair converted by every converter warp of both CTAs
  uint64_t sempty[kGcBufs];  // the tile pair's MMAs done (committed to both CTAs)
  uint64_t acc_full[2];        // accumulator b holds a finished interval (committed to both CTAs)
  uint64_t acc_empty[2];       // even CTA: accumulator b read by both CTAs' epilogues (8 arrivals)
  uint64_t drain;
  uint32_t tmem_base;
  int abort;       // set by this CTA's waits or by the peer's
  int next;        // batched launches: the item both CTAs take next (written by the even CTA)
  int my_abort;    // abort snapshots exchanged between items
  int peer_abort;
  int epi_go;      // the epilogue issuer's wait result for the current interval
};

constexpr int kGcOutCols = 16;  // columns of one drain chunk (kGcOutCols x 128 rows of FP32)
constexpr uint32_t kGcOutBytes = kGcOutCols * kGcRows * 4;
constexpr size_t kGcSmemBytes = 1024 + (size_t)kGcBufs * 2 * kGcTileBytes + (size_t)kGcStages * kGcStageBytes +
                                2 * (size_t)kGcOutBytes + sizeof(GcSmem);

struct GcParams {
  int64_t nA, nB;
  int D, Dp;
  const float* s32;   // pilot shift [D]
  int nclu, ncA;      // clusters; clusters reading A (the rest read B)
  int64_t r0A, r1A, r0B, r1B;  // the rows this launch reads of A and of B
  int clu0;           // the launch's first slot
  float* out;         // [clu0 + nclu] x kGcSlotFloats
  double* sums;       // [clu0 + nclu] x kGcSumsDoubles
  int* status;
  uint64_t timeout_ns;
  // batched launches: clusters take items from the table through an atomic
  // ticket; nullptr for one pair (cluster c is item c of the static split)
  const GcItem* items;
  int nitems;
  int* ticket;
};

// Two-wide FP32 arithmetic on point pairs (f32x2; lo = the first point).
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// The two BF16 halves of v as an FP32 pair (a BF16 is the top half of an FP32).
__device__ __forceinline__ uint64_t f2_from_bf16x2(uint32_t v) {
  return ((uint64_t)(v & 0xffff0000u) << 32) | (uint64_t)(v << 16);
}

// Per converter lane and dimension: the Kahan-compensated set sum of z, and
// the two sums whose difference is the diagonal correction
// sum (z^2 - h^2 - 2hm) = sum e (z + h) - sum h (2m), e = z - h; each holds
// two points' lanes (f32x2).
struct GcAcc {
  float ss, sc;
  uint64_t ezh, hm2;
};

// Splits eight points of one dimension into the {h, 2m} operand rows (16
// bytes each, point i in the low half of pair i/2) and accumulates GcAcc.
// Only the first `nv` points are real when !FULL; the rest contribute zeros.
template <bool FULL>
__device__ __forceinline__ void gc_convert_row(const float* __restrict__ st, uint8_t* __restrict__ dst, float shift,
                                               GcAcc& a, int nv) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float v = st[i * kGcRows];
    x[i] = (FULL || i < nv) ? v : shift;  // padding points centre to exactly zero
  }
  const uint64_t sh = f2_pack(shift, shift);
  uint64_t z[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) z[i] = f2_sub(f2_pack(x[2 * i], x[2 * i + 1]), sh);
  {
    float lo, hi;
    f2_unpack(f2_add(f2_add(z[0], z[1]), f2_add(z[2], z[3])), lo, hi);
    kahan_add(a.ss, a.sc, lo + hi);
  }
  uint32_t h[4], m2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float z0, z1;
    f2_unpack(z[i], z0, z1);
    h[i] = bf16x2_rn(z0, z1);
    const uint64_t hf = f2_from_bf16x2(h[i]);
    const uint64_t e = f2_sub(z[i], hf);  // exact
    float e20, e21;
    f2_unpack(f2_add(e, e), e20, e21);    // 2e, exact
    m2[i] = bf16x2_rn(e20, e21);          // 2m, the exact doubling of bf16(e)
    a.ezh = f2_fma(e, f2_add(z[i], hf), a.ezh);
    a.hm2 = f2_fma(hf, f2_from_bf16x2(m2[i]), a.hm2);  // h (2m) is exact
  }
  *reinterpret_cast<uint4*>(dst) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(dst + kGcTileBytes) = make_uint4(m2[0], m2[1], m2[2], m2[3]);
}

// Waits with the kernel's limit; on failure the peer CTA is told to stop too.
__device__ __forceinline__ bool gc_wait(uint64_t* bar, uint32_t parity, volatile int* abort, uint32_t peer_abort,
                                        uint64_t timeout_ns) {
  if (mbar_wait_bounded(bar, parity, abort, timeout_ns)) return true;
  st_cluster_s32(peer_abort, 1);
  return false;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGcThreads, 1)
    gram_tc_kernel(const GcParams p, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = smem_align<1024>(smem_raw);
  uint8_t* tiles = base;  // [kGcBufs][h, 2m]
  float* stage = reinterpret_cast<float*>(base + kGcBufs * 2 * kGcTileBytes);  // [kGcStages][64][128]
  float* outst = reinterpret_cast<float*>(base + kGcBufs * 2 * kGcTileBytes +
                                          (size_t)kGcStages * kGcStageBytes);  // [2][kGcOutCols][128]
  GcSmem& S = *reinterpret_cast<GcSmem*>(base + kGcBufs * 2 * kGcTileBytes + (size_t)kGcStages * kGcStageBytes +
                                         2 * (size_t)kGcOutBytes);
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &S.abort;
  const uint32_t peer_abort = map_to_cta(&S.abort, rank ^ 1u);
  const bool batched = p.items != nullptr;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGcStages; ++s) {
      mbar_init(&S.ffull[s], 1);
      mbar_init(&S.fempty[s], kGcConv);
    }
    for (int b = 0; b < kGcBufs; ++b) {
      mbar_init(&S.sfull[b], 2 * kGcConv);  // every converter warp of both CTAs
      mbar_init(&S.sempty[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.acc_full[b], 1);
      mbar_init(&S.acc_empty[b], 2 * kGcEpi);
    }
    mbar_init(&S.drain, 1);
    S.abort = 0;
    S.next = 0;
    S.my_abort = 0;
    S.peer_abort = 0;
    fence_mbar_init();
  }
  if (warp == kGcMmaWarp) {
    tc2_alloc(&S.tmem_base, 512);
    tc2_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  // Ring positions and accumulation intervals run on over all items, so
  // every barrier's phase parity follows from two counters.
  uint32_t g0 = 0, f0 = 0;
  const int clu = (int)(blockIdx.x >> 1);

  for (int iter = 0;; ++iter) {
    GcItem w;
    if (!batched) {
      if (iter > 0) break;
      const bool setA = clu < p.ncA;
      const int64_t r0 = setA ? p.r0A : p.r0B, n = (setA ? p.r1A : p.r1B) - r0;
      const int cj = setA ? clu : clu - p.ncA, ncj = setA ? p.ncA : p.nclu - p.ncA;
      w.tm = setA ? &tmA : &tmB;
      w.s32 = p.s32;
      w.out = p.out + (size_t)(p.clu0 + clu) * kGcSlotFloats;
      w.sums = p.sums + (size_t)(p.clu0 + clu) * kGcSumsDoubles;
      w.status = p.status;
      w.p0 = r0 + n * cj / ncj;
      w.p1 = r0 + n * (cj + 1) / ncj;
      w.D = p.D;
      w.Dp = p.Dp;
      w.setA = setA ? 1 : 0;
    } else {
      // both CTAs take the same item and agree on stopping: each publishes
      // its abort state, the even CTA the ticket, then a cluster barrier
      cluster_sync();
      if (threadIdx.x == 0) {
        const int a = *abort;
        S.my_abort = a;
        st_cluster_s32(map_to_cta(&S.peer_abort, rank ^ 1u), a);
        if (leader) {
          const int it = atomicAdd(p.ticket, 1);
          S.next = it;
          st_cluster_s32(map_to_cta(&S.next, 1), it);
        }
      }
      cluster_sync();
      if (S.my_abort | S.peer_abort) break;
      const int it = S.next;
      if (it >= p.nitems) break;
      w = p.items[it];
    }
    const bool split_dims = w.Dp > kGcRows;
    const int64_t span = split_dims ? kGcPts : 2 * kGcPts;           // points per step of the pair
    const int64_t cta_off = split_dims ? 0 : (int64_t)rank * kGcPts;  // this CTA's first point of a step
    const int dim0 = split_dims ? (int)rank * kGcRows : 0;
    const int nsteps = w.p1 > w.p0 ? (int)((w.p1 - w.p0 + span - 1) / span) : 0;
    const int nint = (nsteps + kGcFlush - 1) / kGcFlush;
    const int N = split_dims ? 256 : 2 * w.Dp;           // MMA N
    const int ucol0 = split_dims ? 0 : (int)rank * w.Dp;  // this CTA's useful accumulator columns
    const int ucols = split_dims ? 256 : w.Dp;
    const int urows = split_dims ? kGcRows : w.Dp;        // useful TMEM lanes

    if (warp == kGcTmaWarp) {
      // ---------------- TMA producer ----------------
      if (lane == 0) {
        tma_prefetch_desc(w.tm);
        uint32_t armed = g0;
        for (int c = 0; c < nsteps; ++c) {
          const uint32_t g = g0 + (uint32_t)c;
          const int f = (int)(g % kGcStages);
          if (!gc_wait(&S.fempty[f], ((g / kGcStages) & 1u) ^ 1u, abort, peer_abort, p.timeout_ns)) break;
          mbar_arrive_expect_tx(&S.ffull[f], kGcStageBytes);
          const int64_t y = w.p0 + (int64_t)c * span + cta_off;
          tma_load_2d(stage + (size_t)f * (kGcStageBytes / 4), w.tm, dim0, (int)y, &S.ffull[f]);
          armed = g + 1;
        }
        if (*abort) {
          // error path: let the copies already issued land before the CTA exits
          for (uint32_t g = armed >= g0 + kGcStages ? armed - kGcStages : g0; g < armed; ++g) {
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(&S.ffull[g % kGcStages], (g / kGcStages) & 1u) &&
                   global_timer_ns() - t0 < 2000000ull) {
            }
          }
        }
      }
    } else if (warp < kGcConv) {
      // ---------------- converters: centre, split, transpose ----------------
      // warp w: points 8 (w % 8) .. + 7 of the tile, dimensions lane + 32 t
      // for t = 2 (w / 8), 2 (w / 8) + 1 (tile rows of this CTA)
      const int pg = warp & (kGcPg - 1), th = warp / kGcPg;
      const float* st0 = stage + (size_t)(pg * 8) * kGcRows + lane + 64 * th;
      uint8_t* dst0 = tiles + lane * 128 + ((pg ^ (lane & 7)) * 16) + th * 2 * 4096;
      GcAcc acc[2];
      float shift[2];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        acc[t].ss = acc[t].sc = 0.f;
        acc[t].ezh = acc[t].hm2 = 0ull;
        const int d = dim0 + lane + 32 * (2 * th + t);
        shift[t] = d < w.D ? w.s32[d] : 0.f;
      }
      for (int c = 0; c < nsteps; ++c) {
        const uint32_t g = g0 + (uint32_t)c;
        const int f = (int)(g % kGcStages);
        const int bf = (int)(g % kGcBufs);
        const uint32_t use = g / kGcBufs;  // this buffer's use count: wait for the MMAs of its previous use
        uint8_t* dst = dst0 + (size_t)bf * 2 * kGcTileBytes;
        int got = 1;
        if (lane == 0)
          got = gc_wait(&S.sempty[bf], (use & 1u) ^ 1u, abort, peer_abort, p.timeout_ns) &&
                gc_wait(&S.ffull[f], (g / kGcStages) & 1u, abort, peer_abort, p.timeout_ns);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) break;
        const float* st = st0 + (size_t)f * kGcPts * kGcRows;
        const int64_t left = w.p1 - (w.p0 + (int64_t)c * span + cta_off + pg * 8);
        if (left >= 8) {
#pragma unroll
          for (int t = 0; t < 2; ++t) gc_convert_row<true>(st + 32 * t, dst + t * 4096, shift[t], acc[t], 8);
        } else {
          const int nv = left > 0 ? (int)left : 0;
#pragma unroll
          for (int t = 0; t < 2; ++t) gc_convert_row<false>(st + 32 * t, dst + t * 4096, shift[t], acc[t], nv);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&S.fempty[f]);
          if (leader) mbar_arrive(&S.sfull[bf]);
          else mbar_arrive_remote(map_to_cta(&S.sfull[bf], 0));
        }
      }
      // A non-finite coordinate makes its dimension's running sum non-finite
      // (so does an FP32 overflow of the sum, which would also ruin G).
      bool bad = false;
      double* out = w.sums + (size_t)(rank * kGcPg + pg) * 2 * kGcRows;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int dl = lane + 32 * (2 * th + t);
        float e0, e1, q0, q1;
        f2_unpack(acc[t].ezh, e0, e1);
        f2_unpack(acc[t].hm2, q0, q1);
        bad |= !isfinite(acc[t].ss) || !isfinite(acc[t].sc) || !isfinite(e0 + e1);
        out[dl] = (double)acc[t].ss - (double)acc[t].sc;
        out[kGcRows + dl] = ((double)e0 + (double)e1) - ((double)q0 + (double)q1);
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicMax(w.status, (int)PROHD_ENONFINITE);
    } else if (warp == kGcMmaWarp) {
      // ---------------- MMA issuer (even CTA) ----------------
      if (leader && lane == 0) {
        const uint32_t idesc = idesc_f16(1, 256, N);
        int in_acc = 0;
        uint32_t fi = f0;
        for (int c = 0; c < nsteps; ++c) {
          const uint32_t g = g0 + (uint32_t)c;
          const uint32_t ab = fi & 1u;  // accumulators alternate between intervals
          if (in_acc == 0) {
            if (!gc_wait(&S.acc_empty[ab], ((fi >> 1) & 1u) ^ 1u, abort, peer_abort, p.timeout_ns)) break;
            tc_fence_after();
          }
          const uint32_t dacc = tmem + ab * 256u;
          const int bf = (int)(g % kGcBufs);
          const uint32_t use = g / kGcBufs;
          const uint32_t th = smem_u32(tiles) + (uint32_t)bf * 2 * kGcTileBytes, tm2 = th + kGcTileBytes;
          if (!gc_wait(&S.sfull[bf], use & 1u, abort, peer_abort, p.timeout_ns)) break;
          tc_fence_after();
#pragma unroll
          for (int k = 0; k < kGcSlices; ++k) {
            const uint64_t bh = smem_desc_sw128(th + k * 32);
            tc2_mma_f16(dacc, bh, bh, idesc, (in_acc | k) != 0);
            tc2_mma_f16(dacc, smem_desc_sw128(tm2 + k * 32), bh, idesc, 1u);
          }
          tc2_commit_mc(&S.sempty[bf], 0x3);  // this tile pair may be overwritten in both CTAs
          if (++in_acc == kGcFlush || c == nsteps - 1) {
            tc2_commit_mc(&S.acc_full[ab], 0x3);
            in_acc = 0;
            ++fi;
          }
        }
      }
    } else {
      // ---------------- epilogue: accumulator -> running sum in the item's slot ----------------
      // The slot holds the running sum: the first interval's accumulator is
      // stored, every later one added at the L2 (bulk reduce-add, FP32 round
      // to nearest: the same sum as adding in registers). Chunks of 16
      // columns x 128 rows go through two shared-memory buffers; one thread
      // issues each chunk's bulk copy after the four warps have written it.
      // The accumulator is handed back as soon as it is read, so the MMAs of
      // the next interval (into the other accumulator) never wait for the
      // slot. Intervals of one item reach the slot in order: the issuer
      // waits for the previous interval's copies before the next.
      const int q = warp & 3;  // TMEM lane quarter this warp may access
      const int row = q * 32 + lane;
      const bool useful = q * 32 < urows;
      const bool issuer = warp == kGcConv + 1 && lane == 0;
      const uint32_t acc_empty_leader0 = map_to_cta(&S.acc_empty[0], 0);
      const uint32_t acc_empty_leader1 = map_to_cta(&S.acc_empty[1], 0);
      const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
      float* o = w.out + (size_t)rank * ucols * kGcRows;
      const int nch = ucols / kGcOutCols;
      uint32_t chunk = 0;  // drain chunks so far: staging buffer chunk & 1
      for (int i = 0; i < nint; ++i) {
        const uint32_t fi = f0 + (uint32_t)i;
        const uint32_t ab = fi & 1u;
        // one thread waits; the four warps take its result together (they
        // meet at named barriers below, so they must all go on or all stop)
        if (issuer) {
          S.epi_go = gc_wait(&S.acc_full[ab], (fi >> 1) & 1u, abort, peer_abort, p.timeout_ns) ? 1 : 0;
          if (i > 0) bulk_wait_all();  // the previous interval's adds are performed
        }
        __syncwarp();  // each warp reaches the barrier converged
        named_bar_sync(1, 32 * kGcEpi);
        const int go = S.epi_go;
        named_bar_sync(1, 32 * kGcEpi);  // S.epi_go is read before the next interval rewrites it
        if (!go) break;
        tc_fence_after();
        for (int cc = 0; cc < nch; ++cc, ++chunk) {
          float v[kGcOutCols];
          if (useful) {
            __syncwarp();
            tc_ld_32x32b_x16(lane_base + ab * 256u + (uint32_t)(ucol0 + cc * kGcOutCols), v);
            tc_wait_ld();
          } else {
#pragma unroll
            for (int j = 0; j < kGcOutCols; ++j) v[j] = 0.f;
          }
          if (cc == nch - 1) {
            // this CTA's half of accumulator ab is read: tell the MMA thread
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if (leader) mbar_arrive(&S.acc_empty[ab]);
              else mbar_arrive_remote(ab ? acc_empty_leader1 : acc_empty_leader0);
            }
          }
          float* buf = outst + (size_t)(chunk & 1u) * (kGcOutCols * kGcRows);
          if (issuer) bulk_wait_read<1>();  // the copy that last used this buffer has read it
          __syncwarp();
          named_bar_sync(1, 32 * kGcEpi);
#pragma unroll
          for (int j = 0; j < kGcOutCols; ++j) buf[j * kGcRows + row] = v[j];
          fence_proxy_async();
          __syncwarp();
          named_bar_sync(1, 32 * kGcEpi);
          if (issuer) {
            float* dst = o + (size_t)cc * kGcOutCols * kGcRows;
            if (i == 0) bulk_store_s2g(dst, buf, kGcOutBytes);
            else bulk_add_f32_s2g(dst, buf, kGcOutBytes);
            bulk_commit();
          }
          __syncwarp();
        }
      }
      if (nint == 0) {
        // an empty item's partial product is zero
        for (int cc = 0; cc < nch; ++cc)
#pragma unroll
          for (int j = 0; j < kGcOutCols; ++j) o[(size_t)(cc * kGcOutCols + j) * kGcRows + row] = 0.f;
      }
      if (issuer) bulk_wait_all();
    }
    // the item is finished by every role of this CTA: the rings are idle
    __syncthreads();
    g0 += (uint32_t)nsteps;
    f0 += (uint32_t)nint;
    if (!batched) break;
  }

  // every MMA the pair issued has completed before either CTA moves on
  if (warp == kGcMmaWarp && lane == 0) {
    if (leader) tc2_commit_mc(&S.drain, 0x3);
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(&S.drain, 0) && global_timer_ns() - t0 < 1000000000ull) {
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && S.abort) atomicMax(p.status, (int)PROHD_ETIMEOUT);
  // neither CTA leaves while the other may still read its shared memory or
  // arrive on its barriers; then the pair frees its tensor memory together
  cluster_sync();
  if (warp == kGcMmaWarp) {
    __syncwarp();
    tc_fence_after();
    tc2_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------- reduction

// The partial product X of a list of pair slots: X[i][j] for one slot list
// entry. Split dimensions (Dp > 128): row i lives in CTA i / 128 at lane
// i % 128, all 256 columns. Split points: both CTAs hold rows 0..Dp-1 and
// columns 0..Dp-1 of their own points, so X is their sum.
__device__ __forceinline__ float gc_x(const float* __restrict__ slot, int Dp, int i, int j) {
  if (Dp > kGcRows) return __ldg(slot + (size_t)(i >> 7) * 256 * kGcRows + (size_t)j * kGcRows + (i & 127));
  return __ldg(slot + (size_t)j * kGcRows + i) + __ldg(slot + (size_t)(Dp + j) * kGcRows + i);
}

// Floats of one pair slot's partial products: two CTAs x useful columns x 128 rows.
__host__ __device__ constexpr size_t gc_slot_floats(int Dp) { return (size_t)2 * (Dp > kGcRows ? 256 : Dp) * kGcRows; }

// Reduction of the pair slots, each summed in FP64 in a fixed order:
//  1. Z = sum over slots of X, stored transposed in G's memory
//     (G[j * D + i] = Z(i, j); reads of X are contiguous in i);
//  2. per dimension (one warp each, lane l taking slots l, l + 32, ...,
//     then a fixed butterfly): the set sums of z - s and the diagonal
//     correction sum of z^2 - h^2 - 2hm;
//  3. the upper triangle of G is overwritten in place with
//     (Z(i, j) + Z(j, i)) / 2, plus the correction for i == j. Thread (i, j)
//     reads G[j D + i] and G[i D + j] and writes G[i D + j]; no other thread
//     of the upper triangle reads that location, so the pass is free of races.
template <class SlotOf>
__device__ __forceinline__ void gc_sum_pass(const SlotOf& slot_of, int nslots, int Dp, int D, double* __restrict__ G,
                                            int64_t e0, int64_t estride) {
  const int64_t DD = (int64_t)D * D;
  for (int64_t e = e0; e < DD; e += estride) {
    const int j = (int)(e / D), i = (int)(e % D);
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    int c = 0;
    for (; c + 4 <= nslots; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float* slot;
        const double* sums;
        bool setA;
        slot_of(c + u, slot, sums, setA);
        s4[u] += (double)gc_x(slot, Dp, i, j);
      }
    }
    for (; c < nslots; ++c) {
      const float* slot;
      const double* sums;
      bool setA;
      slot_of(c, slot, sums, setA);
      s4[0] += (double)gc_x(slot, Dp, i, j);
    }
    G[(size_t)j * D + i] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
  }
}

// Warp w0, w0 + wstride, ...: dimension d.
template <class SlotOf>
__device__ __forceinline__ void gc_dims_pass(const SlotOf& slot_of, int nslots, int Dp, int D,
                                             double* __restrict__ sumA, double* __restrict__ sumB,
                                             double* __restrict__ corr, int w0, int wstride) {
  const int lane = threadIdx.x & 31;
  for (int d = w0; d < D; d += wstride) {
    const int r0 = Dp > kGcRows ? (d >> 7) : 0, r1 = Dp > kGcRows ? r0 : 1;
    const int dl = Dp > kGcRows ? (d & 127) : d;
    double sa = 0.0, sb = 0.0, cr = 0.0;
    for (int c = lane; c < nslots; c += 32) {
      const float* slot;
      const double* sums;
      bool setA;
      slot_of(c, slot, sums, setA);
      for (int r = r0; r <= r1; ++r)
        for (int w = 0; w < kGcPg; ++w) {
          const double* sw = sums + (size_t)(r * kGcPg + w) * 2 * kGcRows;
          const double z = __ldg(sw + dl);
          cr += __ldg(sw + kGcRows + dl);
          if (setA) sa += z;
          else sb += z;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
      cr += __shfl_xor_sync(0xffffffffu, cr, o);
    }
    if (lane == 0) {
      sumA[d] = sa;
      sumB[d] = sb;
      corr[d] = cr;
    }
  }
}

__device__ __forceinline__ void gc_sym_pass(int D, double* __restrict__ G, const double* __restrict__ corr,
                                            int64_t e0, int64_t estride) {
  const int64_t DD = (int64_t)D * D;
  for (int64_t e = e0; e < DD; e += estride) {
    const int i = (int)(e / D), j = (int)(e % D);
    if (j < i) continue;
    if (i != j) G[(size_t)i * D + j] = 0.5 * (G[(size_t)j * D + i] + G[(size_t)i * D + j]);
    else G[(size_t)i * D + i] += corr[i];
  }
}

// One pair: blocks [0, nsum) sum X into G, the rest take the dimensions.
__global__ void __launch_bounds__(256) gram_tc_sum_kernel(const GcParams p, int nsum, double* __restrict__ G,
                                                          double* __restrict__ sumA, double* __restrict__ sumB,
                                                          double* __restrict__ corr) {
  auto slot_of = [&](int c, const float*& slot, const double*& sums, bool& setA) {
    slot = p.out + (size_t)c * kGcSlotFloats;
    sums = p.sums + (size_t)c * kGcSumsDoubles;
    setA = c < p.ncA;
  };
  if ((int)blockIdx.x < nsum)
    gc_sum_pass(slot_of, p.nclu, p.Dp, p.D, G, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)nsum * blockDim.x);
  else
    gc_dims_pass(slot_of, p.nclu, p.Dp, p.D, sumA, sumB, corr,
                 (int)((blockIdx.x - nsum) * (blockDim.x >> 5) + (threadIdx.x >> 5)),
                 (int)((gridDim.x - nsum) * (blockDim.x >> 5)));
}

__global__ void __launch_bounds__(256) gram_tc_sym_kernel(int D, double* __restrict__ G,
                                                          const double* __restrict__ corr) {
  gc_sym_pass(D, G, corr, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

bool gram_tc_supported(int D) { return D >= 4 && D <= 2 * kGcRows && D % 4 == 0; }

size_t gram_tc_scratch_doubles(int D, int num_sms, int parts) {
  (void)D;
  const size_t slots = (size_t)(num_sms / 2) * (parts > 1 ? 2 * parts : 1);
  return slots * (kGcSlotFloats / 2 + kGcSumsDoubles) + 2 * kGcRows;
}

cudaError_t gram_tc_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                        const float* s32, double* scratch, double* G, double* sumA, double* sumB, int* status,
                        int64_t timeout_ns, cudaStream_t st, const InputFeed* feed) {
  if (nA < 1 || nB < 1 || nA > INT_MAX || nB > INT_MAX) return cudaErrorInvalidValue;
  const int parts = feed && feed->parts > 1 ? feed->parts : 1;
  GcParams p;
  p.nA = nA;
  p.nB = nB;
  p.D = D;
  p.Dp = (int)round_up(D, 64);
  p.s32 = s32;
  p.nclu = ctx->num_sms / 2;
  {
    // clusters in proportion to the set sizes, at least one per set
    int a = (int)std::lround((double)p.nclu * (double)nA / (double)(nA + nB));
    p.ncA = std::min(std::max(a, 1), p.nclu - 1);
  }
  p.r0A = 0;
  p.r1A = nA;
  p.r0B = 0;
  p.r1B = nB;
  p.clu0 = 0;
  const int nslots = parts > 1 ? 2 * parts * p.nclu : p.nclu;
  p.out = reinterpret_cast<float*>(scratch);
  p.sums = scratch + (size_t)nslots * (kGcSlotFloats / 2);
  p.status = status;
  p.timeout_ns = (uint64_t)timeout_ns;
  p.items = nullptr;
  p.nitems = 0;
  p.ticket = nullptr;
  CUtensorMap tA, tB;
  const uint64_t rowb = (uint64_t)D * 4;
  if (!encode_2d(ctx, &tA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)D, (uint64_t)nA, rowb, kGcRows, kGcPts,
                 CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_2d(ctx, &tB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, B, (uint64_t)D, (uint64_t)nB, rowb, kGcRows, kGcPts,
                 CU_TENSOR_MAP_SWIZZLE_NONE))
    return cudaErrorInvalidValue;
  cudaError_t e =
      cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGcSmemBytes);
  if (e) return e;
  if (parts == 1) {
    if (feed && feed->ready) {
      if ((e = cudaStreamWaitEvent(st, feed->ready[0], 0))) return e;
      if ((e = cudaStreamWaitEvent(st, feed->ready[1], 0))) return e;
    }
    PhaseTimer pt(ctx, PROHD_PH_GRAM, st);
    count_launch();
    gram_tc_kernel<<<2 * p.nclu, kGcThreads, kGcSmemBytes, st>>>(p, tA, tB);
    if ((e = cudaGetLastError())) return e;
  } else {
    // one launch per row range of each set, every cluster on that range,
    // each launch into its own slots (A's ranges first); a range's launch
    // waits for its rows to land
    for (int s = 0; s < 2; ++s)
      for (int k = 0; k < parts; ++k) {
        const int64_t n = s ? nB : nA;
        GcParams q = p;
        q.ncA = s ? 0 : p.nclu;
        if (s) {
          q.r0B = n * k / parts;
          q.r1B = n * (k + 1) / parts;
        } else {
          q.r0A = n * k / parts;
          q.r1A = n * (k + 1) / parts;
        }
        q.clu0 = (s * parts + k) * p.nclu;
        if (feed->ready && (e = cudaStreamWaitEvent(st, feed->ready[s * parts + k], 0))) return e;
        PhaseTimer pt(ctx, PROHD_PH_GRAM, st);
        count_launch();
        gram_tc_kernel<<<2 * p.nclu, kGcThreads, kGcSmemBytes, st>>>(q, tA, tB);
        if ((e = cudaGetLastError())) return e;
      }
    // the reduction sees all slots, A's first
    p.ncA = parts * p.nclu;
    p.nclu = nslots;
  }
  double* corr = p.sums + (size_t)nslots * kGcSumsDoubles;
  const int nsum = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)D * D, 256), (int64_t)ctx->num_sms * 4));
  const int ndim = (int)ceil_div(D, 8);  // 8 warps per block, one dimension each
  count_launch();
  gram_tc_sum_kernel<<<nsum + ndim, 256, 0, st>>>(p, nsum, G, sumA, sumB, corr);
  count_launch();
  gram_tc_sym_kernel<<<nsum, 256, 0, st>>>(D, G, corr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched pairs

// G and the set sums of every pair of a batch from its items' partials, in
// the fixed order of the pair's item list. grid (chunks + dimension blocks, pairs).
__global__ void __launch_bounds__(256) gram_tc_sum_batched_kernel(const BPair* __restrict__ P,
                                                                  const GcItem* __restrict__ items,
                                                                  const int* __restrict__ ids, int nsum) {
  const BPair& q = P[blockIdx.y];
  auto slot_of = [&](int c, const float*& slot, const double*& sums, bool& setA) {
    const GcItem& it = items[ids[q.gi0 + c]];
    slot = it.out;
    sums = it.sums;
    setA = it.setA != 0;
  };
  if ((int)blockIdx.x < nsum)
    gc_sum_pass(slot_of, q.gn0, q.Dp, q.D, q.G, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                (int64_t)nsum * blockDim.x);
  else
    gc_dims_pass(slot_of, q.gn0, q.Dp, q.D, q.sumA, q.sumB, q.gcorr,
                 (int)((blockIdx.x - nsum) * (blockDim.x >> 5) + (threadIdx.x >> 5)),
                 (int)((gridDim.x - nsum) * (blockDim.x >> 5)));
}

__global__ void __launch_bounds__(256) gram_tc_sym_batched_kernel(const BPair* __restrict__ P) {
  const BPair& q = P[blockIdx.y];
  gc_sym_pass(q.D, q.G, q.gcorr, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

size_t gram_tc_smem_batched() { return kGcSmemBytes; }
size_t gram_tc_item_sums_offset(int Dp) { return round_up(gc_slot_floats(Dp) * sizeof(float), 256); }
size_t gram_tc_item_slot_bytes(int Dp) {
  return gram_tc_item_sums_offset(Dp) + round_up((size_t)kGcSumsDoubles * sizeof(double), 256);
}

cudaError_t gram_tc_batched(const GcItem* items, int nitems, int* ticket, int* batch_status, int grid,
                            int64_t timeout_ns, cudaStream_t st) {
  GcParams p{};
  p.items = items;
  p.nitems = nitems;
  p.ticket = ticket;
  p.status = batch_status;
  p.timeout_ns = (uint64_t)timeout_ns;
  p.nclu = grid / 2;
  cudaError_t e =
      cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGcSmemBytes);
  if (e) return e;
  // the tensor maps live in the item table; the kernel's own map parameters are unused
  CUtensorMap none;
  memset(&none, 0, sizeof none);
  count_launch();
  gram_tc_kernel<<<2 * (grid / 2), kGcThreads, kGcSmemBytes, st>>>(p, none, none);
  return cudaGetLastError();
}

cudaError_t gram_reduce_batched(const BPair* P, int npairs, const GcItem* items, const int* ids, int Dmax,
                                cudaStream_t st) {
  const int nsum = (int)std::max<int64_t>(1, std::min<int64_t>(16, ceil_div((int64_t)Dmax * Dmax, 256 * 4)));
  const int ndim = (int)ceil_div(Dmax, 8);
  count_launch();
  gram_tc_sum_batched_kernel<<<dim3(nsum + ndim, npairs), 256, 0, st>>>(P, items, ids, nsum);
  count_launch();
  gram_tc_sym_batched_kernel<<<dim3(nsum, npairs), 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace prohd
