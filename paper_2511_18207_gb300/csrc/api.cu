// C ABI entry points (include/prohd.h): argument checks, workspace layout and
// the order of the kernels of each call. Everything runs asynchronously on
// the caller's stream; nothing here allocates device memory or synchronises.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "internal.h"

namespace prohd {

std::atomic<uint64_t> g_launches{0};

__global__ void set_i64_kernel(int64_t* p, int64_t v) { *p = v; }
__global__ void zero_i32_kernel(int* p, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}
__global__ void finish_estimate_kernel(prohd_result* out, const int64_t* nselA, const int64_t* nselB) {
  out->nsel_a = *nselA;
  out->nsel_b = *nselB;
}

// One-sided refinement (max of the two directed distances of each selected
// set against the whole other set): r1 holds h(A_sel, B) in its h_ab, with
// witness (ab_a mapped to A, ab_b in B); r2 holds h(B_sel, A) likewise with
// the roles of the sets swapped.
__global__ void refine_combine_kernel(const prohd_hd_result* r1, const prohd_hd_result* r2, prohd_result* out) {
  prohd_hd_result r;
  const prohd_hd_result a = *r1, b = *r2;
  r.h_ab = a.h_ab;
  r.h_ba = b.h_ab;
  r.ab_a = a.ab_a;
  r.ab_b = a.ab_b;
  r.ba_b = b.ab_a;
  r.ba_a = b.ab_b;
  r.dir = r.h_ab >= r.h_ba ? 0 : 1;
  r.H = r.dir == 0 ? r.h_ab : r.h_ba;
  r.wit_a = r.dir == 0 ? r.ab_a : r.ba_a;
  r.wit_b = r.dir == 0 ? r.ab_b : r.ba_b;
  r.status = a.status > b.status ? a.status : b.status;
  if (out->hd.status > r.status) r.status = out->hd.status;
  r.H_lowp = fmax(a.H_lowp, b.H_lowp);
  r.n_rescored_a = a.n_rescored_a;
  r.n_rescored_b = b.n_rescored_a;
  out->hd = r;
}

// mask[i] = i < *n_dev and hi[i] >= scale * max(*lb1, *lb2) (lb2 may be null), for i < n_max
__global__ void keep_mask_kernel(const float* __restrict__ hi, const int64_t* n_dev, int64_t n_max, const double* lb1,
                                 const double* lb2, double scale, uint8_t* __restrict__ mask) {
  const int64_t n = *n_dev;
  const double L = scale * (lb2 ? fmax(*lb1, *lb2) : *lb1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_max; i += (int64_t)gridDim.x * blockDim.x)
    mask[i] = (i < n && (double)hi[i] >= L) ? 1 : 0;
}

// S = min(Smax, *n_dev) indices spread evenly over [0, *n_dev): idx[i] = floor(i n / S)
__global__ void strided_dev_kernel(int32_t* __restrict__ idx, int64_t* __restrict__ nS, int64_t Smax,
                                   const int64_t* __restrict__ n_dev) {
  const int64_t n = *n_dev;
  const int64_t S = n < Smax ? n : Smax;
  for (int64_t i = threadIdx.x; i < S; i += blockDim.x) idx[i] = (int32_t)((i * n) / S);
  if (threadIdx.x == 0) *nS = S;
}

// S = min(Smax, *nlist) entries of list spread evenly: idx[i] = list[floor(i nlist / S)]
__global__ void strided_sub_kernel(int32_t* __restrict__ idx, int64_t* __restrict__ nS, int64_t Smax,
                                   const int32_t* __restrict__ list, const int64_t* __restrict__ nlist) {
  const int64_t n = *nlist;
  const int64_t S = n < Smax ? n : Smax;
  for (int64_t i = threadIdx.x; i < S; i += blockDim.x) idx[i] = list[(i * n) / S];
  if (threadIdx.x == 0) *nS = S;
}

// out[i] = map[idx[i]] for i < *n_dev
__global__ void compose_idx_kernel(int32_t* __restrict__ out, const int32_t* __restrict__ idx,
                                   const int32_t* __restrict__ map, const int64_t* __restrict__ n_dev) {
  const int64_t n = *n_dev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = map[idx[i]];
}

// The two directed results of the pruned exact distance: r1 = h(A, B) in its
// h_ab (witness ab_a in A, ab_b in B), r2 = h(B, A) in its h_ab with the sets'
// roles swapped.
__global__ void directed_combine_kernel(const prohd_hd_result* r1, const prohd_hd_result* r2, prohd_hd_result* out) {
  prohd_hd_result r;
  const prohd_hd_result a = *r1, b = *r2;
  r.h_ab = a.h_ab;
  r.h_ba = b.h_ab;
  r.ab_a = a.ab_a;
  r.ab_b = a.ab_b;
  r.ba_b = b.ab_a;
  r.ba_a = b.ab_b;
  r.dir = r.h_ab >= r.h_ba ? 0 : 1;
  r.H = r.dir == 0 ? r.h_ab : r.h_ba;
  r.wit_a = r.dir == 0 ? r.ab_a : r.ba_a;
  r.wit_b = r.dir == 0 ? r.ab_b : r.ba_b;
  r.status = a.status > b.status ? a.status : b.status;
  r.H_lowp = fmax(a.H_lowp, b.H_lowp);
  r.n_rescored_a = a.n_rescored_a;
  r.n_rescored_b = b.n_rescored_a;
  *out = r;
}

cudaError_t set_i64(int64_t* p, int64_t v, cudaStream_t st) {
  count_launch();
  set_i64_kernel<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}
cudaError_t zero_i32(int* p, int n, cudaStream_t st) {
  count_launch();
  zero_i32_kernel<<<1, 32, 0, st>>>(p, n);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_2d(prohd_ctx* ctx, CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t inner,
               uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
  if (!ctx->encode_tiled) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = reinterpret_cast<EncodeTiledFn>(ctx->encode_tiled)(
      map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace prohd

using namespace prohd;

// ---------------------------------------------------------------- helpers

static prohd_status fail(prohd_ctx* ctx, prohd_status s, const char* fmt, const char* detail = "") {
  if (ctx) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, detail);
    ctx->err = buf;
  }
  return s;
}

static prohd_status cuda_fail(prohd_ctx* ctx, cudaError_t e) {
  return fail(ctx, PROHD_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
}

static bool bad_n(int64_t n) { return n < 1 || n >= ((int64_t)1 << 31); }

static int resolve_m(const prohd_params* p, int D) {
  return p->m < 0 ? (int)floor(sqrt((double)D)) : p->m;
}
static double resolve_alpha_p(const prohd_params* p, int m) {
  return p->alpha_p < 0 ? p->alpha_c / (double)std::max(m, 1) : p->alpha_p;
}

static prohd_status check_sets(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D) {
  if (!ctx) return PROHD_EINVAL;
  if (!A || !B) return fail(ctx, PROHD_EINVAL, "null point-set pointer%s");
  if (bad_n(nA) || bad_n(nB)) return fail(ctx, PROHD_EINVAL, "set sizes must be in [1, 2^31)%s");
  if (D < 1 || D > 1024) return fail(ctx, PROHD_EINVAL, "D must be in [1, 1024]%s");
  return PROHD_OK;
}

static prohd_status check_params(prohd_ctx* ctx, const prohd_params* p, int D) {
  if (!p) return fail(ctx, PROHD_EINVAL, "null params%s");
  if (!(p->alpha_c > 0.0 && p->alpha_c < 1.0)) return fail(ctx, PROHD_EINVAL, "alpha_c must be in (0, 1)%s");
  if (p->alpha_p >= 0.0 && !(p->alpha_p > 0.0 && p->alpha_p < 1.0))
    return fail(ctx, PROHD_EINVAL, "alpha_p must be in (0, 1) or negative for alpha_c / m%s");
  const int m = resolve_m(p, D);
  if (m < 0 || m > D || m > 63) return fail(ctx, PROHD_EINVAL, "m must be in [0, min(D, 63)]%s");
  if (p->precision != PROHD_FP32 && p->precision != PROHD_FP16 && p->precision != PROHD_BF16)
    return fail(ctx, PROHD_EINVAL, "unknown precision%s");
  if (p->precision != PROHD_FP32 && !tc_supported_dim(D))
    return fail(ctx, PROHD_ENOTSUP, "tensor-core precisions need D <= 256 (use PROHD_FP32)%s");
  if (p->power_max_iters < 1) return fail(ctx, PROHD_EINVAL, "power_max_iters must be >= 1%s");
  if (p->refine != 0 && p->refine != 1) return fail(ctx, PROHD_EINVAL, "refine must be 0 or 1%s");
  return PROHD_OK;
}

static prohd_status check_ws(prohd_ctx* ctx, void* ws, size_t ws_bytes, size_t need) {
  if (!ws) return fail(ctx, PROHD_EINVAL, "null workspace%s");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, PROHD_EINVAL, "workspace must be 256-byte aligned%s");
  if (ws_bytes < need) return fail(ctx, PROHD_ENOMEM, "workspace too small%s");
  return PROHD_OK;
}

// per-direction k for one set (Algorithms 1-3): k_c for the centroid axis, k_p for the PCs
static void k_list(int64_t n, int nd, double alpha_c, double alpha_p, int64_t* k) {
  for (int d = 0; d < nd; ++d) k[d] = prohd_k_of(d == 0 ? alpha_c : alpha_p, n);
}
static int64_t subset_bound(int64_t n, int nd, const int64_t* k) {
  int64_t s = 0;
  for (int d = 0; d < nd; ++d) s += 2 * std::min(k[d], n);
  return std::min(n, s);
}

// ---------------------------------------------------------------- row pruning (directed distances)

constexpr int64_t kPruneSample = 1024;   // rows of a lower-bound sample
constexpr int64_t kPruneMinRows = 32768; // smaller column sets take the plain contraction
// Smaller contractions (rows x columns) than ctx->prune_min_pairs (default
// 4e9) take the plain path: at 1.9e9 pairs the passes' fixed costs exceed
// the saving, at 7.5e9 pairs the pruning wins.
// A sample's distance is the FP64 length of the FP32 nearest neighbour of
// its row, which can exceed the row's true NN distance by the FP32 rounding
// of D-term squared sums (under 2^-24 D relative); the pruning threshold is
// lowered by 1e-4 relative to stay below the true distance.
constexpr double kPruneScale = 1.0 - 1e-4;

// columns of Y the pruning contraction scans: n_Y / 64, at least 8192, whole tiles
static int64_t prune_prefix(int64_t nY) {
  const int64_t p = std::max<int64_t>(8192, nY / 64);
  return std::min(nY, (p + 255) / 256 * 256);
}

namespace {
// Buffers of the pruned directed distance h(X, Y) for two directions:
// direction d has at most nX[d] rows in X and nY[d] rows in Y.
struct PruneLayout {
  int64_t *nS, *nYp, *nkeep;
  int32_t* sidx;
  float* Xs;
  prohd_hd_result* rs;  // [4]: the two samples' results per direction
  float* hi;            // certified upper bounds of the rows' NN distances
  uint8_t* mask;
  unsigned* counts;
  int64_t* offsets;
  int32_t *kidx, *kmap;
  float* Xk;
  HdShared Ysh;         // the other set's rounded copy, made once per direction
  size_t mark;          // the passes' shared scratch starts here
};
void prune_layout(Arena& a, const int64_t nX[2], const int64_t nY[2], int D, int precision, PruneLayout& L) {
  const int64_t xm = std::max(nX[0], nX[1]);
  const int64_t S = std::min(kPruneSample, xm);
  L.nS = a.take<int64_t>(1);
  L.nYp = a.take<int64_t>(1);
  L.nkeep = a.take<int64_t>(1);
  L.sidx = a.take<int32_t>((size_t)S);
  L.Xs = a.take<float>((size_t)S * D);
  L.rs = a.take<prohd_hd_result>(4);
  L.hi = a.take<float>((size_t)xm);
  L.mask = a.take<uint8_t>((size_t)xm);
  L.counts = a.take<unsigned>((size_t)compact_blocks(xm));
  L.offsets = a.take<int64_t>((size_t)compact_blocks(xm));
  L.kidx = a.take<int32_t>((size_t)xm);
  L.kmap = a.take<int32_t>((size_t)xm);
  L.Xk = a.take<float>((size_t)xm * D);
  hd_shared_layout(a, std::max(nY[0], nY[1]), D, precision, L.Ysh);
  L.mark = (a.off + 255) / 256 * 256;
  size_t end = a.off;
  for (int d = 0; d < 2; ++d) {
    const int64_t Sd = std::min(kPruneSample, nX[d]);
    Arena t = a;
    hd_core_layout(t, Sd, nY[d], D, precision);
    end = std::max(end, t.off);
    t = a;
    hd_prefix_layout(t, nX[d], prune_prefix(nY[d]), D, precision);
    end = std::max(end, t.off);
    t = a;
    hd_core_layout(t, nX[d], nY[d], D, precision);
    end = std::max(end, t.off);
  }
  a.off = end;
}
}  // namespace

// h(X, Y) with row pruning, X holding *nX_dev rows (at most nX_max), Y nY
// rows; the result r carries witness rows of X mapped through `map` (NULL:
// X's own indices). h over an evenly spread sample of rows of X is a lower
// bound LB1; one contraction of every row against the first prune_prefix(nY)
// rows of Y gives each row a certified upper bound of its NN distance; the
// rows whose bound reaches LB1 are the hard ones, and h over an evenly spread
// sample of those is a second, larger lower bound LB2. The exact path then
// runs on the rows whose bound reaches max(LB1, LB2). Every lower bound is a
// row's own distance, so the row attaining h(X, Y) always stays and the
// result equals the plain one. X of at most kPruneSample rows, or Y under
// kPruneMinRows rows, takes the plain path directly.
static cudaError_t pruned_directed(prohd_ctx* ctx, const float* X, const int64_t* nX_dev, int64_t nX_max,
                                   const float* Y, const int64_t* nY_dev, int64_t nY, int D, int precision,
                                   const int32_t* map, PruneLayout& L, int dir, prohd_hd_result* r, int* status,
                                   char* wsb, size_t ws_bytes, int64_t timeout_ns, cudaStream_t st) {
  const int nsm = ctx->num_sms;
  auto phase = [&]() {
    Arena t;
    t.base = wsb;
    t.cap = ws_bytes;
    t.off = L.mark;
    return t;
  };
  if (nX_max <= kPruneSample || nY < kPruneMinRows || (double)nX_max * (double)nY < ctx->prune_min_pairs) {
    // every row is kept
    cudaError_t e0 = cudaMemcpyAsync(L.nkeep, nX_dev, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
    if (e0) return e0;
    Arena t = phase();
    return hd_core(ctx, X, nX_dev, nX_max, Y, nY_dev, nY, D, precision, map, nullptr, r, status, t, timeout_ns, st,
                   true);
  }
  const int64_t S = kPruneSample;
  const int64_t nYp = prune_prefix(nY);
  // rows of X (by index) against all of Y; few rows: the contraction cuts
  // the columns into segments so that every SM works
  auto exact_rows = [&](const int32_t* idx, const int32_t* idx_map, const int64_t* n_dev, int64_t n_max, float* rows,
                        prohd_hd_result* res) {
    cudaError_t e2 = gather_rows(X, D, idx, n_dev, n_max, rows, nsm, st);
    if (e2) return e2;
    Arena t = phase();
    return hd_core(ctx, rows, n_dev, n_max, Y, nY_dev, nY, D, precision, idx_map, nullptr, res, status, t,
                   timeout_ns, st, true, &L.Ysh);
  };
  auto keep = [&](const double* lb2) {
    count_launch();
    keep_mask_kernel<<<nsm * 2, 256, 0, st>>>(L.hi, nX_dev, nX_max, &L.rs[dir].h_ab, lb2, kPruneScale, L.mask);
    cudaError_t e2 = cudaGetLastError();
    return e2 ? e2 : mask_to_indices(L.mask, nX_max, L.kidx, L.nkeep, L.counts, L.offsets, st);
  };
  cudaError_t e = set_i64(L.nYp, nYp, st);
  // Y's rounded copy once for every pass of this direction, with a shift and
  // scale that cover all rows of X
  if (!e) e = hd_shared_prepare(ctx, X, nX_dev, Y, nY_dev, D, precision, L.Ysh, status, st);
  if (!e) {
    count_launch();
    strided_dev_kernel<<<1, 1024, 0, st>>>(L.sidx, L.nS, S, nX_dev);
    e = cudaGetLastError();
  }
  if (!e) e = exact_rows(L.sidx, nullptr, L.nS, S, L.Xs, L.rs + dir);  // LB1
  if (!e) {
    Arena t = phase();
    e = hd_prefix_upper(ctx, X, nX_dev, nX_max, Y, L.nYp, nYp, D, precision, L.hi, status, t, timeout_ns, st,
                        &L.Ysh);
  }
  if (!e) e = keep(nullptr);
  if (!e) {
    count_launch();
    strided_sub_kernel<<<1, 1024, 0, st>>>(L.sidx, L.nS, S, L.kidx, L.nkeep);
    e = cudaGetLastError();
  }
  if (!e) e = exact_rows(L.sidx, nullptr, L.nS, S, L.Xs, L.rs + 2 + dir);  // LB2
  if (!e) e = keep(&L.rs[2 + dir].h_ab);
  const int32_t* final_map = L.kidx;
  if (!e && map) {
    count_launch();
    compose_idx_kernel<<<nsm * 2, 256, 0, st>>>(L.kmap, L.kidx, map, L.nkeep);
    e = cudaGetLastError();
    final_map = L.kmap;
  }
  if (!e) e = exact_rows(L.kidx, final_map, L.nkeep, nX_max, L.Xk, r);
  return e;
}

// ---------------------------------------------------------------- layouts

namespace {

struct HdLayout {
  int* status;
  int64_t *nA, *nB;
};
void hd_layout(Arena& a, int64_t nA, int64_t nB, int D, int precision, HdLayout& L) {
  L.status = a.take<int>(8);
  L.nA = a.take<int64_t>(1);
  L.nB = a.take<int64_t>(1);
  hd_core_layout(a, nA, nB, D, precision);
}

struct EstLayout {
  int* status;
  double* dirs;
  double* eig;
  int32_t *idxA, *idxB;
  int64_t *nselA, *nselB;
  float *As, *Bs;
  int64_t boundA, boundB;
  int nd;
  int64_t kA[64], kB[64];
  size_t mark_dir, mark_sel, mark_hd;  // arena offsets where each phase's scratch starts
  // one-sided refinement: full-set sizes on the device and the two directed results
  bool refine = false, refine_pruned = false;
  bool prune_sub = false;  // the subset distance may take the pruned form
  int64_t *nA_full = nullptr, *nB_full = nullptr;
  prohd_hd_result *r1 = nullptr, *r2 = nullptr;
  PruneLayout P;  // the refinement's row pruning (tensor-core precisions)
  const InputFeed* feed = nullptr;  // host-buffer entry: inputs landing in row ranges
  // the union centroid (from the covariance pass) and max |x - centroid| over
  // the gathered subsets: the subset distance's centre and scale
  float* center = nullptr;
  float* gmax = nullptr;
};

// Layout of an estimate with nd directions and the given k lists; m_dirs >= 0
// reserves the directions phase's scratch (m_dirs components), -1 skips it.
void est_layout_k(Arena& a, int64_t nA, int64_t nB, int D, int nd, const int64_t* kA, const int64_t* kB,
                  int precision, int m_dirs, EstLayout& L, bool refine = false, int gram_parts = 1) {
  L.nd = nd;
  for (int d = 0; d < nd; ++d) {
    L.kA[d] = kA[d];
    L.kB[d] = kB[d];
  }
  L.boundA = subset_bound(nA, L.nd, L.kA);
  L.boundB = subset_bound(nB, L.nd, L.kB);
  L.status = a.take<int>(8);
  L.dirs = a.take<double>((size_t)L.nd * D);
  L.eig = a.take<double>((size_t)std::max(m_dirs, 1));
  L.idxA = a.take<int32_t>((size_t)nA);
  L.idxB = a.take<int32_t>((size_t)nB);
  L.nselA = a.take<int64_t>(1);
  L.nselB = a.take<int64_t>(1);
  L.As = a.take<float>((size_t)L.boundA * D);
  L.Bs = a.take<float>((size_t)L.boundB * D);
  L.center = a.take<float>((size_t)D);
  L.gmax = a.take<float>(1);
  L.refine = refine;
  L.refine_pruned = refine && precision != PROHD_FP32;
  if (refine) {
    L.nA_full = a.take<int64_t>(1);
    L.nB_full = a.take<int64_t>(1);
    L.r1 = a.take<prohd_hd_result>(1);
    L.r2 = a.take<prohd_hd_result>(1);
  }
  if (L.refine_pruned) {
    // its buffers and its own scratch, ahead of the phases' shared region
    const int64_t nX[2] = {L.boundA, L.boundB}, nY[2] = {nB, nA};
    prune_layout(a, nX, nY, D, precision, L.P);
  }
  // the phases run one after another and share the rest of the arena
  const size_t start = a.off;
  size_t end = start;
  L.mark_dir = L.mark_sel = L.mark_hd = (start + 255) / 256 * 256;
  Arena t = a;
  if (m_dirs >= 0) {
    directions_layout(t, nA, nB, D, m_dirs, gram_parts);
    end = std::max(end, t.off);
  }
  t = a;
  select_layout(t, nA, nB, D, L.nd);
  end = std::max(end, t.off);
  t = a;
  hd_core_pruned_layout(t, L.boundA, L.boundB, D, precision);
  L.prune_sub = hd_subset_prunable(L.boundA, L.boundB, D, precision);
  end = std::max(end, t.off);
  if (refine && !L.refine_pruned) {
    // h(A_sel, B) then h(B_sel, A): one after the other in the same region
    t = a;
    hd_core_layout(t, L.boundA, nB, D, precision);
    end = std::max(end, t.off);
    t = a;
    hd_core_layout(t, L.boundB, nA, D, precision);
    end = std::max(end, t.off);
  }
  a.off = end;
}

void est_layout(Arena& a, int64_t nA, int64_t nB, int D, const prohd_params* p, EstLayout& L, int gram_parts = 1) {
  const int m = resolve_m(p, D);
  const int nd = 1 + m;
  const double ap = resolve_alpha_p(p, m);
  int64_t kA[64], kB[64];
  k_list(nA, nd, p->alpha_c, ap, kA);
  k_list(nB, nd, p->alpha_c, ap, kB);
  est_layout_k(a, nA, nB, D, nd, kA, kB, p->precision, m, L, p->refine != 0, gram_parts);
}

// Row ranges per set in which prohd_estimate_host copies its inputs: where
// the tensor-core Gram runs and both sets are large, its launch over each
// range overlaps the copies of the later ranges (2 ranges from 131,072 rows
// per set, 4 from 524,288).
int host_parts(int64_t nA, int64_t nB, int D) {
  if (!gram_tc_supported(D)) return 1;
  const int64_t n = std::min(nA, nB);
  return n >= 524288 ? 4 : (n >= 131072 ? 2 : 1);
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

prohd_status prohd_create(prohd_ctx** out) {
  if (!out) return PROHD_EINVAL;
  *out = nullptr;
  prohd_ctx* c = new (std::nothrow) prohd_ctx();
  if (!c) return PROHD_ENOMEM;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, c->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (e != cudaSuccess) {
    delete c;
    return PROHD_ECUDA;
  }
  if (c->cc_major != 10 || c->cc_minor != 3) {
    delete c;
    return PROHD_ENOTSUP;  // the library is built for sm_103a only
  }
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    c->encode_tiled = fn;
  *out = c;
  return PROHD_OK;
}

void prohd_destroy(prohd_ctx* ctx) {
  if (!ctx) return;
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->feed_start) cudaEventDestroy(ctx->feed_start);
  for (cudaEvent_t ev : ctx->feed_ready)
    if (ev) cudaEventDestroy(ev);
  for (auto& p : ctx->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  delete ctx;
}

const char* prohd_last_error(const prohd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void prohd_params_default(prohd_params* p) {
  if (!p) return;
  *p = prohd_params{};
  p->m = -1;
  p->precision = PROHD_FP16;
  p->alpha_c = 0.01;
  p->alpha_p = -1.0;
  p->power_max_iters = 96;
  p->power_tol = 1e-13;
  p->seed = 0;
  p->wait_timeout_ns = kDefaultTimeoutNs;
}

int64_t prohd_k_of(double alpha, int64_t n) {
  int64_t k = (int64_t)floor(alpha * (double)n);
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

size_t hausdorff_exact_workspace_size(int64_t nA, int64_t nB, int D, int precision) {
  if (bad_n(nA) || bad_n(nB) || D < 1) return 0;
  Arena a;
  HdLayout L;
  hd_layout(a, nA, nB, D, precision, L);
  return a.off + 256;
}

size_t prohd_directions_workspace_size(int64_t nA, int64_t nB, int D, int m) {
  Arena a;
  a.take<int>(8);
  directions_layout(a, nA, nB, D, m < 0 ? (int)floor(sqrt((double)D)) : m);
  return a.off + 256;
}

size_t prohd_select_workspace_size(int64_t nA, int64_t nB, int D, int ndirs) {
  if (bad_n(nA) || bad_n(nB) || ndirs < 1) return 0;
  Arena a;
  a.take<int>(8);
  select_layout(a, nA, nB, D, ndirs);
  return a.off + 256;
}

size_t prohd_estimate_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p) {
  if (!p || bad_n(nA) || bad_n(nB) || D < 1) return 0;
  Arena a;
  EstLayout L;
  est_layout(a, nA, nB, D, p, L);
  return a.off + 256;
}

size_t prohd_estimate_host_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p) {
  if (!p || bad_n(nA) || bad_n(nB) || D < 1) return 0;
  Arena a;
  a.take<float>((size_t)nA * D);
  a.take<float>((size_t)nB * D);
  a.take<prohd_result>(1);
  const size_t base = a.off;
  Arena b;
  EstLayout L;
  est_layout(b, nA, nB, D, p, L, host_parts(nA, nB, D));
  return base + b.off + 512;
}

prohd_status hausdorff_exact(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                             int precision, prohd_hd_result* out, void* ws, size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!out) return fail(ctx, PROHD_EINVAL, "null output%s");
  if (precision != PROHD_FP32 && precision != PROHD_FP16 && precision != PROHD_BF16)
    return fail(ctx, PROHD_EINVAL, "unknown precision%s");
  if (precision != PROHD_FP32 && !tc_supported_dim(D))
    return fail(ctx, PROHD_ENOTSUP, "tensor-core precisions need D <= 256 (use PROHD_FP32)%s");
  if ((s = check_ws(ctx, ws, ws_bytes, hausdorff_exact_workspace_size(nA, nB, D, precision)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  HdLayout L;
  hd_layout(a, nA, nB, D, precision, L);
  Arena run;  // hd_core re-derives its buffers from the same offsets
  run.base = static_cast<char*>(ws);
  run.cap = ws_bytes;
  run.take<int>(8);
  run.take<int64_t>(1);
  run.take<int64_t>(1);
  cudaError_t e = zero_i32(L.status, 8, st);
  if (!e) e = set_i64(L.nA, nA, st);
  if (!e) e = set_i64(L.nB, nB, st);
  if (!e) e = hd_core(ctx, A, L.nA, nA, B, L.nB, nB, D, precision, nullptr, nullptr, out, L.status, run,
                      kDefaultTimeoutNs, st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_directions(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                              const prohd_params* p, double* dirs, double* eig, void* ws, size_t ws_bytes,
                              void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!p) return fail(ctx, PROHD_EINVAL, "null params%s");
  if (!dirs) return fail(ctx, PROHD_EINVAL, "null dirs%s");
  const int m = resolve_m(p, D);
  if (m < 0 || m > D || m > 63) return fail(ctx, PROHD_EINVAL, "m must be in [0, min(D, 63)]%s");
  if (p->power_max_iters < 1) return fail(ctx, PROHD_EINVAL, "power_max_iters must be >= 1%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_directions_workspace_size(nA, nB, D, m)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  int* status = a.take<int>(8);
  cudaError_t e = zero_i32(status, 8, st);
  if (!e)
    e = directions_run(ctx, A, nA, B, nB, D, m, p->power_max_iters, p->power_tol, p->seed, dirs, eig, status, a, st,
                       p->wait_timeout_ns);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

size_t prohd_covariance_workspace_size(int64_t nA, int64_t nB, int D) {
  if (bad_n(nA) || bad_n(nB) || D < 1) return 0;
  Arena a;
  a.take<int>(8);
  covariance_layout(a, D);
  return a.off + 256;
}

prohd_status prohd_covariance(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                              double* C, double* mean, void* ws, size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!C) return fail(ctx, PROHD_EINVAL, "null C%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_covariance_workspace_size(nA, nB, D)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  int* status = a.take<int>(8);
  cudaError_t e = zero_i32(status, 8, st);
  if (!e) e = covariance_run(ctx, A, nA, B, nB, D, C, mean, status, a, st, kDefaultTimeoutNs);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_select(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                          const double* dirs, int ndirs, const int64_t* kA, const int64_t* kB, int32_t* idxA,
                          int64_t* nselA, int32_t* idxB, int64_t* nselB, void* ws, size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!dirs || ndirs < 1 || ndirs > 64) return fail(ctx, PROHD_EINVAL, "need 1..64 directions%s");
  if (!kA || !kB) return fail(ctx, PROHD_EINVAL, "null k lists%s");
  for (int d = 0; d < ndirs; ++d)
    if (kA[d] < 1 || kB[d] < 1) return fail(ctx, PROHD_EINVAL, "k must be >= 1%s");
  if (!idxA || !idxB || !nselA || !nselB) return fail(ctx, PROHD_EINVAL, "null output%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_select_workspace_size(nA, nB, D, ndirs)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  int* status = a.take<int>(8);
  cudaError_t e = zero_i32(status, 8, st);
  if (!e) e = select_run(ctx, A, nA, B, nB, D, dirs, ndirs, kA, kB, idxA, nselA, idxB, nselB, status, a, st,
                         kDefaultTimeoutNs);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

// One-sided refinement after the selection and gather: h(A_sel, B) and
// h(B_sel, A) on the original sets, then their maximum into out->hd (whose
// status field must hold the earlier stages' status, or 0).
static cudaError_t refine_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                              const prohd_params* p, EstLayout& L, prohd_result* out, char* wsb, size_t ws_bytes,
                              cudaStream_t st) {
  Arena t;
  t.base = wsb;
  t.cap = ws_bytes;
  t.off = L.mark_hd;
  const int64_t to = p->wait_timeout_ns > 0 ? p->wait_timeout_ns : kDefaultTimeoutNs;
  cudaError_t e = set_i64(L.nA_full, nA, st);
  if (!e) e = set_i64(L.nB_full, nB, st);
  if (L.refine_pruned) {
    // the same two directed distances with row pruning (equal results)
    if (!e)
      e = pruned_directed(ctx, L.As, L.nselA, L.boundA, B, L.nB_full, nB, D, p->precision, L.idxA, L.P, 0, L.r1,
                          L.status, wsb, ws_bytes, to, st);
    if (!e)
      e = pruned_directed(ctx, L.Bs, L.nselB, L.boundB, A, L.nA_full, nA, D, p->precision, L.idxB, L.P, 1, L.r2,
                          L.status, wsb, ws_bytes, to, st);
    if (!e) {
      count_launch();
      refine_combine_kernel<<<1, 1, 0, st>>>(L.r1, L.r2, out);
      e = cudaGetLastError();
    }
    return e;
  }
  if (!e)
    e = hd_core(ctx, L.As, L.nselA, L.boundA, B, L.nB_full, nB, D, p->precision, L.idxA, nullptr, L.r1, L.status, t,
                to, st);
  t.off = L.mark_hd;
  if (!e)
    e = hd_core(ctx, L.Bs, L.nselB, L.boundB, A, L.nA_full, nA, D, p->precision, L.idxB, nullptr, L.r2, L.status, t,
                to, st);
  if (!e) {
    count_launch();
    refine_combine_kernel<<<1, 1, 0, st>>>(L.r1, L.r2, out);
    e = cudaGetLastError();
  }
  return e;
}

// given_dirs: the caller's directions (nd = L.nd) replace the directions phase.
static prohd_status estimate_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                 const prohd_params* p, EstLayout& L, prohd_result* out, int32_t* idxA,
                                 int32_t* idxB, double* dirs, const double* given_dirs, char* wsb, size_t ws_bytes,
                                 cudaStream_t st) {
  if (idxA) L.idxA = idxA;
  if (idxB) L.idxB = idxB;
  if (dirs) L.dirs = dirs;
  const int m = L.nd - 1;
  auto phase = [&](size_t mark) {
    Arena t;
    t.base = wsb;
    t.cap = ws_bytes;
    t.off = mark;
    return t;
  };
  cudaError_t e = zero_i32(L.status, 8, st);
  const double* use_dirs = given_dirs ? given_dirs : L.dirs;
  if (!e && !given_dirs) {
    Arena t = phase(L.mark_dir);
    e = directions_run(ctx, A, nA, B, nB, D, m, p->power_max_iters, p->power_tol, p->seed, L.dirs, L.eig, L.status, t, st,
                       p->wait_timeout_ns, L.feed, L.center, L.gmax);
  }
  if (!e) {
    Arena t = phase(L.mark_sel);
    e = select_run(ctx, A, nA, B, nB, D, use_dirs, L.nd, L.kA, L.kB, L.idxA, L.nselA, L.idxB, L.nselB, L.status, t,
                   st, p->wait_timeout_ns);
  }
  // with the directions computed here, the gather also takes the subset
  // distance's scale about the union centroid (no centring passes later)
  const bool centred = !given_dirs && p->precision != PROHD_FP32;
  const HdCenter hc{L.center, L.gmax};
  {
    PhaseTimer pt(ctx, PROHD_PH_GATHER, st);
    if (centred) {
      if (!e) e = gather_rows_center(A, D, L.idxA, L.nselA, L.boundA, L.As, L.center, L.gmax, L.status, ctx->num_sms, st);
      if (!e) e = gather_rows_center(B, D, L.idxB, L.nselB, L.boundB, L.Bs, L.center, L.gmax, L.status, ctx->num_sms, st);
    } else {
      if (!e) e = gather_rows(A, D, L.idxA, L.nselA, L.boundA, L.As, ctx->num_sms, st);
      if (!e) e = gather_rows(B, D, L.idxB, L.nselB, L.boundB, L.Bs, ctx->num_sms, st);
    }
  }
  if (!e) {
    Arena t = phase(L.mark_hd);
    const int64_t to = p->wait_timeout_ns > 0 ? p->wait_timeout_ns : kDefaultTimeoutNs;
    // the same result; the pruned form leaves out the subset rows that
    // cannot attain either directed maximum
    if (L.prune_sub && (double)L.boundA * (double)L.boundB >= ctx->subset_prune_min_pairs)
      e = hd_core_pruned(ctx, L.As, L.nselA, L.boundA, L.Bs, L.nselB, L.boundB, D, p->precision, L.idxA, L.idxB,
                         &out->hd, L.status, t, to, st, centred ? &hc : nullptr);
    else
      e = hd_core(ctx, L.As, L.nselA, L.boundA, L.Bs, L.nselB, L.boundB, D, p->precision, L.idxA, L.idxB, &out->hd,
                  L.status, t, to, st, false, nullptr, centred ? &hc : nullptr);
  }
  if (!e && L.refine) e = refine_run(ctx, A, nA, B, nB, D, p, L, out, wsb, ws_bytes, st);
  if (!e) {
    count_launch();
    finish_estimate_kernel<<<1, 1, 0, st>>>(out, L.nselA, L.nselB);
    e = cudaGetLastError();
  }
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

static prohd_status estimate_impl(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                  const prohd_params* p, prohd_result* out, int32_t* idxA, int32_t* idxB,
                                  double* dirs, char* wsb, size_t ws_bytes, cudaStream_t st,
                                  const InputFeed* feed = nullptr) {
  Arena a;
  a.base = wsb;
  a.cap = ws_bytes;
  EstLayout L;
  est_layout(a, nA, nB, D, p, L, feed ? feed->parts : 1);
  L.feed = feed;
  if (a.overflow()) return fail(ctx, PROHD_ENOMEM, "workspace too small%s");
  return estimate_run(ctx, A, nA, B, nB, D, p, L, out, idxA, idxB, dirs, nullptr, wsb, ws_bytes, st);
}

prohd_status prohd_estimate(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                            const prohd_params* p, prohd_result* out, int32_t* idxA, int32_t* idxB, double* dirs,
                            void* ws, size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if ((s = check_params(ctx, p, D))) return s;
  if (!out) return fail(ctx, PROHD_EINVAL, "null output%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_estimate_workspace_size(nA, nB, D, p)))) return s;
  return estimate_impl(ctx, A, nA, B, nB, D, p, out, idxA, idxB, dirs, static_cast<char*>(ws), ws_bytes,
                       reinterpret_cast<cudaStream_t>(stream));
}

prohd_status prohd_estimate_host(prohd_ctx* ctx, const float* A_host, int64_t nA, const float* B_host, int64_t nB,
                                 int D, const prohd_params* p, prohd_result* out_host, void* ws, size_t ws_bytes,
                                 void* stream) {
  prohd_status s = check_sets(ctx, A_host, nA, B_host, nB, D);
  if (s) return s;
  if ((s = check_params(ctx, p, D))) return s;
  if (!out_host) return fail(ctx, PROHD_EINVAL, "null output%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_estimate_host_workspace_size(nA, nB, D, p)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  float* Ad = a.take<float>((size_t)nA * D);
  float* Bd = a.take<float>((size_t)nB * D);
  prohd_result* od = a.take<prohd_result>(1);
  const size_t base = (a.off + 255) / 256 * 256;
  // the copies run on the context's copy stream, in row ranges, each range's
  // event recorded behind it; the Gram waits for each range before reading it
  // (overlapping the later copies), and every later step runs after the Gram
  const int parts = host_parts(nA, nB, D);
  cudaError_t e = cudaSuccess;
  if (!ctx->copy_stream) {
    e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&ctx->feed_start, cudaEventDisableTiming);
    for (int i = 0; i < 8 && !e; ++i) e = cudaEventCreateWithFlags(&ctx->feed_ready[i], cudaEventDisableTiming);
    if (e) return cuda_fail(ctx, e);
  }
  cudaStream_t cs = ctx->copy_stream;
  // the copies may overwrite the workspace only after the stream's earlier work
  if (!e) e = cudaEventRecord(ctx->feed_start, st);
  if (!e) e = cudaStreamWaitEvent(cs, ctx->feed_start, 0);
  for (int set = 0; set < 2 && !e; ++set) {
    const int64_t n = set ? nB : nA;
    const float* src = set ? B_host : A_host;
    float* dst = set ? Bd : Ad;
    for (int k = 0; k < parts && !e; ++k) {
      const int64_t r0 = n * k / parts, r1 = n * (k + 1) / parts;
      e = cudaMemcpyAsync(dst + r0 * D, src + r0 * D, sizeof(float) * (size_t)(r1 - r0) * D, cudaMemcpyHostToDevice,
                          cs);
      if (!e) e = cudaEventRecord(ctx->feed_ready[set * parts + k], cs);
    }
  }
  if (e) return cuda_fail(ctx, e);
  InputFeed feed;
  feed.parts = parts;
  feed.ready = ctx->feed_ready;
  s = estimate_impl(ctx, Ad, nA, Bd, nB, D, p, od, nullptr, nullptr, nullptr, static_cast<char*>(ws) + base,
                    ws_bytes - base, st, &feed);
  // the stream holds the copies whatever happened above
  e = cudaStreamWaitEvent(st, ctx->feed_ready[2 * parts - 1], 0);
  if (s) return s;
  if (e) return cuda_fail(ctx, e);
  e = cudaMemcpyAsync(out_host, od, sizeof(prohd_result), cudaMemcpyDeviceToHost, st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_profile_enable(prohd_ctx* ctx, int on) {
  if (!ctx) return PROHD_EINVAL;
  ctx->profiling = on != 0;
  return PROHD_OK;
}

prohd_status prohd_profile_read(prohd_ctx* ctx, double* ms, int64_t* count, int reset) {
  if (!ctx) return PROHD_EINVAL;
  for (auto& p : ctx->pending) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ctx->ph_ms[p.phase] += t;
      ctx->ph_count[p.phase] += 1;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  ctx->pending.clear();
  for (int i = 0; i < PROHD_PH_COUNT; ++i) {
    if (ms) ms[i] = ctx->ph_ms[i];
    if (count) count[i] = ctx->ph_count[i];
    if (reset) {
      ctx->ph_ms[i] = 0.0;
      ctx->ph_count[i] = 0;
    }
  }
  return PROHD_OK;
}

// ---------------------------------------------------------------- estimate with given directions

static prohd_status check_klist(prohd_ctx* ctx, int nd, const int64_t* kA, const int64_t* kB) {
  if (nd < 1 || nd > 64) return fail(ctx, PROHD_EINVAL, "need 1..64 directions%s");
  if (!kA || !kB) return fail(ctx, PROHD_EINVAL, "null k lists%s");
  for (int d = 0; d < nd; ++d)
    if (kA[d] < 1 || kB[d] < 1) return fail(ctx, PROHD_EINVAL, "k must be >= 1%s");
  return PROHD_OK;
}

size_t prohd_estimate_dirs_workspace_size(int64_t nA, int64_t nB, int D, int nd, const int64_t* kA, const int64_t* kB,
                                          const prohd_params* p) {
  if (nd < 1 || nd > 64 || !kA || !kB || !p) return 0;
  Arena a;
  EstLayout L;
  est_layout_k(a, nA, nB, D, nd, kA, kB, p->precision, -1, L, p->refine != 0);
  return a.off + 256;
}

prohd_status prohd_estimate_dirs(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                 const prohd_params* p, const double* dirs, int nd, const int64_t* kA,
                                 const int64_t* kB, prohd_result* out, int32_t* idxA, int32_t* idxB, void* ws,
                                 size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if ((s = check_params(ctx, p, D))) return s;
  if (!dirs) return fail(ctx, PROHD_EINVAL, "null dirs%s");
  if ((s = check_klist(ctx, nd, kA, kB))) return s;
  if (!out) return fail(ctx, PROHD_EINVAL, "null output%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_estimate_dirs_workspace_size(nA, nB, D, nd, kA, kB, p)))) return s;
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  EstLayout L;
  est_layout_k(a, nA, nB, D, nd, kA, kB, p->precision, -1, L, p->refine != 0);
  return estimate_run(ctx, A, nA, B, nB, D, p, L, out, idxA, idxB, nullptr, dirs, static_cast<char*>(ws), ws_bytes,
                      reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------- exact distance with row pruning

// the pruned layout (workspace) applies by the row counts alone; whether a
// call prunes also depends on the context's pair threshold
static bool prune_applies(int64_t nA, int64_t nB, int precision) {
  return precision != PROHD_FP32 && nA >= kPruneMinRows && nB >= kPruneMinRows;
}

namespace {
struct ExactPruneLayout {
  int* status;
  int64_t *nA, *nB;
  int64_t* kept;        // [2]: rows kept per direction
  prohd_hd_result* rk;  // [2]: h(A, B), h(B, A)
  PruneLayout P;
};
void exact_prune_layout(Arena& a, int64_t nA, int64_t nB, int D, int precision, ExactPruneLayout& L) {
  L.status = a.take<int>(8);
  L.nA = a.take<int64_t>(1);
  L.nB = a.take<int64_t>(1);
  L.kept = a.take<int64_t>(2);
  L.rk = a.take<prohd_hd_result>(2);
  const int64_t nX[2] = {nA, nB}, nY[2] = {nB, nA};
  prune_layout(a, nX, nY, D, precision, L.P);
}
}  // namespace

size_t hausdorff_exact_pruned_workspace_size(int64_t nA, int64_t nB, int D, int precision) {
  if (bad_n(nA) || bad_n(nB) || D < 1) return 0;
  if (!prune_applies(nA, nB, precision)) return hausdorff_exact_workspace_size(nA, nB, D, precision);
  Arena a;
  ExactPruneLayout L;
  exact_prune_layout(a, nA, nB, D, precision, L);
  return a.off + 256;
}

prohd_status hausdorff_exact_pruned(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                    int precision, prohd_hd_result* out, int64_t* kept, void* ws, size_t ws_bytes,
                                    void* stream) {
  if (!prune_applies(nA, nB, precision) || (ctx && (double)nA * (double)nB < ctx->prune_min_pairs)) {
    if (kept) kept[0] = kept[1] = -1;
    return hausdorff_exact(ctx, A, nA, B, nB, D, precision, out, ws, ws_bytes, stream);
  }
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!out) return fail(ctx, PROHD_EINVAL, "null output%s");
  if (precision != PROHD_FP16 && precision != PROHD_BF16) return fail(ctx, PROHD_EINVAL, "unknown precision%s");
  if (!tc_supported_dim(D)) return fail(ctx, PROHD_ENOTSUP, "tensor-core precisions need D <= 256 (use PROHD_FP32)%s");
  if ((s = check_ws(ctx, ws, ws_bytes, hausdorff_exact_pruned_workspace_size(nA, nB, D, precision)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  Arena a;
  a.base = wsb;
  a.cap = ws_bytes;
  ExactPruneLayout L;
  exact_prune_layout(a, nA, nB, D, precision, L);
  if (a.overflow()) return fail(ctx, PROHD_ENOMEM, "workspace too small%s");
  cudaError_t e = zero_i32(L.status, 8, st);
  if (!e) e = set_i64(L.nA, nA, st);
  if (!e) e = set_i64(L.nB, nB, st);
  // kept-row counts: each direction's count is copied (device to device)
  // before the next direction reuses the pruning buffers, and read back once
  for (int dir = 0; dir < 2 && !e; ++dir) {
    e = dir == 0 ? pruned_directed(ctx, A, L.nA, nA, B, L.nB, nB, D, precision, nullptr, L.P, 0, L.rk, L.status, wsb,
                                   ws_bytes, kDefaultTimeoutNs, st)
                 : pruned_directed(ctx, B, L.nB, nB, A, L.nA, nA, D, precision, nullptr, L.P, 1, L.rk + 1, L.status,
                                   wsb, ws_bytes, kDefaultTimeoutNs, st);
    if (!e && kept) e = cudaMemcpyAsync(L.kept + dir, L.P.nkeep, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  }
  if (!e) {
    count_launch();
    directed_combine_kernel<<<1, 1, 0, st>>>(L.rk, L.rk + 1, out);
    e = cudaGetLastError();
  }
  if (kept) {
    int64_t keep_host[2] = {-1, -1};
    if (!e) e = cudaMemcpyAsync(keep_host, L.kept, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    kept[0] = e ? -1 : keep_host[0];
    kept[1] = e ? -1 : keep_host[1];
  }
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_set_prune_min_pairs(prohd_ctx* ctx, double min_pairs) {
  if (!ctx) return PROHD_EINVAL;
  if (!(min_pairs >= 0.0)) return fail(ctx, PROHD_EINVAL, "min_pairs must be >= 0%s");
  ctx->prune_min_pairs = min_pairs;
  return PROHD_OK;
}

prohd_status prohd_set_subset_prune_min_pairs(prohd_ctx* ctx, double min_pairs) {
  if (!ctx) return PROHD_EINVAL;
  if (!(min_pairs >= 0.0)) return fail(ctx, PROHD_EINVAL, "min_pairs must be >= 0%s");
  ctx->subset_prune_min_pairs = min_pairs;
  return PROHD_OK;
}

// ---------------------------------------------------------------- adaptive alpha

// number of doublings the schedule can take: the largest t with alpha_c 2^t <= alpha_max
static int adaptive_last_step(double alpha_c, double alpha_max) {
  int t = 0;
  while (t + 1 < PROHD_ADAPT_MAX_STEPS && alpha_c * ldexp(1.0, t + 1) <= alpha_max) ++t;
  return t;
}

static bool adaptive_layout(Arena& a, int64_t nA, int64_t nB, int D, const prohd_params* p, double alpha_max,
                            EstLayout& L) {
  const int m = resolve_m(p, D);
  const int nd = 1 + m;
  const double ap = resolve_alpha_p(p, m);
  const double sc = ldexp(1.0, adaptive_last_step(p->alpha_c, alpha_max));
  int64_t kA[64], kB[64];
  k_list(nA, nd, p->alpha_c * sc, ap * sc, kA);
  k_list(nB, nd, p->alpha_c * sc, ap * sc, kB);
  est_layout_k(a, nA, nB, D, nd, kA, kB, p->precision, m, L, true);
  return true;
}

size_t prohd_estimate_adaptive_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p,
                                              double alpha_max) {
  if (!p || !(p->alpha_c > 0.0) || !(alpha_max >= p->alpha_c)) return 0;
  Arena a;
  EstLayout L;
  adaptive_layout(a, nA, nB, D, p, alpha_max, L);
  return a.off + 256;
}

prohd_status prohd_estimate_adaptive(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                     const prohd_params* p, double alpha_max, double rel_tol, prohd_result* out,
                                     prohd_adaptive_info* info, int32_t* idxA, int32_t* idxB, double* dirs,
                                     void* ws, size_t ws_bytes, void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if ((s = check_params(ctx, p, D))) return s;
  if (!(alpha_max >= p->alpha_c && alpha_max < 1.0))
    return fail(ctx, PROHD_EINVAL, "alpha_max must be in [alpha_c, 1)%s");
  if (!(rel_tol >= 0.0)) return fail(ctx, PROHD_EINVAL, "rel_tol must be >= 0%s");
  if (!out || !info) return fail(ctx, PROHD_EINVAL, "null output%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_estimate_adaptive_workspace_size(nA, nB, D, p, alpha_max)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  Arena a;
  a.base = wsb;
  a.cap = ws_bytes;
  EstLayout L;
  adaptive_layout(a, nA, nB, D, p, alpha_max, L);
  if (a.overflow()) return fail(ctx, PROHD_ENOMEM, "workspace too small%s");
  if (idxA) L.idxA = idxA;
  if (idxB) L.idxB = idxB;
  if (dirs) L.dirs = dirs;
  const int m = L.nd - 1;
  const double ap = resolve_alpha_p(p, m);
  *info = prohd_adaptive_info{};
  auto phase = [&](size_t mark) {
    Arena t;
    t.base = wsb;
    t.cap = ws_bytes;
    t.off = mark;
    return t;
  };
  cudaError_t e = zero_i32(L.status, 8, st);
  if (!e) {
    Arena t = phase(L.mark_dir);
    e = directions_run(ctx, A, nA, B, nB, D, m, p->power_max_iters, p->power_tol, p->seed, L.dirs, L.eig, L.status, t,
                       st, p->wait_timeout_ns);
  }
  prohd_result h{};
  for (int step = 0; !e; ++step) {
    const double sc = ldexp(1.0, step);
    const double a_t = p->alpha_c * sc, ap_t = ap * sc;
    k_list(nA, L.nd, a_t, ap_t, L.kA);
    k_list(nB, L.nd, a_t, ap_t, L.kB);
    e = cudaMemsetAsync(out, 0, sizeof(prohd_result), st);
    if (!e) {
      Arena t = phase(L.mark_sel);
      e = select_run(ctx, A, nA, B, nB, D, L.dirs, L.nd, L.kA, L.kB, L.idxA, L.nselA, L.idxB, L.nselB, L.status, t,
                     st, p->wait_timeout_ns);
    }
    {
      PhaseTimer pt(ctx, PROHD_PH_GATHER, st);
      if (!e) e = gather_rows(A, D, L.idxA, L.nselA, L.boundA, L.As, ctx->num_sms, st);
      if (!e) e = gather_rows(B, D, L.idxB, L.nselB, L.boundB, L.Bs, ctx->num_sms, st);
    }
    if (!e) e = refine_run(ctx, A, nA, B, nB, D, p, L, out, wsb, ws_bytes, st);
    if (!e) {
      count_launch();
      finish_estimate_kernel<<<1, 1, 0, st>>>(out, L.nselA, L.nselB);
      e = cudaGetLastError();
    }
    // the stop decision needs this step's result on the host
    if (!e) e = cudaMemcpyAsync(&h, out, sizeof(prohd_result), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) break;
    info->steps = step + 1;
    info->alpha_c = a_t;
    info->alpha_p = ap_t;
    info->H[step] = h.hd.H;
    info->nsel_a[step] = h.nsel_a;
    info->nsel_b[step] = h.nsel_b;
    if (h.hd.status != PROHD_OK) break;  // reported through out
    if (h.nsel_a == nA && h.nsel_b == nB) {
      info->reason = PROHD_ADAPT_ALL;
      break;
    }
    if (step >= 1 && info->H[step] - info->H[step - 1] <= rel_tol * info->H[step]) {
      info->reason = PROHD_ADAPT_STABLE;
      break;
    }
    if (p->alpha_c * ldexp(1.0, step + 1) > alpha_max) {
      info->reason = PROHD_ADAPT_BUDGET;
      break;
    }
    if (step + 1 >= PROHD_ADAPT_MAX_STEPS) {
      info->reason = PROHD_ADAPT_STEPS;
      break;
    }
  }
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

// ---------------------------------------------------------------- learned directions

size_t prohd_features_workspace_size(int64_t nA, int64_t nB, int D) {
  Arena a;
  a.take<int>(8);
  directions_layout(a, nA, nB, D, 8);
  return a.off + 256;
}

prohd_status prohd_features(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                            const prohd_params* p, float* feat, double* dirs, double* eig, void* ws, size_t ws_bytes,
                            void* stream) {
  prohd_status s = check_sets(ctx, A, nA, B, nB, D);
  if (s) return s;
  if (!p || !feat || !dirs || !eig) return fail(ctx, PROHD_EINVAL, "null argument%s");
  if (D < 8) return fail(ctx, PROHD_EINVAL, "features need D >= 8 (8 components)%s");
  if (p->power_max_iters < 1) return fail(ctx, PROHD_EINVAL, "power_max_iters must be >= 1%s");
  if ((s = check_ws(ctx, ws, ws_bytes, prohd_features_workspace_size(nA, nB, D)))) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Arena a;
  a.base = static_cast<char*>(ws);
  a.cap = ws_bytes;
  int* status = a.take<int>(8);
  cudaError_t e = zero_i32(status, 8, st);
  if (!e) e = directions_features(ctx, A, nA, B, nB, D, p->power_max_iters, p->power_tol, p->seed, dirs, eig, feat,
                                  status, a, st, p->wait_timeout_ns);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

size_t prohd_mlp_param_count(int D) { return D >= 1 ? mlp_shape(D).nparam : 0; }
size_t prohd_mlp_state_bytes(int D) { return D >= 1 ? 3 * mlp_shape(D).nparam * sizeof(float) : 0; }
size_t prohd_mlp_scratch_bytes(int D, int batch) {
  return (D >= 1 && batch >= 1) ? mlp_scratch_floats(D, batch) * sizeof(float) + 256 : 0;
}

static prohd_status check_mlp(prohd_ctx* ctx, int D, int batch, int precision, const void* state, void* scratch,
                              size_t scratch_bytes) {
  if (!ctx) return PROHD_EINVAL;
  if (D < 8 || D > 1024) return fail(ctx, PROHD_EINVAL, "the network needs 8 <= D <= 1024%s");
  if (batch < 1 || batch > 65535) return fail(ctx, PROHD_EINVAL, "batch must be in [1, 65535]%s");
  if (precision != PROHD_FP32 && precision != PROHD_BF16)
    return fail(ctx, PROHD_EINVAL, "network precision is PROHD_FP32 or PROHD_BF16%s");
  if (!state) return fail(ctx, PROHD_EINVAL, "null state%s");
  if (scratch && ((reinterpret_cast<uintptr_t>(scratch) & 255) || scratch_bytes < prohd_mlp_scratch_bytes(D, batch)))
    return fail(ctx, PROHD_ENOMEM, "scratch too small or misaligned%s");
  if (!scratch) return fail(ctx, PROHD_EINVAL, "null scratch%s");
  return PROHD_OK;
}

prohd_status prohd_mlp_init(prohd_ctx* ctx, int D, uint64_t seed, void* state, void* stream) {
  if (!ctx) return PROHD_EINVAL;
  if (D < 8 || D > 1024 || !state) return fail(ctx, PROHD_EINVAL, "bad network arguments%s");
  cudaError_t e = mlp_init(mlp_shape(D), static_cast<float*>(state), seed, reinterpret_cast<cudaStream_t>(stream));
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_mlp_forward(prohd_ctx* ctx, int D, const void* state, const float* feat, int batch, int precision,
                               float* dirs32, double* dirs64, void* scratch, size_t scratch_bytes, void* stream) {
  prohd_status s = check_mlp(ctx, D, batch, precision, state, scratch, scratch_bytes);
  if (s) return s;
  if (!feat) return fail(ctx, PROHD_EINVAL, "null features%s");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const MlpShape sh = mlp_shape(D);
  float* sc = static_cast<float*>(scratch);
  cudaError_t e = mlp_forward(sh, static_cast<const float*>(state), feat, batch, precision, sc, nullptr, st);
  const MlpActsView v = mlp_acts_view(D, batch, sc);
  if (!e && dirs32)
    e = cudaMemcpyAsync(dirs32, v.u, sizeof(float) * (size_t)batch * sh.n_out, cudaMemcpyDeviceToDevice, st);
  if (!e && dirs64) e = mlp_dirs64(v.u, batch * 4, D, dirs64, st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_mlp_loss_grad(prohd_ctx* ctx, int D, const void* state, const float* feat, const float* label,
                                 int batch, int precision, float* loss, float* grad, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  prohd_status s = check_mlp(ctx, D, batch, precision, state, scratch, scratch_bytes);
  if (s) return s;
  if (!feat || !label) return fail(ctx, PROHD_EINVAL, "null features or labels%s");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const MlpShape sh = mlp_shape(D);
  float* sc = static_cast<float*>(scratch);
  const float* P = static_cast<const float*>(state);
  cudaError_t e = mlp_forward(sh, P, feat, batch, precision, sc, label, st);
  if (!e && grad) e = mlp_backward(sh, P, feat, batch, precision, sc, st);
  const MlpActsView v = mlp_acts_view(D, batch, sc);
  if (!e && loss) e = cudaMemcpyAsync(loss, v.lmean, sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (!e && grad) e = cudaMemcpyAsync(grad, v.grad, sizeof(float) * sh.nparam, cudaMemcpyDeviceToDevice, st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_mlp_train_step(prohd_ctx* ctx, int D, void* state, const float* feat, const float* label, int batch,
                                  int precision, float lr, int64_t step, float* loss, void* scratch,
                                  size_t scratch_bytes, void* stream) {
  prohd_status s = check_mlp(ctx, D, batch, precision, state, scratch, scratch_bytes);
  if (s) return s;
  if (!feat || !label) return fail(ctx, PROHD_EINVAL, "null features or labels%s");
  if (step < 1) return fail(ctx, PROHD_EINVAL, "step counts from 1%s");
  if (!(lr > 0.f)) return fail(ctx, PROHD_EINVAL, "learning rate must be positive%s");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const MlpShape sh = mlp_shape(D);
  float* sc = static_cast<float*>(scratch);
  float* P = static_cast<float*>(state);
  cudaError_t e = mlp_forward(sh, P, feat, batch, precision, sc, label, st);
  if (!e) e = mlp_backward(sh, P, feat, batch, precision, sc, st);
  const MlpActsView v = mlp_acts_view(D, batch, sc);
  if (!e) e = mlp_adam(sh, P, v.grad, lr, step, st);
  if (!e && loss) e = cudaMemcpyAsync(loss, v.lmean, sizeof(float), cudaMemcpyDeviceToDevice, st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

prohd_status prohd_mlp_adam_step(prohd_ctx* ctx, int D, void* state, const float* grad, float lr, int64_t step,
                                 void* stream) {
  if (!ctx) return PROHD_EINVAL;
  if (D < 8 || D > 1024 || !state || !grad) return fail(ctx, PROHD_EINVAL, "bad network arguments%s");
  if (step < 1) return fail(ctx, PROHD_EINVAL, "step counts from 1%s");
  if (!(lr > 0.f)) return fail(ctx, PROHD_EINVAL, "learning rate must be positive%s");
  cudaError_t e = mlp_adam(mlp_shape(D), static_cast<float*>(state), grad, lr, step,
                           reinterpret_cast<cudaStream_t>(stream));
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

// Checkpoint file: "PHDMLP01", int32 D, int64 step, int64 parameter count,
// int64 extra-byte count (all little-endian, unpadded), the extra bytes,
// then params | Adam m | Adam v as FP32.
static const char kMlpMagic[8] = {'P', 'H', 'D', 'M', 'L', 'P', '0', '1'};

prohd_status prohd_mlp_save(prohd_ctx* ctx, const char* path, int D, int64_t step, const void* state,
                            const void* extra, int64_t extra_bytes, void* stream) {
  if (!ctx) return PROHD_EINVAL;
  if (!path || D < 8 || D > 1024 || !state || step < 0 || extra_bytes < 0 || (extra_bytes > 0 && !extra))
    return fail(ctx, PROHD_EINVAL, "bad checkpoint arguments%s");
  const int64_t np = (int64_t)mlp_shape(D).nparam;
  std::vector<float> body((size_t)(3 * np));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(body.data(), state, body.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(ctx, e);
  unsigned char head[8 + 4 + 3 * 8];
  const int32_t d32 = D;
  memcpy(head, kMlpMagic, 8);
  memcpy(head + 8, &d32, 4);
  memcpy(head + 12, &step, 8);
  memcpy(head + 20, &np, 8);
  memcpy(head + 28, &extra_bytes, 8);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(ctx, PROHD_EINVAL, "cannot open the checkpoint file for writing%s");
  bool ok = fwrite(head, 1, sizeof head, f) == sizeof head;
  if (ok && extra_bytes > 0) ok = fwrite(extra, 1, (size_t)extra_bytes, f) == (size_t)extra_bytes;
  if (ok) ok = fwrite(body.data(), sizeof(float), body.size(), f) == body.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? PROHD_OK : fail(ctx, PROHD_EINVAL, "writing the checkpoint failed%s");
}

prohd_status prohd_mlp_load(prohd_ctx* ctx, const char* path, int* D_out, int64_t* step_out, void* state,
                            void* extra, int64_t extra_cap, int64_t* extra_bytes, void* stream) {
  if (!ctx) return PROHD_EINVAL;
  if (!path || !D_out || !step_out || extra_cap < 0) return fail(ctx, PROHD_EINVAL, "bad checkpoint arguments%s");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(ctx, PROHD_EINVAL, "cannot open the checkpoint file%s");
  unsigned char head[8 + 4 + 3 * 8];
  int32_t d32 = 0;
  int64_t step = 0, np = 0, nx = 0;
  bool ok = fread(head, 1, sizeof head, f) == sizeof head && memcmp(head, kMlpMagic, 8) == 0;
  if (ok) {
    memcpy(&d32, head + 8, 4);
    memcpy(&step, head + 12, 8);
    memcpy(&np, head + 20, 8);
    memcpy(&nx, head + 28, 8);
    ok = d32 >= 8 && d32 <= 1024 && np == (int64_t)mlp_shape(d32).nparam && nx >= 0 && step >= 0;
  }
  if (!ok) {
    fclose(f);
    return fail(ctx, PROHD_EINVAL, "not a network checkpoint of this version%s");
  }
  *D_out = d32;
  *step_out = step;
  if (extra_bytes) *extra_bytes = nx;
  if (!state) {  // header only
    fclose(f);
    return PROHD_OK;
  }
  if (nx > extra_cap || (nx > 0 && !extra)) {
    fclose(f);
    return fail(ctx, PROHD_EINVAL, "the extra-byte buffer is smaller than the checkpoint's%s");
  }
  if (nx > 0) ok = fread(extra, 1, (size_t)nx, f) == (size_t)nx;
  std::vector<float> body((size_t)(3 * np));
  if (ok) ok = fread(body.data(), sizeof(float), body.size(), f) == body.size();
  fclose(f);
  if (!ok) return fail(ctx, PROHD_EINVAL, "the checkpoint file is truncated%s");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(state, body.data(), body.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);
  return e ? cuda_fail(ctx, e) : PROHD_OK;
}

uint64_t prohd_launch_count(void) { return g_launches.load(); }

}  // extern "C"
