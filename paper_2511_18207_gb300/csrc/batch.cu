// Batched ProHD (Algorithm 3 for many independent pairs of uneven sizes).
//
// A plan, built once on the host, lays the whole batch out in one workspace
// and writes the device tables every stage reads: a descriptor per pair, the
// tensor-core Gram work items with their tensor maps, the projection items,
// the selection problems, and per-D-class pair lists. Each stage then runs as
// ONE launch over all pairs:
//   pilot shift -> Gram (persistent, atomic ticket over items, largest first)
//   -> Gram reduction -> covariance + centroid axis -> block iteration (one
//   CTA per pair, one launch per D class) -> FP64 clean-up + Rayleigh
//   quotients -> projection (one block per item) -> radix select + band
//   resolution (every (pair, set, direction) problem) -> compaction + gather
//   -> subset HD -> [one-sided refinement] -> finalize. The subset HD runs
//   either on the tensor cores (FP16/BF16 tiles over (pair, row block) items,
//   margins, FP32 rescoring of the candidates) or as FP32 direct differences
//   (persistent, atomic ticket over 128 x 128 tiles), as params.precision
//   asks. With params.refine = 1 each pair adds two row-set-vs-set pairs
//   (its selected rows of A against all of B, of B against all of A) that
//   the same stage runs after the subsets, rows' distances only.
// The sequence is captured once into a CUDA graph and replayed. Item sizes
// (Gram points per item, projection rows per item, selection keys per
// block) come from an autotuner that times candidates on the batch itself.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>

#include "common.cuh"
#include "internal.h"

using namespace prohd;

namespace {

constexpr int kBatchMaxPairs = 1 << 16;
constexpr int kTuneGramPts[] = {4096, 8192, 16384, 32768};
constexpr int kTuneProjRows[] = {4096, 8192, 32768};
constexpr int kTuneSelChunk[] = {4096, 16384, 131072};
constexpr int kMinGramPts = 4096;
constexpr int kMinProjRows = 4096;
constexpr int kCompactItemsB = 4096;  // mask bytes per compaction block (select.cu)

int resolve_m_b(const prohd_params* p, int D) { return p->m < 0 ? (int)floor(sqrt((double)D)) : p->m; }
double resolve_ap_b(const prohd_params* p, int m) {
  return p->alpha_p < 0 ? p->alpha_c / (double)std::max(m, 1) : p->alpha_p;
}

struct PairPlan {
  int D, Dp, m, nd;
  int64_t nA, nB, boundA, boundB;
};

// Host-side layout of the batch workspace. With a null base it only measures.
struct BatchLayout {
  // tables
  BPair* P;
  GcItem* items;
  int* ids;
  CUtensorMap* maps;
  ProjItem* pitems;
  void* probs;
  double* alpha_of;
  unsigned* hist;
  int* order;
  int* cls;  // [npairs] pair ids grouped by D class
  int64_t* prefix;
  // cleared every run
  char* zero_base;
  size_t zero_bytes;
  char* ones_base;
  size_t ones_bytes;
  unsigned* colmin_base;
  int64_t colmin_count;
  int* gticket;
  unsigned long long* hticket;
  int* bstatus;
  // Gram partial slots
  char* slots;
  size_t slot_bytes;
  // per-pair regions (filled into the BPair table)
  std::vector<BPair> hp;
  // one-sided refinement (params.refine = 1): per pair two virtual pairs, the
  // selected rows of one set against the whole other set (v = 2 i: A_sel vs
  // B; v = 2 i + 1: B_sel vs A), run through the subset-distance stage
  BPair* R = nullptr;
  int* rorder = nullptr;
  int64_t* rprefix = nullptr;
  int64_t* rn = nullptr;         // [2 np][2]: selected rows (set at run time), columns
  prohd_result* rout = nullptr;  // [2 np]
  unsigned long long* rticket = nullptr;
  std::vector<BPair> hr;
  size_t end;
};


int64_t items_for(int64_t n, int pts) { return ceil_div(n, pts); }

// Upper bounds of the tables that depend on the tunables.
void table_caps(const std::vector<PairPlan>& pp, bool tensor, bool refine, int64_t& max_items,
                int64_t& max_pitems, size_t& slot_cap, int& nmaps) {
  max_items = 0;
  max_pitems = 0;
  slot_cap = 0;
  nmaps = 0;
  for (const auto& q : pp) {
    const int64_t ni = items_for(q.nA, kMinGramPts) + items_for(q.nB, kMinGramPts);
    max_items += ni;
    slot_cap += (size_t)ni * gram_tc_item_slot_bytes(q.Dp);
    nmaps += 2;
    max_pitems += items_for(q.nA, kMinProjRows) + items_for(q.nB, kMinProjRows);
    if (tensor) nmaps += refine ? 12 : 4;  // subset distance: A, B and their norm operands (x3 refined)
  }
}

// Buffers of one contraction of `rows` (at most) rows against `cols` columns
// on the tensor-core path, as the subset-distance stage reads them.
void hd_bufs(Arena& a, BPair& b, int64_t rows, int64_t cols, int D, int Dp) {
  b.hd_nA_pad = round_up(rows, 128);
  b.hd_nB_pad = round_up(cols, 256);
  b.hd_At = a.take<uint16_t>((size_t)b.hd_nA_pad * Dp, 1024);
  b.hd_Bt = a.take<uint16_t>((size_t)b.hd_nB_pad * Dp, 1024);
  b.hd_nA8 = a.take<float>((size_t)b.hd_nA_pad * 8, 1024);
  b.hd_nB8 = a.take<float>((size_t)b.hd_nB_pad * 8, 1024);
  b.hd_nA2 = a.take<float>((size_t)b.hd_nA_pad);
  b.hd_nB2 = a.take<float>((size_t)b.hd_nB_pad);
  b.hd_epsA = a.take<float>((size_t)b.hd_nA_pad);
  b.hd_epsB = a.take<float>((size_t)b.hd_nB_pad);
  b.hd_rowmin = a.take<float>((size_t)b.hd_nA_pad);
  b.hd_candA = a.take<int32_t>((size_t)rows);
  b.hd_candB = a.take<int32_t>((size_t)cols);
  b.hd_shift = a.take<float>((size_t)D);
  b.hd_spart = a.take<double>((size_t)16 * D);
}

void batch_layout(Arena& a, const std::vector<PairPlan>& pp, const prohd_pair_desc* pairs, bool tensor, bool refine,
                  BatchLayout& L) {
  const int np = (int)pp.size();
  int64_t max_items, max_pitems;
  size_t slot_cap;
  int nmaps;
  table_caps(pp, tensor, refine, max_items, max_pitems, slot_cap, nmaps);
  int64_t nprob = 0;
  for (const auto& q : pp) nprob += 2 * q.nd;

  L.P = a.take<BPair>((size_t)np);
  L.items = a.take<GcItem>((size_t)max_items);
  L.ids = a.take<int>((size_t)max_items);
  L.maps = a.take<CUtensorMap>((size_t)std::max(nmaps, 1));
  L.pitems = a.take<ProjItem>((size_t)max_pitems);
  L.probs = a.take<char>((size_t)nprob * sel_prob_bytes());
  L.alpha_of = a.take<double>((size_t)nprob);
  L.hist = a.take<unsigned>((size_t)nprob * 512);
  L.order = a.take<int>((size_t)np);
  L.cls = a.take<int>((size_t)np);
  L.prefix = a.take<int64_t>((size_t)np + 1);
  L.slots = a.take<char>(slot_cap);
  L.slot_bytes = slot_cap;

  L.hp.assign((size_t)np, BPair{});
  // per-pair arrays that the stages overwrite completely
  for (int i = 0; i < np; ++i) {
    const PairPlan& q = pp[i];
    BPair& b = L.hp[i];
    b.A = pairs ? pairs[i].A : nullptr;
    b.B = pairs ? pairs[i].B : nullptr;
    b.nA = q.nA;
    b.nB = q.nB;
    b.D = q.D;
    b.Dp = q.Dp;
    b.m = q.m;
    b.nd = q.nd;
    const size_t DD = (size_t)q.D * q.D, mD = (size_t)std::max(q.m, 1) * q.D;
    b.s32 = a.take<float>((size_t)q.D);
    b.pilot_part = a.take<double>(pilot_part_doubles(q.D));
    b.G = a.take<double>(DD);
    b.sumA = a.take<double>((size_t)q.D);
    b.sumB = a.take<double>((size_t)q.D);
    b.gcorr = a.take<double>((size_t)q.D);
    b.C64 = a.take<double>(DD);
    b.C32 = a.take<float>(DD);
    b.U = a.take<double>(mD);
    b.rpart = a.take<double>(mD);
    b.dirs = a.take<double>((size_t)q.nd * q.D);
    b.eig = a.take<double>((size_t)std::max(q.m, 1));
    b.qA = a.take<float>((size_t)q.nd * q.nA);
    b.qB = a.take<float>((size_t)q.nd * q.nB);
    b.idxA = a.take<int32_t>((size_t)q.nA);
    b.idxB = a.take<int32_t>((size_t)q.nB);
    b.nsel = a.take<int64_t>(2);
    b.nblkA = (int)ceil_div(q.nA, kCompactItemsB);
    b.nblkB = (int)ceil_div(q.nB, kCompactItemsB);
    b.counts = a.take<unsigned>((size_t)b.nblkA + b.nblkB);
    b.offsets = a.take<int64_t>((size_t)b.nblkA + b.nblkB);
    b.As = a.take<float>((size_t)q.boundA * q.D);
    b.Bs = a.take<float>((size_t)q.boundB * q.D);
    // tensor-core subset distance: 16-bit copies padded to whole tiles
    if (tensor) hd_bufs(a, b, q.boundA, q.boundB, q.D, q.Dp);
  }
  L.hr.clear();
  if (refine) {
    L.R = a.take<BPair>((size_t)2 * np);
    L.rorder = a.take<int>((size_t)2 * np);
    L.rprefix = a.take<int64_t>((size_t)2 * np + 1);
    L.rn = a.take<int64_t>((size_t)4 * np);
    L.rout = a.take<prohd_result>((size_t)2 * np);
    L.hr.assign((size_t)2 * np, BPair{});
    for (int i = 0; i < np; ++i)
      for (int s = 0; s < 2; ++s) {
        const PairPlan& q = pp[i];
        const BPair& bp = L.hp[i];
        BPair& r = L.hr[(size_t)2 * i + s];
        const int64_t rows = s ? q.boundB : q.boundA, cols = s ? q.nA : q.nB;
        r.D = q.D;
        r.Dp = q.Dp;
        r.nA = rows;
        r.nB = cols;
        r.As = s ? bp.Bs : bp.As;
        // the subset-distance stage only reads Bs
        r.Bs = pairs ? const_cast<float*>(s ? pairs[i].A : pairs[i].B) : nullptr;
        r.nsel = L.rn ? L.rn + (size_t)4 * i + 2 * s : nullptr;
        r.idxA = s ? bp.idxB : bp.idxA;
        r.idxB = nullptr;  // columns are rows of the whole set
        r.out = L.rout ? L.rout + (size_t)2 * i + s : nullptr;
        r.rows_only = 1;
        if (tensor) hd_bufs(a, r, rows, cols, q.D, q.Dp);
      }
  }
  // band lists (any size up to the set's)
  L.end = 0;
  // regions cleared to zero every run: statuses, maxnorms, masks, tickets
  a.off = round_up(a.off, 256);
  L.zero_base = a.base ? a.base + a.off : nullptr;
  const size_t z0 = a.off;
  L.gticket = a.take<int>(1, 16);
  L.hticket = a.take<unsigned long long>(1, 16);
  L.rticket = a.take<unsigned long long>(1, 16);
  L.bstatus = a.take<int>(1, 16);
  for (int i = 0; i < np; ++i) {
    BPair& b = L.hp[i];
    b.status = a.take<int>(1, 16);
    b.iters_out = a.take<int>(1, 16);
    b.maxnorm = a.take<float>(2, 16);
    if (tensor) b.hd_sc = a.take<char>(hd_scalars_bytes(), 16);
  }
  for (auto& r : L.hr)
    if (tensor) r.hd_sc = a.take<char>(hd_scalars_bytes(), 16);
  for (int i = 0; i < np; ++i) {
    BPair& b = L.hp[i];
    b.maskA = a.take<uint8_t>((size_t)pp[i].nA, 16);
    b.maskB = a.take<uint8_t>((size_t)pp[i].nB, 16);
  }
  a.off = round_up(a.off, 256);
  L.zero_bytes = a.off - z0;
  // region filled with all-ones bytes every run: packed (d^2, index) minima
  L.ones_base = a.base ? a.base + a.off : nullptr;
  const size_t o0 = a.off;
  for (int i = 0; i < np; ++i) {
    BPair& b = L.hp[i];
    b.bestA = a.take<unsigned long long>((size_t)pp[i].boundA, 16);
    b.bestB = a.take<unsigned long long>((size_t)pp[i].boundB, 16);
  }
  for (auto& r : L.hr) {
    r.bestA = a.take<unsigned long long>((size_t)r.nA, 16);
    r.bestB = a.take<unsigned long long>((size_t)r.nB, 16);
  }
  a.off = round_up(a.off, 256);
  L.ones_bytes = a.off - o0;
  // column minima of the contraction, +inf (as bits) every run
  L.colmin_base = a.base ? reinterpret_cast<unsigned*>(a.base + a.off) : nullptr;
  const size_t c0 = a.off;
  if (tensor) {
    for (int i = 0; i < np; ++i) L.hp[i].hd_colmin = a.take<unsigned>((size_t)L.hp[i].hd_nB_pad, 4);
    for (auto& r : L.hr) r.hd_colmin = a.take<unsigned>((size_t)r.hd_nB_pad, 4);
  }
  L.colmin_count = (int64_t)((a.off - c0) / sizeof(unsigned));
  // the virtual pairs report into their pair's status word
  for (size_t v = 0; v < L.hr.size(); ++v) L.hr[v].status = L.hp[v / 2].status;
}

// Band lists per selection problem and side, n entries each (a band can hold
// the whole set when keys tie).
void band_layout(Arena& a, const std::vector<PairPlan>& pp, std::vector<int32_t*>& band,
                 std::vector<uint64_t*>& bkey) {
  band.clear();
  bkey.clear();
  for (const auto& q : pp)
    for (int set = 0; set < 2; ++set)
      for (int d = 0; d < q.nd; ++d)
        for (int side = 0; side < 2; ++side) {
          const int64_t n = set ? q.nB : q.nA;
          band.push_back(a.take<int32_t>((size_t)n));
          bkey.push_back(a.take<uint64_t>((size_t)n));
        }
}

prohd_status bfail(prohd_ctx* ctx, prohd_status s, const char* msg) {
  if (ctx) ctx->err = msg;
  return s;
}

prohd_status check_batch(prohd_ctx* ctx, const prohd_pair_desc* pairs, int npairs, const prohd_params* p,
                         std::vector<PairPlan>& pp) {
  if (!pairs || npairs < 1 || npairs > kBatchMaxPairs) return bfail(ctx, PROHD_EINVAL, "npairs must be in [1, 65536]");
  if (!p) return bfail(ctx, PROHD_EINVAL, "null params");
  if (!(p->alpha_c > 0.0 && p->alpha_c < 1.0)) return bfail(ctx, PROHD_EINVAL, "alpha_c must be in (0, 1)");
  if (p->alpha_p >= 0.0 && !(p->alpha_p > 0.0 && p->alpha_p < 1.0))
    return bfail(ctx, PROHD_EINVAL, "alpha_p must be in (0, 1) or negative for alpha_c / m");
  if (p->power_max_iters < 1) return bfail(ctx, PROHD_EINVAL, "power_max_iters must be >= 1");
  if (p->precision != PROHD_FP32 && p->precision != PROHD_FP16 && p->precision != PROHD_BF16)
    return bfail(ctx, PROHD_EINVAL, "unknown precision");
  if (p->refine != 0 && p->refine != 1) return bfail(ctx, PROHD_EINVAL, "refine must be 0 or 1");
  pp.resize((size_t)npairs);
  int64_t nprob = 0;
  for (int i = 0; i < npairs; ++i) {
    const prohd_pair_desc& d = pairs[i];
    if (!d.A || !d.B) return bfail(ctx, PROHD_EINVAL, "null point-set pointer in a pair");
    if (d.nA < 1 || d.nB < 1 || d.nA >= ((int64_t)1 << 31) || d.nB >= ((int64_t)1 << 31))
      return bfail(ctx, PROHD_EINVAL, "set sizes must be in [1, 2^31)");
    if (d.D < 4 || d.D > 256 || d.D % 4 != 0)
      return bfail(ctx, PROHD_ENOTSUP, "batched pairs need D % 4 == 0 and 4 <= D <= 256");
    if (((reinterpret_cast<uintptr_t>(d.A) | reinterpret_cast<uintptr_t>(d.B)) & 15) != 0)
      return bfail(ctx, PROHD_EINVAL, "batched point sets need 16-byte aligned bases");
    PairPlan& q = pp[i];
    q.D = d.D;
    q.Dp = (int)round_up(d.D, 64);
    q.m = resolve_m_b(p, d.D);
    if (q.m < 1 || q.m > 24 || q.m > d.D) return bfail(ctx, PROHD_ENOTSUP, "batched pairs need 1 <= m <= min(24, D)");
    q.nd = 1 + q.m;
    q.nA = d.nA;
    q.nB = d.nB;
    const double ap = resolve_ap_b(p, q.m);
    int64_t sa = 0, sb = 0;
    for (int k = 0; k < q.nd; ++k) {
      const double al = k == 0 ? p->alpha_c : ap;
      sa += 2 * std::min(prohd_k_of(al, q.nA), q.nA);
      sb += 2 * std::min(prohd_k_of(al, q.nB), q.nB);
    }
    q.boundA = std::min(q.nA, sa);
    q.boundB = std::min(q.nB, sb);
    nprob += 2 * q.nd;
  }
  if (nprob > 32767) return bfail(ctx, PROHD_ENOTSUP, "too many selection problems in one batch (2 x sum of 1 + m)");
  return PROHD_OK;
}

__global__ void finish_batched_kernel(const BPair* __restrict__ P, int npairs, const int* __restrict__ bstatus) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const BPair& q = P[i];
  q.out->nsel_a = q.nsel[0];
  q.out->nsel_b = q.nsel[1];
  const int bs = *bstatus;
  if (bs > q.out->hd.status) q.out->hd.status = bs;
}

// Row counts of the refinement's virtual pairs: v = 2 i + s takes the size of
// set s's selection of pair i.
__global__ void refine_rows_batched_kernel(const BPair* __restrict__ P, int64_t* __restrict__ rn, int nv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) rn[2 * v] = P[v >> 1].nsel[v & 1];
}

// h(A_sel, B) from virtual pair 2 i and h(B_sel, A) from 2 i + 1 (each as its
// rows' directed distance) into pair i's result.
__global__ void refine_combine_batched_kernel(const BPair* __restrict__ P, const prohd_result* __restrict__ rout,
                                              int npairs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const prohd_hd_result a = rout[2 * i].hd, c = rout[2 * i + 1].hd;
  prohd_hd_result& o = P[i].out->hd;
  prohd_hd_result r;
  r.h_ab = a.h_ab;
  r.h_ba = c.h_ab;
  r.ab_a = a.ab_a;
  r.ab_b = a.ab_b;
  r.ba_b = c.ab_a;
  r.ba_a = c.ab_b;
  r.dir = r.h_ab >= r.h_ba ? 0 : 1;
  r.H = r.dir == 0 ? r.h_ab : r.h_ba;
  r.wit_a = r.dir == 0 ? r.ab_a : r.ba_a;
  r.wit_b = r.dir == 0 ? r.ab_b : r.ba_b;
  r.status = max(max(a.status, c.status), o.status);
  r.H_lowp = fmax(a.H_lowp, c.H_lowp);
  r.n_rescored_a = a.n_rescored_a;
  r.n_rescored_b = c.n_rescored_a;
  o = r;
}

__global__ void set_out_kernel(BPair* __restrict__ P, int npairs, prohd_result* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npairs) P[i].out = out + i;
}

}  // namespace

struct prohd_batch {
  prohd_ctx* ctx = nullptr;
  int npairs = 0;
  prohd_params p{};
  std::vector<prohd_pair_desc> pairs;
  std::vector<PairPlan> pp;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  BatchLayout L;
  // tunables
  int gram_pts = 16384, proj_rows = 8192, sel_chunk = 16384;
  // table extents for the current tunables
  int nitems = 0, npitems = 0, nprob = 0;
  int ncls[3] = {0, 0, 0};
  int cls_off[3] = {0, 0, 0};
  int Dmax = 0, ndmax = 0, mmax = 0, nblk_max = 0;
  int64_t nmax = 0;
  int grid_gram = 0;
  bool tensor = false;  // subset HD on the tensor-core path (FP16 / BF16)
  // side streams and events of the fork-join around the block iteration
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  // graph
  bool use_graph = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  prohd_result* gout = nullptr;
  uint64_t graph_launches = 0;
};

namespace {

// Writes the tunable-dependent tables (Gram items, projection items) and the
// fixed ones (pairs, problems, class lists, orders) into the workspace.
prohd_status write_tables(prohd_batch* b) {
  prohd_ctx* ctx = b->ctx;
  BatchLayout& L = b->L;
  const int np = b->npairs;
  const auto& pp = b->pp;
  // ---- tensor maps: per (pair, set), FP32 boxes of 128 dimensions x 64 points
  std::vector<CUtensorMap> maps;
  std::vector<int> map_of((size_t)np * 2, -1);
  for (int i = 0; i < np; ++i) {
    const PairPlan& q = pp[i];
    for (int set = 0; set < 2; ++set) {
      CUtensorMap m;
      const float* X = set ? b->pairs[i].B : b->pairs[i].A;
      const int64_t n = set ? q.nB : q.nA;
      if (!encode_2d(ctx, &m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, X, (uint64_t)q.D, (uint64_t)n, (uint64_t)q.D * 4, 128,
                     64, CU_TENSOR_MAP_SWIZZLE_NONE))
        return bfail(ctx, PROHD_ECUDA, "tensor-map encoding failed for a batched pair");
      map_of[(size_t)i * 2 + set] = (int)maps.size();
      maps.push_back(m);
    }
  }
  // ---- subset-distance maps (tensor path): A, B tiles and their norm operands
  if (b->tensor) {
    const CUtensorMapDataType dt =
        b->p.precision == PROHD_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    for (size_t i = 0; i < (size_t)np + L.hr.size(); ++i) {
      BPair& q = i < (size_t)np ? L.hp[i] : L.hr[i - np];
      CUtensorMap m[4];
      const uint64_t Dp = (uint64_t)q.Dp;
      if (!encode_2d(ctx, &m[0], dt, q.hd_At, Dp, (uint64_t)q.hd_nA_pad, Dp * 2, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B) ||
          !encode_2d(ctx, &m[1], dt, q.hd_Bt, Dp, (uint64_t)q.hd_nB_pad, Dp * 2, 64, 256, CU_TENSOR_MAP_SWIZZLE_128B) ||
          !encode_2d(ctx, &m[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, q.hd_nA8, 8, (uint64_t)q.hd_nA_pad, 32, 8, 128,
                     CU_TENSOR_MAP_SWIZZLE_32B) ||
          !encode_2d(ctx, &m[3], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, q.hd_nB8, 8, (uint64_t)q.hd_nB_pad, 32, 8, 256,
                     CU_TENSOR_MAP_SWIZZLE_32B))
        return bfail(ctx, PROHD_ECUDA, "tensor-map encoding failed for a batched subset");
      q.hd_map = (int)maps.size();
      for (int k = 0; k < 4; ++k) maps.push_back(m[k]);
    }
  }
  // ---- Gram items (a point range of one set, run by a CTA pair), largest first
  struct HItem {
    GcItem it;
    double cost;
  };
  std::vector<HItem> hitems;
  std::vector<int> item_pair;
  size_t slot_off = 0;
  for (int i = 0; i < np; ++i) {
    const PairPlan& q = pp[i];
    for (int set = 0; set < 2; ++set) {
      const int64_t n = set ? q.nB : q.nA;
      const int64_t ni = items_for(n, b->gram_pts);
      for (int64_t k = 0; k < ni; ++k) {
        HItem h;
        h.it.tm = L.maps + map_of[(size_t)i * 2 + set];
        h.it.s32 = L.hp[i].s32;
        h.it.out = reinterpret_cast<float*>(L.slots + slot_off);
        h.it.sums = reinterpret_cast<double*>(L.slots + slot_off + gram_tc_item_sums_offset(q.Dp));
        slot_off += gram_tc_item_slot_bytes(q.Dp);
        h.it.status = L.hp[i].status;
        h.it.p0 = n * k / ni;
        h.it.p1 = n * (k + 1) / ni;
        h.it.D = q.D;
        h.it.Dp = q.Dp;
        h.it.setA = set ? 0 : 1;
        // steps of the pair: 64 points each for D > 128 (the CTAs split the
        // dimensions), 128 points for D <= 128 (they split the points)
        h.cost = (double)(h.it.p1 - h.it.p0) / (q.Dp > 128 ? 64.0 : 128.0);
        hitems.push_back(h);
        item_pair.push_back(i);
      }
    }
  }
  if (slot_off > L.slot_bytes) return bfail(ctx, PROHD_ENOMEM, "batch Gram slots exceed the workspace");
  // execution order: decreasing cost (ticket order)
  std::vector<int> perm(hitems.size());
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return hitems[x].cost > hitems[y].cost; });
  std::vector<GcItem> items(hitems.size());
  std::vector<int> pos(hitems.size());
  for (size_t r = 0; r < perm.size(); ++r) {
    items[r] = hitems[perm[r]].it;
    pos[perm[r]] = (int)r;
  }
  // id list: per pair, its items in creation order (set A, then set B)
  std::vector<int> ids;
  ids.reserve(hitems.size());
  for (int i = 0; i < np; ++i) {
    BPair& bp = L.hp[i];
    const int start = (int)ids.size();
    for (size_t h = 0; h < hitems.size(); ++h)
      if (item_pair[h] == i) ids.push_back(pos[h]);
    bp.gi0 = start;
    bp.gn0 = (int)ids.size() - start;
  }
  b->nitems = (int)items.size();
  // ---- projection items, largest first
  std::vector<ProjItem> pitems;
  for (int i = 0; i < np; ++i)
    for (int set = 0; set < 2; ++set) {
      const int64_t n = set ? pp[i].nB : pp[i].nA;
      const int64_t ni = items_for(n, b->proj_rows);
      for (int64_t k = 0; k < ni; ++k) {
        ProjItem it;
        it.pair = i;
        it.set = set;
        // row ranges start on 256-row tile boundaries
        it.r0 = std::min(n, round_up(n * k / ni, 256));
        it.r1 = std::min(n, round_up(n * (k + 1) / ni, 256));
        if (k == ni - 1) it.r1 = n;
        if (it.r1 > it.r0) pitems.push_back(it);
      }
    }
  std::stable_sort(pitems.begin(), pitems.end(), [&](const ProjItem& x, const ProjItem& y) {
    return (x.r1 - x.r0) * (int64_t)pp[x.pair].D > (y.r1 - y.r0) * (int64_t)pp[y.pair].D;
  });
  b->npitems = (int)pitems.size();
  // ---- selection problems
  Arena ba;
  ba.base = b->ws;
  ba.off = L.end;
  ba.cap = b->ws_bytes;
  std::vector<int32_t*> band;
  std::vector<uint64_t*> bkey;
  band_layout(ba, pp, band, bkey);
  if (ba.overflow()) return bfail(ctx, PROHD_ENOMEM, "workspace too small for the batch");
  const size_t pb = sel_prob_bytes();
  std::vector<char> probs;
  std::vector<double> alpha_of;
  int prob = 0;
  for (int i = 0; i < np; ++i) {
    const PairPlan& q = pp[i];
    BPair& bp = L.hp[i];
    bp.prob0 = prob;
    const double ap = resolve_ap_b(&b->p, q.m);
    for (int set = 0; set < 2; ++set)
      for (int d = 0; d < q.nd; ++d) {
        const int64_t n = set ? q.nB : q.nA;
        probs.resize(probs.size() + pb);
        const size_t bi = (size_t)prob * 2;
        sel_prob_fill(probs.data() + (size_t)prob * pb, (set ? bp.qB : bp.qA) + (size_t)d * n, n,
                      set ? bp.B : bp.A, bp.dirs + (size_t)d * q.D, set ? bp.maskB : bp.maskA, bp.maxnorm + set,
                      q.D, band[bi], band[bi + 1], bkey[bi], bkey[bi + 1]);
        alpha_of.push_back(d == 0 ? b->p.alpha_c : ap);
        ++prob;
      }
  }
  b->nprob = prob;
  // ---- D classes and the subset-HD order
  std::vector<int> cls;
  for (int c = 0; c < 3; ++c) {
    b->cls_off[c] = (int)cls.size();
    const int lo = c == 0 ? 0 : (c == 1 ? 64 : 128), hi = c == 0 ? 64 : (c == 1 ? 128 : 256);
    for (int i = 0; i < np; ++i)
      if (pp[i].D > lo && pp[i].D <= hi) cls.push_back(i);
    b->ncls[c] = (int)cls.size() - b->cls_off[c];
  }
  std::vector<int> order((size_t)np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return pp[x].boundA * pp[x].boundB * pp[x].D > pp[y].boundA * pp[y].boundB * pp[y].D;
  });
  // refinement: virtual pairs largest first; their column counts are fixed
  std::vector<int> rorder(L.hr.size());
  std::vector<int64_t> rn(L.hr.size() * 2, 0);
  std::iota(rorder.begin(), rorder.end(), 0);
  std::stable_sort(rorder.begin(), rorder.end(), [&](int x, int y) {
    return L.hr[x].nA * L.hr[x].nB * L.hr[x].D > L.hr[y].nA * L.hr[y].nB * L.hr[y].D;
  });
  for (size_t v = 0; v < L.hr.size(); ++v) rn[2 * v + 1] = L.hr[v].nB;
  for (int i = 0; i < np; ++i) {
    L.hp[i].iters = b->p.power_max_iters;
    L.hp[i].out = nullptr;
  }
  // ---- upload (planning is allowed to synchronise)
  cudaError_t e = cudaSuccess;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(L.P, L.hp.data(), sizeof(BPair) * np);
  up(L.items, items.data(), sizeof(GcItem) * items.size());
  up(L.ids, ids.data(), sizeof(int) * ids.size());
  up(L.maps, maps.data(), sizeof(CUtensorMap) * maps.size());
  up(L.pitems, pitems.data(), sizeof(ProjItem) * pitems.size());
  up(L.probs, probs.data(), probs.size());
  up(L.alpha_of, alpha_of.data(), sizeof(double) * alpha_of.size());
  up(L.order, order.data(), sizeof(int) * order.size());
  if (!L.hr.empty()) {
    up(L.R, L.hr.data(), sizeof(BPair) * L.hr.size());
    up(L.rorder, rorder.data(), sizeof(int) * rorder.size());
    up(L.rn, rn.data(), sizeof(int64_t) * rn.size());
  }
  up(L.cls, cls.data(), sizeof(int) * cls.size());
  if (e) {
    ctx->err = std::string("CUDA error while planning the batch: ") + cudaGetErrorString(e);
    return PROHD_ECUDA;
  }
  // any graph built on the old tables is stale
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->gout = nullptr;
  }
  return PROHD_OK;
}

cudaError_t enqueue(prohd_batch* b, prohd_result* out, cudaStream_t st) {
  BatchLayout& L = b->L;
  prohd_ctx* ctx = b->ctx;
  const int np = b->npairs;
  cudaError_t e;
  count_launch();
  set_out_kernel<<<(np + 255) / 256, 256, 0, st>>>(L.P, np, out);
  if ((e = cudaMemsetAsync(L.zero_base, 0, L.zero_bytes, st))) return e;
  if ((e = cudaMemsetAsync(L.ones_base, 0xff, L.ones_bytes, st))) return e;
  {
    PhaseTimer pt(ctx, PROHD_PH_GRAM, st);
    if ((e = pilot_batched(L.P, np, st))) return e;
    if ((e = gram_tc_batched(L.items, b->nitems, L.gticket, L.bstatus, b->grid_gram, b->p.wait_timeout_ns, st)))
      return e;
    if ((e = gram_reduce_batched(L.P, np, L.items, L.ids, b->Dmax, st))) return e;
  }
  {
    PhaseTimer pt(ctx, PROHD_PH_POWER, st);
    if ((e = covariance_batched(L.P, np, b->Dmax, st))) return e;
    const int* lists[3] = {L.cls + b->cls_off[0], L.cls + b->cls_off[1], L.cls + b->cls_off[2]};
    // the three D classes run side by side: fork two streams off `st`, join them back
    const cudaStream_t cs[3] = {st, b->side[0], b->side[1]};
    if ((e = cudaEventRecord(b->ev_fork, st))) return e;
    for (int k = 0; k < 2; ++k)
      if ((e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0))) return e;
    if ((e = subspace_batched(L.P, lists, b->ncls, np, b->Dmax, b->mmax, b->p.power_tol, b->p.seed, cs))) return e;
    for (int k = 0; k < 2; ++k) {
      if ((e = cudaEventRecord(b->ev_join[k], b->side[k]))) return e;
      if ((e = cudaStreamWaitEvent(st, b->ev_join[k], 0))) return e;
    }
    if ((e = subspace_batched_finish(L.P, np, b->Dmax, b->mmax, st))) return e;
  }
  {
    PhaseTimer pt(ctx, PROHD_PH_PROJECT, st);
    if ((e = proj_batched(L.P, L.pitems, b->npitems, b->ndmax, L.bstatus, st))) return e;
  }
  {
    PhaseTimer pt(ctx, PROHD_PH_SELECT, st);
    if ((e = select_batched(reinterpret_cast<SelProb*>(L.probs), b->nprob, L.alpha_of, L.hist, b->nmax, b->sel_chunk,
                            st)))
      return e;
  }
  {
    PhaseTimer pt(ctx, PROHD_PH_GATHER, st);
    if ((e = compact_gather_batched(L.P, np, b->nblk_max, b->nmax, st))) return e;
  }
  {
    PhaseTimer pt(ctx, PROHD_PH_HD_CONTRACT, st);
    if (b->tensor) {
      if ((e = fill_u32_region(L.colmin_base, L.colmin_count, 0x7f800000u, ctx->num_sms, st))) return e;
      if ((e = hd_tc_batched(L.P, L.order, np, L.prefix, L.maps, b->Dmax, b->p.precision == PROHD_BF16 ? 1 : 0,
                             L.bstatus, ctx->num_sms, b->p.wait_timeout_ns, st)))
        return e;
    } else if ((e = hd_simt_batched(L.P, L.order, np, L.prefix, L.hticket, ctx->num_sms, st))) {
      return e;
    }
  }
  if (!L.hr.empty()) {
    // one-sided refinement: the selected rows of each set against the whole
    // other set, as 2 np virtual pairs through the same stage, then per pair
    // h(A_sel, B) and h(B_sel, A) into its result
    PhaseTimer pt(ctx, PROHD_PH_HD_RESCORE, st);
    const int nv = 2 * np;
    count_launch();
    refine_rows_batched_kernel<<<(nv + 255) / 256, 256, 0, st>>>(L.P, L.rn, nv);
    if ((e = cudaGetLastError())) return e;
    if (b->tensor) {
      // the column side holds whole sets: blocks per set for about 1,024 rows each
      const int bx = (int)std::min<int64_t>(128, std::max<int64_t>(4, ceil_div(b->nmax, 1024)));
      if ((e = hd_tc_batched(L.R, L.rorder, nv, L.rprefix, L.maps, b->Dmax, b->p.precision == PROHD_BF16 ? 1 : 0,
                             L.bstatus, ctx->num_sms, b->p.wait_timeout_ns, st, bx)))
        return e;
    } else if ((e = hd_simt_batched(L.R, L.rorder, nv, L.rprefix, L.rticket, ctx->num_sms, st))) {
      return e;
    }
    count_launch();
    refine_combine_batched_kernel<<<(np + 255) / 256, 256, 0, st>>>(L.P, L.rout, np);
    if ((e = cudaGetLastError())) return e;
  }
  count_launch();
  finish_batched_kernel<<<(np + 255) / 256, 256, 0, st>>>(L.P, np, L.bstatus);
  return cudaGetLastError();
}

size_t batch_bytes(const std::vector<PairPlan>& pp, bool tensor, bool refine) {
  Arena a;
  BatchLayout L;
  batch_layout(a, pp, nullptr, tensor, refine, L);
  std::vector<int32_t*> band;
  std::vector<uint64_t*> bkey;
  band_layout(a, pp, band, bkey);
  return a.off + 256;
}

}  // namespace

extern "C" {

size_t prohd_batch_workspace_size(const prohd_pair_desc* pairs, int npairs, const prohd_params* p) {
  std::vector<PairPlan> pp;
  if (check_batch(nullptr, pairs, npairs, p, pp) != PROHD_OK) return 0;
  return batch_bytes(pp, p->precision != PROHD_FP32, p->refine == 1);
}

prohd_status prohd_batch_plan(prohd_ctx* ctx, const prohd_pair_desc* pairs, int npairs, const prohd_params* p,
                              void* ws, size_t ws_bytes, prohd_batch** out) {
  if (!ctx || !out) return PROHD_EINVAL;
  *out = nullptr;
  std::vector<PairPlan> pp;
  prohd_status s = check_batch(ctx, pairs, npairs, p, pp);
  if (s != PROHD_OK) return s;
  if (!ctx->encode_tiled) return bfail(ctx, PROHD_ENOTSUP, "driver has no tensor-map encoder");
  if (ctx->num_sms > kMaxSms) return bfail(ctx, PROHD_ENOTSUP, "more SMs than the library sizes its scratch for");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return bfail(ctx, PROHD_EINVAL, "workspace must be 256-byte aligned");
  const bool tensor = p->precision != PROHD_FP32;
  if (ws_bytes < batch_bytes(pp, tensor, p->refine == 1))
    return bfail(ctx, PROHD_ENOMEM, "workspace too small for the batch");
  prohd_batch* b = new (std::nothrow) prohd_batch();
  if (!b) return PROHD_ENOMEM;
  b->ctx = ctx;
  b->npairs = npairs;
  b->p = *p;
  if (b->p.wait_timeout_ns <= 0) b->p.wait_timeout_ns = kDefaultTimeoutNs;
  b->pairs.assign(pairs, pairs + npairs);
  b->pp = pp;
  b->ws = static_cast<char*>(ws);
  b->ws_bytes = ws_bytes;
  Arena a;
  a.base = b->ws;
  a.cap = ws_bytes;
  b->tensor = tensor;
  batch_layout(a, pp, pairs, tensor, p->refine == 1, b->L);
  b->L.end = a.off;
  for (const auto& q : pp) {
    b->Dmax = std::max(b->Dmax, q.D);
    b->ndmax = std::max(b->ndmax, q.nd);
    b->mmax = std::max(b->mmax, q.m);
    b->nmax = std::max(b->nmax, std::max(q.nA, q.nB));
    b->nblk_max = std::max(b->nblk_max, (int)ceil_div(std::max(q.nA, q.nB), kCompactItemsB));
  }
  b->grid_gram = ctx->num_sms;
  if (ctx->batch_tuned) {
    b->gram_pts = ctx->batch_gram_pts;
    b->proj_rows = ctx->batch_proj_rows;
    b->sel_chunk = ctx->batch_sel_chunk;
  }
  bool ok = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 2 && ok; ++k) {
    ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
  }
  ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    prohd_batch_destroy(b);
    return bfail(ctx, PROHD_ECUDA, "could not create the batch's streams and events");
  }
  s = write_tables(b);
  if (s != PROHD_OK) {
    prohd_batch_destroy(b);
    return s;
  }
  *out = b;
  return PROHD_OK;
}

void prohd_batch_destroy(prohd_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (int k = 0; k < 2; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
}

prohd_status prohd_batch_use_graph(prohd_batch* b, int on) {
  if (!b) return PROHD_EINVAL;
  b->use_graph = on != 0;
  return PROHD_OK;
}

prohd_status prohd_estimate_batched(prohd_ctx* ctx, prohd_batch* b, prohd_result* out, void* stream) {
  if (!ctx || !b || !out || b->ctx != ctx) return bfail(ctx, PROHD_EINVAL, "bad batch arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (!b->use_graph || ctx->profiling) {
    if ((e = enqueue(b, out, st))) {
      ctx->err = std::string("CUDA error: ") + cudaGetErrorString(e);
      return PROHD_ECUDA;
    }
    return PROHD_OK;
  }
  if (!b->gexec || b->gout != out) {
    // capture the whole batch once on the plan's own stream; replays go to `stream`
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    const uint64_t l0 = g_launches.load();
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (!e) {
      cudaError_t e2 = enqueue(b, out, b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &g);
      if (!e) e = e2;
    }
    if (!e) e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    // kernels enqueued during capture run only when the graph is launched
    const uint64_t in_graph = g_launches.load() - l0;
    g_launches.fetch_sub(in_graph);
    if (e) {
      b->gexec = nullptr;
      ctx->err = std::string("CUDA error while capturing the batch: ") + cudaGetErrorString(e);
      return PROHD_ECUDA;
    }
    b->graph_launches = in_graph;
    b->gout = out;
  }
  if ((e = cudaGraphLaunch(b->gexec, st))) {
    ctx->err = std::string("CUDA error: ") + cudaGetErrorString(e);
    return PROHD_ECUDA;
  }
  count_launch((int)b->graph_launches);
  return PROHD_OK;
}

// Coordinate search over the three tunables, timing the whole batch with
// CUDA events on `stream` (synchronises). The best values are kept in the
// plan and as the context's defaults for later plans.
prohd_status prohd_batch_autotune(prohd_ctx* ctx, prohd_batch* b, prohd_result* out, void* stream, double* best_ms) {
  if (!ctx || !b || !out) return bfail(ctx, PROHD_EINVAL, "bad batch arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto time_once = [&](float& ms) -> prohd_status {
    prohd_status s = write_tables(b);
    if (s != PROHD_OK) return s;
    for (int rep = 0; rep < 3; ++rep) {
      if (rep == 1) cudaEventRecord(e0, st);
      if (enqueue(b, out, st)) return bfail(ctx, PROHD_ECUDA, "launch failed while tuning");
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return bfail(ctx, PROHD_ECUDA, "tuning run failed");
    cudaEventElapsedTime(&ms, e0, e1);
    ms *= 0.5f;
    return PROHD_OK;
  };
  float best = 1e30f;
  prohd_status s = PROHD_OK;
  for (int round = 0; round < 3 && s == PROHD_OK; ++round) {
    const int* cand = round == 0 ? kTuneGramPts : (round == 1 ? kTuneProjRows : kTuneSelChunk);
    const int nc = round == 0 ? 4 : 3;
    int* knob = round == 0 ? &b->gram_pts : (round == 1 ? &b->proj_rows : &b->sel_chunk);
    int keep = *knob;
    for (int c = 0; c < nc && s == PROHD_OK; ++c) {
      *knob = cand[c];
      float ms = 0.f;
      s = time_once(ms);
      if (s == PROHD_OK && ms < best) {
        best = ms;
        keep = cand[c];
      }
    }
    *knob = keep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PROHD_OK) return s;
  s = write_tables(b);
  if (s != PROHD_OK) return s;
  ctx->batch_tuned = true;
  ctx->batch_gram_pts = b->gram_pts;
  ctx->batch_proj_rows = b->proj_rows;
  ctx->batch_sel_chunk = b->sel_chunk;
  if (best_ms) *best_ms = best;
  return PROHD_OK;
}

prohd_status prohd_batch_get_tunables(const prohd_batch* b, int32_t* gram_pts, int32_t* proj_rows, int32_t* sel_chunk) {
  if (!b) return PROHD_EINVAL;
  if (gram_pts) *gram_pts = b->gram_pts;
  if (proj_rows) *proj_rows = b->proj_rows;
  if (sel_chunk) *sel_chunk = b->sel_chunk;
  return PROHD_OK;
}

prohd_status prohd_batch_set_tunables(prohd_batch* b, int32_t gram_pts, int32_t proj_rows, int32_t sel_chunk) {
  if (!b) return PROHD_EINVAL;
  if (gram_pts < kMinGramPts || proj_rows < kMinProjRows || sel_chunk < 256)
    return bfail(b->ctx, PROHD_EINVAL, "tunables below their minimum");
  b->gram_pts = gram_pts;
  b->proj_rows = proj_rows;
  b->sel_chunk = sel_chunk;
  return write_tables(b);
}

// The tuning table: one text file per device type, keyed by the device name,
// SM count and compute capability, holding the batch item sizes the
// autotuner chose (the context's defaults for new plans).
static bool device_key(const prohd_ctx* ctx, char* name, size_t cap) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) return false;
  snprintf(name, cap, "%s", prop.name);
  for (char* c = name; *c; ++c)
    if (*c == ' ' || *c == '\t' || *c == '\n') *c = '_';
  return true;
}

prohd_status prohd_tunables_save(prohd_ctx* ctx, const char* path) {
  if (!ctx || !path) return PROHD_EINVAL;
  char name[256];
  if (!device_key(ctx, name, sizeof name)) return bfail(ctx, PROHD_ECUDA, "device properties unavailable");
  FILE* f = fopen(path, "w");
  if (!f) return bfail(ctx, PROHD_EINVAL, "cannot open the tuning table for writing");
  const int ok = fprintf(f, "prohd-tunables 1\ndevice %s sms %d cc %d.%d\n", name, ctx->num_sms, ctx->cc_major,
                         ctx->cc_minor) > 0 &&
                 fprintf(f, "batch_gram_pts %d\nbatch_proj_rows %d\nbatch_sel_chunk %d\n", ctx->batch_gram_pts,
                         ctx->batch_proj_rows, ctx->batch_sel_chunk) > 0;
  if (fclose(f) != 0 || !ok) return bfail(ctx, PROHD_EINVAL, "writing the tuning table failed");
  return PROHD_OK;
}

prohd_status prohd_tunables_load(prohd_ctx* ctx, const char* path) {
  if (!ctx || !path) return PROHD_EINVAL;
  char name[256], fname[256];
  if (!device_key(ctx, name, sizeof name)) return bfail(ctx, PROHD_ECUDA, "device properties unavailable");
  FILE* f = fopen(path, "r");
  if (!f) return bfail(ctx, PROHD_EINVAL, "cannot open the tuning table");
  int version = 0, sms = 0, ccM = 0, ccm = 0, g = 0, pr = 0, sc = 0;
  const int n = fscanf(f, "prohd-tunables %d device %255s sms %d cc %d.%d batch_gram_pts %d batch_proj_rows %d "
                       "batch_sel_chunk %d", &version, fname, &sms, &ccM, &ccm, &g, &pr, &sc);
  fclose(f);
  if (n != 8 || version != 1) return bfail(ctx, PROHD_EINVAL, "not a tuning table");
  if (strcmp(fname, name) != 0 || sms != ctx->num_sms || ccM != ctx->cc_major || ccm != ctx->cc_minor)
    return bfail(ctx, PROHD_EINVAL, "the tuning table is for another device");
  if (g < kMinGramPts || pr < kMinProjRows || sc < 256) return bfail(ctx, PROHD_EINVAL, "tunables below their minimum");
  ctx->batch_tuned = true;
  ctx->batch_gram_pts = g;
  ctx->batch_proj_rows = pr;
  ctx->batch_sel_chunk = sc;
  return PROHD_OK;
}

prohd_status prohd_batch_pair_outputs(const prohd_batch* b, int pair, double** dirs, int32_t** idxA, int32_t** idxB,
                                      int32_t** iters) {
  if (!b || pair < 0 || pair >= b->npairs) return PROHD_EINVAL;
  const BPair& q = b->L.hp[(size_t)pair];
  if (dirs) *dirs = q.dirs;
  if (idxA) *idxA = q.idxA;
  if (idxB) *idxB = q.idxB;
  if (iters) *iters = q.iters_out;
  return PROHD_OK;
}

}  // extern "C"
