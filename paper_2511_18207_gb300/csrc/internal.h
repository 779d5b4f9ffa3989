// Internal host-side interfaces between the ProHD translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/prohd.h"

struct prohd_ctx {
  int device = 0;
  int num_sms = 0;
  int cc_major = 0, cc_minor = 0;
  int smem_optin = 0;
  void* encode_tiled = nullptr;  // cuTensorMapEncodeTiled from the driver
  std::string err;
  // profiler
  bool profiling = false;
  struct Pending {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double ph_ms[PROHD_PH_COUNT] = {};
  int64_t ph_count[PROHD_PH_COUNT] = {};
  // batched-pair tunables found by prohd_batch_autotune (defaults for new plans)
  bool batch_tuned = false;
  int batch_gram_pts = 16384, batch_proj_rows = 8192, batch_sel_chunk = 16384;
  // row pruning of directed distances only for contractions of at least this
  // many (row, column) pairs (prohd_set_prune_min_pairs)
  double prune_min_pairs = 4e9;
  // the estimate's subset distance takes the pruned form when the subset
  // bounds give at least this many (row, column) pairs
  // (prohd_set_subset_prune_min_pairs)
  double subset_prune_min_pairs = 1e9;
  // host-buffer estimates: the copy stream and the events of its row ranges
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t feed_start = nullptr;
  cudaEvent_t feed_ready[8] = {};
};

namespace prohd {

extern std::atomic<uint64_t> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Records an event pair around a phase on `st` when the context profiles.
struct PhaseTimer {
  prohd_ctx* ctx;
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  PhaseTimer(prohd_ctx* c, int ph, cudaStream_t s) : ctx(c), phase(ph), st(s) {
    if (ctx && ctx->profiling && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
  }
  void stop() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, st);
      ctx->pending.push_back({phase, a, b});
    } else {
      cudaEventDestroy(a);
    }
    a = nullptr;
  }
  ~PhaseTimer() { stop(); }
};

// Bump allocator over the caller's workspace. With base == nullptr it only
// measures, so the size queries and the entry points share one layout.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  size_t cap = 0;
  template <typename T>
  T* take(size_t count, size_t align = 256) {
    off = (off + align - 1) / align * align;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  bool overflow() const { return base && off > cap; }
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

constexpr int64_t kDefaultTimeoutNs = 4000000000LL;

// ---- distance contraction (hd.cu) ----
// Sizes may live on the device (n*_dev) with host upper bounds (n*_max); the
// index maps translate row numbers to caller indices for the witnesses.
void hd_core_layout(Arena& ws, int64_t nA_max, int64_t nB_max, int D, int precision);
struct HdShared;
// A centre for the rounded copies and a bound max |x - shift| over both row
// sets (FP32), known before the subset distance (the estimate: the union
// centroid from the covariance pass, the bound taken while gathering the
// subsets), so that the copies skip their own centring passes.
struct HdCenter {
  const float* shift;   // [D]
  const float* maxabs;  // [1]
};
cudaError_t hd_core(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, int64_t nA_max, const float* B,
                    const int64_t* nB_dev, int64_t nB_max, int D, int precision, const int32_t* mapA,
                    const int32_t* mapB, prohd_hd_result* out, int* status_dev, Arena& ws, int64_t timeout_ns,
                    cudaStream_t st, bool few_rows = false, const HdShared* shared = nullptr,
                    const HdCenter* center = nullptr);
bool tc_supported_dim(int D);
// The same result as hd_core (tensor-core precisions), with the rows that
// cannot attain either directed maximum left out of the full contractions;
// applies where hd_subset_prunable holds (its layout: hd_core_pruned_layout,
// which is hd_core_layout plus the pruning buffers where it applies).
bool hd_subset_prunable(int64_t nA_max, int64_t nB_max, int D, int precision);
void hd_core_pruned_layout(Arena& ws, int64_t nA_max, int64_t nB_max, int D, int precision);
cudaError_t hd_core_pruned(prohd_ctx* ctx, const float* A, const int64_t* nA_dev, int64_t nA_max, const float* B,
                           const int64_t* nB_dev, int64_t nB_max, int D, int precision, const int32_t* mapA,
                           const int32_t* mapB, prohd_hd_result* out, int* status_dev, Arena& ws, int64_t timeout_ns,
                           cudaStream_t st, const HdCenter* center = nullptr);

// ---- selection (select.cu) ----
void select_layout(Arena& ws, int64_t nA, int64_t nB, int D, int ndirs);
cudaError_t select_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                       const double* dirs, int ndirs, const int64_t* kA, const int64_t* kB, int32_t* idxA,
                       int64_t* nselA, int32_t* idxB, int64_t* nselB, int* status_dev, Arena& ws,
                       cudaStream_t st, int64_t timeout_ns);
cudaError_t gather_rows(const float* X, int D, const int32_t* idx, const int64_t* n_dev, int64_t n_max, float* out,
                        int num_sms, cudaStream_t st);
// The same gather, also raising *maxabs to max |x - center| over the gathered
// values (FP32, atomic; *maxabs starts at 0) and flagging non-finite values.
cudaError_t gather_rows_center(const float* X, int D, const int32_t* idx, const int64_t* n_dev, int64_t n_max,
                               float* out, const float* center, float* maxabs, int* status, int num_sms,
                               cudaStream_t st);

// ---- directions (directions.cu) ----
// Inputs that land while the work runs (the host-buffer entry point): each
// set arrives in `parts` row ranges [n k / parts, n (k+1) / parts), range k of
// set s complete once ready[s * parts + k] has completed. The tensor-core Gram
// reads range k only after waiting for its event, so it overlaps the copies of
// the later ranges; every other reader runs after the Gram.
struct InputFeed {
  int parts = 1;
  const cudaEvent_t* ready = nullptr;
};
void directions_layout(Arena& ws, int64_t nA, int64_t nB, int D, int m, int gram_parts = 1);
// center32 (optional): the union centroid in FP32 [D]; zero1 (optional): one
// float set to 0 in the same launch.
cudaError_t directions_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D, int m,
                           int max_iters, double tol, uint64_t seed, double* dirs, double* eig, int* status_dev,
                           Arena& ws, cudaStream_t st, int64_t timeout_ns, const InputFeed* feed = nullptr,
                           float* center32 = nullptr, float* zero1 = nullptr);

// Union covariance C (FP64, D x D, 1/N) and mean of [A; B] (directions.cu).
void covariance_layout(Arena& ws, int D);
cudaError_t covariance_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D, double* C,
                           double* mean, int* status, Arena& ws, cudaStream_t st, int64_t timeout_ns);

// ---- tensor-core Gram (gram_tc.cu) ----
constexpr int kMaxSms = 192;  // upper bound used to size per-CTA scratch
// Top-m eigenvectors by block iteration with Rayleigh-Ritz (subspace.cu).
bool subspace_supported(int D, int m);
size_t subspace_scratch_doubles(int D, int m);
cudaError_t subspace_run(prohd_ctx* ctx, const float* C32, const double* C64, int D, int m, int max_iters, double tol,
                         uint64_t seed, double* dirs, double* eig, double* scratch, cudaStream_t st);
bool gram_tc_supported(int D);
// parts > 1: one launch per row range of each set (InputFeed), partials
// summed together
size_t gram_tc_scratch_doubles(int D, int num_sms, int parts = 1);
cudaError_t gram_tc_run(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                        const float* s32, double* scratch, double* G, double* sumA, double* sumB, int* status,
                        int64_t timeout_ns, cudaStream_t st, const InputFeed* feed = nullptr);

// ---- batched pairs (batch.cu drives these; each stage is one launch for all pairs) ----

// One unit of tensor-core Gram work for a CTA pair: a point range of one
// set. The tensor map (box 128 dimensions x 64 points) lives in device memory.
struct GcItem {
  const CUtensorMap* tm;  // FP32 tiles of the set
  const float* s32;       // pilot shift of the pair [D]
  float* out;             // [2 CTAs][useful columns: 256, or Dp if Dp <= 128][128 rows] partial products
  double* sums;           // [2 CTAs][8 warps][set sum | diagonal correction][128 dims]
  int* status;            // the pair's status
  int64_t p0, p1;         // point range [p0, p1) of the set
  int D, Dp, setA;
};

// Device-side descriptor of one pair of a batch: its inputs, parameters and
// the slices of the batch workspace that each stage reads and writes.
struct BPair {
  const float* A;
  const float* B;
  int64_t nA, nB;
  int D, Dp, m, nd;
  // directions
  float* s32;
  double* pilot_part;  // [16][D] slice sums of the pilot shift
  double *G, *sumA, *sumB, *C64;
  double* gcorr;  // [D] diagonal corrections of the tensor-core Gram
  float* C32;
  double* U;      // [m][D] Ritz vectors before the FP64 clean-up
  double* rpart;  // [m][D] Rayleigh-quotient partials
  double* dirs;   // [nd][D]
  double* eig;    // [max(m,1)]
  int iters;      // block-iteration cap
  int* iters_out; // block-iteration steps taken
  // selection
  float *qA, *qB;  // [nd][n] FP32 projections
  float* maxnorm;  // [2]
  uint8_t *maskA, *maskB;
  int32_t *idxA, *idxB;
  int64_t* nsel;       // [2]
  unsigned* counts;    // [2][nblk] compaction block counts
  int64_t* offsets;    // [2][nblk]
  int nblkA, nblkB;
  // subset distance
  float *As, *Bs;
  unsigned long long *bestA, *bestB;
  int* status;
  prohd_result* out;
  // tensor-core subset distance (FP16 / BF16 batches): rounded copies, norms,
  // margins, minima, candidate lists, shift, scalars; four tensor maps from hd_map
  void *hd_At, *hd_Bt;
  float *hd_nA2, *hd_nB2, *hd_epsA, *hd_epsB, *hd_rowmin, *hd_shift, *hd_nA8, *hd_nB8;
  unsigned* hd_colmin;
  int32_t *hd_candA, *hd_candB;
  double* hd_spart;
  void* hd_sc;
  int64_t hd_nA_pad, hd_nB_pad;
  int hd_map;
  int rows_only;  // only the rows' directed distance is wanted (refinement pairs)
  // Gram items of this pair (both sets), as positions in the batch's item-id list
  int gi0, gn0;
  int prob0;  // first selection problem of this pair (set-major: set * nd + d)
};

// One unit of projection work: rows [r0, r1) of one set of one pair.
struct ProjItem {
  int pair, set;
  int64_t r0, r1;
};

size_t gram_tc_smem_batched();
size_t gram_tc_item_slot_bytes(int Dp);   // output slot of one item (partial products, then sums)
size_t gram_tc_item_sums_offset(int Dp);  // byte offset of the sums within a slot
cudaError_t gram_tc_batched(const GcItem* items, int nitems, int* ticket, int* batch_status, int grid,
                            int64_t timeout_ns, cudaStream_t st);
cudaError_t gram_reduce_batched(const BPair* P, int npairs, const GcItem* items, const int* ids, int Dmax,
                                cudaStream_t st);
cudaError_t pilot_batched(const BPair* P, int npairs, cudaStream_t st);
size_t pilot_part_doubles(int D);
cudaError_t covariance_batched(const BPair* P, int npairs, int Dmax, cudaStream_t st);
// Block iteration with one CTA per pair, one launch per D class (D <= 64, 128, 256),
// each on its own stream; then the FP64 clean-up and Rayleigh quotients.
cudaError_t subspace_batched(const BPair* P, const int* const cls_pairs[3], const int ncls[3], int npairs, int Dmax,
                             int mmax, double tol, uint64_t seed, const cudaStream_t cls_st[3]);
cudaError_t subspace_batched_finish(const BPair* P, int npairs, int Dmax, int mmax, cudaStream_t st);
cudaError_t proj_batched(const BPair* P, const ProjItem* items, int nitems, int ndmax, int* batch_status,
                         cudaStream_t st);
struct SelProb;
size_t sel_prob_bytes();
cudaError_t select_batched(SelProb* probs, int nprob, const double* alpha_of, unsigned* hist, int64_t nmax, int chunk,
                           cudaStream_t st);
// Fills the data fields of one selection problem (host side, at planning).
void sel_prob_fill(void* dst, const float* q, int64_t n, const float* X, const double* u, uint8_t* mask,
                   const float* maxnorm, int D, int32_t* band0, int32_t* band1, uint64_t* key0, uint64_t* key1);
// Ascending indices of the set bytes of mask[0..n) into idx, their count
// into *nsel (device); counts / offsets hold compact_blocks(n) entries.
int64_t compact_blocks(int64_t n);
cudaError_t mask_to_indices(const uint8_t* mask, int64_t n, int32_t* idx, int64_t* nsel, unsigned* counts,
                            int64_t* offsets, cudaStream_t st);
// One set's rounded copy (with its norms and margins) and the shift and
// scale it was made with, prepared once for several contractions against
// row sets drawn from one set X (hd_shared_prepare covers X and Y).
struct HdShared {
  void* Yt = nullptr;
  float *n2 = nullptr, *eps = nullptr, *n8 = nullptr, *shift = nullptr;
  double* spart = nullptr;
  void* sc = nullptr;
  int64_t pad = 0;
  int Dp = 0;
};
void hd_shared_layout(Arena& ws, int64_t nY_max, int D, int precision, HdShared& s);
cudaError_t hd_shared_prepare(prohd_ctx* ctx, const float* X, const int64_t* nX_dev, const float* Y,
                              const int64_t* nY_dev, int D, int precision, HdShared& s, int* status_dev,
                              cudaStream_t st);
// Row pruning for the exact distance: rows of X (nX_dev of at most nX_max)
// against the first nYp_dev rows of Y on tensor cores; hi[i] receives a
// certified upper bound of row i's NN distance over those rows (so over Y).
void hd_prefix_layout(Arena& ws, int64_t nX_max, int64_t nYp_max, int D, int precision);
cudaError_t hd_prefix_upper(prohd_ctx* ctx, const float* X, const int64_t* nX_dev, int64_t nX_max, const float* Y,
                            const int64_t* nYp_dev, int64_t nYp_max, int D, int precision, float* hi, int* status_dev,
                            Arena& ws, int64_t timeout_ns, cudaStream_t st, const HdShared* shared = nullptr);
cudaError_t compact_gather_batched(const BPair* P, int npairs, int nblk_max, int64_t nmax, cudaStream_t st);
size_t hd_scalars_bytes();
size_t hd_tc_row_block();   // rows of A per contraction item (128)
// Tensor-core subset HD of every pair: prep, contraction over (pair, row block)
// items, margins, FP32 rescoring of candidates, FP64 witnesses. `bx` blocks
// per (pair, set) run the max |x - s| and rounded-copy passes (the largest
// set's rows decide).
cudaError_t hd_tc_batched(const BPair* P, const int* order, int npairs, int64_t* prefix, const CUtensorMap* maps,
                          int Dmax, int bf16, int* batch_status, int num_sms, int64_t timeout_ns, cudaStream_t st,
                          int bx = 4);
cudaError_t fill_u32_region(unsigned* p, int64_t n, unsigned v, int num_sms, cudaStream_t st);
cudaError_t hd_simt_batched(const BPair* P, const int* order, int npairs, int64_t* prefix, unsigned long long* ticket,
                            int num_sms, cudaStream_t st);

// ---- learned directions (mlp.cu) ----
// Parameter layout (FP32, offsets in floats, each block 64-aligned):
// W1 [10D x 256], b1, W2 [256 x 256], b2, W3 [256 x 4D], b3. The training
// state is params | Adam m | Adam v (3 * nparam floats).
struct MlpShape {
  int D, n_in, h, n_out;
  size_t w1, b1, w2, b2, w3, b3, nparam;
};
MlpShape mlp_shape(int D);
size_t mlp_scratch_floats(int D, int B);
struct MlpActsView {
  float *u, *loss, *lmean, *grad;
};
MlpActsView mlp_acts_view(int D, int B, float* scratch);
cudaError_t mlp_init(const MlpShape& s, float* state, uint64_t seed, cudaStream_t st);
// Forward pass of B samples; with labels W it also forms the loss and the
// gradient of the head (kept in the scratch for mlp_backward).
cudaError_t mlp_forward(const MlpShape& s, const float* P, const float* X, int B, int prec, float* scratch,
                        const float* W, cudaStream_t st);
cudaError_t mlp_backward(const MlpShape& s, const float* P, const float* X, int B, int prec, float* scratch,
                         cudaStream_t st);
cudaError_t mlp_adam(const MlpShape& s, float* state, const float* grad, float lr, int64_t step, cudaStream_t st);
cudaError_t mlp_features(const double* sumA, const double* sumB, int64_t nA, int64_t nB, const double* C64,
                         const double* dirs, const double* eig, int D, float* feat, cudaStream_t st);
cudaError_t mlp_dirs64(const float* U, int count, int D, double* out, cudaStream_t st);
// Directions (m = 8) and the network's input features of one pair.
cudaError_t directions_features(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                int max_iters, double tol, uint64_t seed, double* dirs, double* eig, float* feat,
                                int* status, Arena& ws, cudaStream_t st, int64_t timeout_ns);

// ---- small utilities (api.cu) ----
cudaError_t set_i64(int64_t* p, int64_t v, cudaStream_t st);
cudaError_t zero_i32(int* p, int n, cudaStream_t st);

// Tensor-map encoder (driver entry point fetched through the runtime).
bool encode_2d(prohd_ctx* ctx, CUtensorMap* map, CUtensorMapDataType dtype, const void* base, uint64_t inner,
               uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz);

}  // namespace prohd
