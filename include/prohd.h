/*
 * prohd.h - C ABI of the GB300 (sm_103a) ProHD library.
 *
 * ProHD (arxiv 2511.18207) approximates the Hausdorff distance
 *   H(A,B) = max{ h(A,B), h(B,A) },  h(A,B) = max_{a in A} min_{b in B} ||a - b||_2   (Eq. 1)
 * by projecting both sets onto a few directions (the centroid axis, Algorithm 1,
 * and the top-m principal components of [A;B], Algorithm 2), keeping the k
 * smallest and k largest projections of each set per direction, and computing
 * the exact Hausdorff distance of the two selected subsets (Algorithm 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Point sets are FP32, row-major, contiguous: point i of A is A[i*D .. i*D+D-1].
 *   1 <= n < 2^31 points per set, 1 <= D <= 1024.
 * - Unless a parameter says "host", every array pointer is a DEVICE pointer
 *   owned by the caller. The library never frees or retains them.
 * - Point indices are 0-based int32 (the paper counts from 1).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls are asynchronous on that stream: they enqueue kernels and return.
 *   They never synchronise the device and never allocate device memory.
 * - Scratch memory is a caller-owned device buffer `ws` of at least the size
 *   returned by the matching *_workspace_size query, 256-byte aligned.
 *   Its contents on entry are ignored; on return it holds intermediate data
 *   that the next call may overwrite. Two calls that run concurrently must
 *   not share a workspace.
 * - Results land in device memory; read them after synchronising `stream`.
 *   Each result struct carries a device-side status (see prohd_status): a
 *   non-finite input value or a bounded device wait that ran out is reported
 *   there, not as the return value.
 * - Return value: PROHD_OK when the work was enqueued; otherwise nothing was
 *   enqueued and prohd_last_error(ctx) describes the problem.
 * - Every non-sequential arithmetic path in the library is on the GPU; there
 *   is no CPU fallback.
 */
#ifndef PROHD_H
#define PROHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PROHD_OK = 0,
  PROHD_EINVAL = 1,      /* invalid argument: null pointer, size out of range, bad alpha */
  PROHD_ENOMEM = 2,      /* workspace smaller than the *_workspace_size query */
  PROHD_ECUDA = 3,       /* a CUDA runtime call failed (message in prohd_last_error) */
  PROHD_ETIMEOUT = 4,    /* device-side: a bounded wait in a kernel ran out */
  PROHD_ENONFINITE = 5,  /* device-side: the input holds NaN or Inf */
  PROHD_ENOTSUP = 6      /* valid request the library does not support (e.g. GPU older than sm_103a) */
} prohd_status;

/* Tile precision of the distance contraction (Methodology – Algorithms, "exact HD on the subsets"). */
enum {
  PROHD_FP32 = 0, /* direct-difference FP32 on CUDA cores; exact to FP32 rounding */
  PROHD_FP16 = 1, /* FP16 tensor-core tiles, FP32 accumulation, rigorous margin + FP32 rescoring */
  PROHD_BF16 = 2  /* BF16 tensor-core tiles, same refinement */
};

/* Opaque library context: device properties, tensor-map encoder, last error text. */
typedef struct prohd_ctx prohd_ctx;

/*
 * ProHD parameters (Algorithm 3 and Evaluation – Datasets and Experimental Setup).
 *   m            number of principal components; m < 0 selects floor(sqrt(D))
 *   alpha_c      fraction kept per side on the centroid axis, 0 < alpha_c < 1:
 *                k_c = max(1, floor(alpha_c * n)) per set (Algorithm 1)
 *   alpha_p      fraction per side per component; alpha_p < 0 selects alpha_c / m
 *                (Algorithm 3: alpha' = alpha / m), k_p = max(1, floor(alpha_p * n))
 *   power_max_iters, power_tol
 *                the eigenvector iteration stops when its residuals meet
 *                power_tol (the power-iteration test 1 - |<v_t, v_{t-1}>| <
 *                power_tol, as a residual bound), or after power_max_iters
 *                steps (defaults 96 and 1e-13; a truncated-SVD budget: well
 *                separated spectra converge in 15-30 steps)
 *   seed         seed of the SplitMix64 start vectors of the power iteration
 *   precision    PROHD_FP32 / PROHD_FP16 / PROHD_BF16 for the subset HD
 *   refine       0: H_hat = H(A_sel, B_sel) as Algorithm 3 states (default);
 *                1: one-sided refinement H_hat = max(h(A_sel, B), h(B_sel, A)),
 *                   each selected point against the whole other set. It never
 *                   exceeds H(A, B) (the selected points are points of A and B),
 *                   at the cost of two subset-vs-set contractions
 *                   (prohd_estimate / prohd_estimate_dirs / prohd_estimate_host,
 *                   and batched plans)
 *   wait_timeout_ns  limit of every bounded device wait (default 4e9 ns)
 */
typedef struct {
  int32_t m;
  int32_t precision;
  double alpha_c;
  double alpha_p;
  int32_t power_max_iters;
  int32_t refine;
  double power_tol;
  uint64_t seed;
  int64_t wait_timeout_ns;
  int64_t reserved[4];
} prohd_params;

/*
 * Result of an exact Hausdorff distance (Eq. 1). Distances are FP64 values of
 * the witness pairs; the pairs are chosen from FP32 distances (exact rescoring
 * of every candidate the low-precision pass could not rule out).
 *   H, h_ab, h_ba   H = max(h_ab, h_ba)
 *   wit_a, wit_b    witness of H: index into A and index into B
 *   ab_a, ab_b      witness of h(A,B) (a and its nearest b)
 *   ba_b, ba_a      witness of h(B,A) (b and its nearest a)
 *   dir             0 if h_ab >= h_ba, else 1
 *   status          prohd_status of the device work (OK, ETIMEOUT, ENONFINITE)
 *   H_lowp          tensor paths: H from the low-precision tiles before any
 *                   rescoring; FP32 path: same as H
 *   n_rescored_a/b  rows of A / columns of B rescored in FP32 (0 on the FP32 path)
 */
typedef struct {
  double H, h_ab, h_ba;
  int64_t wit_a, wit_b;
  int64_t ab_a, ab_b;
  int64_t ba_b, ba_a;
  int32_t dir;
  int32_t status;
  double H_lowp;
  int64_t n_rescored_a, n_rescored_b;
} prohd_hd_result;

/* Result of prohd_estimate (Algorithm 3): hd is H_hat = H(A_sel, B_sel), with
 * witness indices mapped back to A and B; nsel_a = |I^A|, nsel_b = |I^B|. */
typedef struct {
  prohd_hd_result hd;
  int64_t nsel_a, nsel_b;
} prohd_result;

/* ---------------------------------------------------------------- context */

/* Creates a context bound to the current CUDA device. Checks the device is
 * sm_103 (else PROHD_ENOTSUP). Allocates host memory only. */
prohd_status prohd_create(prohd_ctx** out);
void prohd_destroy(prohd_ctx* ctx);
/* Text of the last error reported through ctx (empty string if none). */
const char* prohd_last_error(const prohd_ctx* ctx);
/* Fills the defaults listed above (m = -1, alpha_c = 0.01, alpha_p = -1, FP16). */
void prohd_params_default(prohd_params* p);
/* k = max(1, floor(alpha * n)) computed in FP64, clamped to n (Algorithms 1-2). */
int64_t prohd_k_of(double alpha, int64_t n);

/* --------------------------------------------------------- workspace sizes */

size_t hausdorff_exact_workspace_size(int64_t nA, int64_t nB, int D, int precision);
size_t prohd_directions_workspace_size(int64_t nA, int64_t nB, int D, int m);
size_t prohd_select_workspace_size(int64_t nA, int64_t nB, int D, int ndirs);
size_t prohd_estimate_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p);
/* prohd_estimate_host also stages A and B in the workspace. */
size_t prohd_estimate_host_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p);

/* ------------------------------------------------------------ entry points */

/*
 * Exact Hausdorff distance H(A,B) (Eq. 1; the paper computes it with a Faiss
 * flat index, Methodology – Algorithms and Evaluation – Datasets and Experimental Setup "ANN-Exact").
 *   A [nA*D], B [nB*D]   device FP32 point sets
 *   precision            PROHD_FP32, PROHD_FP16 or PROHD_BF16 (tile dtype)
 *   out                  device pointer to one prohd_hd_result
 * FP16/BF16: tensor-core tiles give every point's nearest-neighbour distance
 * up to a rigorous rounding margin; every row and column whose margin
 * interval reaches the largest lower bound is rescored in FP32, so the result
 * equals the FP32 path's up to FP32 rounding. Tensor paths need D <= 256.
 */
prohd_status hausdorff_exact(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB,
                             int D, int precision, prohd_hd_result* out, void* ws, size_t ws_bytes,
                             void* stream);

/*
 * The same exact distance with row pruning: the early-break idea of the exact
 * Hausdorff algorithms the paper compares with (Related Work), as whole-set passes.
 * For each direction h(X, Y):
 *   1. an exact pass over 1,024 evenly spread rows of X gives a lower bound
 *      LB1 of h(X, Y);
 *   2. one tensor-core contraction of every row of X against the first
 *      max(8192, n_Y / 64) rows of Y gives every row a certified upper bound
 *      of its NN distance;
 *   3. an exact pass over 1,024 evenly spread rows among those whose bound
 *      reaches LB1 gives LB2;
 *   4. the exact path of hausdorff_exact runs on the rows whose bound reaches
 *      max(LB1, LB2), lowered by 1e-4 relative.
 * The row attaining h(X, Y) always stays, so out equals hausdorff_exact's
 * result up to the FP32 argmin of rows within 1e-4 of the maximum.
 * Arguments as for hausdorff_exact, plus
 *   kept    HOST int64_t[2] or NULL: the rows left in each direction
 *           ({-1, -1} when the plain path ran). Non-NULL synchronises
 *           `stream` once, after all the work is enqueued, so it must be
 *           NULL while `stream` is being captured into a CUDA graph.
 * Pruning applies with FP16/BF16 tiles, nA, nB >= 32768 and nA * nB at least
 * the context's pair threshold; otherwise (and for PROHD_FP32) the call is
 * hausdorff_exact. The one-sided refinement (params.refine) prunes its two
 * directed distances by the same rule, its rows being the subset and its
 * columns the other full set. The workspace size depends on the row counts
 * only.
 */
size_t hausdorff_exact_pruned_workspace_size(int64_t nA, int64_t nB, int D, int precision);
prohd_status hausdorff_exact_pruned(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                    int precision, prohd_hd_result* out, int64_t* kept, void* ws, size_t ws_bytes,
                                    void* stream);
/* Pair threshold of the row pruning (default 4e9; >= 0, else PROHD_EINVAL;
 * 0 prunes whenever the row counts allow). Smaller contractions take the
 * plain path, whose fixed costs are lower: measured, the plain path is faster
 * at 1.9e9 pairs and the pruned one at 7.5e9. */
prohd_status prohd_set_prune_min_pairs(prohd_ctx* ctx, double min_pairs);
/* Pair threshold of the estimate's pruned subset distance (default 1e9;
 * >= 0, else PROHD_EINVAL; 0 prunes whenever the subsets allow). The subset
 * HD of prohd_estimate (and of prohd_estimate_dirs / _adaptive / _host) is
 * Eq. 1 on A_sel and B_sel, computed exactly either way. With FP16/BF16 tiles,
 * D <= 256 and both subset bounds (2 sum_d k_d per set) of at least 8,192
 * rows, and their product at least this threshold, it leaves out the subset
 * rows that cannot attain either directed maximum: every row of one subset is
 * contracted against the first 2,048 rows of the other (an upper bound of its
 * NN distance), the first 2,048 rows of each against the whole other subset
 * (lower bounds of h by the intervals' lower ends), then, twice, 1,024
 * evenly spread rows among those whose upper bound reaches the current bound
 * (a larger lower bound), and only the rows whose upper bound reaches the last
 * bound (and row 0) run the full contraction, with the same intervals,
 * candidates and FP32 rescoring. The
 * result is the plain contraction's in every field (H, both directed
 * distances, witnesses, H_lowp, rescored counts). */
prohd_status prohd_set_subset_prune_min_pairs(prohd_ctx* ctx, double min_pairs);

/*
 * Projection directions (Algorithm 1 step 2 and Algorithm 2 step 2):
 *   dirs[0]      centroid axis u = (ybar - xbar)/||ybar - xbar||, or e_1 when
 *                ||ybar - xbar|| < 1e-9
 *   dirs[1..m]   top-m principal components of the stacked set [A;B]: unit
 *                eigenvectors of the union covariance C = (1/N) sum (z-mu)(z-mu)^T
 *                by power iteration with deflation, largest-magnitude entry
 *                made positive
 *   eig[0..m-1]  their Rayleigh quotients (may be NULL)
 * dirs is a device FP64 array [(1+m) * D]; m comes from p (m < 0: floor(sqrt D)).
 * Centroid sums and the covariance are accumulated in FP64 across blocks.
 */
prohd_status prohd_directions(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB,
                              int D, const prohd_params* p, double* dirs, double* eig, void* ws,
                              size_t ws_bytes, void* stream);

/*
 * Union covariance of the stacked set [A; B] (Algorithm 2 step 2: the
 * principal components are eigenvectors of this matrix), the same matrix
 * prohd_directions iterates on:
 *   C      device FP64 [D * D], row-major: C = (1/N) sum_z (z - mu)(z - mu)^T
 *          over the N = nA + nB points
 *   mean   device FP64 [D] receiving mu, or NULL
 * For D <= 256 with D % 4 == 0 and 16-byte aligned sets the products come
 * from BF16 tensor-core tiles (a two-part split of each centred FP32 value,
 * FP32 accumulation of 512 points, FP64 across blocks); otherwise from FP32
 * CUDA-core tiles with FP64 accumulation.
 */
size_t prohd_covariance_workspace_size(int64_t nA, int64_t nB, int D);
prohd_status prohd_covariance(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                              double* C, double* mean, void* ws, size_t ws_bytes, void* stream);

/*
 * Extreme selection for given directions (Algorithms 1-2, steps "argsort",
 * "keep bottom-k and top-k", "unique"; Algorithm 3 step 4, union):
 *   dirs       device FP64 [ndirs * D] (any vectors; the projection is x^T u)
 *   kA, kB     HOST int64 [ndirs]: k per direction for A and for B (clamped to n)
 *   idxA       device int32 [nA]: receives the sorted unique selected indices
 *   nselA      device int64 scalar: receives |I^A|; same for B
 * Point i is kept for direction d if it is among the first k of the ascending
 * order of (x_i^T u_d, i) or of the descending order of x_i^T u_d with
 * ascending i on ties. The order uses the FP64 projection summed over
 * k = 0..D-1 with separately rounded products and sums, so the result is
 * identical to a sequential FP64 full sort.
 */
prohd_status prohd_select(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB,
                          int D, const double* dirs, int ndirs, const int64_t* kA, const int64_t* kB,
                          int32_t* idxA, int64_t* nselA, int32_t* idxB, int64_t* nselB, void* ws,
                          size_t ws_bytes, void* stream);

/*
 * ProHD estimate H_hat(A,B) (Algorithm 3): directions, selection, and the exact
 * Hausdorff distance of A_sel = A[I^A] and B_sel = B[I^B].
 *   out        device pointer to one prohd_result
 *   idxA/idxB  optional device int32 [nA]/[nB] receiving I^A, I^B (may be NULL)
 *   dirs       optional device FP64 [(1+m) * D] receiving the directions (may be NULL)
 */
prohd_status prohd_estimate(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB,
                            int D, const prohd_params* p, prohd_result* out, int32_t* idxA,
                            int32_t* idxB, double* dirs, void* ws, size_t ws_bytes, void* stream);

/*
 * prohd_estimate for HOST inputs: copies A_host and B_host (pinned memory
 * recommended) into the workspace with cudaMemcpyAsync on `stream`, runs
 * prohd_estimate, and copies the result into *out_host. Asynchronous: read
 * *out_host after synchronising `stream`. The host buffers must stay valid
 * until then. Uses prohd_estimate_host_workspace_size bytes of workspace.
 */
prohd_status prohd_estimate_host(prohd_ctx* ctx, const float* A_host, int64_t nA, const float* B_host,
                                 int64_t nB, int D, const prohd_params* p, prohd_result* out_host,
                                 void* ws, size_t ws_bytes, void* stream);

/*
 * hausdorff_exact without a workspace, for callers that cannot allocate
 * device memory (code running under someone else's stream capture, plugins
 * whose host framework owns the allocator, programs that forbid allocation
 * after start-up). The paper has no counterpart; this is a deployment aid.
 * Same result as hausdorff_exact(..., PROHD_FP32, ...); scratch is a fixed
 * 2 MiB __device__ array inside the library (held by every GPU that loads
 * it), so nA + nB is limited to about 262,000 points and larger inputs return
 * PROHD_EINVAL. The first call on a device looks up the array's address
 * (cudaGetSymbolAddress): make it before any stream capture. After
 * cudaDeviceReset the next call on that device looks the address up again
 * (the reset unloads the array), so it too must come before any capture.
 * All calls share the array: calls whose GPU work overlaps race; serialise
 * them.
 */
prohd_status hausdorff_exact_noalloc(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB,
                                     int D, prohd_hd_result* out, void* stream);

/* ------------------------------------------------------------ observability */

/* Phases timed by the profiler (one kernel each unless noted). */
typedef enum {
  PROHD_PH_GRAM = 0,      /* union Gram + centroid sums (gram_kernel), Algorithm 2 step 2 */
  PROHD_PH_POWER = 1,     /* power iteration (one cluster launch) */
  PROHD_PH_PROJECT = 2,   /* FP32 projections of both sets (two launches) */
  PROHD_PH_SELECT = 3,    /* radix select, band, FP64 band ranking, compaction (several) */
  PROHD_PH_GATHER = 4,    /* subset gather (two launches) */
  PROHD_PH_HD_PREP = 5,   /* centring, scale, rounded copies (several) */
  PROHD_PH_HD_CONTRACT = 6, /* the distance contraction: hd_tc_kernel, or the FP32 tile kernel */
  PROHD_PH_HD_RESCORE = 7,  /* margins, candidate rescoring, FP64 witnesses (several);
                               batched plans: the one-sided refinement */
  PROHD_PH_COUNT = 8
} prohd_phase;

/* While on, every call records a CUDA event pair on its stream around each
 * phase (host-side event objects only; no device allocation). */
prohd_status prohd_profile_enable(prohd_ctx* ctx, int on);
/* Waits for the recorded events, adds their durations to per-phase totals and
 * copies the totals: ms[PROHD_PH_COUNT] (milliseconds) and count[PROHD_PH_COUNT]
 * (phase instances). reset != 0 clears the totals afterwards. Host arrays. */
prohd_status prohd_profile_read(prohd_ctx* ctx, double* ms, int64_t* count, int reset);
/* Number of kernels this library has launched in this process. */
uint64_t prohd_launch_count(void);

/* ---------------------------------------------------------------- batched pairs
 *
 * ProHD for many independent pairs (Algorithm 3 applied to each pair; the
 * paper runs its class pairs one at a time). A plan lays the batch out in one
 * workspace and writes the device tables every stage reads; each stage then
 * runs as one launch over all pairs, and the whole sequence is captured into
 * a CUDA graph on first use and replayed.
 *
 * Pairs: A, B device pointers, FP32 row-major, 16-byte aligned bases;
 * 1 <= nA, nB < 2^31; 4 <= D <= 256 with D % 4 == 0; 1 <= m <= min(24, D)
 * after resolving m < 0 to floor(sqrt(D)). params.precision picks the subset
 * HD as in prohd_estimate: PROHD_FP16 / PROHD_BF16 tensor-core tiles with the
 * rigorous margin and FP32 rescoring, or PROHD_FP32 direct differences.
 */
typedef struct {
  const float* A;
  int64_t nA;
  const float* B;
  int64_t nB;
  int32_t D;
  int32_t reserved;
} prohd_pair_desc;

typedef struct prohd_batch prohd_batch;

/* Bytes of workspace a plan of these pairs needs (0 if the pairs are invalid). */
size_t prohd_batch_workspace_size(const prohd_pair_desc* pairs, int npairs, const prohd_params* p);

/* Plans the batch: copies the pair list (host array of device pointers),
 * validates it, lays it out in `ws` (device, 256-byte aligned, at least the
 * size above; owned by the caller and bound to the plan until it is
 * destroyed), encodes the tensor maps and uploads the tables. Planning
 * synchronises the device (synchronous copies); running does not.
 * params.refine = 1 adds, per pair, the one-sided refinement: the selected
 * rows of each set against the whole other set, run as two more row-set
 * pairs through the subset-distance stage; the workspace then also holds
 * their rounded copies (tensor precisions: about 2 (nA + nB) Dp 2 bytes per
 * pair). refine must be 0 or 1 (PROHD_EINVAL otherwise). */
prohd_status prohd_batch_plan(prohd_ctx* ctx, const prohd_pair_desc* pairs, int npairs, const prohd_params* p,
                              void* ws, size_t ws_bytes, prohd_batch** out);
void prohd_batch_destroy(prohd_batch* b);

/* Runs the batch on `stream`: out is a device array of npairs results (pair
 * i's H_hat, witnesses mapped to indices into its own A and B, |I^A|, |I^B|,
 * status). With graphs on (the default), the first call for a given `out`
 * captures the sequence on the plan's private stream; every call launches
 * the graph on `stream`. Asynchronous. */
prohd_status prohd_estimate_batched(prohd_ctx* ctx, prohd_batch* b, prohd_result* out, void* stream);
prohd_status prohd_batch_use_graph(prohd_batch* b, int on);

/* Autotuner: times the batch for candidate item sizes (Gram points per work
 * item, projection rows per item, selection keys per block), one knob at a
 * time, with CUDA events on `stream`; keeps the fastest in the plan and as
 * the context's defaults for later plans. Synchronises. best_ms may be NULL. */
prohd_status prohd_batch_autotune(prohd_ctx* ctx, prohd_batch* b, prohd_result* out, void* stream, double* best_ms);
prohd_status prohd_batch_get_tunables(const prohd_batch* b, int32_t* gram_pts, int32_t* proj_rows, int32_t* sel_chunk);
prohd_status prohd_batch_set_tunables(prohd_batch* b, int32_t gram_pts, int32_t proj_rows, int32_t sel_chunk);

/* The tuning table, persisted: prohd_tunables_save writes the context's
 * batch item sizes (those prohd_batch_autotune left, else the defaults) to a
 * small text file at `path` (host path), keyed by the device name, SM count
 * and compute capability; prohd_tunables_load reads one back into the
 * context, whose later plans then start from those sizes. Load returns
 * PROHD_EINVAL for a missing or malformed file, a table of another device
 * (name, SM count or compute capability differ) or values below the
 * minimums, and leaves the context unchanged. No device work; no stream.
 * The kernels' tile shapes (operand rings, stages, TMEM buffers) are fixed
 * at compile time from offline sweeps; the runtime table holds the item
 * sizes, which depend on the batch. */
prohd_status prohd_tunables_save(prohd_ctx* ctx, const char* path);
prohd_status prohd_tunables_load(prohd_ctx* ctx, const char* path);

/* Device pointers (inside the plan's workspace) of pair `pair`'s directions
 * [1+m][D] (FP64), candidate indices (int32, the first nsel_a / nsel_b
 * entries are valid after a run) and block-iteration step count (one int32).
 * Any output pointer may be NULL. */
prohd_status prohd_batch_pair_outputs(const prohd_batch* b, int pair, double** dirs, int32_t** idxA, int32_t** idxB,
                                      int32_t** iters);

/* ---------------------------------------------------------------- given directions
 *
 * Algorithm 3 from the selection on: the caller's directions dirs [nd][D]
 * (device, FP64, unit rows; row 0 conventionally the centroid axis) with
 * per-direction k lists kA, kB (HOST arrays of nd values >= 1; a direction
 * keeps its kA[d] smallest and kA[d] largest projections of A). Selection,
 * union, gather and the subset HD run as in prohd_estimate (params.precision
 * picks the tiles and params.refine the one-sided refinement; m, alpha are
 * not used). idxA / idxB may be NULL. */
size_t prohd_estimate_dirs_workspace_size(int64_t nA, int64_t nB, int D, int nd, const int64_t* kA, const int64_t* kB,
                                          const prohd_params* p);
prohd_status prohd_estimate_dirs(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                 const prohd_params* p, const double* dirs, int nd, const int64_t* kA,
                                 const int64_t* kB, prohd_result* out, int32_t* idxA, int32_t* idxB, void* ws,
                                 size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- adaptive alpha
 *
 * The adaptive alpha schedule Conclusion and Future Work proposes for strict error budgets, read
 * as doubling alpha on the one-sided refined estimate: the directions are
 * computed once (as prohd_estimate computes them); step t = 0, 1, ... keeps
 * alpha_t = alpha_c 2^t per side on the centroid axis and alpha_p 2^t on each
 * component (alpha_p < 0: alpha_c / m), selects as Algorithm 3, and takes
 * H_t = max(h(A_sel, B), h(B_sel, A)) (params.refine = 1 semantics). The
 * candidate sets grow with t, so H_t never decreases and never exceeds H.
 * The schedule stops, checked in this order, when every point of both sets is
 * selected (H_t = H: PROHD_ADAPT_ALL), when t >= 1 and H_t - H_{t-1} <=
 * rel_tol H_t (PROHD_ADAPT_STABLE), when alpha_c 2^(t+1) > alpha_max
 * (PROHD_ADAPT_BUDGET), or after PROHD_ADAPT_MAX_STEPS steps.
 *
 * params.refine is ignored (always the refined estimate); alpha_max must be
 * in [alpha_c, 1), rel_tol >= 0. out (device) holds the last step's result,
 * dirs (device, [1+m][D] FP64) the directions, idxA / idxB (device) the last
 * step's candidate indices; each may be NULL but out. info (HOST) receives
 * the schedule. The stop decision is taken on the host: the call
 * synchronises `stream` once per step, so it cannot be captured in a CUDA
 * graph. The workspace holds the largest step's subsets. */
#define PROHD_ADAPT_MAX_STEPS 32
enum { PROHD_ADAPT_ALL = 0, PROHD_ADAPT_STABLE = 1, PROHD_ADAPT_BUDGET = 2, PROHD_ADAPT_STEPS = 3 };
typedef struct prohd_adaptive_info {
  int32_t steps;                          /* steps run (>= 1) */
  int32_t reason;                         /* PROHD_ADAPT_* */
  double alpha_c, alpha_p;                /* the last step's fractions */
  double H[PROHD_ADAPT_MAX_STEPS];        /* H_t per step */
  int64_t nsel_a[PROHD_ADAPT_MAX_STEPS];  /* |A_sel| per step */
  int64_t nsel_b[PROHD_ADAPT_MAX_STEPS];  /* |B_sel| per step */
} prohd_adaptive_info;

size_t prohd_estimate_adaptive_workspace_size(int64_t nA, int64_t nB, int D, const prohd_params* p,
                                              double alpha_max);
prohd_status prohd_estimate_adaptive(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                                     const prohd_params* p, double alpha_max, double rel_tol, prohd_result* out,
                                     prohd_adaptive_info* info, int32_t* idxA, int32_t* idxB, double* dirs,
                                     void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- learned directions
 *
 * A small network proposes 4 extra unit directions per pair from cheap set
 * statistics (the learned direction dictionary of Conclusion and Future Work, future work in the
 * paper). It only adds directions, so plain ProHD is its fallback.
 *
 * Features (prohd_features), x [10 D] FP32: the centroid difference
 * ybar - xbar, the 8 leading components scaled by sqrt(lambda), and the
 * per-dimension union variances, divided by s = sqrt(trace(C)/D) (the
 * variances by s^2). The call also returns the directions [9][D] (centroid
 * axis + 8 components, as prohd_directions with m = 8) and eig [8].
 *
 * Network: h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), z = h2 W3 + b3 with
 * W1 [10D x 256], W2 [256 x 256], W3 [256 x 4D]; the 4 vectors of z are
 * normalised. Loss against a unit label w (the witness direction
 * (a* - b*)/||a* - b*|| of the exact HD): 1 - (1/10) log sum_j exp(10 (u_j . w)^2),
 * averaged over the batch.
 *
 * State: params | Adam m | Adam v, FP32, prohd_mlp_state_bytes(D) bytes of
 * device memory owned by the caller (prohd_mlp_param_count(D) floats per
 * block; layout W1, b1, W2, b2, W3, b3, each row-major and 64-float aligned).
 * precision: PROHD_FP32 (CUDA-core FP32 GEMMs) or PROHD_BF16 (operands
 * rounded to BF16, tensor-core products, FP32 accumulation). Every call
 * needs a scratch buffer of prohd_mlp_scratch_bytes(D, batch) (256-byte
 * aligned). feat [batch][10 D], label [batch][D], outputs [batch][4][D].
 */
size_t prohd_features_workspace_size(int64_t nA, int64_t nB, int D);
prohd_status prohd_features(prohd_ctx* ctx, const float* A, int64_t nA, const float* B, int64_t nB, int D,
                            const prohd_params* p, float* feat, double* dirs, double* eig, void* ws, size_t ws_bytes,
                            void* stream);
size_t prohd_mlp_param_count(int D);
size_t prohd_mlp_state_bytes(int D);
size_t prohd_mlp_scratch_bytes(int D, int batch);
/* Weights uniform on +-sqrt(6 / fan_in) from SplitMix64 (seed, layer 101..103,
 * element index); biases and Adam moments zero. */
prohd_status prohd_mlp_init(prohd_ctx* ctx, int D, uint64_t seed, void* state, void* stream);
/* Unit directions of a batch: FP32 [batch][4][D] and/or FP64 (renormalised) [batch][4][D]; either may be NULL. */
prohd_status prohd_mlp_forward(prohd_ctx* ctx, int D, const void* state, const float* feat, int batch, int precision,
                               float* dirs32, double* dirs64, void* scratch, size_t scratch_bytes, void* stream);
/* Mean loss (device float) and, if grad != NULL, its gradient [param_count] (no update). */
prohd_status prohd_mlp_loss_grad(prohd_ctx* ctx, int D, const void* state, const float* feat, const float* label,
                                 int batch, int precision, float* loss, float* grad, void* scratch,
                                 size_t scratch_bytes, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected with `step`,
 * counting from 1) on the mean loss of the batch; loss may be NULL. */
prohd_status prohd_mlp_train_step(prohd_ctx* ctx, int D, void* state, const float* feat, const float* label, int batch,
                                  int precision, float lr, int64_t step, float* loss, void* scratch,
                                  size_t scratch_bytes, void* stream);
/* The Adam update alone, with a caller gradient [param_count] (device FP32). */
prohd_status prohd_mlp_adam_step(prohd_ctx* ctx, int D, void* state, const float* grad, float lr, int64_t step,
                                 void* stream);
/* Checkpoint of a network's state, so training can resume exactly. File:
 * "PHDMLP01", int32 D, int64 step, int64 parameter count, int64 extra-byte
 * count (little-endian, unpadded), the caller's extra bytes (e.g. the state
 * of its training-data sampler), then params | Adam m | Adam v as FP32.
 * `state` is the device state; save copies it to the host and synchronises
 * `stream`. PROHD_EINVAL if the file cannot be written. */
prohd_status prohd_mlp_save(prohd_ctx* ctx, const char* path, int D, int64_t step, const void* state,
                            const void* extra, int64_t extra_bytes, void* stream);
/* Reads a checkpoint: D and step into *D_out / *step_out and the extra-byte
 * count into *extra_bytes (may be NULL). state == NULL reads the header only;
 * otherwise state (device, prohd_mlp_state_bytes(*D_out) bytes) receives
 * params | m | v and extra (host, extra_cap bytes) the extra bytes, and the
 * call synchronises `stream`. PROHD_EINVAL for a missing, foreign, truncated
 * or mismatched file, or an extra buffer smaller than the file's. */
prohd_status prohd_mlp_load(prohd_ctx* ctx, const char* path, int* D_out, int64_t* step_out, void* state,
                            void* extra, int64_t extra_cap, int64_t* extra_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PROHD_H */
