/*
 * ntt.h -- C ABI of the GB300 non-negative tensor-train (nTT) library.
 *
 * The library computes the nTT of a dense non-negative tensor by the chain of
 * non-negative matrix factorisations of Algorithm 2 ("distnTT") of Bhattarai
 * et al., "Distributed Non-Negative Tensor Train Decomposition": stage l
 * factors the unfolding X_l (r_{l-1} n_l x prod_{j>l} n_j) as W H with
 * W, H >= 0; W becomes TT core G_l (r_{l-1} x n_l x r_l) and H becomes the
 * next unfolding; the last core is the final H.  Each NMF is iterated with
 * the Lee-Seung multiplicative updates the paper times in Section IV:
 *     H <- max(0, H o (W^T X) / (W^T W H + eps))
 *     W <- max(0, W o (X H^T) / (W H H^T + eps))
 * TT ranks are given, or chosen stage by stage by Algorithm 2's rule on the
 * singular values of each unfolding (ranks == NULL, eps_rank > 0).
 *
 * Conventions for every entry point:
 *  - All arrays are dense, row-major (C order).  Device pointers must point to
 *    memory of the current CUDA device; host pointers are ordinary host memory
 *    (pinned memory makes the host variants asynchronous).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is enqueued on it and the call returns without waiting,
 *    unless stated otherwise.
 *  - The caller allocates and frees every device buffer (tensor, cores,
 *    factors, workspace).  The library owns only plan objects (host memory and
 *    cached CUDA graphs) and never allocates device memory.
 *  - Argument, shape and rank-feasibility errors are returned synchronously
 *    and nothing is launched.  Device-side errors (a bounded wait that timed
 *    out) are written to a status word in the workspace and reported by
 *    ntt_plan_get_stats / ntt_status_of_workspace after the stream is synced.
 *  - No call ever falls back to a CPU implementation.
 */
#ifndef NTT_H
#define NTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NTT_MAX_D 16      /* maximum tensor order d */
#define NTT_MAX_RANK 32   /* maximum TT rank r_k */
#define NTT_MAX_ROWS 512  /* maximum unfolding height r_{k-1} n_k */
#define NTT_MAX_TALL_ROWS 16384  /* maximum NMF height of the grouped entry points (row blocks of 512) */

typedef enum {
  NTT_OK = 0,
  NTT_ERR_INVALID_ARG = 1,      /* NULL pointer, bad size, bad enum */
  NTT_ERR_RANK_INFEASIBLE = 2,  /* r_k > min(r_{k-1} n_k, prod_{j>k} n_j) (Alg. 2: N = min(m, n)) */
  NTT_ERR_OOM = 3,              /* workspace too small / host allocation failed */
  NTT_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  NTT_ERR_TIMEOUT = 5,          /* a bounded device wait gave up (device status word) */
  NTT_ERR_UNSUPPORTED = 6       /* shape or option outside what is built */
} ntt_status;

typedef enum { NTT_F32 = 0, NTT_BF16 = 1 } ntt_dtype;

typedef struct ntt_plan_s* ntt_plan;

/* Kernel routing of the MU loops.  NTT_ROUTE_AUTO takes, per unfolding shape,
 * the kernel measured fastest on GB300; the others restrict the choice (for
 * comparisons and tests).  A route that does not apply to a stage's shape
 * leaves that stage on the automatic choice among what remains allowed. */
typedef enum {
  NTT_ROUTE_AUTO = 0,      /* measured-fastest kernel per stage */
  NTT_ROUTE_PASS = 1,      /* single-problem passes only (no grouped engine) */
  NTT_ROUTE_GROUPED = 2,   /* the grouped engine wherever it applies */
  NTT_ROUTE_FMA = 3,       /* CUDA-core (FMA) kernels only: no tensor-core pass */
  NTT_ROUTE_GENERIC = 4,   /* the generic FMA pass only */
  NTT_ROUTE_TC = 5         /* a tensor-core pass wherever one applies, including the
                              forms that are slower than the FMA kernels on GB300 */
} ntt_route;

/* ntt_plan_desc.solver: the NMF of every stage */
#define NTT_SOLVER_MU 0     /* Lee-Seung multiplicative updates (the default) */
#define NTT_SOLVER_BCD 1    /* Algorithm 3, block coordinate descent (FP32 X, no stopping test) */

/* ntt_plan_desc.flags */
#define NTT_PLAN_EAGER 1u   /* enqueue every launch on each call instead of replaying a
                               cached CUDA graph (debugging; each call then first waits for
                               the previous call of the plan to finish) */

/* Plan description (Algorithm 2's inputs). */
typedef struct {
  int d;                 /* tensor order, 2 <= d <= NTT_MAX_D */
  const int64_t* dims;   /* d mode sizes n_1..n_d (host) */
  const int64_t* ranks;  /* d+1 TT ranks r_0..r_d with r_0 = r_d = 1 (host), or NULL:
                            Algorithm 2's rank rule with eps_rank (see below) */
  int iters;             /* multiplicative-update iterations per stage (>= 1) */
  float eps_mu;          /* epsilon added to both MU denominators (e.g. 1e-12) */
  ntt_dtype x_dtype;     /* NTT_F32, or NTT_BF16: each unfolding is cast to BF16 and
                            iterated with FP32 accumulation, then refined in FP32 */
  int refine_iters;      /* FP32 iterations after the BF16 ones (BF16 form only) */
  uint64_t seed;         /* seed of the counter-based initialisation */
  double tol;            /* stopping test of each stage's main MU loop (Algorithm 3's loop
                            tracks the objective f = 1/2||X-WH||^2 and runs to a maximum
                            count): 0 runs `iters` iterations; > 0 stops after iteration u,
                            u a multiple of check_every and u >= 2 check_every, once
                            f_{u-K} - f_u <= tol |f_{u-K}| (f in FP64, Gram form).  The
                            refinement iterations always run.  >= 0. */
  int check_every;       /* K of that test; >= 1 when tol > 0 */
  int route;             /* ntt_route of every stage (0 = NTT_ROUTE_AUTO) */
  unsigned flags;        /* NTT_PLAN_* bits (0: cached CUDA graph) */
  double eps_rank;       /* ranks == NULL: Algorithm 2's threshold.  Before stage l's NMF,
                            r_l = the smallest k >= 1 with
                              sqrt(s_{k+1}^2 + ... + s_N^2) / sqrt(s_1^2 + ... + s_N^2) <= eps_rank,
                            s_i the singular values of X_l, N = min(m, n); > 0 */
  int rank_cap;          /* ranks == NULL: upper bound of every chosen rank (0: NTT_MAX_RANK).
                            The rule's rank is also capped at NTT_MAX_RANK and at
                            NTT_MAX_ROWS / n_{l+1}, so that the next unfolding fits the
                            built height (ntt_plan_get_ranks reports these bounds). */
  int solver;            /* NTT_SOLVER_MU or NTT_SOLVER_BCD; `iters` counts its iterations */
} ntt_plan_desc;

/* Per-stage statistics, filled by ntt_plan_get_stats after the last call. */
typedef struct {
  int d;                            /* tensor order of the plan */
  int status;                       /* device status word (ntt_status) */
  int iters[NTT_MAX_D];             /* MU iterations run per stage (BF16 + FP32; fewer than
                                       iters + refine_iters when the stopping test fired) */
  int64_t m[NTT_MAX_D], n[NTT_MAX_D], r[NTT_MAX_D];   /* unfolding shapes */
  double xnorm2[NTT_MAX_D];         /* ||X_l||_F^2 (FP64 reduction) */
  double obj_first[NTT_MAX_D];      /* 1/2||X-WH||^2 after the first iteration (Gram form) */
  double obj_last[NTT_MAX_D];       /* same after the last iteration (Gram form) */
  double resid[NTT_MAX_D];          /* 1/2||X-WH||^2 at stage end, direct FP64 pass */
  float stage_ms[NTT_MAX_D];        /* device time of each stage (CUDA events) */
  float iter_ms[NTT_MAX_D];         /* device time of the stage's MU iteration loop */
  float total_ms;                   /* device time of the whole decomposition */
  double alg_bytes[NTT_MAX_D];      /* algorithmic bytes of one MU iteration of the stage:
                                       m n sizeof(X) + 8 r n (X read once, H read+written) */
  int64_t launches;                 /* kernels launched by one decomposition */
  int engine[NTT_MAX_D];            /* kernel of the stage's main MU loop: NTT_ENGINE_* */
} ntt_stats;

#define NTT_ENGINE_FMA_PASS 0         /* single-problem fused pass, packed FP32 FMAs */
#define NTT_ENGINE_GROUPED 1          /* grouped engine (register-tiled FMA pass) */
#define NTT_ENGINE_TC_BF16 2          /* BF16-X tensor-core pass (tcgen05 kind::f16) */
#define NTT_ENGINE_TC_TF32 3          /* retired (a 3xTF32 pass, slower than the split form) */
#define NTT_ENGINE_FMA_NARROW 4       /* warp-streamed FMA pass: <= 32 rows, rank <= 8, FP32 X */
#define NTT_ENGINE_BCD_PASS 5         /* the fused pass in its BCD (Algorithm 3) mode */
#define NTT_ENGINE_TC_SPLIT 6         /* FP32 X split in two BF16 matrices on the tensor-core pass */
#define NTT_ENGINE_TC_NARROW 7        /* warp-level BF16 MMAs: FP32 X of 17..32 rows at rank <= 8 split in two
                                         BF16 terms, or BF16 X of <= 16 rows at rank 9..16 */

/* Human-readable name of a status code (static string). */
const char* ntt_status_string(ntt_status s);

/* Library version string (static). */
const char* ntt_version(void);

/* Validate `desc` and build a plan (host only, no device work).  Checks the
 * ranks against Algorithm 2's feasibility bound r_k <= min(r_{k-1} n_k,
 * prod_{j>k} n_j), r_k <= NTT_MAX_RANK and r_{k-1} n_k <= NTT_MAX_ROWS.
 * With ranks == NULL the workspace and the core buffers are sized for the
 * largest ranks the rule may choose (ntt_plan_get_ranks before any call).
 * On success *out owns a plan to be released with ntt_plan_destroy. */
ntt_status ntt_plan_create(const ntt_plan_desc* desc, ntt_plan* out);

/* The plan's d+1 TT ranks: the given ones; with the rank rule, the ranks the
 * last ntt_decompose chose, or before any call the largest the rule may
 * choose (core k then needs r_k n_{k+1} r_{k+1} floats of those bounds). */
ntt_status ntt_plan_get_ranks(ntt_plan plan, int64_t* ranks);

/* Device workspace bytes needed by ntt_decompose with this plan. */
ntt_status ntt_plan_workspace_size(ntt_plan plan, size_t* bytes);

/* Device workspace bytes needed by ntt_decompose_host (adds room for two
 * copies of A, the cores and the Eq. (3) scratch). */
ntt_status ntt_plan_workspace_size_host(ntt_plan plan, size_t* bytes);

/* Algorithm 2 on the device.
 *   A         device, prod(dims) FP32 entries, C order, >= 0; read only.
 *   cores     host array of d device pointers; core k (0-based) receives
 *             G_{k+1} as r_k x n_{k+1} x r_{k+1} FP32 (written).
 *   workspace device, >= ntt_plan_workspace_size bytes, 256-byte aligned;
 *             overwritten.
 * Stage l uses W = core l as its m x r factor and H in the workspace (the
 * last stage writes H straight into the last core), so no reshape copies are
 * made: each reshape of Algorithm 1/2 is a C-order view.
 * With the rank rule (ranks == NULL) each stage first computes the singular
 * values of its unfolding and picks r_l on the device, then the host reads
 * r_l (the call synchronises `stream` once per stage) and enqueues the
 * stage's NMF; core k is written packed as r_k x n_{k+1} x r_{k+1} of the
 * chosen ranks at the start of its buffer (sized for the bounds), and the
 * call returns after the last stage has been enqueued (not finished).
 * Otherwise the whole decomposition is one cached CUDA graph per (A, cores, workspace) triple
 * (two triples are kept), launched on `stream`; the graph contains kernel
 * nodes only.  Capturing a third triple first waits for the last launch of
 * the graph it replaces. */
ntt_status ntt_decompose(ntt_plan plan, const float* A, float* const* cores,
                         void* workspace, void* stream);

/* Stage-level checkpoint and resume (the paper keeps the tensor and the
 * intermediate factors in a store between the stages of Algorithm 2,
 * Section III-B).  Runs stages s0 .. s1-1 of the plan (0 <= s0 < s1 <= d-1;
 * stage s computes core s and the next unfolding) on `stream`, without a
 * graph:
 *   X_in   device FP32: A when s0 == 0, else the unfolding H_{s0}
 *          (ntt_unfolding_size floats, r_{s0} x n_{s0}, row-major) that an
 *          earlier call returned in H_out;
 *   cores  device pointers of all d cores; cores s0 .. s1-1 are written (and
 *          core d-1 when s1 == d-1), the others are not touched;
 *   H_out  device FP32 (nullable when s1 == d-1): receives H_{s1}, the input
 *          of a later call with s0 = s1.
 * Stage s draws its initial factors from (seed, s) only, so the cores of
 * runs split at any stages are bitwise those of one ntt_decompose call.
 * Plans with the rank rule (ranks == NULL) return NTT_ERR_UNSUPPORTED.
 * The stage statistics cover the stages of the last call. */
ntt_status ntt_decompose_stages(ntt_plan plan, int s0, int s1, const float* X_in, float* const* cores,
                                float* H_out, void* workspace, void* stream);

/* Floats of the unfolding H_s that stage s reads (1 <= s <= d-2):
 * r_s x prod_{j >= s} n_j. */
ntt_status ntt_unfolding_size(ntt_plan plan, int s, int64_t* floats);

/* Same as ntt_decompose with A and the cores in HOST memory: A is copied to
 * the workspace, the decomposition runs, the cores are copied back, all on
 * `stream` (asynchronous with pinned host memory; sync before reading).
 * err_host (nullable, 3 doubles) receives Eq. (3) of the result as
 * ntt_rel_error reports it.  workspace: ntt_plan_workspace_size_host bytes.
 * Successive calls alternate between two input slots of the workspace: a
 * call's host-to-device copy runs on the plan's own copy stream, waits only
 * for the call two back to finish reading that slot, and so overlaps the
 * previous call's decomposition; the decomposition waits for its copy.
 * The slot events belong to the plan: successive host calls of one plan must
 * use the same workspace (or synchronise `stream` before switching).
 * A_host must stay unchanged until `stream` has passed the call. */
ntt_status ntt_decompose_host(ntt_plan plan, const float* A_host, float* const* cores_host,
                              double* err_host, void* workspace, void* stream);

/* Synchronise the stream of the last decomposition and read its statistics. */
ntt_status ntt_plan_get_stats(ntt_plan plan, ntt_stats* out);

/* Release a plan and its cached graphs. */
ntt_status ntt_plan_destroy(ntt_plan plan);

/* Workspace bytes for nmf_mu_step on an m x n problem of rank r. */
ntt_status nmf_mu_workspace_size(int64_t m, int64_t n, int r, ntt_dtype x_dtype, size_t* bytes);

/* `iters` multiplicative-update iterations (H first, then W) of one NMF,
 * in place on W and H -- the inner loop of every stage of Algorithm 2.
 *   X       device m x n, FP32 (x_dtype NTT_F32) or BF16 (NTT_BF16), >= 0.
 *   W       device m x r FP32 (in/out), H device r x n FP32 (in/out).
 *   obj_dev device array of `iters` doubles or NULL; obj_dev[t] receives
 *           1/2||X - W_{t+1} H_{t+1}||_F^2 in the expanded Gram form
 *           ||X||^2 - 2<W, X H^T> + <W^T W, H H^T>, reduced in FP64.
 *   ws      device workspace of nmf_mu_workspace_size bytes (overwritten).
 * 1 <= r <= NTT_MAX_RANK, 1 <= m <= NTT_MAX_ROWS, n >= 1. */
ntt_status nmf_mu_step(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype,
                       float* W, float* H, int iters, float eps_mu, double* obj_dev,
                       void* ws, void* stream);

/* ------------------------------------------------------------------------
 * Out-of-core multiplicative updates: X larger than device memory (the
 * paper's Section IV runs a 550 GB synthetic tensor) stays in host memory and
 * every iteration streams it to the device in column chunks of chunk_cols
 * columns (a multiple of 4) through two device buffers; the copy of the next
 * chunk (host row pitch n) overlaps the fused pass over the current one, whose
 * H columns are read and written in place.  Each chunk's [P ; Q] is reduced in
 * FP64 and added in chunk order, then W is updated once per iteration.  Pinned
 * host memory (cudaHostAlloc / cudaHostRegister) is needed for the copies to
 * run asynchronously at the link rate.  With n <= chunk_cols X is copied once.
 * m <= NTT_MAX_ROWS, r <= NTT_MAX_RANK.
 * ------------------------------------------------------------------------ */
ntt_status nmf_mu_host_workspace_size(int64_t m, int64_t n, int r, int64_t chunk_cols, size_t* bytes);

/* `iters` MU iterations with X_host (host m x n FP32, C order) streamed; W
 * (m x r) and H (r x n) device FP32, in place; obj_dev (nullable, `iters`
 * doubles) the FP64 Gram-form objective after each iteration.  ws: device,
 * nmf_mu_host_workspace_size bytes (two chunk buffers of 4 m chunk_cols bytes
 * dominate).  Returns after enqueueing; X_host must stay unchanged until the
 * stream has passed the call. */
ntt_status nmf_mu_step_host(int64_t m, int64_t n, int r, const float* X_host, float* W, float* H, int iters,
                            float eps_mu, double* obj_dev, int64_t chunk_cols, void* ws, void* stream);

/* ------------------------------------------------------------------------
 * Column-sharded multiplicative updates: the 1-D column distribution of
 * Section III-B with one GPU per shard.  Every rank holds a contiguous block of
 * n_shard columns of X (m x n_shard FP32, device) and of H (r x n_shard) and a
 * replica of W (m x r).  One iteration:
 *   nmf_mu_shard_pass   (local)  H update of the local columns, then the
 *                                local [P ; Q] = [X ; H] H^T reduced into FP64
 *   all-reduce (sum) of [P ; Q] over the ranks -- the caller's collective, the
 *                                exchange step of Algorithms 4-6
 *   nmf_mu_shard_update (replicated) W <- max(0, W o P / (W Q + eps)) and the
 *                                objective 1/2 (||X||^2 - 2 <W,P> + <W^T W, Q>)
 * The shards exchange neither X nor H.  [P ; Q] is pq_count doubles in the
 * library's layout (nmf_mu_shard_sizes); m <= NTT_MAX_ROWS, r <= NTT_MAX_RANK.
 * ------------------------------------------------------------------------ */
ntt_status nmf_mu_shard_sizes(int64_t m, int64_t n_shard, int r, size_t* ws_bytes, size_t* pq_count);

/* out_dev (device, one double) = ||X||_F^2 of the local columns (FP64 sum);
 * its all-reduce gives the xnorm2 of nmf_mu_shard_update.  ws: as below. */
ntt_status nmf_mu_shard_norm(int64_t m, int64_t n_shard, const float* X, double* out_dev, void* ws, void* stream);

/* The local half-iteration.  W: device m x r (read); H: device r x n_shard
 * (updated); pq_out: device pq_count doubles (written); ws: ws_bytes. */
ntt_status nmf_mu_shard_pass(int64_t m, int64_t n_shard, int r, const float* X, const float* W, float* H,
                             float eps_mu, double* pq_out, void* ws, void* stream);

/* The replicated W half from the all-reduced pq (device, pq_count doubles).
 * xnorm2: ||X||_F^2 of the whole (unsharded) X; obj_dev (nullable): one
 * double receiving the objective of (W_new, H).  ws: as for the pass. */
ntt_status nmf_mu_shard_update(int64_t m, int r, const double* pq, float* W, float eps_mu, double xnorm2,
                               double* obj_dev, void* ws, void* stream);

/* ------------------------------------------------------------------------
 * Algorithm 3 (distBCDnmf) on one GPU: block coordinate descent with
 * prox-linear block steps, extrapolation and the correction test, as the
 * APG-BCD method the paper cites defines them:
 *   W_new = max(0, W_m - (W_m H H^T - X H^T) / ||H H^T||_2)
 *   H_new = max(0, H_m - (W^T W H_m - W^T X) / ||W^T W||_2)      (W = W_new)
 * An iteration whose objective 1/2||X - W H||^2 is not below the last
 * accepted one is rejected: the next steps start from the last accepted
 * iterate without extrapolation.  Otherwise t <- (1 + sqrt(1 + 4t^2))/2,
 * w = (t_old - 1)/t and each block is extrapolated from its accepted iterate,
 * X_m = X_new + min(w, 0.9999 sqrt(L_prev / L)) (X_new - X_acc).  The
 * initial W and H are first scaled to Frobenius norm sqrt(||X||_F) each.
 * Each iteration reads X once (the H step and X H^T, H H^T of the new H
 * from the same tile); FP32 X, m <= NTT_MAX_ROWS, r <= NTT_MAX_RANK.
 * ------------------------------------------------------------------------ */
ntt_status nmf_bcd_workspace_size(int64_t m, int64_t n, int r, size_t* bytes);

/* `iters` BCD iterations on the m x n FP32 X (device), W (m x r) and H
 * (r x n) device FP32: initial factors in, the last accepted iterate out.
 * obj_dev (nullable): `iters` doubles, obj_dev[t] = the last accepted
 * objective after iteration t.  The objective of each new iterate is the
 * direct residual 1/2||X - W H||^2 that the pass sums over the tiles it holds
 * (FP32 within a tile, FP64 across tiles), so the acceptance test sees no
 * cancellation.  ws: device,
 * nmf_bcd_workspace_size bytes, 256-byte aligned (overwritten). */
ntt_status nmf_bcd_step(int64_t m, int64_t n, int r, const float* X, float* W, float* H, int iters,
                        double* obj_dev, void* ws, void* stream);

/* Workspace bytes of nmf_mu_step_route: it adds 4 m n bytes for two BF16
 * terms of an FP32 X (X = bf16(X) + bf16(X - bf16(X))) where a tensor-core
 * form that reads them may run -- with NTT_ROUTE_TC on 128 or 256 rows at rank
 * 9..32 (n a multiple of 8), and on every route but NTT_ROUTE_FMA, _GENERIC
 * and _TC on 17..32 rows at rank <= 8 (n a multiple of 64, the warp-level MMA
 * form); otherwise as nmf_mu_workspace_size.  The plain nmf_mu_step never
 * takes those forms. */
ntt_status nmf_mu_workspace_size_route(int64_t m, int64_t n, int r, ntt_dtype x_dtype, int route,
                                      size_t* bytes);

/* nmf_mu_step with its kernel choice restricted by `route` (ntt_route; the
 * plan's routes other than NTT_ROUTE_GROUPED, which is a plan-level choice and
 * acts here as NTT_ROUTE_AUTO).  *engine_out (nullable) receives the
 * NTT_ENGINE_* of the pass that ran.  ws: nmf_mu_workspace_size_route bytes.
 * Other arguments as for nmf_mu_step. */
ntt_status nmf_mu_step_route(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype,
                             float* W, float* H, int iters, float eps_mu, double* obj_dev,
                             void* ws, void* stream, int route, int* engine_out);

/* nmf_mu_step without a workspace argument, for callers that cannot allocate
 * device memory (for instance a plugin running inside a host process whose own
 * runtime owns every device allocation, or a control loop that must not take
 * the implicit synchronisation of cudaMalloc).  The paper has no counterpart:
 * this is an interface convenience of the library.
 *   Scratch: one file-scope device array of 8 MiB (8 << 20 bytes), held by
 *   every GPU that loads the library until the process exits.  Shapes whose
 *   nmf_mu_workspace_size exceeds 8 MiB return NTT_ERR_OOM and launch nothing
 *   (m <= 512 with r <= 16 always fit; m = 512 with r = 32 does not).
 *   All calls on a device share the array and it keeps the last call's
 *   contents; each call clears the words that must start at zero.  Calls whose
 *   device work overlaps (different streams or host threads) race: serialise
 *   them.  The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.  No allocation of any kind is made.
 * Other arguments and results as for nmf_mu_step. */
ntt_status nmf_mu_step_noalloc(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype,
                               float* W, float* H, int iters, float eps_mu, double* obj_dev,
                               void* stream);

/* Many independent NMFs in one call: problem i is X_i ~ W_i H_i with X_i
 * m[i] x n[i] FP32 (device, row-major, >= 0), W_i m[i] x r[i] and H_i
 * r[i] x n[i] FP32 (device, initial factors in, iterates out), and `iters`
 * multiplicative-update iterations (H first, then W) run on every problem, as
 * nmf_mu_step does on one.  All problems advance together: per iteration one
 * pass launch per (height, rank) bucket and one combine launch for all.
 * Heights above NTT_MAX_ROWS (up to NTT_MAX_TALL_ROWS) run as row blocks of
 * 512: a W^T X partial per block, a fixed-order sum of the blocks for the H
 * update, then a second read of X for X H^T (two reads of X per iteration
 * instead of one).  Every reduction of a problem runs in an order fixed by its
 * own shape, so a problem's iterates are bitwise the same alone or in any mix.
 * Host arrays m, n, r, X, W, H of `count` entries; 1 <= r[i] <= NTT_MAX_RANK.
 * ws: device, nmf_mu_many_workspace_size bytes, 256-byte aligned (overwritten).
 * The grouped pass computes the H half of Algorithm 3's update with one read
 * of X per iteration, like nmf_mu_step; the paper has no many-problem form. */
ntt_status nmf_mu_many_workspace_size(int count, const int64_t* m, const int64_t* n, const int* r,
                                      size_t* bytes);
ntt_status nmf_mu_many(int count, const int64_t* m, const int64_t* n, const int* r, const float* const* X,
                       float* const* W, float* const* H, int iters, float eps_mu, void* ws, void* stream);

/* Device status word left in an nmf_mu_step workspace (sync first). */
ntt_status ntt_status_of_workspace(const void* ws, ntt_status* out);

/* ------------------------------------------------------------------------
 * Algorithm 2's rank rule on its own.  X: device m x n FP32 (C order),
 * min(m, n) <= NTT_MAX_ROWS.  The singular values are the square roots of the
 * eigenvalues of the min(m, n)-sided Gram matrix (X X^T or X^T X), formed from
 * FP32 products summed in runs of 256 and accumulated in FP64, then reduced to
 * tridiagonal form and solved by bisection in FP64.
 * ------------------------------------------------------------------------ */
/* Workspace bytes of ntt_singular_values / ntt_select_rank. */
ntt_status ntt_rank_workspace_size(int64_t m, int64_t n, size_t* bytes);

/* sigma_dev: device, min(m, n) doubles, receives the singular values of X in
 * non-increasing order.  ws: ntt_rank_workspace_size bytes, 256-byte aligned. */
ntt_status ntt_singular_values(int64_t m, int64_t n, const float* X, double* sigma_dev, void* ws,
                               void* stream);

/* rank_dev: device int, receives the smallest k >= 1 with
 * sqrt(sum_{i>k} s_i^2) / sqrt(sum_i s_i^2) <= eps_rank (Algorithm 2), capped
 * at rank_cap when rank_cap > 0; an all-zero X gives 1.  sigma_dev
 * (nullable) receives the singular values as above. */
ntt_status ntt_select_rank(int64_t m, int64_t n, const float* X, double eps_rank, int rank_cap,
                           int* rank_dev, double* sigma_dev, void* ws, void* stream);

/* Failure-detection probe of the bounded device waits (Section III's
 * distributed design has no counterpart; every kernel of this library bounds
 * its waits so that a stuck copy or peer ends the kernel with a status word
 * instead of a hang).  Enqueues one single-CTA kernel on `stream` that starts
 * a real 256-byte bulk copy from `ws`, waits at most limit_ns (>= 0) for an
 * mbarrier phase that nothing completes, drains its own copy (bounded by 2 s)
 * and writes NTT_ERR_TIMEOUT into the workspace's status word -- the path a
 * pass kernel takes when one of its waits gives up.  ws: an nmf_mu_step
 * workspace (>= 256 bytes, 256-byte aligned).  A later nmf_mu_step on the
 * same workspace clears the word. */
ntt_status ntt_wait_probe(void* ws, int64_t limit_ns, void* stream);

/* Counter-based U[0,1) fill: out[i] = (SplitMix64(key) output i >> 40) * 2^-24
 * with key = SplitMix64(seed) output (stage * 2^20 + restart * 2 + matrix)
 * (Steele, Lea & Flood 2014).  This is the initialisation of W (matrix 0)
 * and H (matrix 1) in every stage.  out: device, `count` FP32. */
ntt_status ntt_uniform_init(uint64_t seed, int stage, int restart, int matrix, int64_t count,
                            float* out, void* stream);

/* Workspace bytes of ntt_reconstruct / ntt_rel_error for these cores. */
ntt_status ntt_reconstruct_workspace_size(int d, const int64_t* dims, const int64_t* ranks,
                                          size_t* bytes);

/* Eq. (2): the full tensor of a TT.  cores: host array of d device pointers
 * (core k is r_k x n_{k+1} x r_{k+1} FP32); A_out device prod(dims) FP32.
 * The chain is split at the mode s that balances the two halves: the
 * products G_1..G_s and G_{s+1}..G_d are formed first, then multiplied. */
ntt_status ntt_reconstruct(int d, const int64_t* dims, const int64_t* ranks,
                           const float* const* cores, float* A_out, void* ws, void* stream);

/* Eq. (3): err_dev[0] = ||A - A~||_F / ||A||_F (FP64), A~ the TT of `cores`,
 * computed without materialising A~ (split-chain product fused with the
 * difference and an FP64 reduction).  A: device prod(dims) FP32.
 * err_dev[1] and err_dev[2] receive ||A - A~||^2 and ||A||^2. */
ntt_status ntt_rel_error(int d, const int64_t* dims, const int64_t* ranks,
                         const float* const* cores, const float* A, double* err_dev,
                         void* ws, void* stream);

/* ------------------------------------------------------------------------
 * Batched form: B independent nTTs, each stage solved from `restarts` random
 * initialisations (restart j of stage s of instance i uses the init streams
 * (seed + i, s, j, 0/1)); the restart with the lowest final 1/2||X - WH||^2
 * is kept (ties: lowest index), hand-off normalised, and its H becomes the
 * next unfolding (Algorithm 2 per instance).  Small unfoldings are solved one
 * NMF per CTA in shared memory; large ones run several restarts side by side
 * in one streaming pass (restarts are independent blocks of one NMF).
 * ------------------------------------------------------------------------ */
typedef struct ntt_batch_s* ntt_batch;

/* d[i] (B entries), dims (sum d[i] entries), ranks (sum (d[i]+1) entries),
 * all host arrays, instance after instance.  Validates like ntt_plan_create. */
ntt_status ntt_batch_create(int B, const int* d, const int64_t* dims, const int64_t* ranks,
                            int iters, int restarts, float eps_mu, uint64_t seed, ntt_batch* out);

/* Sizes of the packed input (floats), packed cores (floats) and workspace (bytes). */
ntt_status ntt_batch_sizes(ntt_batch b, size_t* input_floats, size_t* core_floats,
                           size_t* workspace_bytes);

/* Offsets (in floats) of each instance's tensor in the packed input (B entries)
 * and of each core in the packed cores (sum d[i] entries, instance after instance). */
ntt_status ntt_batch_offsets(ntt_batch b, int64_t* input_off, int64_t* core_off);

/* Decompose all instances.  A: device packed tensors (C order each); cores:
 * device packed cores (core k of instance i is r_k x n_{k+1} x r_{k+1});
 * workspace: device, ntt_batch_sizes bytes, 256-byte aligned.  The whole
 * batch -- every stage's small NMFs, grouped engine launches, residuals and
 * selections -- is one cached CUDA graph per (A, cores, workspace) triple (two
 * triples are kept; replacing one first waits for its last launch), launched
 * on `stream`; the call returns without waiting.  The graph holds kernel nodes
 * only: its tables live in the batch's mapped pinned host memory, written once
 * at capture, and are uploaded by kernels on every launch.  The device status
 * word is the first word of the workspace (ntt_status_of_workspace after a
 * stream synchronisation). */
ntt_status ntt_decompose_batched(ntt_batch b, const float* A, float* cores, void* workspace,
                                 void* stream);

/* Autotuner of the batched form: for every stage with grouped (large)
 * unfoldings, the CTA split of the grouped engine -- how many CTAs problems
 * sharing a launch get: 1/split of one wave's tile share each, split in
 * {1, 2, 4, 8} -- is taken from `cache_path` when that file holds an entry
 * for the stage's signature (a hash of its problem shapes and the SM count),
 * else timed: the batch runs eagerly on the caller's buffers once per
 * candidate with probe_iters iterations per stage (CUDA events around each
 * stage's grouped iterations), the fastest split is kept and appended to
 * cache_path (nullable: no file).  Synchronises `stream`; the outputs of the
 * probe runs are overwritten by the next ntt_decompose_batched.  Cached
 * graphs are dropped and recaptured with the chosen splits.  The workspace
 * size does not depend on the choice. */
ntt_status ntt_batch_tune(ntt_batch b, const float* A, float* cores, void* workspace, void* stream,
                          int probe_iters, const char* cache_path);

/* The split of each stage (max_stages entries; 0 for stages without grouped
 * work) and how many stages took theirs from the cache file / were timed by
 * the last ntt_batch_tune. */
ntt_status ntt_batch_get_tuning(ntt_batch b, int max_stages, int* split, int* from_cache, int* timed);

ntt_status ntt_batch_destroy(ntt_batch b);

/* ------------------------------------------------------------------------
 * Serving form: continuous batching of nTT jobs (Algorithm 2 per job, one
 * initialisation per stage, fixed iterations per stage).  Jobs wait in FIFO
 * order; the head is admitted while a job slot is free and its device
 * footprint (ntt_server_job_footprint) fits the HBM budget, an arena the
 * server allocates once.  Resident jobs advance together in ticks of
 * tick_iters multiplicative-update iterations of their current stage through
 * the grouped engine of nmf_mu_many; at a stage end (stage_iters divisible by
 * tick_iters) the job takes the column-L1 hand-off, and after its last stage
 * its cores are copied to the caller's host buffer.  Initial factors of stage
 * s come from the streams (seed, s, 0, 0/1) of the job's own seed, and every
 * reduction runs in an order fixed by the job's own shapes: a job's cores are
 * bitwise the same alone or among any others.  The paper has no serving form.
 * ------------------------------------------------------------------------ */
typedef struct ntt_server_s* ntt_server;

typedef struct {
  size_t hbm_budget_bytes;   /* device arena for jobs (>= 1 MiB); engine tables are extra */
  int max_jobs;              /* resident job slots */
  int tick_iters;            /* MU iterations per tick; divides stage_iters */
  int stage_iters;           /* MU iterations per stage */
  float eps_mu;
} ntt_server_config;

#define NTT_JOB_QUEUED 0
#define NTT_JOB_RUNNING 1
#define NTT_JOB_DONE 2
#define NTT_JOB_FAILED 3

typedef struct {
  int state;                 /* NTT_JOB_* */
  ntt_status status;         /* NTT_OK, or why the job failed */
  int stage;                 /* stage in progress (d - 1 when done) */
  double t_submit, t_admit, t_done;   /* seconds on the server's steady clock; -1 if not yet */
  size_t footprint_bytes;    /* arena bytes the job holds while resident */
} ntt_job_info;

typedef struct {
  int64_t submitted, completed, failed, ticks;
  int resident, queued;
  size_t bytes_in_use, peak_bytes, capacity_bytes;
  double busy_s;             /* engine time spent in ticks */
} ntt_server_stats;

/* Allocates the arena, starts the engine thread on the current device. */
ntt_status ntt_server_create(const ntt_server_config* cfg, ntt_server* out);

/* Device bytes a job of this shape holds while resident (input in FP32, plus
 * its BF16 copy for NTT_BF16 jobs, ping-pong unfoldings, cores, engine scratch). */
ntt_status ntt_server_job_footprint(int d, const int64_t* dims, const int64_t* ranks, ntt_dtype dtype,
                                    size_t* bytes);

/* Queue one job.  A_host: host tensor, prod(dims) entries of FP32 or BF16
 * (C order), read when the job is admitted -- keep it unchanged until the job
 * is done; pinned memory makes the copy asynchronous.  cores_host: host buffer
 * of sum_k r_{k-1} n_k r_k floats that receives the cores, core after core.
 * Returns NTT_ERR_OOM at once when the footprint exceeds the whole budget. */
ntt_status ntt_server_submit(ntt_server s, int d, const int64_t* dims, const int64_t* ranks, const void* A_host,
                             ntt_dtype dtype, uint64_t seed, float* cores_host, int64_t* job_id);

/* State of a job (non-blocking). */
ntt_status ntt_server_poll(ntt_server s, int64_t job_id, ntt_job_info* info);

/* Block until the job is done or failed (timeout_s < 0: no limit; on timeout
 * NTT_ERR_TIMEOUT and the job stays known).  Returns the job's status and
 * forgets the job. */
ntt_status ntt_server_wait(ntt_server s, int64_t job_id, double timeout_s, ntt_job_info* info);

ntt_status ntt_server_get_stats(ntt_server s, ntt_server_stats* out);

/* Stops the engine after its current tick; queued and resident jobs are dropped. */
ntt_status ntt_server_destroy(ntt_server s);

/* Eq. (4): prod n_i / sum n_i r_{i-1} r_i (host arithmetic). */
double ntt_compression_ratio(int d, const int64_t* dims, const int64_t* ranks);

#ifdef __cplusplus
}
#endif

#endif /* NTT_H */
