// C ABI of libntt: plans, workspace layout, the stage loop of Algorithm 2,
// CUDA-graph capture of the whole decomposition, statistics, and the
// reconstruction / relative-error entry points (Eq. (2)-(4)).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "group_engine.cuh"

#define NTT_CUDA_TRY_NS(expr)                      \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return NTT_ERR_CUDA;                         \
    }                                              \
  } while (0)
#define NTT_TRY_NS(expr)             \
  do {                               \
    ntt_status s_ = (expr);          \
    if (s_ != NTT_OK) return s_;     \
  } while (0)

using namespace ntt;

namespace ntt {

// Launch the gram and `iters` (pass, combine) pairs of one NMF.
ntt_status run_mu_iters(const MuShape& shp, const MuDev& dev, float eps, int iters, int t0,
                        cudaStream_t st, int* engine) {
  CUtensorMap mx, mh;
  std::memset(&mx, 0, sizeof(mx));
  std::memset(&mh, 0, sizeof(mh));
  MuShape s = shp;
  s.split_ok = dev.xs != nullptr && !s.bf16;
  mu_finalize_shape(&s, dev.X, dev.H, device_sms());
  if (engine)
    *engine = s.tcs ? NTT_ENGINE_TC_SPLIT
                    : (s.tcw ? NTT_ENGINE_TC_NARROW
                             : (s.tcb ? NTT_ENGINE_TC_BF16
                                      : (s.narrow ? NTT_ENGINE_FMA_NARROW : NTT_ENGINE_FMA_PASS)));
  MuDev d = dev;
  if (s.tcs && s.MP <= 32) {
    // the stacked form: X = X1 + X2 (bf16(X) and bf16(X - bf16(X))), once for the whole loop
    const int64_t mn = s.m * s.n;
    NTT_CUDA_TRY_NS(launch_split_bf16x2(reinterpret_cast<const float*>(dev.X), dev.xs, dev.xs + mn, mn, st));
    d.X = dev.xs;
    d.X2 = dev.xs + mn;
  } else if (s.tcs) {
    // the same two terms as the tile-major image of the pass's stages
    NTT_CUDA_TRY_NS(launch_split_blocked(reinterpret_cast<const float*>(dev.X), dev.xs, s.m, s.n, s.MP, st));
    d.X = dev.xs;
    d.X2 = nullptr;
  }
  if (s.tcw && s.bf16) {
    NTT_TRY_NS(encode_tcwb_maps(s, dev.X, dev.H, &mx, &mh));
  } else if (s.tcw) {
    // the same two terms, interleaved by 64-column segments, once for the whole loop
    NTT_CUDA_TRY_NS(launch_split_x12(reinterpret_cast<const float*>(dev.X), dev.xs, s.m, s.n, st));
    NTT_TRY_NS(encode_tcw_maps(s, dev.xs, dev.H, &mx, &mh));
    d.X = dev.xs;
  }
  if (s.tma && !s.tcs && !s.tcw) NTT_TRY_NS(mu_encode_maps(s, dev.X, dev.H, &mx, &mh));
  for (int t = 0; t < iters; ++t) {
    NTT_CUDA_TRY_NS(launch_mu_pass(s, d, eps, mx, mh, st));
    NTT_CUDA_TRY_NS(launch_mu_combine(s, d, eps, t0 + t, st));
  }
  return NTT_OK;
}

ntt_status resid_into(const void* X, int xbf16, const float* L, const float* Rm, int64_t M,
                      int64_t N, int r, int mode, double scale, double* acc, double* rel,
                      double* part64, unsigned* ticket, cudaStream_t st) {
  ResidArgs a;
  a.X = X;
  a.xbf16 = xbf16;
  a.L = L;
  a.Rm = Rm;
  a.M = M;
  a.N = N;
  a.r = r;
  a.mode = mode;
  a.part64 = part64;
  a.ticket = ticket;
  a.acc = acc;
  a.rel = rel;
  a.scale = scale;
  int blocks = resid_blocks(device_sms());
  if (blocks > kMaxResidBlocks) blocks = kMaxResidBlocks;
  NTT_CUDA_TRY_NS(launch_resid(a, blocks, st));
  return NTT_OK;
}


}  // namespace ntt

namespace {


size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  }
};

int64_t prod(const int64_t* v, int a, int b) {  // prod v[a..b)
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= v[i];
  return p;
}

#define NTT_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return NTT_ERR_CUDA;                         \
    }                                              \
  } while (0)

#define NTT_TRY(expr)                \
  do {                               \
    ntt_status s_ = (expr);          \
    if (s_ != NTT_OK) return s_;     \
  } while (0)

// Scratch of one multiplicative-update NMF (shared by nmf_mu_step and stages).
struct MuWs {
  size_t status, tickets, scal, G, red, part, part64, xs;
};

size_t mu_partial_floats(const MuShape& s) { return (size_t)s.grid_cap * s.part_stride(); }

int split_point(int d, const int64_t* dims) {
  double total = 0.0;
  for (int i = 0; i < d; ++i) total += std::log((double)dims[i]);
  int best_s = 1;
  double best = 1e300;
  double left = 0.0;
  for (int s = 1; s < d; ++s) {
    left += std::log((double)dims[s - 1]);
    const double score = std::fabs(left - 0.5 * total);
    if (score < best) {
      best = score;
      best_s = s;
    }
  }
  return best_s;
}

ntt_status check_tt(int d, const int64_t* dims, const int64_t* ranks) {
  if (d < 2 || d > NTT_MAX_D || !dims || !ranks) return NTT_ERR_INVALID_ARG;
  if (ranks[0] != 1 || ranks[d] != 1) return NTT_ERR_INVALID_ARG;
  for (int i = 0; i < d; ++i)
    if (dims[i] < 1) return NTT_ERR_INVALID_ARG;
  for (int i = 1; i < d; ++i)
    if (ranks[i] < 1 || ranks[i] > NTT_MAX_RANK) return NTT_ERR_UNSUPPORTED;
  return NTT_OK;
}

// Layout of the reconstruction workspace: chain buffers for L and R.
struct ChainWs {
  int s = 1;
  int64_t rows = 0, cols = 0;   // L is rows x r_s, R is r_s x cols
  size_t L[2], R[2], part64, ticket, acc, total;
};

ChainWs chain_layout(int d, const int64_t* dims, const int64_t* ranks) {
  ChainWs c;
  c.s = split_point(d, dims);
  Arena ar;
  size_t lmax = 1, rmax = 1;
  for (int k = 2; k <= c.s; ++k) {  // L_k = G_1..G_k : prod_{i<=k} n_i x r_k
    const size_t sz = (size_t)prod(dims, 0, k) * ranks[k];
    if (sz > lmax) lmax = sz;
  }
  for (int k = c.s + 1; k <= d - 1; ++k) {  // R_k = G_k..G_d: r_{k-1} x prod_{i>=k} n_i
    const size_t sz = (size_t)ranks[k - 1] * prod(dims, k - 1, d);
    if (sz > rmax) rmax = sz;
  }
  c.rows = prod(dims, 0, c.s);
  c.cols = prod(dims, c.s, d);
  c.L[0] = ar.take(lmax * 4);
  c.L[1] = ar.take(lmax * 4);
  c.R[0] = ar.take(rmax * 4);
  c.R[1] = ar.take(rmax * 4);
  c.part64 = ar.take(2 * kMaxResidBlocks * sizeof(double));
  c.ticket = ar.take(64);
  c.acc = ar.take(8 * sizeof(double));
  c.total = ar.off;
  return c;
}

// Form L = G_1..G_s and R = G_{s+1}..G_d in the chain workspace.
ntt_status build_chain(int d, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                       const ChainWs& c, char* ws, const float** Lout, const float** Rout,
                       cudaStream_t st) {
  const float* L = cores[0];  // n_1 x r_1
  int64_t rows = dims[0];
  int li = 0;
  for (int k = 2; k <= c.s; ++k) {
    float* dst = reinterpret_cast<float*>(ws + c.L[li]);
    // (rows x r_{k-1}) @ (r_{k-1} x n_k r_k)
    NTT_CUDA_TRY(launch_small_mm(L, cores[k - 1], dst, rows, (int)ranks[k - 1], dims[k - 1] * ranks[k], st));
    rows *= dims[k - 1];
    L = dst;
    li ^= 1;
  }
  const float* R = cores[d - 1];  // r_{d-1} x n_d
  int64_t cols = dims[d - 1];
  int ri = 0;
  for (int k = d - 1; k >= c.s + 1; --k) {
    float* dst = reinterpret_cast<float*>(ws + c.R[ri]);
    // (r_{k-1} n_k x r_k) @ (r_k x cols)
    NTT_CUDA_TRY(launch_small_mm(cores[k - 1], R, dst, ranks[k - 1] * dims[k - 1], (int)ranks[k], cols, st));
    cols *= dims[k - 1];
    R = dst;
    ri ^= 1;
  }
  *Lout = L;
  *Rout = R;
  return NTT_OK;
}

}  // namespace

// ===========================================================================
// Plan
// ===========================================================================
struct ntt_plan_s {
  int d = 0;
  std::vector<int64_t> dims, ranks;
  int iters = 0;
  float eps = 1e-12f;
  ntt_dtype xdt = NTT_F32;
  int refine = 0;
  uint64_t seed = 0;
  double tol = 0.0;              // stopping test of each stage's main loop (0: fixed count)
  int check = 0;
  int route = NTT_ROUTE_AUTO;    // ntt_route of every stage
  bool eager = false;            // NTT_PLAN_EAGER: enqueue every call, no graph
  // Algorithm 2's rank rule: ranks chosen stage by stage at run time
  bool auto_rank = false;
  double eps_rank = 0.0;
  std::vector<int64_t> ranks_max;   // the largest ranks the rule may pick (workspace sizing)
  size_t off_rank = 0, rank_bytes = 0;
  size_t grp_bytes = 0;             // grouped-engine scratch reserved in the layout
  int solver = NTT_SOLVER_MU;       // NMF of every stage
  size_t off_bcd = 0;               // BCD scratch (solver == NTT_SOLVER_BCD)
  size_t off_xs = 0;                // the two BF16 terms of a split-form stage's X
  size_t off_stop = 0;           // one stop word per stage

  // A stage's MU loop runs either on the single-problem pass (TMA, phase
  // split) or on the grouped engine with this one problem, whichever measured
  // faster for its shape (plan_route_group).
  struct Route {
    bool on = false;
    ntt::GroupPlan gp;
    size_t host_off = 0;   // pinned host tables of this route
  };
  struct Stage {
    int64_t m, n;
    int r;
    MuShape f32, bf16;
    Route gf32, gbf16;
    int iters_total;
    size_t obj_off;  // index into the objective array
    double alg_bytes;
    int engine = NTT_ENGINE_FMA_PASS;   // kernel of the main MU loop (set when enqueued)
  };
  std::vector<Stage> st;
  // workspace layout
  size_t off_status = 0, off_tickets = 0, off_scal = 0, off_obj = 0, off_G = 0, off_red = 0,
         off_part = 0, off_part64 = 0, off_hs = 0, off_H[2] = {0, 0}, off_xb = 0, ws_bytes = 0;
  size_t off_A[2] = {0, 0}, off_cores = 0, ws_bytes_host = 0;   // two input slots (host variant)
  std::vector<size_t> core_off;
  size_t obj_total = 0;
  // graph cache: two entries, so the host variant's two input slots both stay
  // captured.  Each entry owns the mapped pinned host tables of its routed
  // stages (written once, at capture; a kernel node of its graph uploads them
  // into the workspace on every launch) and an event recorded after its last
  // launch, waited for before the entry is recaptured.
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    const void* A = nullptr;
    void* ws = nullptr;
    std::vector<float*> cores;
    char* h_tab = nullptr;         // host address of the tables
    char* h_tab_dev = nullptr;     // device address of the same memory
    cudaEvent_t done = nullptr;
    bool launched = false;
  };
  Graph graphs[2];
  int graph_victim = 0;
  cudaStream_t cap = nullptr;
  // host variant: the copy of the next call's input overlaps this call's compute
  cudaStream_t copy_st = nullptr;
  cudaEvent_t slot_ready[2] = {nullptr, nullptr}, slot_free[2] = {nullptr, nullptr};
  int host_slot = 0;
  std::vector<cudaEvent_t> ev;   // 4 per stage + 2 total
  int64_t launches = 0;          // kernels per decomposition
  size_t off_chain = 0, off_err = 0;
  size_t off_grp = 0;            // grouped-engine scratch shared by the routed stages
  char* h_eager = nullptr;       // tables of the eager path (host / device address)
  char* h_eager_dev = nullptr;
  size_t h_bytes = 0;            // table bytes of all routed stages
  cudaStream_t last_stream = nullptr;
  void* last_ws = nullptr;
  bool ran = false;

  ~ntt_plan_s() {
    for (auto& g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.done) cudaEventDestroy(g.done);
      if (g.h_tab) cudaFreeHost(g.h_tab);
    }
    if (cap) cudaStreamDestroy(cap);
    if (copy_st) cudaStreamDestroy(copy_st);
    for (int i = 0; i < 2; ++i) {
      if (slot_ready[i]) cudaEventDestroy(slot_ready[i]);
      if (slot_free[i]) cudaEventDestroy(slot_free[i]);
    }
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    if (h_eager) cudaFreeHost(h_eager);
    cudaGetLastError();
  }
};

namespace {

// Which MU loop a stage runs: the grouped engine when its height bucket is at
// most 256 rows and its rank bucket at least 16 (where it measured faster than
// the single-problem pass on GB300), else the pass; BF16 stages the tensor-core
// pass takes (128/256 rows; with NTT_ROUTE_TC also 16/32 rows) stay on the
// single-problem path.  The plan's route restricts the choice (ntt_route).
// split_ok: the split tensor-core form may take FP32 stages (not in precision-form
// plans, whose FP32 refinement iterations exist to restore full FP32 X).
bool plan_route_group(int64_t m, int64_t n, int r, bool xbf16, int route, bool split_ok = true) {
  const int MP = group_mp_bucket((int)m), R = group_r_bucket(r);
  if (MP < 0 || R < 0) return false;
  if (xbf16 && (!gpass_bf16_supported(MP, R) || n % 8 != 0)) return false;
  if (route == NTT_ROUTE_PASS || route == NTT_ROUTE_GENERIC) return false;
  if (route == NTT_ROUTE_GROUPED) return true;
  if (route == NTT_ROUTE_TC && xbf16 && tcb_pass_supported(MP, R)) return false;
  // FP32 stages of 128/256 rows at rank 16/32: the split tensor-core form
  if (!xbf16 && split_ok && tcs_route_ok(m, n, r, route)) return false;
  if (route != NTT_ROUTE_FMA && xbf16 && tcb_pass_supported(MP, R) && MP >= 128) return false;
  // BF16 stages of <= 16 rows at rank 9..16: the warp-level MMA form
  if (xbf16 && tcwb_route_ok(m, n, r, route)) return false;
  return MP <= 256 && R >= 16;
}

// Record the whole decomposition on stream `st` (captured or eager).
// Shapes of stage s from the plan's current ranks (not its routes).
ntt_status make_stage(ntt_plan p, int s, int sms, ntt_plan_s::Stage* out) {
  ntt_plan_s::Stage S;
  const int d = p->d;
  S.m = p->ranks[s] * p->dims[s];
  S.n = prod(p->dims.data(), s + 1, d);
  S.r = (int)p->ranks[s + 1];
  ntt_status e = mu_choose_shape(S.m, S.n, S.r, 0, sms, &S.f32);
  if (e == NTT_OK && p->xdt == NTT_BF16) e = mu_choose_shape(S.m, S.n, S.r, 1, sms, &S.bf16);
  if (e != NTT_OK) return e;
  S.f32.route = p->route;
  S.bf16.route = p->route;
  S.iters_total = p->iters + p->refine;
  S.obj_off = (size_t)s * S.iters_total;
  const double xs = p->xdt == NTT_BF16 ? 2.0 : 4.0;
  S.alg_bytes = (double)S.m * S.n * xs + 8.0 * S.r * S.n;
  *out = S;
  return NTT_OK;
}

// Grouped-engine routes of a stage, planned at scratch offset `base`; host
// table offsets from *h_off on.  Returns the largest scratch end offset.
size_t plan_stage_routes(ntt_plan p, ntt_plan_s::Stage& S, int sms, size_t base, size_t* h_off) {
  size_t end = 0;
  for (int xb = 0; xb < 2; ++xb) {
    ntt_plan_s::Route& rt = xb ? S.gbf16 : S.gf32;
    rt.on = false;
    if (p->solver != NTT_SOLVER_MU) continue;   // the grouped engine runs multiplicative updates only
    if (xb && p->xdt != NTT_BF16) continue;
    if (xb == 0 && p->xdt == NTT_BF16 && p->refine == 0) continue;
    if (!plan_route_group(S.m, S.n, S.r, xb != 0, p->route, p->xdt == NTT_F32)) continue;
    // a main loop with a stopping test runs on the single-problem passes
    const bool main_loop = xb != 0 || p->xdt != NTT_BF16;
    if (main_loop && p->tol > 0.0) continue;
    GroupShape sh;
    sh.n = S.n;
    sh.m = (int)S.m;
    sh.re = S.r;
    sh.blk = S.r;
    sh.xbf16 = xb;
    if (group_plan({sh}, sms, base, false, true, &rt.gp) != NTT_OK) continue;
    rt.on = true;
    end = std::max(end, rt.gp.bytes);
    rt.host_off = *h_off;
    *h_off += (rt.gp.table_bytes + 255) / 256 * 256;
  }
  return end;
}

struct EnqueueCtx {
  bool capturing = false;
  int64_t launches = 0;
};

// Timing event i of the plan on `st` (external event nodes when capturing: a
// plain record on a capturing stream would only mark a capture dependency and
// put no timing node into the graph; a plain record otherwise).
cudaError_t plan_record(ntt_plan p, int i, cudaStream_t st, const EnqueueCtx& c) {
  if (p->ev.empty()) return cudaSuccess;
  return c.capturing ? cudaEventRecordWithFlags(p->ev[i], st, cudaEventRecordExternal)
                     : cudaEventRecord(p->ev[i], st);
}

ntt_status enqueue_begin(ntt_plan p, char* ws, cudaStream_t st, EnqueueCtx* c) {
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  NTT_CUDA_TRY(cudaStreamIsCapturing(st, &cap_status));
  c->capturing = cap_status == cudaStreamCaptureStatusActive;
  // status word, tickets and stop words are consecutive in the layout
  NTT_CUDA_TRY(launch_zero(ws + p->off_status, p->off_stop + NTT_MAX_D * sizeof(int) - p->off_status, st));
  c->launches = 1;
  NTT_CUDA_TRY(plan_record(p, 4 * p->d, st, *c));
  return NTT_OK;
}

// Stage s of Algorithm 2 (init, ||X||^2, Gram, the MU loops, direct objective, hand-off).
ntt_status enqueue_stage(ntt_plan p, int s, const float* A, float* const* cores, char* ws, cudaStream_t st,
                         char* tab, const char* tab_dev, EnqueueCtx* c) {
  int* status = reinterpret_cast<int*>(ws + p->off_status);
  unsigned* tickets = reinterpret_cast<unsigned*>(ws + p->off_tickets);
  double* scal = reinterpret_cast<double*>(ws + p->off_scal);
  double* obj = reinterpret_cast<double*>(ws + p->off_obj);
  int* stop = reinterpret_cast<int*>(ws + p->off_stop);
  const int d = p->d;
  int64_t& launches = c->launches;
  auto rec = [&](int i) { return plan_record(p, i, st, *c); };
  const auto& S = p->st[s];
  NTT_CUDA_TRY(rec(4 * s));
  const float* X = (s == 0) ? A : reinterpret_cast<const float*>(ws + p->off_H[(s - 1) % 2]);
  float* W = cores[s];
  float* H = (s == d - 2) ? cores[d - 1] : reinterpret_cast<float*>(ws + p->off_H[s % 2]);
  NTT_CUDA_TRY(launch_uniform(stream_key(p->seed, s, 0, 0), S.m * S.r, W, st));
  NTT_CUDA_TRY(launch_uniform(stream_key(p->seed, s, 0, 1), (int64_t)S.r * S.n, H, st));
  double* xnorm2 = scal + s;
  NTT_TRY(resid_into(X, 0, nullptr, nullptr, S.m, S.n, 0, 0, 1.0, xnorm2, nullptr,
                     reinterpret_cast<double*>(ws + p->off_part64), tickets + 1, st));
  MuDev dev;
  dev.W = W;
  dev.H = H;
  dev.G = reinterpret_cast<float*>(ws + p->off_G);
  dev.part = reinterpret_cast<float*>(ws + p->off_part);
  dev.red = reinterpret_cast<float*>(ws + p->off_red);
  dev.ticket = tickets;
  dev.obj = obj + S.obj_off;
  dev.xnorm2 = xnorm2;
  dev.status = status;
  dev.part64 = reinterpret_cast<double*>(ws + p->off_part64);
  NTT_CUDA_TRY(launch_gram(S.f32, dev, st));
  launches += 4;
  auto mu = [&](const ntt_plan_s::Route& rt, const MuShape& shp, const void* Xv, int iters,
                int t0) -> ntt_status {
    if (iters <= 0) return NTT_OK;
    const bool main_loop = t0 == 0;
    if (!rt.on) {
      dev.X = Xv;
      // the split tensor-core form on FP32 unfoldings, when the layout reserved its terms
      dev.xs = (p->off_xs && Xv == (const void*)X) ? reinterpret_cast<__nv_bfloat16*>(ws + p->off_xs) : nullptr;
      dev.stop = main_loop && p->tol > 0.0 ? stop + s : nullptr;
      dev.tol = p->tol;
      dev.check = p->check;
      dev.loop_t0 = t0;
      int eng = NTT_ENGINE_FMA_PASS;
      const ntt_status e = run_mu_iters(shp, dev, p->eps, iters, t0, st, &eng);
      if (main_loop) p->st[s].engine = eng;
      // per iteration the pass and the combine's two launches; the split form's
      // X1, X2 once per loop
      launches += 3LL * iters + (eng == NTT_ENGINE_TC_SPLIT || (eng == NTT_ENGINE_TC_NARROW && !shp.bf16) ? 1 : 0);
      return e;
    }
    if (main_loop) p->st[s].engine = NTT_ENGINE_GROUPED;
    GroupPtrs g;
    g.X = Xv;
    g.H = H;
    g.W = W;
    g.scratch = nullptr;
    g.obj = obj + S.obj_off;
    g.xnorm2 = xnorm2;
    group_fill_tables(rt.gp, &g, ws, tab + rt.host_off);
    NTT_CUDA_TRY(launch_copy_words(ws + rt.gp.off_tables, tab_dev + rt.host_off, rt.gp.table_bytes, st));
    launches += 3 + 2LL * iters;   // table upload, ticket reset, Gram; per iteration pass and combine
    return group_launch(rt.gp, ws, ws + rt.gp.off_tables, iters, p->eps, st, t0);
  };
  if (p->solver == NTT_SOLVER_BCD) {
    NTT_CUDA_TRY(rec(4 * s + 2));
    dev.X = X;
    p->st[s].engine = NTT_ENGINE_BCD_PASS;
    NTT_TRY(run_bcd_iters(S.f32, dev, bcd_ws_layout(S.f32), ws + p->off_bcd, p->iters, 0, st));
    launches += 6;   // three norms, scaling, Gram, H copy; the init pass and combine below
  } else if (p->xdt == NTT_BF16) {
    __nv_bfloat16* xb = reinterpret_cast<__nv_bfloat16*>(ws + p->off_xb);
    NTT_CUDA_TRY(launch_cast_bf16(X, xb, S.m * S.n, st));
    launches += 1;
    NTT_CUDA_TRY(rec(4 * s + 2));
    NTT_TRY(mu(S.gbf16, S.bf16, xb, p->iters, 0));
    NTT_TRY(mu(S.gf32, S.f32, X, p->refine, p->iters));
  } else {
    NTT_CUDA_TRY(rec(4 * s + 2));
    NTT_TRY(mu(S.gf32, S.f32, X, p->iters, 0));
  }
  NTT_CUDA_TRY(rec(4 * s + 3));
  if (p->solver == NTT_SOLVER_BCD) launches += 2LL * S.iters_total + 2;
  // stage-end objective, direct FP64 pass: 1/2 ||X - W H||^2
  NTT_TRY(resid_into(X, 0, W, H, S.m, S.n, S.r, 1, 0.5, scal + NTT_MAX_D + s, nullptr,
                     reinterpret_cast<double*>(ws + p->off_part64), tickets + 1, st));
  NTT_CUDA_TRY(launch_handoff(W, H, S.m, S.n, S.r, reinterpret_cast<float*>(ws + p->off_hs), st));
  launches += 3;
  NTT_CUDA_TRY(rec(4 * s + 1));
  return NTT_OK;
}

ntt_status enqueue_end(ntt_plan p, cudaStream_t st, EnqueueCtx* c) {
  NTT_CUDA_TRY(plan_record(p, 4 * p->d + 1, st, *c));
  p->launches = c->launches;
  return NTT_OK;
}

// tab / tab_dev: host and device addresses of the mapped pinned tables of
// the routed stages (written here; uploaded by a kernel at each stage).
ntt_status enqueue_decompose(ntt_plan p, const float* A, float* const* cores, char* ws,
                             cudaStream_t st, char* tab, const char* tab_dev) {
  EnqueueCtx c;
  NTT_TRY(enqueue_begin(p, ws, st, &c));
  for (int s = 0; s < p->d - 1; ++s) NTT_TRY(enqueue_stage(p, s, A, cores, ws, st, tab, tab_dev, &c));
  return enqueue_end(p, st, &c);
}

// Mapped pinned host memory: *host for the host, *dev for kernels.
ntt_status alloc_mapped(size_t bytes, char** host, char** dev) {
  void* h = nullptr;
  void* d = nullptr;
  if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_OOM;
  }
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    return NTT_ERR_CUDA;
  }
  *host = reinterpret_cast<char*>(h);
  *dev = reinterpret_cast<char*>(d);
  return NTT_OK;
}

// Algorithm 2 with the rank rule: per stage, the rank of X_l on the device,
// read by the host (one stream synchronisation), then the stage's NMF
// enqueued with that rank.  Launches are enqueued directly (no graph).
ntt_status decompose_auto_rank(ntt_plan p, const float* A, float* const* cores, char* ws, cudaStream_t st) {
  if (p->ran && p->last_stream) NTT_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  const int d = p->d, sms = device_sms();
  if (p->h_bytes && !p->h_eager) NTT_TRY(alloc_mapped(p->h_bytes, &p->h_eager, &p->h_eager_dev));
  p->ranks = p->ranks_max;
  p->ranks[0] = 1;
  EnqueueCtx c;
  NTT_TRY(enqueue_begin(p, ws, st, &c));
  int* rank_dev = reinterpret_cast<int*>(ws + p->off_scal + 3 * NTT_MAX_D * sizeof(double));
  for (int s = 0; s < d - 1; ++s) {
    const int64_t m = p->ranks[s] * p->dims[s];
    const int64_t n = prod(p->dims.data(), s + 1, d);
    const float* X = (s == 0) ? A : reinterpret_cast<const float*>(ws + p->off_H[(s - 1) % 2]);
    const RankWs w = rank_ws_layout(m, n, sms);
    if (w.bytes > p->rank_bytes) return NTT_ERR_OOM;
    NTT_CUDA_TRY(launch_rank_select(X, m, n, p->eps_rank, (int)p->ranks_max[s + 1], w, ws + p->off_rank, nullptr,
                                    rank_dev + s, st));
    int k = 0;
    NTT_CUDA_TRY(cudaMemcpyAsync(&k, rank_dev + s, sizeof(int), cudaMemcpyDeviceToHost, st));
    NTT_CUDA_TRY(cudaStreamSynchronize(st));
    if (k < 1 || k > p->ranks_max[s + 1]) return NTT_ERR_CUDA;
    p->ranks[s + 1] = k;
    c.launches += 4;
    NTT_TRY(make_stage(p, s, sms, &p->st[s]));
    size_t h = 0;
    if (p->off_grp) {
      const size_t end = plan_stage_routes(p, p->st[s], sms, p->off_grp, &h);
      if (end > p->off_grp + p->grp_bytes || h > p->h_bytes) {
        p->st[s].gf32.on = false;
        p->st[s].gbf16.on = false;
      }
    }
    NTT_TRY(enqueue_stage(p, s, A, cores, ws, st, p->h_eager, p->h_eager_dev, &c));
  }
  return enqueue_end(p, st, &c);
}

}  // namespace

extern "C" {

const char* ntt_status_string(ntt_status s) {
  switch (s) {
    case NTT_OK: return "NTT_OK";
    case NTT_ERR_INVALID_ARG: return "NTT_ERR_INVALID_ARG";
    case NTT_ERR_RANK_INFEASIBLE: return "NTT_ERR_RANK_INFEASIBLE";
    case NTT_ERR_OOM: return "NTT_ERR_OOM";
    case NTT_ERR_CUDA: return "NTT_ERR_CUDA";
    case NTT_ERR_TIMEOUT: return "NTT_ERR_TIMEOUT";
    case NTT_ERR_UNSUPPORTED: return "NTT_ERR_UNSUPPORTED";
  }
  return "NTT_ERR_UNKNOWN";
}

const char* ntt_version(void) { return "libntt 0.1 (sm_103a)"; }

double ntt_compression_ratio(int d, const int64_t* dims, const int64_t* ranks) {
  if (d < 1 || !dims || !ranks) return 0.0;
  double num = 1.0, den = 0.0;
  for (int i = 0; i < d; ++i) {
    num *= (double)dims[i];
    den += (double)dims[i] * (double)ranks[i] * (double)ranks[i + 1];
  }
  return den > 0.0 ? num / den : 0.0;
}

ntt_status ntt_plan_create(const ntt_plan_desc* desc, ntt_plan* out) {
  if (!desc || !out) return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  const int d = desc->d;
  if (d < 2 || d > NTT_MAX_D || !desc->dims) return NTT_ERR_INVALID_ARG;
  const bool auto_rank = desc->ranks == nullptr;
  if (auto_rank && !(desc->eps_rank > 0.0 && desc->eps_rank <= 1e300)) return NTT_ERR_INVALID_ARG;
  if (desc->rank_cap < 0) return NTT_ERR_INVALID_ARG;
  if (desc->iters < 1 || !(desc->eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  if (desc->x_dtype != NTT_F32 && desc->x_dtype != NTT_BF16) return NTT_ERR_INVALID_ARG;
  if (desc->refine_iters < 0) return NTT_ERR_INVALID_ARG;
  if (!(desc->tol >= 0.0) || desc->tol > 1e300) return NTT_ERR_INVALID_ARG;
  if (desc->route < NTT_ROUTE_AUTO || desc->route > NTT_ROUTE_TC) return NTT_ERR_INVALID_ARG;
  if (desc->flags & ~NTT_PLAN_EAGER) return NTT_ERR_INVALID_ARG;
  if (desc->tol > 0.0 && desc->check_every < 1) return NTT_ERR_INVALID_ARG;
  if (desc->solver != NTT_SOLVER_MU && desc->solver != NTT_SOLVER_BCD) return NTT_ERR_INVALID_ARG;
  if (desc->solver == NTT_SOLVER_BCD && (desc->x_dtype != NTT_F32 || desc->tol > 0.0)) return NTT_ERR_UNSUPPORTED;
  const int64_t* dims = desc->dims;
  for (int i = 0; i < d; ++i)
    if (dims[i] < 1) return NTT_ERR_INVALID_ARG;
  std::vector<int64_t> rk(d + 1, 1);
  if (auto_rank) {
    // Largest rank the rule may pick at each stage: min(m, n) (Algorithm 2's
    // N), the built maximum, the caller's cap, and a height of the next
    // unfolding r_l n_{l+1} <= NTT_MAX_ROWS.
    const int64_t cap = desc->rank_cap > 0 ? std::min<int64_t>(desc->rank_cap, NTT_MAX_RANK) : NTT_MAX_RANK;
    if (dims[0] > NTT_MAX_ROWS) return NTT_ERR_UNSUPPORTED;
    for (int k = 1; k < d; ++k) {
      const int64_t m = rk[k - 1] * dims[k - 1];
      const int64_t n = prod(dims, k, d);
      int64_t r = std::min(std::min(m, n), cap);
      if (k < d - 1) r = std::min<int64_t>(r, NTT_MAX_ROWS / dims[k]);
      if (r < 1) return NTT_ERR_UNSUPPORTED;
      rk[k] = r;
    }
  } else {
    const int64_t* ranks = desc->ranks;
    if (ranks[0] != 1 || ranks[d] != 1) return NTT_ERR_INVALID_ARG;
    for (int k = 1; k < d; ++k) {
      const int64_t m = ranks[k - 1] * dims[k - 1];
      const int64_t n = prod(dims, k, d);
      if (ranks[k] < 1) return NTT_ERR_INVALID_ARG;
      if (ranks[k] > m || ranks[k] > n) return NTT_ERR_RANK_INFEASIBLE;
      if (ranks[k] > NTT_MAX_RANK || m > NTT_MAX_ROWS) return NTT_ERR_UNSUPPORTED;
    }
    rk.assign(ranks, ranks + d + 1);
  }
  ntt_plan p = new (std::nothrow) ntt_plan_s();
  if (!p) return NTT_ERR_OOM;
  p->d = d;
  p->dims.assign(dims, dims + d);
  p->ranks = rk;
  p->auto_rank = auto_rank;
  p->eps_rank = desc->eps_rank;
  p->ranks_max = rk;
  p->iters = desc->iters;
  p->eps = desc->eps_mu;
  p->xdt = desc->x_dtype;
  p->refine = desc->x_dtype == NTT_BF16 ? desc->refine_iters : 0;
  p->seed = desc->seed;
  p->tol = desc->tol;
  p->check = desc->tol > 0.0 ? desc->check_every : 0;
  p->route = desc->route;
  p->solver = desc->solver;
  p->eager = auto_rank || (desc->flags & NTT_PLAN_EAGER) != 0;
  const int sms = device_sms();
  size_t max_part = 1, max_red = 1, maxH[2] = {1, 1}, max_xb = 1;
  for (int s = 0; s < d - 1; ++s) {
    ntt_plan_s::Stage S;
    const ntt_status e = make_stage(p, s, sms, &S);
    if (e != NTT_OK) {
      delete p;
      return e;
    }
    p->obj_total += S.iters_total;
    size_t pf = mu_partial_floats(S.f32);
    if (p->xdt == NTT_BF16 && mu_partial_floats(S.bf16) > pf) pf = mu_partial_floats(S.bf16);
    if (pf > max_part) max_part = pf;
    if ((size_t)S.f32.part_stride() > max_red) max_red = S.f32.part_stride();
    if (s < d - 2 && (size_t)(S.r * S.n) > maxH[s % 2]) maxH[s % 2] = (size_t)S.r * S.n;
    if ((size_t)(S.m * S.n) > max_xb) max_xb = (size_t)(S.m * S.n);
    p->st.push_back(S);
  }
  // grouped-engine routes: plan each at offset 0 for its size; one scratch
  // region shared by the routed stages follows the device layout.  With the
  // rank rule, every rank up to the stage's maximum is sized for.
  size_t grp = 0, hb = 0;
  for (int s = 0; s < d - 1; ++s) {
    if (!auto_rank) {
      grp = std::max(grp, plan_stage_routes(p, p->st[s], sms, 0, &hb));
      continue;
    }
    size_t hmax = 0;
    for (int64_t r = 1; r <= p->ranks_max[s + 1]; ++r) {
      ntt_plan_s::Stage S;
      p->ranks[s + 1] = r;
      if (make_stage(p, s, sms, &S) != NTT_OK) continue;
      size_t h = 0;
      grp = std::max(grp, plan_stage_routes(p, S, sms, 0, &h));
      hmax = std::max(hmax, h);
    }
    p->ranks[s + 1] = p->ranks_max[s + 1];
    hb = std::max(hb, hmax);
  }
  p->h_bytes = hb;
  // split-form terms (2 m n BF16) for FP32 stages the split tensor-core pass may take
  size_t xs_bytes = 0;
  if (p->solver == NTT_SOLVER_MU && p->xdt == NTT_F32)
    for (int s = 0; s < d - 1; ++s) {
      const int64_t n = prod(dims, s + 1, d);
      for (int64_t rp = auto_rank ? 1 : p->ranks_max[s]; rp <= p->ranks_max[s]; ++rp) {
        const int64_t m = rp * dims[s];
        for (int64_t r = auto_rank ? 1 : p->ranks_max[s + 1]; r <= p->ranks_max[s + 1]; ++r)
          if ((tcs_route_ok(m, n, (int)r, p->route) || tcw_route_ok(m, n, (int)r, p->route)) &&
              !plan_route_group(m, n, (int)r, false, p->route))
            xs_bytes = std::max(xs_bytes, split_scratch_bytes(m, n));
      }
    }
  size_t bcd_bytes = 0;
  if (p->solver == NTT_SOLVER_BCD)
    for (int s = 0; s < d - 1; ++s) {
      if (!auto_rank) {
        bcd_bytes = std::max(bcd_bytes, bcd_ws_layout(p->st[s].f32).bytes);
        continue;
      }
      for (int64_t r = 1; r <= p->ranks_max[s + 1]; ++r)
        for (int64_t rp = 1; rp <= p->ranks_max[s]; ++rp) {
          MuShape sh;
          if (mu_choose_shape(rp * dims[s], prod(dims, s + 1, d), (int)r, 0, sms, &sh) == NTT_OK)
            bcd_bytes = std::max(bcd_bytes, bcd_ws_layout(sh).bytes);
        }
    }
  size_t rank_bytes = 0;
  if (auto_rank)
    for (int s = 0; s < d - 1; ++s) {
      const int64_t n = prod(dims, s + 1, d);
      for (int64_t r = 1; r <= p->ranks_max[s]; ++r)
        rank_bytes = std::max(rank_bytes, rank_ws_layout(r * dims[s], n, sms).bytes);
    }
  Arena ar;
  p->off_status = ar.take(64);
  p->off_tickets = ar.take(64);
  p->off_stop = ar.take(NTT_MAX_D * sizeof(int));
  p->off_scal = ar.take(4 * NTT_MAX_D * sizeof(double));
  p->off_obj = ar.take(p->obj_total * sizeof(double));
  p->off_G = ar.take(NTT_MAX_RANK * NTT_MAX_RANK * 4);
  p->off_red = ar.take(max_red * 4);
  p->off_part = ar.take(max_part * 4);
  p->off_part64 = ar.take(2 * kMaxResidBlocks * sizeof(double));
  p->off_hs = ar.take(NTT_MAX_RANK * 4);
  p->off_H[0] = ar.take(maxH[0] * 4);
  p->off_H[1] = ar.take(maxH[1] * 4);
  if (p->xdt == NTT_BF16) p->off_xb = ar.take(max_xb * 2);
  if (auto_rank) {
    p->off_rank = ar.take(rank_bytes);
    p->rank_bytes = rank_bytes;
  }
  if (grp) p->off_grp = ar.take(grp);
  p->grp_bytes = grp;
  if (bcd_bytes) p->off_bcd = ar.take(bcd_bytes);
  if (xs_bytes) p->off_xs = ar.take(xs_bytes);
  p->ws_bytes = ar.off;
  p->off_A[0] = ar.take((size_t)prod(dims, 0, d) * 4);
  p->off_A[1] = ar.take((size_t)prod(dims, 0, d) * 4);
  for (int k = 0; k < d; ++k)
    p->core_off.push_back(ar.take((size_t)rk[k] * dims[k] * rk[k + 1] * 4));
  p->off_err = ar.take(8 * sizeof(double));
  p->off_chain = ar.take(chain_layout(d, dims, rk.data()).total);
  p->ws_bytes_host = ar.off;
  if (!auto_rank && p->off_grp) {
    size_t h = 0;
    for (auto& S : p->st) plan_stage_routes(p, S, sms, p->off_grp, &h);
  }
  *out = p;
  return NTT_OK;
}

ntt_status ntt_plan_get_ranks(ntt_plan plan, int64_t* ranks) {
  if (!plan || !ranks) return NTT_ERR_INVALID_ARG;
  for (int k = 0; k <= plan->d; ++k) ranks[k] = plan->ranks[k];
  return NTT_OK;
}

ntt_status ntt_rank_workspace_size(int64_t m, int64_t n, size_t* bytes) {
  if (!bytes || m < 1 || n < 1) return NTT_ERR_INVALID_ARG;
  if (std::min(m, n) > NTT_MAX_ROWS) return NTT_ERR_UNSUPPORTED;
  *bytes = rank_ws_layout(m, n, device_sms()).bytes;
  return NTT_OK;
}

ntt_status ntt_select_rank(int64_t m, int64_t n, const float* X, double eps_rank, int rank_cap, int* rank_dev,
                           double* sigma_dev, void* ws, void* stream) {
  if (!X || !ws || m < 1 || n < 1 || rank_cap < 0) return NTT_ERR_INVALID_ARG;
  if (rank_dev && !(eps_rank >= 0.0)) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  if (std::min(m, n) > NTT_MAX_ROWS) return NTT_ERR_UNSUPPORTED;
  const RankWs w = rank_ws_layout(m, n, device_sms());
  NTT_CUDA_TRY(launch_rank_select(X, m, n, eps_rank, rank_cap, w, reinterpret_cast<char*>(ws), sigma_dev, rank_dev,
                                  reinterpret_cast<cudaStream_t>(stream)));
  return NTT_OK;
}

ntt_status ntt_singular_values(int64_t m, int64_t n, const float* X, double* sigma_dev, void* ws, void* stream) {
  if (!sigma_dev) return NTT_ERR_INVALID_ARG;
  return ntt_select_rank(m, n, X, 0.0, 0, nullptr, sigma_dev, ws, stream);
}

ntt_status ntt_plan_workspace_size(ntt_plan plan, size_t* bytes) {
  if (!plan || !bytes) return NTT_ERR_INVALID_ARG;
  *bytes = plan->ws_bytes;
  return NTT_OK;
}

ntt_status ntt_plan_workspace_size_host(ntt_plan plan, size_t* bytes) {
  if (!plan || !bytes) return NTT_ERR_INVALID_ARG;
  *bytes = plan->ws_bytes_host;
  return NTT_OK;
}

ntt_status ntt_plan_destroy(ntt_plan plan) {
  if (!plan) return NTT_ERR_INVALID_ARG;
  delete plan;
  return NTT_OK;
}

ntt_status ntt_decompose(ntt_plan p, const float* A, float* const* cores, void* workspace,
                         void* stream) {
  if (!p || !A || !cores || !workspace) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return NTT_ERR_INVALID_ARG;
  for (int k = 0; k < p->d; ++k)
    if (!cores[k]) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  const int d = p->d;
  if (p->ev.empty()) {
    p->ev.assign(4 * d + 2, nullptr);
    for (auto& e : p->ev) NTT_CUDA_TRY(cudaEventCreate(&e));
  }
  if (p->auto_rank) {
    NTT_TRY(decompose_auto_rank(p, A, cores, ws, st));
  } else if (p->eager) {
    // the eager tables are rewritten: the previous run must have read them
    if (p->ran && p->last_stream) NTT_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
    if (p->h_bytes && !p->h_eager) NTT_TRY(alloc_mapped(p->h_bytes, &p->h_eager, &p->h_eager_dev));
    NTT_TRY(enqueue_decompose(p, A, cores, ws, st, p->h_eager, p->h_eager_dev));
  } else {
    ntt_plan_s::Graph* G = nullptr;
    for (auto& g : p->graphs) {
      bool hit = g.exec && g.A == A && g.ws == workspace && g.cores.size() == (size_t)d;
      for (int k = 0; hit && k < d; ++k) hit = g.cores[k] == cores[k];
      if (hit) G = &g;
    }
    if (!G) {
      G = &p->graphs[p->graph_victim];
      p->graph_victim ^= 1;
      // the entry's tables are rewritten by the capture: its last launch must be done
      if (G->launched) NTT_CUDA_TRY(cudaEventSynchronize(G->done));
      G->launched = false;
      if (G->exec) {
        cudaGraphExecDestroy(G->exec);
        G->exec = nullptr;
      }
      if (!G->done) NTT_CUDA_TRY(cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming));
      if (p->h_bytes && !G->h_tab) NTT_TRY(alloc_mapped(p->h_bytes, &G->h_tab, &G->h_tab_dev));
      if (!p->cap) NTT_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
      cudaGraph_t g = nullptr;
      NTT_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
      ntt_status e = enqueue_decompose(p, A, cores, ws, p->cap, G->h_tab, G->h_tab_dev);
      cudaError_t ce = cudaStreamEndCapture(p->cap, &g);
      if (e != NTT_OK) {
        if (g) cudaGraphDestroy(g);
        return e;
      }
      if (ce != cudaSuccess) {
        cudaGetLastError();
        return NTT_ERR_CUDA;
      }
      cudaError_t ie = cudaGraphInstantiate(&G->exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        cudaGetLastError();
        G->exec = nullptr;
        return NTT_ERR_CUDA;
      }
      G->A = A;
      G->ws = workspace;
      G->cores.assign(cores, cores + d);
    }
    NTT_CUDA_TRY(cudaGraphLaunch(G->exec, st));
    NTT_CUDA_TRY(cudaEventRecord(G->done, st));
    G->launched = true;
  }
  p->last_stream = st;
  p->last_ws = workspace;
  p->ran = true;
  return NTT_OK;
}

ntt_status ntt_unfolding_size(ntt_plan p, int s, int64_t* floats) {
  if (!p || !floats || s < 1 || s > p->d - 2) return NTT_ERR_INVALID_ARG;
  *floats = p->ranks[s] * prod(p->dims.data(), s, p->d);
  return NTT_OK;
}

ntt_status ntt_decompose_stages(ntt_plan p, int s0, int s1, const float* X_in, float* const* cores,
                                float* H_out, void* workspace, void* stream) {
  if (!p || !X_in || !cores || !workspace) return NTT_ERR_INVALID_ARG;
  const int d = p->d;
  if (s0 < 0 || s1 <= s0 || s1 > d - 1) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return NTT_ERR_INVALID_ARG;
  if (p->auto_rank) return NTT_ERR_UNSUPPORTED;
  for (int k = s0; k < s1; ++k)
    if (!cores[k]) return NTT_ERR_INVALID_ARG;
  if (s1 == d - 1 && !cores[d - 1]) return NTT_ERR_INVALID_ARG;
  if (s1 < d - 1 && !H_out) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  if (p->ev.empty()) {
    p->ev.assign(4 * d + 2, nullptr);
    for (auto& e : p->ev) NTT_CUDA_TRY(cudaEventCreate(&e));
  }
  // eager launches; the eager tables are rewritten: the previous run must have read them
  if (p->ran && p->last_stream) NTT_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  if (p->h_bytes && !p->h_eager) NTT_TRY(alloc_mapped(p->h_bytes, &p->h_eager, &p->h_eager_dev));
  EnqueueCtx c;
  NTT_TRY(enqueue_begin(p, ws, st, &c));
  if (s0 > 0) {
    // the saved unfolding where stage s0 reads its X
    const size_t bytes = (size_t)(p->ranks[s0] * prod(p->dims.data(), s0, d)) * 4;
    NTT_CUDA_TRY(cudaMemcpyAsync(ws + p->off_H[(s0 - 1) % 2], X_in, bytes, cudaMemcpyDeviceToDevice, st));
  }
  for (int s = s0; s < s1; ++s) NTT_TRY(enqueue_stage(p, s, X_in, cores, ws, st, p->h_eager, p->h_eager_dev, &c));
  if (s1 < d - 1) {
    const size_t bytes = (size_t)(p->ranks[s1] * prod(p->dims.data(), s1, d)) * 4;
    NTT_CUDA_TRY(cudaMemcpyAsync(H_out, ws + p->off_H[(s1 - 1) % 2], bytes, cudaMemcpyDeviceToDevice, st));
  }
  NTT_TRY(enqueue_end(p, st, &c));
  p->last_stream = st;
  p->last_ws = workspace;
  p->ran = true;
  return NTT_OK;
}

ntt_status ntt_decompose_host(ntt_plan p, const float* A_host, float* const* cores_host,
                              double* err_host, void* workspace, void* stream) {
  if (!p || !A_host || !cores_host || !workspace) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  const int d = p->d;
  // Two input slots alternate: this call's copy runs on the plan's copy stream
  // and waits only until the call two back has finished reading its slot, so
  // it overlaps the previous call's compute; the compute waits for the copy.
  if (!p->copy_st) {
    NTT_CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      NTT_CUDA_TRY(cudaEventCreateWithFlags(&p->slot_ready[i], cudaEventDisableTiming));
      NTT_CUDA_TRY(cudaEventCreateWithFlags(&p->slot_free[i], cudaEventDisableTiming));
    }
  }
  const int slot = p->host_slot;
  p->host_slot ^= 1;
  float* A_dev = reinterpret_cast<float*>(ws + p->off_A[slot]);
  std::vector<float*> cdev(d);
  for (int k = 0; k < d; ++k) cdev[k] = reinterpret_cast<float*>(ws + p->core_off[k]);
  const size_t abytes = (size_t)prod(p->dims.data(), 0, d) * 4;
  NTT_CUDA_TRY(cudaStreamWaitEvent(p->copy_st, p->slot_free[slot], 0));   // never recorded: no wait
  NTT_CUDA_TRY(cudaMemcpyAsync(A_dev, A_host, abytes, cudaMemcpyHostToDevice, p->copy_st));
  NTT_CUDA_TRY(cudaEventRecord(p->slot_ready[slot], p->copy_st));
  // From here on the slot's free event is recorded on every return path: the
  // next copy into this slot must wait for whatever of this call was enqueued.
  auto body = [&]() -> ntt_status {
    NTT_CUDA_TRY(cudaStreamWaitEvent(st, p->slot_ready[slot], 0));
    NTT_TRY(ntt_decompose(p, A_dev, cdev.data(), workspace, stream));
    if (err_host) {
      double* err_dev = reinterpret_cast<double*>(ws + p->off_err);
      NTT_TRY(ntt_rel_error(d, p->dims.data(), p->ranks.data(), cdev.data(), A_dev, err_dev,
                            ws + p->off_chain, stream));
      NTT_CUDA_TRY(cudaMemcpyAsync(err_host, err_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    for (int k = 0; k < d; ++k) {
      const size_t cb = (size_t)p->ranks[k] * p->dims[k] * p->ranks[k + 1] * 4;
      NTT_CUDA_TRY(cudaMemcpyAsync(cores_host[k], cdev[k], cb, cudaMemcpyDeviceToHost, st));
    }
    return NTT_OK;
  };
  const ntt_status res = body();
  // slot read by the graph and Eq. (3); recorded even when the call failed
  if (cudaEventRecord(p->slot_free[slot], st) != cudaSuccess) {
    cudaGetLastError();
    if (res == NTT_OK) return NTT_ERR_CUDA;
  }
  return res;
}

ntt_status ntt_plan_get_stats(ntt_plan p, ntt_stats* out) {
  if (!p || !out) return NTT_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->d = p->d;
  for (int s = 0; s < p->d - 1; ++s) {
    out->m[s] = p->st[s].m;
    out->n[s] = p->st[s].n;
    out->r[s] = p->st[s].r;
    out->iters[s] = p->st[s].iters_total;
    out->alg_bytes[s] = p->st[s].alg_bytes;
    out->engine[s] = p->st[s].engine;
  }
  if (!p->ran) return NTT_OK;
  NTT_CUDA_TRY(cudaStreamSynchronize(p->last_stream));
  const char* ws = reinterpret_cast<const char*>(p->last_ws);
  int status = 0;
  NTT_CUDA_TRY(cudaMemcpy(&status, ws + p->off_status, sizeof(int), cudaMemcpyDeviceToHost));
  out->status = status;
  std::vector<double> scal(4 * NTT_MAX_D);
  NTT_CUDA_TRY(cudaMemcpy(scal.data(), ws + p->off_scal, scal.size() * 8, cudaMemcpyDeviceToHost));
  std::vector<double> obj(p->obj_total ? p->obj_total : 1);
  if (p->obj_total)
    NTT_CUDA_TRY(cudaMemcpy(obj.data(), ws + p->off_obj, p->obj_total * 8, cudaMemcpyDeviceToHost));
  int stopw[NTT_MAX_D];
  NTT_CUDA_TRY(cudaMemcpy(stopw, ws + p->off_stop, sizeof(stopw), cudaMemcpyDeviceToHost));
  for (int s = 0; s < p->d - 1; ++s) {
    out->xnorm2[s] = scal[s];
    out->resid[s] = scal[NTT_MAX_D + s];
    const auto& S = p->st[s];
    // iterations run: the main loop's count (cut by the stopping test) + refinement
    const int main_run = (p->tol > 0.0 && stopw[s] > 0) ? stopw[s] : p->iters;
    out->iters[s] = main_run + p->refine;
    out->obj_first[s] = obj[S.obj_off];
    out->obj_last[s] = obj[S.obj_off + (p->refine > 0 ? S.iters_total : main_run) - 1];
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p->ev[4 * s], p->ev[4 * s + 1]) == cudaSuccess)
      out->stage_ms[s] = ms;
    if (cudaEventElapsedTime(&ms, p->ev[4 * s + 2], p->ev[4 * s + 3]) == cudaSuccess)
      out->iter_ms[s] = ms;
    cudaGetLastError();
  }
  float tot = 0.0f;
  if (cudaEventElapsedTime(&tot, p->ev[4 * p->d], p->ev[4 * p->d + 1]) == cudaSuccess)
    out->total_ms = tot;
  out->launches = p->launches;
  cudaGetLastError();
  return status == 0 ? NTT_OK : (ntt_status)status;
}

// ---------------------------------------------------------------------------
// Single NMF
// ---------------------------------------------------------------------------
// Whether the single-NMF workspace holds the two BF16 terms of X: the split
// tensor-core form with NTT_ROUTE_TC, the warp-level MMA form of <= 32 rows
// wherever its route allows it.
static bool mu_split_scratch(int64_t m, int64_t n, int r, ntt_dtype x_dtype, int route) {
  if (x_dtype != NTT_F32) return false;
  return (route == NTT_ROUTE_TC && tcs_route_ok(m, n, r, route)) || tcw_route_ok(m, n, r, route);
}

static MuWs mu_ws_layout(const MuShape& s, size_t* total, bool split = false) {
  Arena ar;
  MuWs w;
  w.status = ar.take(64);
  w.tickets = ar.take(64);
  w.scal = ar.take(8 * sizeof(double));
  w.G = ar.take(NTT_MAX_RANK * NTT_MAX_RANK * 4);
  w.red = ar.take((size_t)s.part_stride() * 4);
  w.part = ar.take(mu_partial_floats(s) * 4);
  w.part64 = ar.take(2 * kMaxResidBlocks * sizeof(double));
  w.xs = split ? ar.take(split_scratch_bytes(s.m, s.n)) : 0;
  *total = ar.off;
  return w;
}

ntt_status nmf_mu_workspace_size_route(int64_t m, int64_t n, int r, ntt_dtype x_dtype, int route,
                                      size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  if (x_dtype != NTT_F32 && x_dtype != NTT_BF16) return NTT_ERR_INVALID_ARG;
  if (route < NTT_ROUTE_AUTO || route > NTT_ROUTE_TC) return NTT_ERR_INVALID_ARG;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n, r, x_dtype == NTT_BF16, device_sms(), &s));
  mu_ws_layout(s, bytes, mu_split_scratch(m, n, r, x_dtype, route));
  return NTT_OK;
}

ntt_status nmf_mu_workspace_size(int64_t m, int64_t n, int r, ntt_dtype x_dtype, size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  if (x_dtype != NTT_F32 && x_dtype != NTT_BF16) return NTT_ERR_INVALID_ARG;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n, r, x_dtype == NTT_BF16, device_sms(), &s));
  mu_ws_layout(s, bytes);
  return NTT_OK;
}

static ntt_status nmf_mu_step_impl(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype, float* W,
                                   float* H, int iters, float eps_mu, double* obj_dev, void* ws,
                                   void* stream, int route, int* engine_out, bool split_ws);

// The plain entry point keeps the workspace of nmf_mu_workspace_size (no
// split X: the tensor-core forms that need one are left out).
ntt_status nmf_mu_step(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype, float* W,
                       float* H, int iters, float eps_mu, double* obj_dev, void* ws,
                       void* stream) {
  return nmf_mu_step_impl(m, n, r, X, x_dtype, W, H, iters, eps_mu, obj_dev, ws, stream,
                          NTT_ROUTE_AUTO, nullptr, false);
}

ntt_status nmf_mu_step_route(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype, float* W,
                             float* H, int iters, float eps_mu, double* obj_dev, void* ws,
                             void* stream, int route, int* engine_out) {
  return nmf_mu_step_impl(m, n, r, X, x_dtype, W, H, iters, eps_mu, obj_dev, ws, stream, route,
                          engine_out, true);
}

static ntt_status nmf_mu_step_impl(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype, float* W,
                                   float* H, int iters, float eps_mu, double* obj_dev, void* ws,
                                   void* stream, int route, int* engine_out, bool split_ws) {
  if (!X || !W || !H || !ws || iters < 0 || !(eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  if (route < NTT_ROUTE_AUTO || route > NTT_ROUTE_TC) return NTT_ERR_INVALID_ARG;
  if (x_dtype != NTT_F32 && x_dtype != NTT_BF16) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  if (r > m || r > n) return NTT_ERR_RANK_INFEASIBLE;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n, r, x_dtype == NTT_BF16, device_sms(), &s));
  size_t total = 0;
  // the split X of the tensor-core forms takes 4 m n bytes of workspace
  const bool split = split_ws && mu_split_scratch(m, n, r, x_dtype, route);
  MuWs L = mu_ws_layout(s, &total, split);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  // status word and tickets are consecutive in the layout
  NTT_CUDA_TRY(launch_zero(w + L.status, L.tickets + 64 - L.status, st));
  unsigned* tickets = reinterpret_cast<unsigned*>(w + L.tickets);
  double* scal = reinterpret_cast<double*>(w + L.scal);
  if (obj_dev)
    NTT_TRY(resid_into(X, s.bf16, nullptr, nullptr, m, n, 0, 0, 1.0, scal, nullptr,
                       reinterpret_cast<double*>(w + L.part64), tickets + 1, st));
  MuDev dev;
  dev.X = X;
  dev.W = W;
  dev.H = H;
  dev.G = reinterpret_cast<float*>(w + L.G);
  dev.part = reinterpret_cast<float*>(w + L.part);
  dev.red = reinterpret_cast<float*>(w + L.red);
  dev.ticket = tickets;
  dev.obj = obj_dev;
  dev.xnorm2 = scal;
  dev.status = reinterpret_cast<int*>(w + L.status);
  dev.xs = split ? reinterpret_cast<__nv_bfloat16*>(w + L.xs) : nullptr;
  NTT_CUDA_TRY(launch_gram(s, dev, st));
  s.route = route;
  return run_mu_iters(s, dev, eps_mu, iters, 0, st, engine_out);
}

ntt_status nmf_mu_shard_sizes(int64_t m, int64_t n_shard, int r, size_t* ws_bytes, size_t* pq_count) {
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n_shard, r, 0, device_sms(), &s));
  size_t total = 0;
  mu_ws_layout(s, &total);
  if (ws_bytes) *ws_bytes = total;
  if (pq_count) *pq_count = (size_t)s.part_stride();
  return NTT_OK;
}

ntt_status nmf_mu_shard_norm(int64_t m, int64_t n_shard, const float* X, double* out_dev, void* ws, void* stream) {
  if (!X || !out_dev || !ws || m < 1 || n_shard < 1) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n_shard, 1, 0, device_sms(), &s));
  size_t total = 0;
  MuWs L = mu_ws_layout(s, &total);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  unsigned* tickets = reinterpret_cast<unsigned*>(w + L.tickets);
  NTT_CUDA_TRY(launch_zero(tickets, 64, st));
  return resid_into(X, 0, nullptr, nullptr, m, n_shard, 0, 0, 1.0, out_dev, nullptr,
                    reinterpret_cast<double*>(w + L.part64), tickets + 1, st);
}

ntt_status nmf_mu_shard_pass(int64_t m, int64_t n_shard, int r, const float* X, const float* W, float* H,
                             float eps_mu, double* pq_out, void* ws, void* stream) {
  if (!X || !W || !H || !pq_out || !ws || !(eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  if (r > m) return NTT_ERR_RANK_INFEASIBLE;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n_shard, r, 0, device_sms(), &s));
  size_t total = 0;
  MuWs L = mu_ws_layout(s, &total);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  NTT_CUDA_TRY(launch_zero(w + L.status, L.tickets + 64 - L.status, st));
  MuDev dev;
  dev.X = X;
  dev.W = const_cast<float*>(W);
  dev.H = H;
  dev.G = reinterpret_cast<float*>(w + L.G);
  dev.part = reinterpret_cast<float*>(w + L.part);
  dev.red = reinterpret_cast<float*>(w + L.red);
  dev.ticket = reinterpret_cast<unsigned*>(w + L.tickets);
  dev.status = reinterpret_cast<int*>(w + L.status);
  NTT_CUDA_TRY(launch_gram(s, dev, st));
  mu_finalize_shape(&s, X, H, device_sms());
  CUtensorMap mx, mh;
  std::memset(&mx, 0, sizeof(mx));
  std::memset(&mh, 0, sizeof(mh));
  if (s.tma) NTT_TRY(mu_encode_maps(s, X, H, &mx, &mh));
  NTT_CUDA_TRY(launch_mu_pass(s, dev, eps_mu, mx, mh, st));
  NTT_CUDA_TRY(launch_shard_reduce(dev.part, s.grid, s.part_stride(), pq_out, st));
  return NTT_OK;
}

ntt_status nmf_mu_shard_update(int64_t m, int r, const double* pq, float* W, float eps_mu, double xnorm2,
                               double* obj_dev, void* ws, void* stream) {
  if (!pq || !W || !ws || !(eps_mu >= 0.0f) || m < 1 || r < 1) return NTT_ERR_INVALID_ARG;
  if (m > NTT_MAX_ROWS || r > NTT_MAX_RANK) return NTT_ERR_UNSUPPORTED;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, 1 << 20, r, 0, device_sms(), &s));   // MP, R of the [P ; Q] layout
  size_t total = 0;
  MuWs L = mu_ws_layout(s, &total);
  char* w = reinterpret_cast<char*>(ws);
  NTT_CUDA_TRY(launch_shard_update(pq, (int)m, r, s.MP, s.R, W, reinterpret_cast<float*>(w + L.G), eps_mu, xnorm2,
                                   obj_dev, reinterpret_cast<cudaStream_t>(stream)));
  return NTT_OK;
}

ntt_status nmf_mu_host_workspace_size(int64_t m, int64_t n, int r, int64_t chunk_cols, size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  return stream_ws_size(m, n, r, chunk_cols, bytes);
}

ntt_status nmf_mu_step_host(int64_t m, int64_t n, int r, const float* X_host, float* W, float* H, int iters,
                            float eps_mu, double* obj_dev, int64_t chunk_cols, void* ws, void* stream) {
  if (!X_host || !W || !H || !ws || iters < 0 || !(eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  if (r > m || r > n) return NTT_ERR_RANK_INFEASIBLE;
  return stream_mu(m, n, r, X_host, W, H, iters, eps_mu, obj_dev, chunk_cols, ws,
                   reinterpret_cast<cudaStream_t>(stream));
}

ntt_status nmf_bcd_workspace_size(int64_t m, int64_t n, int r, size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n, r, 0, device_sms(), &s));
  size_t mu = 0;
  mu_ws_layout(s, &mu);
  *bytes = mu + bcd_ws_layout(s).bytes;
  return NTT_OK;
}

ntt_status nmf_bcd_step(int64_t m, int64_t n, int r, const float* X, float* W, float* H, int iters,
                        double* obj_dev, void* ws, void* stream) {
  if (!X || !W || !H || !ws || iters < 0) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  if (r > m || r > n) return NTT_ERR_RANK_INFEASIBLE;
  MuShape s;
  NTT_TRY(mu_choose_shape(m, n, r, 0, device_sms(), &s));
  size_t total = 0;
  MuWs L = mu_ws_layout(s, &total);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = reinterpret_cast<char*>(ws);
  NTT_CUDA_TRY(launch_zero(w + L.status, L.tickets + 64 - L.status, st));
  MuDev dev;
  dev.X = X;
  dev.W = W;
  dev.H = H;
  dev.G = reinterpret_cast<float*>(w + L.G);
  dev.part = reinterpret_cast<float*>(w + L.part);
  dev.red = reinterpret_cast<float*>(w + L.red);
  dev.ticket = reinterpret_cast<unsigned*>(w + L.tickets);
  dev.obj = obj_dev;
  dev.status = reinterpret_cast<int*>(w + L.status);
  dev.part64 = reinterpret_cast<double*>(w + L.part64);
  return run_bcd_iters(s, dev, bcd_ws_layout(s), w + total, iters, 0, st);
}

ntt_status ntt_status_of_workspace(const void* ws, ntt_status* out) {
  if (!ws || !out) return NTT_ERR_INVALID_ARG;
  int v = 0;
  NTT_CUDA_TRY(cudaMemcpy(&v, ws, sizeof(int), cudaMemcpyDeviceToHost));
  *out = (ntt_status)v;
  return NTT_OK;
}

ntt_status ntt_wait_probe(void* ws, int64_t limit_ns, void* stream) {
  if (!ws || limit_ns < 0 || (reinterpret_cast<uintptr_t>(ws) % 256)) return NTT_ERR_INVALID_ARG;
  // the status word is the first word of an nmf_mu_step workspace; the probe
  // copies the 256 bytes that start there
  NTT_CUDA_TRY(launch_wait_probe(ws, reinterpret_cast<int*>(ws), (long long)limit_ns,
                                 reinterpret_cast<cudaStream_t>(stream)));
  return NTT_OK;
}

ntt_status ntt_uniform_init(uint64_t seed, int stage, int restart, int matrix, int64_t count,
                            float* out, void* stream) {
  if (!out || count < 0 || stage < 0 || restart < 0 || (matrix != 0 && matrix != 1))
    return NTT_ERR_INVALID_ARG;
  NTT_CUDA_TRY(launch_uniform(stream_key(seed, stage, restart, matrix), count, out,
                              reinterpret_cast<cudaStream_t>(stream)));
  return NTT_OK;
}

// ---------------------------------------------------------------------------
// Reconstruction and relative error
// ---------------------------------------------------------------------------
ntt_status ntt_reconstruct_workspace_size(int d, const int64_t* dims, const int64_t* ranks,
                                          size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  NTT_TRY(check_tt(d, dims, ranks));
  *bytes = chain_layout(d, dims, ranks).total;
  return NTT_OK;
}

ntt_status ntt_reconstruct(int d, const int64_t* dims, const int64_t* ranks,
                           const float* const* cores, float* A_out, void* ws, void* stream) {
  NTT_TRY(check_tt(d, dims, ranks));
  if (!cores || !A_out || !ws) return NTT_ERR_INVALID_ARG;
  for (int k = 0; k < d; ++k)
    if (!cores[k]) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const ChainWs c = chain_layout(d, dims, ranks);
  char* w = reinterpret_cast<char*>(ws);
  const float *L, *R;
  NTT_TRY(build_chain(d, dims, ranks, cores, c, w, &L, &R, st));
  ResidArgs a;
  a.L = L;
  a.Rm = R;
  a.out = A_out;
  a.M = c.rows;
  a.N = c.cols;
  a.r = (int)ranks[c.s];
  a.mode = 2;
  NTT_CUDA_TRY(launch_resid(a, resid_blocks(device_sms()), st));
  return NTT_OK;
}

ntt_status ntt_rel_error(int d, const int64_t* dims, const int64_t* ranks,
                         const float* const* cores, const float* A, double* err_dev, void* ws,
                         void* stream) {
  NTT_TRY(check_tt(d, dims, ranks));
  if (!cores || !A || !err_dev || !ws) return NTT_ERR_INVALID_ARG;
  for (int k = 0; k < d; ++k)
    if (!cores[k]) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const ChainWs c = chain_layout(d, dims, ranks);
  char* w = reinterpret_cast<char*>(ws);
  const float *L, *R;
  NTT_TRY(build_chain(d, dims, ranks, cores, c, w, &L, &R, st));
  unsigned* ticket = reinterpret_cast<unsigned*>(w + c.ticket);
  NTT_CUDA_TRY(launch_zero(ticket, 64, st));
  return resid_into(A, 0, L, R, c.rows, c.cols, (int)ranks[c.s], 1, 1.0,
                    reinterpret_cast<double*>(w + c.acc), err_dev,
                    reinterpret_cast<double*>(w + c.part64), ticket, st);
}

}  // extern "C"
