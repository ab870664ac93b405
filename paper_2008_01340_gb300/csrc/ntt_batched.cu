// Batched form: many non-negative tensor trains with random restarts.
//
// Every instance runs Algorithm 2 with its own ranks; every stage of every
// instance is solved from `restarts` independent initialisations (restart j
// uses the init stream (seed_i, stage, j)) and the restart with the lowest
// final objective 1/2||X - WH||^2 (ties: lowest index) is kept, hand-off
// normalised, and its H becomes the next unfolding.
//
// Work per stage:
//   * small unfoldings (X, H and the update buffers fit in shared memory):
//     one launch of small_nmf_kernel over all (instance, restart) tasks of the
//     stage; one CTA owns one NMF for all of its iterations, X read from HBM
//     once per task;
//   * large unfoldings: the restarts run side by side as one NMF of rank
//     g*r with W^T W and H H^T kept on the diagonal r x r blocks (the only
//     coupling between columns of W), g = floor(32 / r), and every group of
//     every large instance of the stage advances together in the grouped MU
//     engine -- one pass launch per shape bucket and one combine launch per
//     iteration for all of them, one read of X serving g restarts;
//   * per-restart objectives by one grouped FP64 residual pass;
//   * select_kernel: best restart, column-L1 hand-off into the core and the
//     next unfolding, for all instances of the stage at once.
// The small-unfolding launch runs on a second stream, beside the large work.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "group_engine.cuh"

namespace ntt {
namespace {

#define NTT_TRY_B(expr)          \
  do {                           \
    ntt_status s_ = (expr);      \
    if (s_ != NTT_OK) return s_; \
  } while (0)

constexpr int kSmallThreads = 256;
constexpr int kSmallMaxR = 16;
constexpr size_t kSmallSmemCap = 200 * 1024;
constexpr int kMaxRestarts = 16;

struct SmallTask {
  const float* X;
  float* W;
  float* H;
  double* obj;
  uint64_t keyW, keyH;
  int m, n, r, pad;
};

__host__ __device__ inline size_t small_smem_bytes(int m, int n, int r) {
  // X (m x (n+1)), Y, H, Hn (r x (n+1) each), W, Wn, P (m x r), Q, G (r x r), reduction doubles
  return 4 * ((size_t)m * (n + 1) + 3 * (size_t)r * (n + 1) + 3 * (size_t)m * r + 2 * (size_t)r * r) +
         8 * kSmallThreads + 64;
}

// One CTA = one NMF: all multiplicative-update iterations in shared memory.
__global__ void __launch_bounds__(kSmallThreads) small_nmf_kernel(const SmallTask* tasks,
                                                                  int ntasks, int iters,
                                                                  float eps) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const SmallTask tk = tasks[t];
    const int m = tk.m, n = tk.n, r = tk.r, ld = n + 1;
    float* Xs = sm;
    float* Ys = Xs + (size_t)m * ld;
    float* Hs = Ys + (size_t)r * ld;
    float* Hn = Hs + (size_t)r * ld;
    float* Ws = Hn + (size_t)r * ld;
    float* Wn = Ws + (size_t)m * r;
    float* Ps = Wn + (size_t)m * r;
    float* Qs = Ps + (size_t)m * r;
    float* Gs = Qs + (size_t)r * r;
    double* dred = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(Gs + r * r) + 7) & ~uintptr_t(7));
    __syncthreads();
    for (int e = tid; e < m * n; e += NT) Xs[(e / n) * ld + e % n] = tk.X[e];
    for (int e = tid; e < m * r; e += NT) Ws[e] = uniform24(tk.keyW, (uint64_t)e);
    for (int e = tid; e < r * n; e += NT) Hs[(e / n) * ld + e % n] = uniform24(tk.keyH, (uint64_t)e);
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
      // G = W^T W
      for (int kl = tid; kl < r * r; kl += NT) {
        const int k = kl / r, l = kl % r;
        float g = 0.0f;
        for (int i = 0; i < m; ++i) g = fmaf(Ws[i * r + k], Ws[i * r + l], g);
        Gs[kl] = g;
      }
      // Y = W^T X
      for (int e = tid; e < r * n; e += NT) {
        const int k = e / n, c = e % n;
        float y = 0.0f;
        for (int i = 0; i < m; ++i) y = fmaf(Ws[i * r + k], Xs[i * ld + c], y);
        Ys[k * ld + c] = y;
      }
      __syncthreads();
      // H <- max(0, H o Y / (G H + eps))
      for (int e = tid; e < r * n; e += NT) {
        const int k = e / n, c = e % n;
        float gh = 0.0f;
        for (int l = 0; l < r; ++l) gh = fmaf(Gs[k * r + l], Hs[l * ld + c], gh);
        Hn[k * ld + c] = fmaxf(0.0f, __fdividef(Hs[k * ld + c] * Ys[k * ld + c], gh + eps));
      }
      __syncthreads();
      // P = X H^T, Q = H H^T
      for (int e = tid; e < m * r + r * r; e += NT) {
        const float* a;
        int k;
        if (e < m * r) {
          a = Xs + (e / r) * ld;
          k = e % r;
        } else {
          a = Hn + ((e - m * r) / r) * ld;
          k = (e - m * r) % r;
        }
        const float* b = Hn + k * ld;
        float s0 = 0.0f, s1 = 0.0f;
        int c = 0;
        for (; c + 1 < n; c += 2) {
          s0 = fmaf(a[c], b[c], s0);
          s1 = fmaf(a[c + 1], b[c + 1], s1);
        }
        if (c < n) s0 = fmaf(a[c], b[c], s0);
        if (e < m * r) Ps[e] = s0 + s1; else Qs[e - m * r] = s0 + s1;
      }
      __syncthreads();
      // W <- max(0, W o P / (W Q + eps)); H <- H_new
      for (int e = tid; e < m * r; e += NT) {
        const int i = e / r, k = e % r;
        float wq = 0.0f;
        for (int l = 0; l < r; ++l) wq = fmaf(Ws[i * r + l], Qs[l * r + k], wq);
        Wn[e] = fmaxf(0.0f, __fdiv_rn(Ws[e] * Ps[e], wq + eps));
      }
      __syncthreads();
      for (int e = tid; e < m * r; e += NT) Ws[e] = Wn[e];
      for (int e = tid; e < r * n; e += NT) Hs[(e / n) * ld + e % n] = Hn[(e / n) * ld + e % n];
      __syncthreads();
    }
    // final objective 1/2 ||X - W H||^2 (FP32 products, FP64 sums, fixed order)
    double acc = 0.0;
    for (int e = tid; e < m * n; e += NT) {
      const int i = e / n, c = e % n;
      float v = 0.0f;
      for (int k = 0; k < r; ++k) v = fmaf(Ws[i * r + k], Hs[k * ld + c], v);
      const float d = Xs[i * ld + c] - v;
      acc += (double)(d * d);
    }
    dred[tid] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
      if (tid < s) dred[tid] += dred[tid + s];
      __syncthreads();
    }
    if (tid == 0) *tk.obj = 0.5 * dred[0];
    for (int e = tid; e < m * r; e += NT) tk.W[e] = Ws[e];
    for (int e = tid; e < r * n; e += NT) tk.H[e] = Hs[(e / n) * ld + e % n];
    __syncthreads();
  }
}


// Initial factors of one group of g side-by-side restarts: W_group (m x g r,
// restart q in columns q r .. q r + r - 1) and H rows q r .. of the group,
// each restart from its own stream.  One table entry per group.
struct InitJob {
  float* W;
  float* H;
  int64_t n;
  int m, r, g, pad;
  uint64_t kw[kMaxRestarts], kh[kMaxRestarts];
};

__global__ void init_groups_kernel(const InitJob* jobs) {
  const InitJob& J = jobs[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int re = J.g * J.r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)J.m * re; e += stride) {
    const int i = (int)(e / re), q = (int)(e % re), j = q / J.r, k = q % J.r;
    J.W[e] = uniform24(J.kw[j], (uint64_t)(i * J.r + k));
  }
  const int64_t rn = (int64_t)J.r * J.n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)re * J.n; e += stride) {
    const int j = (int)(e / rn);
    J.H[e] = uniform24(J.kh[j], (uint64_t)(e - (int64_t)j * rn));
  }
}

// W_j (m x r, contiguous) <- columns j r .. of W_group, for the g restarts of a group.
struct SplitJob {
  const float* Wg;
  float* Wall;
  int m, r, g, pad;
};

__global__ void split_groups_kernel(const SplitJob* jobs) {
  const SplitJob J = jobs[blockIdx.y];
  const int re = J.g * J.r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J.m * re; e += gridDim.x * blockDim.x) {
    const int i = e / re, q = e % re, j = q / J.r, k = q % J.r;
    J.Wall[(size_t)j * J.m * J.r + i * J.r + k] = J.Wg[e];
  }
}

// 1/2 ||X - W H||_F^2 of one restart: FP32 products, FP64 sums in a fixed
// order.  Blocks cover kResCols columns each; block partials are summed in
// block order by resid_reduce_kernel.
constexpr int kResCols = 2048;
struct ResJob {
  const float* X;
  const float* W;   // m x r
  const float* H;   // r x n
  double* out;
  int64_t n;
  int m, r, blk0, nblk;
};

__global__ void __launch_bounds__(256) resid_groups_kernel(const ResJob* __restrict__ jobs,
                                                           const int* __restrict__ blk_job,
                                                           double* __restrict__ partial) {
  extern __shared__ float wsm[];
  __shared__ double dred[256];
  const ResJob J = jobs[blk_job[blockIdx.x]];
  const int tid = threadIdx.x;
  for (int e = tid; e < J.m * J.r; e += blockDim.x) wsm[e] = J.W[e];
  __syncthreads();
  const int64_t c0 = (int64_t)(blockIdx.x - J.blk0) * kResCols;
  const int64_t c1 = c0 + kResCols < J.n ? c0 + kResCols : J.n;
  double acc = 0.0;
  for (int64_t c = c0 + tid; c < c1; c += blockDim.x) {
    float h[NTT_MAX_RANK];
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) h[k] = k < J.r ? J.H[(int64_t)k * J.n + c] : 0.0f;
    for (int i = 0; i < J.m; ++i) {
      float v = 0.0f;
#pragma unroll
      for (int k = 0; k < NTT_MAX_RANK; ++k)
        if (k < J.r) v = fmaf(wsm[i * J.r + k], h[k], v);
      const float d = J.X[(int64_t)i * J.n + c] - v;
      acc += (double)(d * d);
    }
  }
  dred[tid] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) dred[tid] += dred[tid + s];
    __syncthreads();
  }
  if (tid == 0) partial[blockIdx.x] = dred[0];
}

__global__ void resid_reduce_kernel(const ResJob* jobs, int njobs, const double* partial) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  const ResJob J = jobs[j];
  double s = 0.0;
  for (int b = 0; b < J.nblk; ++b) s += partial[J.blk0 + b];
  *J.out = 0.5 * s;
}

struct SelectJob {
  const float* Wc;   // restart candidates: restart j's W at Wc + j * w_stride
  const float* Hc;   // restart j's H at Hc + j * h_stride
  int64_t w_stride, h_stride;
  const double* obj;
  float* core;       // W of the kept restart, column-L1 normalised (m x r)
  float* next;       // H of the kept restart, rows scaled by the norms (r x n)
  int64_t n;
  int m, r, restarts, pad;
};

// One select job on the calling block: every block picks the same restart,
// computes the column norms, block x == 0 writes the core, all blocks scale
// their chunk of H.
__global__ void select_kernel(const SelectJob* jobs) {
  __shared__ float snorm[NTT_MAX_RANK];
  __shared__ int sbest;
  const SelectJob jb = jobs[blockIdx.y];
  const int tid = threadIdx.x;
  if (tid == 0) {
    int best = 0;
    double bv = jb.obj[0];
    for (int j = 1; j < jb.restarts; ++j)
      if (jb.obj[j] < bv) {
        bv = jb.obj[j];
        best = j;
      }
    sbest = best;
  }
  __syncthreads();
  const float* W = jb.Wc + (size_t)sbest * jb.w_stride;
  const float* H = jb.Hc + (size_t)sbest * jb.h_stride;
  if (tid < jb.r) {
    float s = 0.0f;
    for (int i = 0; i < jb.m; ++i) s += W[i * jb.r + tid];
    snorm[tid] = s;
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int e = tid; e < jb.m * jb.r; e += blockDim.x) {
      const float s = snorm[e % jb.r];
      jb.core[e] = s > 0.0f ? __fdiv_rn(W[e], s) : W[e];
    }
  const int64_t total = (int64_t)jb.r * jb.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < total; e += stride) {
    const float s = snorm[e / jb.n];
    jb.next[e] = s > 0.0f ? H[e] * s : H[e];
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }
size_t align64f(size_t x) { return (x + 63) / 64 * 64; }   // floats, 256-byte steps
int64_t prod64(const std::vector<int64_t>& v, int a, int b) {
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= v[i];
  return p;
}

bool is_small(int64_t m, int64_t n, int r) {
  return r <= kSmallMaxR && n < (1 << 20) && small_smem_bytes((int)m, (int)n, r) <= kSmallSmemCap;
}

}  // namespace
}  // namespace ntt

using namespace ntt;

struct ntt_batch_s {
  struct Inst {
    int d;
    std::vector<int64_t> dims, ranks;
    size_t a_off;                    // floats into the packed input
    std::vector<size_t> core_off;    // floats into the packed cores
    size_t x_off[2];                 // floats into the workspace (next-unfolding ping-pong)
    uint64_t seed;
  };
  // Large unfoldings of one stage: per instance its restart factors, per
  // group of g restarts one problem of the grouped engine.
  struct Stage {
    std::vector<int> large;                       // instances
    std::vector<size_t> wall_off, hall_off;       // per large instance, bytes
    std::vector<int> prob_inst, prob_j0, prob_g;  // per problem
    std::vector<size_t> wg_off;                   // per problem, bytes
    ntt::GroupPlan gp;
    int nres = 0, res_blocks = 0, res_smem = 0;
    size_t off_init, off_split, off_res, off_resmap, off_respart, off_sel;   // bytes, device tables
    size_t tab_bytes = 0;                          // bytes of those tables (one copy)
    size_t host_off = 0;                           // pinned host offset of this stage
    size_t host_bytes = 0;                         // bytes of its tables + the engine's (uploaded per call)
    std::vector<GroupShape> shapes;                // grouped problems of the stage
    size_t gp_base = 0;                            // scratch offset of the engine plan
    int split = 4;                                 // CTA split of the engine (autotuned)
    uint64_t sig = 0;                              // signature of the stage's problem shapes
    bool tuned = false;
    int sel_grid = 1;
    // small tasks and their select jobs
    size_t task_base = 0, ntasks = 0, job_base = 0, njobs = 0, small_floats = 0;
    size_t small_smem = 0;
  };
  std::vector<Inst> inst;
  std::vector<Stage> stage;
  int iters = 0, restarts = 1;
  float eps = 1e-12f;
  size_t a_total = 0, cores_total = 0;
  // workspace layout (bytes)
  size_t off_status, off_obj, off_tasks, off_jobs, off_small, off_x, off_stage, bytes;
  size_t n_tasks = 0, n_jobs = 0;
  int max_stages = 0;
  // host tables (small tasks, small select jobs, per-stage tables): h_bytes per
  // copy; every cached graph owns a mapped pinned copy written once at capture
  // and uploaded by kernel nodes on each launch
  size_t h_bytes = 0, h_tasks_off = 0, h_jobs_off = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    const float* A = nullptr;
    float* cores = nullptr;
    void* ws = nullptr;
    char* h = nullptr;        // host address of the tables
    char* hdev = nullptr;     // device address of the same memory
    cudaEvent_t done = nullptr;
    bool launched = false;
  };
  Graph graphs[2];
  int victim = 0;
  cudaStream_t cap = nullptr;
  char* h_tune = nullptr;     // tables of the autotuner's eager runs
  char* h_tune_dev = nullptr;
  int tuned_from_cache = 0;   // stages whose split came from the cache file
  int tuned_timed = 0;        // stages whose split was timed
  void drop_graphs() {
    for (auto& g : graphs) {
      if (g.launched) cudaEventSynchronize(g.done);
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      g.launched = false;
      g.A = nullptr;
      g.cores = nullptr;
      g.ws = nullptr;
    }
  }
  ~ntt_batch_s() {
    drop_graphs();
    for (auto& g : graphs) {
      if (g.done) cudaEventDestroy(g.done);
      if (g.h) cudaFreeHost(g.h);
    }
    if (h_tune) cudaFreeHost(h_tune);
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    cudaGetLastError();
  }
};

namespace {

const float* stage_input(ntt_batch b, int i, int s, const float* A, char* ws) {
  const auto& I = b->inst[i];
  return (s == 0) ? A + I.a_off : reinterpret_cast<const float*>(ws + b->off_x) + I.x_off[(s - 1) & 1];
}

float* stage_next(ntt_batch b, int i, int s, float* cores, char* ws) {
  const auto& I = b->inst[i];
  return (s == I.d - 2) ? cores + I.core_off[I.d - 1]
                        : reinterpret_cast<float*>(ws + b->off_x) + I.x_off[s & 1];
}

// Host tables of stage s's small tasks and their selection jobs (into h).
void fill_small_tables(ntt_batch b, int s, const float* A, float* cores, char* ws, char* h) {
  const auto& S = b->stage[s];
  const int R = b->restarts;
  double* obj = reinterpret_cast<double*>(ws + b->off_obj);
  SmallTask* tasks = reinterpret_cast<SmallTask*>(h + b->h_tasks_off);
  SelectJob* jobs = reinterpret_cast<SelectJob*>(h + b->h_jobs_off);
  size_t t = S.task_base, jn = S.job_base, off = 0;
  for (int i = 0; i < (int)b->inst.size(); ++i) {
    auto& I = b->inst[i];
    if (s >= I.d - 1) continue;
    const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
    const int r = (int)I.ranks[s + 1];
    if (!is_small(m, n, r)) continue;
    const float* X = stage_input(b, i, s, A, ws);
    float* base = reinterpret_cast<float*>(ws + b->off_small) + off;
    for (int j = 0; j < R; ++j) {
      SmallTask& tk = tasks[t++];
      tk.X = X;
      tk.W = base + (size_t)j * (m * r + r * n);
      tk.H = tk.W + m * r;
      tk.obj = obj + (size_t)i * R + j;
      tk.keyW = stream_key(I.seed, s, j, 0);
      tk.keyH = stream_key(I.seed, s, j, 1);
      tk.m = (int)m;
      tk.n = (int)n;
      tk.r = r;
      tk.pad = 0;
    }
    SelectJob& jb = jobs[jn++];
    jb.Wc = base;
    jb.Hc = base + m * r;
    jb.w_stride = m * r + r * n;
    jb.h_stride = m * r + r * n;
    jb.obj = obj + (size_t)i * R;
    jb.core = cores + I.core_off[s];
    jb.next = stage_next(b, i, s, cores, ws);
    jb.n = n;
    jb.m = (int)m;
    jb.r = r;
    jb.restarts = R;
    jb.pad = 0;
    off += (size_t)R * (m * r + r * n);
  }
}

// Large unfoldings of stage s: init tables, grouped iterations, split,
// residuals, selection -- all on stream st.  hb / hbdev: host and device
// addresses of the mapped pinned tables; ev (nullable): two events around the
// grouped iterations.
ntt_status enqueue_large_stage(ntt_batch b, int s, const float* A, float* cores, char* ws, cudaStream_t st,
                               int sms, char* hb, const char* hbdev, int iters, cudaEvent_t* ev) {
  auto& S = b->stage[s];
  if (S.large.empty()) return NTT_OK;
  const int R = b->restarts;
  double* obj = reinterpret_cast<double*>(ws + b->off_obj);
  char* h = hb + S.host_off;
  InitJob* hi = reinterpret_cast<InitJob*>(h + (S.off_init - b->off_stage));
  SplitJob* hs = reinterpret_cast<SplitJob*>(h + (S.off_split - b->off_stage));
  ResJob* hr = reinterpret_cast<ResJob*>(h + (S.off_res - b->off_stage));
  int* hrm = reinterpret_cast<int*>(h + (S.off_resmap - b->off_stage));
  SelectJob* hsel = reinterpret_cast<SelectJob*>(h + (S.off_sel - b->off_stage));
  const int np = (int)S.prob_inst.size();
  std::vector<GroupPtrs> ptrs(np);
  int rj = 0, rb = 0;
  for (int li = 0; li < (int)S.large.size(); ++li) {
    const int i = S.large[li];
    const auto& I = b->inst[i];
    const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
    const int r = (int)I.ranks[s + 1];
    const float* X = stage_input(b, i, s, A, ws);
    float* Wall = reinterpret_cast<float*>(ws + S.wall_off[li]);
    float* Hall = reinterpret_cast<float*>(ws + S.hall_off[li]);
    for (int j = 0; j < R; ++j, ++rj) {
      ResJob& J = hr[rj];
      J.X = X;
      J.W = Wall + (size_t)j * m * r;
      J.H = Hall + (size_t)j * r * n;
      J.out = obj + (size_t)i * R + j;
      J.n = n;
      J.m = (int)m;
      J.r = r;
      J.nblk = (int)((n + kResCols - 1) / kResCols);
      J.blk0 = rb;
      for (int q = 0; q < J.nblk; ++q) hrm[rb + q] = rj;
      rb += J.nblk;
    }
    SelectJob& jb = hsel[li];
    jb.Wc = Wall;
    jb.Hc = Hall;
    jb.w_stride = m * r;
    jb.h_stride = (int64_t)r * n;
    jb.obj = obj + (size_t)i * R;
    jb.core = cores + I.core_off[s];
    jb.next = stage_next(b, i, s, cores, ws);
    jb.n = n;
    jb.m = (int)m;
    jb.r = r;
    jb.restarts = R;
    jb.pad = 0;
  }
  for (int p = 0; p < np; ++p) {
    const int i = S.prob_inst[p], j0 = S.prob_j0[p], g = S.prob_g[p];
    const int li = (int)(std::find(S.large.begin(), S.large.end(), i) - S.large.begin());
    const auto& I = b->inst[i];
    const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
    const int r = (int)I.ranks[s + 1];
    float* Wg = reinterpret_cast<float*>(ws + S.wg_off[p]);
    float* Hg = reinterpret_cast<float*>(ws + S.hall_off[li]) + (size_t)j0 * r * n;
    InitJob& ij = hi[p];
    std::memset(&ij, 0, sizeof(ij));
    ij.W = Wg;
    ij.H = Hg;
    ij.n = n;
    ij.m = (int)m;
    ij.r = r;
    ij.g = g;
    for (int q = 0; q < g; ++q) {
      ij.kw[q] = stream_key(I.seed, s, j0 + q, 0);
      ij.kh[q] = stream_key(I.seed, s, j0 + q, 1);
    }
    SplitJob& sj = hs[p];
    sj.Wg = Wg;
    sj.Wall = reinterpret_cast<float*>(ws + S.wall_off[li]) + (size_t)j0 * m * r;
    sj.m = (int)m;
    sj.r = r;
    sj.g = g;
    sj.pad = 0;
    ptrs[p].X = stage_input(b, i, s, A, ws);
    ptrs[p].H = Hg;
    ptrs[p].W = Wg;
    ptrs[p].scratch = nullptr;
  }
  // the engine's tables follow the stage's own in the host block: one upload
  group_fill_tables(S.gp, ptrs.data(), ws, h + (S.gp.off_tables - b->off_stage));
  if (launch_copy_words(ws + b->off_stage, hbdev + S.host_off, S.host_bytes, st) != cudaSuccess)
    return NTT_ERR_CUDA;
  const InitJob* di = reinterpret_cast<const InitJob*>(ws + S.off_init);
  const SplitJob* dsp = reinterpret_cast<const SplitJob*>(ws + S.off_split);
  const ResJob* dr = reinterpret_cast<const ResJob*>(ws + S.off_res);
  const int* drm = reinterpret_cast<const int*>(ws + S.off_resmap);
  double* drp = reinterpret_cast<double*>(ws + S.off_respart);
  const SelectJob* dsel = reinterpret_cast<const SelectJob*>(ws + S.off_sel);
  init_groups_kernel<<<dim3(sms, np), 256, 0, st>>>(di);
  if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return NTT_ERR_CUDA;
  NTT_TRY_B(group_launch(S.gp, ws, ws + S.gp.off_tables, iters, b->eps, st));
  if (ev && cudaEventRecord(ev[1], st) != cudaSuccess) return NTT_ERR_CUDA;
  split_groups_kernel<<<dim3(8, np), 256, 0, st>>>(dsp);
  resid_groups_kernel<<<S.res_blocks, 256, S.res_smem, st>>>(dr, drm, drp);
  resid_reduce_kernel<<<(S.nres + 127) / 128, 128, 0, st>>>(dr, S.nres, drp);
  select_kernel<<<dim3(S.sel_grid, (unsigned)S.large.size()), 256, 0, st>>>(dsel);
  return cudaGetLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

ntt_status batch_setup(ntt_batch b) {
  if (b->side) return NTT_OK;
  if (cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return NTT_ERR_CUDA;
  if (cudaFuncSetAttribute(small_nmf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSmallSmemCap + 1024) != cudaSuccess ||
      cudaFuncSetAttribute(resid_groups_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           NTT_MAX_ROWS * NTT_MAX_RANK * 4) != cudaSuccess)
    return NTT_ERR_CUDA;
  return NTT_OK;
}

// The whole batch on stream st (captured or eager): every stage's small tasks
// on the side stream beside its large work, then the selections.  h / hdev:
// the mapped pinned tables this enqueue writes and its kernels upload.
// ev (nullable): 2 events per stage around the grouped iterations.
ntt_status enqueue_batch(ntt_batch b, const float* A, float* cores, char* ws, cudaStream_t st, char* h,
                         const char* hdev, int iters, cudaEvent_t* ev) {
  if (launch_zero(ws + b->off_status, 64, st) != cudaSuccess) return NTT_ERR_CUDA;
  NTT_TRY_B(batch_setup(b));
  for (int s = 0; s < b->max_stages; ++s) fill_small_tables(b, s, A, cores, ws, h);
  SmallTask* dtasks = reinterpret_cast<SmallTask*>(ws + b->off_tasks);
  SelectJob* djobs = reinterpret_cast<SelectJob*>(ws + b->off_jobs);
  if (b->n_tasks && launch_copy_words(dtasks, hdev + b->h_tasks_off, b->n_tasks * sizeof(SmallTask), st) != cudaSuccess)
    return NTT_ERR_CUDA;
  if (b->n_jobs && launch_copy_words(djobs, hdev + b->h_jobs_off, b->n_jobs * sizeof(SelectJob), st) != cudaSuccess)
    return NTT_ERR_CUDA;
  const int sms = device_sms();
  for (int s = 0; s < b->max_stages; ++s) {
    const auto& S = b->stage[s];
    // small tasks on the side stream, after everything the caller's stream holds
    if (S.ntasks) {
      if (cudaEventRecord(b->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(b->side, b->ev_fork, 0) != cudaSuccess)
        return NTT_ERR_CUDA;
      const int grid = (int)std::min<size_t>(S.ntasks, (size_t)sms * (S.small_smem > 110 * 1024 ? 1 : 2));
      small_nmf_kernel<<<grid, kSmallThreads, S.small_smem, b->side>>>(dtasks + S.task_base, (int)S.ntasks,
                                                                        iters, b->eps);
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(b->ev_join, b->side) != cudaSuccess)
        return NTT_ERR_CUDA;
    }
    NTT_TRY_B(enqueue_large_stage(b, s, A, cores, ws, st, sms, h, hdev, iters, ev ? ev + 2 * s : nullptr));
    if (S.ntasks) {
      if (cudaStreamWaitEvent(st, b->ev_join, 0) != cudaSuccess) return NTT_ERR_CUDA;
      select_kernel<<<dim3(1, (unsigned)S.njobs), 256, 0, st>>>(djobs + S.job_base);
      if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    }
  }
  return NTT_OK;
}

ntt_status alloc_mapped_b(size_t bytes, char** host, char** dev) {
  void* hp = nullptr;
  void* dp = nullptr;
  if (cudaHostAlloc(&hp, bytes, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_OOM;
  }
  if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(hp);
    return NTT_ERR_CUDA;
  }
  *host = reinterpret_cast<char*>(hp);
  *dev = reinterpret_cast<char*>(dp);
  return NTT_OK;
}

}  // namespace

extern "C" {

ntt_status ntt_batch_create(int B, const int* d, const int64_t* dims, const int64_t* ranks,
                            int iters, int restarts, float eps_mu, uint64_t seed, ntt_batch* out) {
  if (!out || B < 1 || !d || !dims || !ranks || iters < 1 || restarts < 1 ||
      restarts > kMaxRestarts || !(eps_mu >= 0.0f))
    return NTT_ERR_INVALID_ARG;
  *out = nullptr;
  ntt_batch b = new (std::nothrow) ntt_batch_s();
  if (!b) return NTT_ERR_OOM;
  b->iters = iters;
  b->restarts = restarts;
  b->eps = eps_mu;
  size_t dpos = 0, rpos = 0, a_total = 0, c_total = 0, x_total = 0;
  for (int i = 0; i < B; ++i) {
    ntt_batch_s::Inst I;
    I.d = d[i];
    if (I.d < 2 || I.d > NTT_MAX_D) {
      delete b;
      return NTT_ERR_INVALID_ARG;
    }
    I.dims.assign(dims + dpos, dims + dpos + I.d);
    I.ranks.assign(ranks + rpos, ranks + rpos + I.d + 1);
    dpos += I.d;
    rpos += I.d + 1;
    if (I.ranks[0] != 1 || I.ranks[I.d] != 1) {
      delete b;
      return NTT_ERR_INVALID_ARG;
    }
    for (int k = 0; k < I.d; ++k)
      if (I.dims[k] < 1) {
        delete b;
        return NTT_ERR_INVALID_ARG;
      }
    I.seed = seed + (uint64_t)i;
    I.a_off = a_total;
    a_total = align64f(a_total + (size_t)prod64(I.dims, 0, I.d));
    size_t hmax[2] = {0, 0};
    for (int k = 0; k < I.d; ++k) {
      I.core_off.push_back(c_total);
      c_total += (size_t)(I.ranks[k] * I.dims[k] * I.ranks[k + 1]);
    }
    for (int s = 0; s < I.d - 1; ++s) {
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
      const int64_t r = I.ranks[s + 1];
      if (r < 1 || r > m || r > n) {
        delete b;
        return NTT_ERR_RANK_INFEASIBLE;
      }
      if (r > NTT_MAX_RANK || m > NTT_MAX_ROWS) {
        delete b;
        return NTT_ERR_UNSUPPORTED;
      }
      if (s < I.d - 2) hmax[s & 1] = std::max(hmax[s & 1], (size_t)(r * n));
    }
    I.x_off[0] = x_total;
    x_total = align64f(x_total + hmax[0] + 1);
    I.x_off[1] = x_total;
    x_total = align64f(x_total + hmax[1] + 1);
    b->max_stages = std::max(b->max_stages, I.d - 1);
    b->inst.push_back(I);
  }
  b->a_total = a_total;
  b->cores_total = c_total;
  const int R = restarts;
  const int sms = device_sms();
  // ---- per stage: small tasks, large problems
  b->stage.resize(b->max_stages);
  size_t small_max = 0;
  for (int s = 0; s < b->max_stages; ++s) {
    auto& S = b->stage[s];
    S.task_base = b->n_tasks;
    S.job_base = b->n_jobs;
    for (int i = 0; i < B; ++i) {
      const auto& I = b->inst[i];
      if (s >= I.d - 1) continue;
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
      const int r = (int)I.ranks[s + 1];
      if (is_small(m, n, r)) {
        S.ntasks += R;
        S.njobs += 1;
        S.small_floats += (size_t)R * (m * r + r * n);
        S.small_smem = std::max(S.small_smem, small_smem_bytes((int)m, (int)n, r));
      } else {
        S.large.push_back(i);
      }
    }
    b->n_tasks += S.ntasks;
    b->n_jobs += S.njobs;
    small_max = std::max(small_max, S.small_floats);
  }
  // ---- workspace: fixed regions, then the stage region (reused by every stage)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + (bytes ? bytes : 1));
    return o;
  };
  b->off_status = take(64);
  b->off_obj = take((size_t)B * R * sizeof(double));
  b->off_tasks = take(std::max<size_t>(1, b->n_tasks) * sizeof(SmallTask));
  b->off_jobs = take(std::max<size_t>(1, b->n_jobs) * sizeof(SelectJob));
  b->off_small = take(small_max * 4);
  b->off_x = take(x_total * 4);
  b->off_stage = off;
  size_t stage_max = 0, host_total = 0;
  for (int s = 0; s < b->max_stages; ++s) {
    auto& S = b->stage[s];
    if (S.large.empty()) continue;
    // tables first (one host-to-device copy), then factors and engine scratch
    size_t so = b->off_stage;
    auto stake = [&](size_t bytes) {
      const size_t o = so;
      so = align256(so + (bytes ? bytes : 1));
      return o;
    };
    std::vector<GroupShape> shapes;
    for (int i : S.large) {
      const auto& I = b->inst[i];
      const int r = (int)I.ranks[s + 1];
      const int g = std::max(1, std::min(R, NTT_MAX_RANK / r));
      for (int j0 = 0; j0 < R; j0 += g) {
        const int gj = std::min(g, R - j0);
        S.prob_inst.push_back(i);
        S.prob_j0.push_back(j0);
        S.prob_g.push_back(gj);
        GroupShape sh;
        sh.n = prod64(I.dims, s + 1, I.d);
        sh.m = (int)(I.ranks[s] * I.dims[s]);
        sh.re = gj * r;
        sh.blk = r;
        shapes.push_back(sh);
      }
    }
    const int np = (int)shapes.size();
    S.nres = (int)S.large.size() * R;
    int64_t max_rn = 1;
    S.res_blocks = 0;
    int res_w = 1;
    for (int i : S.large) {
      const auto& I = b->inst[i];
      const int64_t n = prod64(I.dims, s + 1, I.d);
      const int64_t m = I.ranks[s] * I.dims[s], r = I.ranks[s + 1];
      S.res_blocks += R * (int)((n + kResCols - 1) / kResCols);
      max_rn = std::max(max_rn, r * n);
      res_w = std::max(res_w, (int)(m * r));
    }
    S.res_smem = res_w * 4;
    S.sel_grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (max_rn + 4095) / 4096));
    S.off_init = stake((size_t)np * sizeof(InitJob));
    S.off_split = stake((size_t)np * sizeof(SplitJob));
    S.off_res = stake((size_t)S.nres * sizeof(ResJob));
    S.off_resmap = stake((size_t)S.res_blocks * sizeof(int));
    S.off_sel = stake(S.large.size() * sizeof(SelectJob));
    S.tab_bytes = so - b->off_stage;
    // the engine's own tables follow directly, so the host staging stays one
    // block; sized for every CTA split the autotuner may choose
    S.shapes = shapes;
    S.gp_base = so;
    size_t gp_end = 0, host_bytes = 0;
    for (int div : {1, 2, 4, 8}) {
      GroupPlan g;
      if (group_plan(shapes, sms, so, false, true, &g, div) != NTT_OK) {
        delete b;
        return NTT_ERR_UNSUPPORTED;
      }
      gp_end = std::max(gp_end, g.bytes);
      host_bytes = std::max(host_bytes, align256(g.off_tables + g.table_bytes - b->off_stage));
    }
    if (group_plan(shapes, sms, so, false, true, &S.gp, S.split) != NTT_OK) {
      delete b;
      return NTT_ERR_UNSUPPORTED;
    }
    // signature of the stage's grouped problems (FNV-1a over their shapes)
    uint64_t sig = 1469598103934665603ULL;
    auto mixin = [&](uint64_t v) {
      for (int k = 0; k < 8; ++k) {
        sig ^= (v >> (8 * k)) & 0xFF;
        sig *= 1099511628211ULL;
      }
    };
    mixin((uint64_t)sms);
    for (const auto& sh : shapes) {
      mixin((uint64_t)sh.n);
      mixin((uint64_t)sh.m);
      mixin((uint64_t)sh.re);
      mixin((uint64_t)sh.blk);
    }
    S.sig = sig;
    so = gp_end;
    S.host_bytes = align256(S.gp.off_tables + S.gp.table_bytes - b->off_stage);
    S.off_respart = stake((size_t)S.res_blocks * sizeof(double));
    for (size_t li = 0; li < S.large.size(); ++li) {
      const auto& I = b->inst[S.large[li]];
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d), r = I.ranks[s + 1];
      S.wall_off.push_back(stake((size_t)R * m * r * 4));
      S.hall_off.push_back(stake((size_t)R * r * n * 4));
    }
    for (int p = 0; p < np; ++p) S.wg_off.push_back(stake((size_t)shapes[p].m * shapes[p].re * 4));
    stage_max = std::max(stage_max, so - b->off_stage);
    S.host_off = host_total;
    host_total += host_bytes;
  }
  off = b->off_stage + stage_max;
  b->bytes = align256(off);
  // ---- host tables (allocated per cached graph, mapped pinned)
  b->h_tasks_off = host_total;
  b->h_jobs_off = align256(b->h_tasks_off + b->n_tasks * sizeof(SmallTask));
  b->h_bytes = align256(b->h_jobs_off + b->n_jobs * sizeof(SelectJob)) + 256;
  *out = b;
  return NTT_OK;
}

ntt_status ntt_batch_sizes(ntt_batch b, size_t* input_floats, size_t* core_floats,
                           size_t* workspace_bytes) {
  if (!b) return NTT_ERR_INVALID_ARG;
  if (input_floats) *input_floats = b->a_total;
  if (core_floats) *core_floats = b->cores_total;
  if (workspace_bytes) *workspace_bytes = b->bytes;
  return NTT_OK;
}

ntt_status ntt_batch_offsets(ntt_batch b, int64_t* input_off, int64_t* core_off) {
  if (!b) return NTT_ERR_INVALID_ARG;
  size_t c = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) {
    if (input_off) input_off[i] = (int64_t)b->inst[i].a_off;
    for (int k = 0; k < b->inst[i].d; ++k)
      if (core_off) core_off[c++] = (int64_t)b->inst[i].core_off[k];
  }
  return NTT_OK;
}

ntt_status ntt_decompose_batched(ntt_batch b, const float* A, float* cores, void* workspace,
                                 void* stream) {
  if (!b || !A || !cores || !workspace) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  NTT_TRY_B(batch_setup(b));
  ntt_batch_s::Graph* G = nullptr;
  for (auto& g : b->graphs)
    if (g.exec && g.A == A && g.cores == cores && g.ws == workspace) G = &g;
  if (!G) {
    G = &b->graphs[b->victim];
    b->victim ^= 1;
    // the entry's tables are rewritten by the capture: its last launch must be done
    if (G->launched && cudaEventSynchronize(G->done) != cudaSuccess) return NTT_ERR_CUDA;
    G->launched = false;
    if (G->exec) {
      cudaGraphExecDestroy(G->exec);
      G->exec = nullptr;
    }
    if (!G->done && cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming) != cudaSuccess) return NTT_ERR_CUDA;
    if (!G->h) NTT_TRY_B(alloc_mapped_b(b->h_bytes, &G->h, &G->hdev));
    if (!b->cap && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return NTT_ERR_CUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return NTT_ERR_CUDA;
    const ntt_status e = enqueue_batch(b, A, cores, ws, b->cap, G->h, G->hdev, b->iters, nullptr);
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (e != NTT_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return e != NTT_OK ? e : NTT_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&G->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      G->exec = nullptr;
      return NTT_ERR_CUDA;
    }
    G->A = A;
    G->cores = cores;
    G->ws = workspace;
  }
  if (cudaGraphLaunch(G->exec, st) != cudaSuccess || cudaEventRecord(G->done, st) != cudaSuccess) {
    cudaGetLastError();
    return NTT_ERR_CUDA;
  }
  G->launched = true;
  return NTT_OK;
}

namespace {

bool read_tuning_cache(const char* path, uint64_t sig, int* split) {
  if (!path || !path[0]) return false;
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  // one entry per line: "gsplit <signature hex> <split> <probe ms>"
  while (std::fgets(line, sizeof(line), f)) {
    char tag[32];
    unsigned long long key = 0;
    int val = 0;
    if (std::sscanf(line, "%31s %llx %d", tag, &key, &val) == 3 && std::strcmp(tag, "gsplit") == 0 &&
        key == sig && (val == 1 || val == 2 || val == 4 || val == 8)) {
      *split = val;   // the last entry for a signature wins
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void append_tuning_cache(const char* path, uint64_t sig, int split, float ms) {
  if (!path || !path[0]) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "gsplit %016llx %d %.4f\n", (unsigned long long)sig, split, ms);
  std::fclose(f);
}

}  // namespace

ntt_status ntt_batch_tune(ntt_batch b, const float* A, float* cores, void* workspace, void* stream,
                          int probe_iters, const char* cache_path) {
  if (!b || !A || !cores || !workspace || probe_iters < 1) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return NTT_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = reinterpret_cast<char*>(workspace);
  NTT_TRY_B(batch_setup(b));
  const int sms = device_sms();
  b->tuned_from_cache = 0;
  b->tuned_timed = 0;
  std::vector<int> todo;
  for (int s = 0; s < b->max_stages; ++s) {
    auto& S = b->stage[s];
    if (S.large.empty()) continue;
    int split = 0;
    if (read_tuning_cache(cache_path, S.sig, &split)) {
      S.split = split;
      S.tuned = true;
      ++b->tuned_from_cache;
    } else {
      todo.push_back(s);
    }
  }
  // the cached graphs hold tables of the old splits
  b->drop_graphs();
  auto replan = [&](int s) -> ntt_status {
    auto& S = b->stage[s];
    if (group_plan(S.shapes, sms, S.gp_base, false, true, &S.gp, S.split) != NTT_OK) return NTT_ERR_UNSUPPORTED;
    S.host_bytes = align256(S.gp.off_tables + S.gp.table_bytes - b->off_stage);
    return NTT_OK;
  };
  for (int s = 0; s < b->max_stages; ++s)
    if (!b->stage[s].large.empty()) NTT_TRY_B(replan(s));
  if (todo.empty()) return NTT_OK;
  if (!b->h_tune) NTT_TRY_B(alloc_mapped_b(b->h_bytes, &b->h_tune, &b->h_tune_dev));
  std::vector<cudaEvent_t> ev(2 * b->max_stages, nullptr);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return NTT_ERR_CUDA;
  auto free_ev = [&]() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    cudaGetLastError();
  };
  const int cands[4] = {1, 2, 4, 8};
  std::vector<float> best(b->max_stages, 1e30f);
  std::vector<int> best_split(b->max_stages, 4);
  // eager runs of the whole batch with probe_iters iterations, every untuned
  // stage on candidate c; the grouped iterations of each stage timed by events
  for (int c : cands) {
    for (int s : todo) {
      b->stage[s].split = c;
      const ntt_status e = replan(s);
      if (e != NTT_OK) {
        free_ev();
        return e;
      }
    }
    ntt_status e = enqueue_batch(b, A, cores, ws, st, b->h_tune, b->h_tune_dev, probe_iters, ev.data());
    if (e == NTT_OK && cudaStreamSynchronize(st) != cudaSuccess) e = NTT_ERR_CUDA;
    if (e != NTT_OK) {
      free_ev();
      return e;
    }
    for (int s : todo) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ev[2 * s], ev[2 * s + 1]) != cudaSuccess) {
        free_ev();
        return NTT_ERR_CUDA;
      }
      if (ms < best[s]) {
        best[s] = ms;
        best_split[s] = c;
      }
    }
  }
  free_ev();
  for (int s : todo) {
    auto& S = b->stage[s];
    S.split = best_split[s];
    S.tuned = true;
    NTT_TRY_B(replan(s));
    append_tuning_cache(cache_path, S.sig, S.split, best[s]);
    ++b->tuned_timed;
  }
  return NTT_OK;
}

ntt_status ntt_batch_get_tuning(ntt_batch b, int max_stages, int* split, int* from_cache, int* timed) {
  if (!b || max_stages < 0 || (max_stages > 0 && !split)) return NTT_ERR_INVALID_ARG;
  for (int s = 0; s < max_stages; ++s)
    split[s] = s < b->max_stages && !b->stage[s].large.empty() ? b->stage[s].split : 0;
  if (from_cache) *from_cache = b->tuned_from_cache;
  if (timed) *timed = b->tuned_timed;
  return NTT_OK;
}

ntt_status ntt_batch_destroy(ntt_batch b) {
  if (!b) return NTT_ERR_INVALID_ARG;
  delete b;
  return NTT_OK;
}

}  // extern "C"
