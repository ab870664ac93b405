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
//     g*r with W^T W and H H^T masked to diagonal r x r blocks (the only
//     coupling between columns of W), g = floor(32 / r), through the streaming
//     pass -- one read of X serves g restarts;
//   * select_kernel: best restart, column-L1 hand-off into the core and the
//     next unfolding, for all instances of the stage at once.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ntt_internal.cuh"

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
constexpr int kStreams = 16;

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

// Initial factors of g side-by-side restarts: W_group (m x g r, restart j in
// columns j r .. j r + r - 1) and H rows j r .. of H_group, from each restart's stream.
struct GroupKeys {
  uint64_t w[kMaxRestarts], h[kMaxRestarts];
};
__global__ void init_group_kernel(float* Wg, float* Hg, int m, int64_t n, int r, int g,
                                  GroupKeys keys) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int re = g * r;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)m * re; e += stride) {
    const int i = (int)(e / re), q = (int)(e % re), j = q / r, k = q % r;
    Wg[e] = uniform24(keys.w[j], (uint64_t)(i * r + k));
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)re * n; e += stride) {
    const int j = (int)(e / ((int64_t)r * n));
    Hg[e] = uniform24(keys.h[j], (uint64_t)(e - (int64_t)j * r * n));
  }
}

// W_j (m x r, contiguous) <- columns j r .. of W_group, for all g restarts.
__global__ void split_group_w_kernel(const float* Wg, float* Wall, int m, int r, int g) {
  const int re = g * r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * re; e += gridDim.x * blockDim.x) {
    const int i = e / re, q = e % re, j = q / r, k = q % r;
    Wall[(size_t)j * m * r + i * r + k] = Wg[e];
  }
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

// grid = (column chunks, jobs): every block picks the same restart, computes
// the column norms, block x == 0 writes the core, all blocks scale their chunk of H.
__global__ void select_kernel(const SelectJob* jobs, int njobs) {
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
int64_t prod64(const std::vector<int64_t>& v, int a, int b) {
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= v[i];
  return p;
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
  std::vector<Inst> inst;
  // large stages run on kStreams streams, instance i on stream i % kStreams,
  // each stream with its own scratch slice
  struct Lane {
    size_t G, red, part, part64, tickets, scal, rtmp, lW, lH, lWg, job;
  };
  std::vector<Lane> lane;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  int iters = 0, restarts = 1;
  float eps = 1e-12f;
  size_t a_total = 0, cores_total = 0;
  // workspace layout (bytes)
  size_t off_status, off_tickets, off_scal, off_obj, off_tasks, off_jobs, off_small, off_x, bytes;
  size_t max_tasks = 0, max_jobs = 0;
  int max_stages = 0;
  std::vector<SmallTask> h_tasks;
  std::vector<SelectJob> h_jobs;
  cudaStream_t last_stream = nullptr;
  void* last_ws = nullptr;
  ~ntt_batch_s() {
    for (auto st : streams)
      if (st) cudaStreamDestroy(st);
    for (auto e : ev_join)
      if (e) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    cudaGetLastError();
  }
};

namespace {

bool is_small(int64_t m, int64_t n, int r) {
  return r <= kSmallMaxR && n < (1 << 20) && small_smem_bytes((int)m, (int)n, r) <= kSmallSmemCap;
}

ntt_status enqueue_batch(ntt_batch b, const float* A, float* cores, char* ws, cudaStream_t st) {
  int* status = reinterpret_cast<int*>(ws + b->off_status);
  unsigned* tickets = reinterpret_cast<unsigned*>(ws + b->off_tickets);
  double* scal = reinterpret_cast<double*>(ws + b->off_scal);
  double* obj = reinterpret_cast<double*>(ws + b->off_obj);
  if (cudaMemsetAsync(status, 0, 64, st) != cudaSuccess || cudaMemsetAsync(tickets, 0, 64, st) != cudaSuccess)
    return NTT_ERR_CUDA;
  if (b->streams.empty()) {
    b->streams.assign(kStreams, nullptr);
    b->ev_join.assign(kStreams, nullptr);
    for (int l = 0; l < kStreams; ++l)
      if (cudaStreamCreateWithFlags(&b->streams[l], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_join[l], cudaEventDisableTiming) != cudaSuccess)
        return NTT_ERR_CUDA;
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess) return NTT_ERR_CUDA;
  }
  for (const auto& L : b->lane)
    if (cudaMemsetAsync(ws + L.tickets, 0, 64, st) != cudaSuccess) return NTT_ERR_CUDA;
  const int R = b->restarts;
  const int sms = device_sms();
  for (int s = 0; s < b->max_stages; ++s) {
    // ---- small tasks of this stage
    b->h_tasks.clear();
    size_t small_off = 0;
    std::vector<int> large;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
      auto& I = b->inst[i];
      if (s >= I.d - 1) continue;
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
      const int r = (int)I.ranks[s + 1];
      if (!is_small(m, n, r)) {
        large.push_back(i);
        continue;
      }
      const float* X = (s == 0) ? A + I.a_off
                                : reinterpret_cast<const float*>(ws + b->off_x) + I.x_off[(s - 1) & 1];
      for (int j = 0; j < R; ++j) {
        SmallTask t;
        t.X = X;
        t.W = reinterpret_cast<float*>(ws + b->off_small) + small_off;
        t.H = t.W + m * r;
        small_off += (size_t)(m * r + r * n);
        t.obj = obj + (size_t)i * R + j;
        t.keyW = stream_key(I.seed, s, j, 0);
        t.keyH = stream_key(I.seed, s, j, 1);
        t.m = (int)m;
        t.n = (int)n;
        t.r = r;
        t.pad = 0;
        b->h_tasks.push_back(t);
      }
    }
    if (!b->h_tasks.empty()) {
      SmallTask* dtasks = reinterpret_cast<SmallTask*>(ws + b->off_tasks);
      if (cudaMemcpyAsync(dtasks, b->h_tasks.data(), b->h_tasks.size() * sizeof(SmallTask),
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NTT_ERR_CUDA;
      size_t smem = 0;
      for (auto& t : b->h_tasks) smem = std::max(smem, small_smem_bytes(t.m, t.n, t.r));
      static bool attr = false;
      if (!attr) {
        if (cudaFuncSetAttribute(small_nmf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmallSmemCap + 1024) != cudaSuccess)
          return NTT_ERR_CUDA;
        attr = true;
      }
      int grid = (int)std::min<size_t>(b->h_tasks.size(), (size_t)sms * (smem > 110 * 1024 ? 1 : 2));
      small_nmf_kernel<<<grid, kSmallThreads, smem, st>>>(dtasks, (int)b->h_tasks.size(), b->iters,
                                                          b->eps);
      if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    }
    // ---- large tasks: instance i on lane i % kStreams, g restarts side by side
    if (!large.empty()) {
      if (cudaEventRecord(b->ev_fork, st) != cudaSuccess) return NTT_ERR_CUDA;
      for (int l = 0; l < kStreams; ++l)
        if (cudaStreamWaitEvent(b->streams[l], b->ev_fork, 0) != cudaSuccess) return NTT_ERR_CUDA;
    }
    for (int i : large) {
      auto& I = b->inst[i];
      const int lid = i % kStreams;
      const auto& L = b->lane[lid];
      cudaStream_t ls = b->streams[lid];
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
      const int r = (int)I.ranks[s + 1];
      const float* X = (s == 0) ? A + I.a_off
                                : reinterpret_cast<const float*>(ws + b->off_x) + I.x_off[(s - 1) & 1];
      float* Wall = reinterpret_cast<float*>(ws + L.lW);
      float* Hall = reinterpret_cast<float*>(ws + L.lH);
      float* Wg = reinterpret_cast<float*>(ws + L.lWg);
      unsigned* lt = reinterpret_cast<unsigned*>(ws + L.tickets);
      double* xn2 = reinterpret_cast<double*>(ws + L.scal);
      double* part64 = reinterpret_cast<double*>(ws + L.part64);
      NTT_TRY_B(resid_into(X, 0, nullptr, nullptr, m, n, 0, 0, 1.0, xn2, nullptr, part64, lt + 1, ls));
      const int g = std::max(1, std::min(R, NTT_MAX_RANK / r));
      for (int j0 = 0; j0 < R; j0 += g) {
        const int gj = std::min(g, R - j0);
        GroupKeys keys;
        std::memset(&keys, 0, sizeof(keys));
        for (int q = 0; q < gj; ++q) {
          keys.w[q] = stream_key(I.seed, s, j0 + q, 0);
          keys.h[q] = stream_key(I.seed, s, j0 + q, 1);
        }
        float* Hg = Hall + (size_t)j0 * r * n;
        init_group_kernel<<<sms * 2, 256, 0, ls>>>(Wg, Hg, (int)m, n, r, gj, keys);
        if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
        MuShape shp;
        NTT_TRY_B(mu_choose_shape(m, n, gj * r, 0, sms, &shp));
        MuDev dev;
        dev.X = X;
        dev.W = Wg;
        dev.H = Hg;
        dev.G = reinterpret_cast<float*>(ws + L.G);
        dev.part = reinterpret_cast<float*>(ws + L.part);
        dev.red = reinterpret_cast<float*>(ws + L.red);
        dev.ticket = lt;
        dev.obj = nullptr;
        dev.xnorm2 = xn2;
        dev.status = status;
        dev.blk = r;
        if (launch_gram(shp, dev, ls) != cudaSuccess) return NTT_ERR_CUDA;
        NTT_TRY_B(run_mu_iters(shp, dev, b->eps, b->iters, 0, ls));
        split_group_w_kernel<<<64, 256, 0, ls>>>(Wg, Wall + (size_t)j0 * m * r, (int)m, r, gj);
        if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
        double* rtmp = reinterpret_cast<double*>(ws + L.rtmp);
        for (int q = 0; q < gj; ++q) {
          NTT_TRY_B(resid_into(X, 0, Wall + (size_t)(j0 + q) * m * r, Hg + (size_t)q * r * n, m, n, r, 1,
                               0.5, rtmp + 2 * q, nullptr, part64, lt + 1, ls));
          if (cudaMemcpyAsync(obj + (size_t)i * R + j0 + q, rtmp + 2 * q, sizeof(double),
                              cudaMemcpyDeviceToDevice, ls) != cudaSuccess)
            return NTT_ERR_CUDA;
        }
      }
      SelectJob jb;
      jb.Wc = Wall;
      jb.Hc = Hall;
      jb.w_stride = m * r;
      jb.h_stride = (int64_t)r * n;
      jb.obj = obj + (size_t)i * R;
      jb.core = cores + I.core_off[s];
      jb.next = (s == I.d - 2) ? cores + I.core_off[I.d - 1]
                               : reinterpret_cast<float*>(ws + b->off_x) + I.x_off[s & 1];
      jb.n = n;
      jb.m = (int)m;
      jb.r = r;
      jb.restarts = R;
      jb.pad = 0;
      SelectJob* dj = reinterpret_cast<SelectJob*>(ws + L.job);
      if (cudaMemcpyAsync(dj, &jb, sizeof(jb), cudaMemcpyHostToDevice, ls) != cudaSuccess)
        return NTT_ERR_CUDA;
      select_kernel<<<dim3(std::max<int64_t>(1, std::min<int64_t>(sms * 4, (r * n + 1023) / 1024)), 1),
                      256, 0, ls>>>(dj, 1);
      if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    }
    if (!large.empty())
      for (int l = 0; l < kStreams; ++l) {
        if (cudaEventRecord(b->ev_join[l], b->streams[l]) != cudaSuccess ||
            cudaStreamWaitEvent(st, b->ev_join[l], 0) != cudaSuccess)
          return NTT_ERR_CUDA;
      }
    // ---- selection for the small instances of this stage
    b->h_jobs.clear();
    {
      size_t off = 0;
      for (int i = 0; i < (int)b->inst.size(); ++i) {
        auto& I = b->inst[i];
        if (s >= I.d - 1) continue;
        const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
        const int r = (int)I.ranks[s + 1];
        if (!is_small(m, n, r)) continue;
        SelectJob jb;
        jb.Wc = reinterpret_cast<float*>(ws + b->off_small) + off;
        jb.Hc = jb.Wc + m * r;
        jb.w_stride = m * r + r * n;
        jb.h_stride = m * r + r * n;
        off += (size_t)R * (m * r + r * n);
        jb.obj = obj + (size_t)i * R;
        jb.core = cores + I.core_off[s];
        jb.next = (s == I.d - 2) ? cores + I.core_off[I.d - 1]
                                 : reinterpret_cast<float*>(ws + b->off_x) + I.x_off[s & 1];
        jb.n = n;
        jb.m = (int)m;
        jb.r = r;
        jb.restarts = R;
        jb.pad = 0;
        b->h_jobs.push_back(jb);
      }
    }
    if (!b->h_jobs.empty()) {
      SelectJob* dj = reinterpret_cast<SelectJob*>(ws + b->off_jobs);
      if (cudaMemcpyAsync(dj, b->h_jobs.data(), b->h_jobs.size() * sizeof(SelectJob),
                          cudaMemcpyHostToDevice, st) != cudaSuccess)
        return NTT_ERR_CUDA;
      select_kernel<<<dim3(1, (unsigned)b->h_jobs.size()), 256, 0, st>>>(dj, (int)b->h_jobs.size());
      if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
    }
    // pageable host-to-device copies are staged before cudaMemcpyAsync returns,
    // so the host vectors can be rebuilt for the next stage right away
  }
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
  size_t small_max = 0;
  std::vector<size_t> lW(kStreams, 1), lH(kStreams, 1), lWg(kStreams, 1), part_max(kStreams, 1),
      red_max(kStreams, 1);
  std::vector<size_t> small_per_stage(NTT_MAX_D, 0), tasks_per_stage(NTT_MAX_D, 0),
      jobs_per_stage(NTT_MAX_D, 0);
  const int sms = device_sms();
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
    I.seed = seed + (uint64_t)i;
    I.a_off = a_total;
    a_total += (size_t)prod64(I.dims, 0, I.d);
    size_t hmax[2] = {0, 0};
    for (int k = 0; k < I.d; ++k) {
      I.core_off.push_back(c_total);
      c_total += (size_t)(I.ranks[k] * I.dims[k] * I.ranks[k + 1]);
    }
    for (int s = 0; s < I.d - 1; ++s) {
      const int64_t m = I.ranks[s] * I.dims[s], n = prod64(I.dims, s + 1, I.d);
      const int r = (int)I.ranks[s + 1];
      if (I.dims[s] < 1 || r < 1 || r > m || r > n) {
        delete b;
        return NTT_ERR_RANK_INFEASIBLE;
      }
      if (r > NTT_MAX_RANK || m > NTT_MAX_ROWS) {
        delete b;
        return NTT_ERR_UNSUPPORTED;
      }
      if (s < I.d - 2) hmax[s & 1] = std::max(hmax[s & 1], (size_t)(r * n));
      if (is_small(m, n, r)) {
        small_per_stage[s] += (size_t)restarts * (m * r + r * n);
        tasks_per_stage[s] += restarts;
      } else {
        const int l = i % kStreams;
        lW[l] = std::max(lW[l], (size_t)restarts * m * r);
        lH[l] = std::max(lH[l], (size_t)restarts * r * n);
        const int g = std::max(1, std::min(restarts, NTT_MAX_RANK / r));
        lWg[l] = std::max(lWg[l], (size_t)m * g * r);
        MuShape shp;
        if (mu_choose_shape(m, n, g * r, 0, sms, &shp) != NTT_OK) {
          delete b;
          return NTT_ERR_UNSUPPORTED;
        }
        part_max[l] = std::max(part_max[l], (size_t)shp.grid_cap * shp.part_stride());
        red_max[l] = std::max(red_max[l], (size_t)shp.part_stride());
      }
      jobs_per_stage[s] += 1;
    }
    I.x_off[0] = x_total;
    x_total += hmax[0] + 1;
    I.x_off[1] = x_total;
    x_total += hmax[1] + 1;
    b->max_stages = std::max(b->max_stages, I.d - 1);
    b->inst.push_back(I);
  }
  for (int s = 0; s < NTT_MAX_D; ++s) {
    small_max = std::max(small_max, small_per_stage[s]);
    b->max_tasks = std::max(b->max_tasks, tasks_per_stage[s]);
    b->max_jobs = std::max(b->max_jobs, jobs_per_stage[s]);
  }
  b->a_total = a_total;
  b->cores_total = c_total;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + (bytes ? bytes : 1));
    return o;
  };
  b->off_status = take(64);
  b->off_tickets = take(64);
  b->off_scal = take(8 * sizeof(double));
  b->off_obj = take((size_t)B * restarts * sizeof(double));
  b->off_tasks = take(std::max<size_t>(1, b->max_tasks) * sizeof(SmallTask));
  b->off_jobs = take((b->max_jobs + 1) * sizeof(SelectJob));
  b->off_small = take(small_max * 4);
  b->off_x = take(x_total * 4);
  b->lane.resize(kStreams);
  for (int l = 0; l < kStreams; ++l) {
    auto& L = b->lane[l];
    L.tickets = take(64);
    L.scal = take(8 * sizeof(double));
    L.G = take(NTT_MAX_RANK * NTT_MAX_RANK * 4);
    L.red = take(red_max[l] * 4);
    L.part = take(part_max[l] * 4);
    L.part64 = take(2 * kMaxResidBlocks * sizeof(double));
    L.rtmp = take(2 * kMaxRestarts * sizeof(double));
    L.lW = take(lW[l] * 4);
    L.lH = take(lH[l] * 4);
    L.lWg = take(lWg[l] * 4);
    L.job = take(sizeof(SelectJob));
  }
  b->bytes = off;
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
  const ntt_status e = enqueue_batch(b, A, cores, reinterpret_cast<char*>(workspace), st);
  b->last_stream = st;
  b->last_ws = workspace;
  if (e != NTT_OK) return e;
  int status = 0;
  if (cudaMemcpyAsync(&status, reinterpret_cast<char*>(workspace) + b->off_status, sizeof(int),
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NTT_ERR_CUDA;
  return status == 0 ? NTT_OK : (ntt_status)status;
}

ntt_status ntt_batch_destroy(ntt_batch b) {
  if (!b) return NTT_ERR_INVALID_ARG;
  delete b;
  return NTT_OK;
}

}  // extern "C"
