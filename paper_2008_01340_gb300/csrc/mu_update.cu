// Cross-CTA reduction of the pass partials and the W half of the MU iteration.
//
//   [P ; Q] = sum over pass CTAs of their partials            (fixed order)
//   W      <- max(0, W o P / (W Q + eps))                     (spec W update)
//   G_W    <- W^T W                                           (Gram, Algorithm 4)
//   f      <- 1/2 (||X||^2 - 2 <W, P> + <G_W, Q>)              (objective, FP64)
//
// The reduction is the single-GPU replacement of the all-reduce of
// Algorithm 4 and the reduce-scatter of Algorithm 5.  Every block reduces 32
// entries with 8 partial-chunks per entry (FP32 within a chunk, FP64 across
// chunks, fixed order); the last block to finish (ticket counter, no spin)
// performs the W update, the Gram and the objective and resets the ticket.
#include "ntt_internal.cuh"

namespace ntt {

namespace {

constexpr int kEntriesPerBlock = 32;
constexpr int kChunks = kAuxThreads / kEntriesPerBlock;  // 8

struct CombineParams {
  const float* part;
  int nb;
  int MP, R, m, r;
  float* W;
  float* G;
  float* red;
  unsigned* ticket;
  double* obj;
  int t;
  const double* xnorm2;
  float eps;
  int blk;   // > 0: W^T W and H H^T masked to diagonal blocks of this size
};

// Deterministic FP64 block sum of one value per thread (tree over smem).
__device__ double block_sum_f64(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  const double out = sh[0];
  __syncthreads();
  return out;
}

// G = W^T W (R x R, zero outside r x r) from W (m x r) by the whole block.
// Eight independent partial sums per entry (fixed order) keep the FMA chain short.
// blk > 0 keeps only the diagonal blk x blk blocks: the columns of W are then
// independent restarts of rank blk solved side by side (their updates only
// ever couple through these Gram matrices).
__device__ void gram_block(const float* W, int m, int r, int R, float* G, float* Gs, int blk) {
  for (int kl = threadIdx.x; kl < R * R; kl += blockDim.x) {
    const int k = kl / R, l = kl % R;
    float g = 0.0f;
    if (k < r && l < r && (blk <= 0 || k / blk == l / blk)) {
      float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int i = 0;
      for (; i + 8 <= m; i += 8)
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fmaf(W[(i + u) * r + k], W[(i + u) * r + l], a[u]);
      for (; i < m; ++i) a[0] = fmaf(W[i * r + k], W[i * r + l], a[0]);
      g = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    G[kl] = g;
    if (Gs) Gs[kl] = g;
  }
}

__global__ void __launch_bounds__(kAuxThreads) mu_combine_kernel(const CombineParams p) {
  extern __shared__ float sm[];
  __shared__ float chunk[kChunks][kEntriesPerBlock];
  __shared__ double dsh[kAuxThreads];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int E = (p.MP + p.R) * p.R;

  // ---- 1. reduce 32 entries over all partials: 8 chunks x FP32, then FP64
  {
    const int el = tid % kEntriesPerBlock;
    const int j = tid / kEntriesPerBlock;
    const int e = blockIdx.x * kEntriesPerBlock + el;
    const int per = (p.nb + kChunks - 1) / kChunks;
    const int b0 = j * per;
    const int b1 = min(p.nb, b0 + per);
    float s = 0.0f;
    if (e < E) {
#pragma unroll 8
      for (int b = b0; b < b1; ++b) s += __ldcg(&p.part[(size_t)b * E + e]);
    }
    chunk[j][el] = s;
    __syncthreads();
    if (tid < kEntriesPerBlock && e < E) {
      double tot = 0.0;
#pragma unroll
      for (int c = 0; c < kChunks; ++c) tot += (double)chunk[c][tid];
      p.red[e] = (float)tot;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---- 2. last block: W update, Gram, objective
  const int m = p.m, r = p.r, R = p.R, MP = p.MP;
  float* red_s = sm;                 // E
  float* Wn = red_s + E;             // m * r
  float* Gs = Wn + m * r;            // R * R
  for (int e = tid; e < E; e += blockDim.x) red_s[e] = __ldcg(&p.red[e]);
  __syncthreads();
  for (int i = tid; i < m; i += blockDim.x) {
    float w[NTT_MAX_RANK];
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) w[k] = (k < r) ? p.W[i * r + k] : 0.0f;
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) {
      if (k < r) {
        float wq = 0.0f;
#pragma unroll
        for (int j = 0; j < NTT_MAX_RANK; ++j)
          if (j < r && (p.blk <= 0 || j / p.blk == k / p.blk))
            wq = fmaf(w[j], red_s[(MP + j) * R + k], wq);
        Wn[i * r + k] = fmaxf(0.0f, __fdiv_rn(w[k] * red_s[i * R + k], wq + p.eps));
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < m * r; e += blockDim.x) p.W[e] = Wn[e];
  gram_block(Wn, m, r, R, p.G, Gs, p.blk);
  __syncthreads();
  if (p.obj) {
    double a = 0.0, b = 0.0;
    for (int e = tid; e < m * r; e += blockDim.x) {
      const int i = e / r, k = e % r;
      a += (double)Wn[e] * (double)red_s[i * R + k];
    }
    for (int kl = tid; kl < r * r; kl += blockDim.x) {
      const int k = kl / r, l = kl % r;
      if (p.blk <= 0 || k / p.blk == l / p.blk)
        b += (double)Gs[k * R + l] * (double)red_s[(MP + k) * R + l];
    }
    const double A = block_sum_f64(a, dsh);
    const double B = block_sum_f64(b, dsh);
    if (tid == 0) p.obj[p.t] = 0.5 * (*p.xnorm2 - 2.0 * A + B);
  }
  if (tid == 0) *p.ticket = 0u;
}

__global__ void __launch_bounds__(kAuxThreads) gram_kernel(const float* W, int m, int r, int R,
                                                           float* G, int blk) {
  gram_block(W, m, r, R, G, nullptr, blk);
}

}  // namespace

cudaError_t launch_mu_combine(const MuShape& s, const MuDev& d, float eps, int t, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_combine_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CombineParams p;
  p.part = d.part;
  p.nb = s.grid;
  p.MP = s.MP;
  p.R = s.R;
  p.m = (int)s.m;
  p.r = s.r;
  p.W = d.W;
  p.G = d.G;
  p.red = d.red;
  p.ticket = d.ticket;
  p.obj = d.obj;
  p.t = t;
  p.xnorm2 = d.xnorm2;
  p.eps = eps;
  p.blk = d.blk;
  const int E = s.part_stride();
  const int blocks = (E + kEntriesPerBlock - 1) / kEntriesPerBlock;
  const size_t smem = (size_t)(E + s.m * s.r + s.R * s.R) * sizeof(float);
  mu_combine_kernel<<<blocks, kAuxThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gram(const MuShape& s, const MuDev& d, cudaStream_t st) {
  gram_kernel<<<1, kAuxThreads, 0, st>>>(d.W, (int)s.m, s.r, s.R, d.G, d.blk);
  return cudaGetLastError();
}

}  // namespace ntt
