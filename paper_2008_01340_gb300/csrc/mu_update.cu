// Cross-CTA reduction of the pass partials and the W half of the MU iteration.
//
//   [P ; Q] = sum over pass CTAs of their partials            (fixed order)
//   W      <- max(0, W o P / (W Q + eps))                     (Lee-Seung W update)
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
  int* stop;   // nullable stop word of the loop (see MuDev)
  double tol;
  int check, t0;
};

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

// W <- max(0, W o P / (W Q + eps)) for the rows of W in shared memory (in place;
// a thread owns whole rows).  RM bounds the rank so the rank loops unroll to the
// padded bucket; the sum over j runs in index order.  blk > 0 keeps Q's diagonal
// blk x blk blocks only.
template <int RM>
__device__ __forceinline__ void w_update_rows(const float* red_s, float* Wn, int m, int r, int R, int MP,
                                              int blk, float eps) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float w[RM];
#pragma unroll
    for (int k = 0; k < RM; ++k) w[k] = (k < r) ? Wn[i * r + k] : 0.0f;
#pragma unroll
    for (int k = 0; k < RM; ++k) {
      if (k < r) {
        float wq = 0.0f;
        if (blk <= 0) {
#pragma unroll
          for (int j = 0; j < RM; ++j)
            if (j < r) wq = fmaf(w[j], red_s[(MP + j) * R + k], wq);
        } else {
          const int g = k / blk;
#pragma unroll
          for (int j = 0; j < RM; ++j)
            if (j < r && j / blk == g) wq = fmaf(w[j], red_s[(MP + j) * R + k], wq);
        }
        Wn[i * r + k] = fmaxf(0.0f, __fdiv_rn(w[k] * red_s[i * R + k], wq + eps));
      }
    }
  }
}

__global__ void __launch_bounds__(kAuxThreads) mu_combine_kernel(const CombineParams p) {
  extern __shared__ float sm[];
  __shared__ float chunk[kChunks][kEntriesPerBlock];
  __shared__ double dsh[kAuxThreads];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int E = (p.MP + p.R) * p.R;
  if (p.stop && __ldcg(p.stop)) return;   // the loop's stopping test has fired

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
      // batches of eight independent loads, summed in partial order
      constexpr int U = 8;
      for (int bb = b0; bb < b1; bb += U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = bb + u < b1 ? __ldcg(&p.part[(size_t)(bb + u) * E + e]) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (bb + u < b1) s += v[u];
      }
    }
    chunk[j][el] = s;
    __syncthreads();
    if (tid < kEntriesPerBlock && e < E) {
      // pairwise FP64 sum of the eight chunks (fixed order)
      double t[kChunks];
#pragma unroll
      for (int c = 0; c < kChunks; ++c) t[c] = (double)chunk[c][tid];
#pragma unroll
      for (int w = 1; w < kChunks; w *= 2)
#pragma unroll
        for (int c = 0; c + w < kChunks; c += 2 * w) t[c] += t[c + w];
      p.red[e] = (float)t[0];
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
  float* Wn = red_s + E;             // m * r: the current W, updated in place row by row
  float* Gs = Wn + m * r;            // R * R
  // [P ; Q] and W into shared memory, eight independent loads per batch
  {
    constexpr int U = 8;
    const int mr = m * r;
    for (int e0 = tid; e0 < E; e0 += U * kAuxThreads) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = e0 + u * kAuxThreads < E ? __ldcg(&p.red[e0 + u * kAuxThreads]) : 0.0f;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e0 + u * kAuxThreads < E) red_s[e0 + u * kAuxThreads] = v[u];
    }
    for (int e0 = tid; e0 < mr; e0 += U * kAuxThreads) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = e0 + u * kAuxThreads < mr ? p.W[e0 + u * kAuxThreads] : 0.0f;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e0 + u * kAuxThreads < mr) Wn[e0 + u * kAuxThreads] = v[u];
    }
  }
  __syncthreads();
  if (R <= 8)
    w_update_rows<8>(red_s, Wn, m, r, R, MP, p.blk, p.eps);
  else if (R <= 16)
    w_update_rows<16>(red_s, Wn, m, r, R, MP, p.blk, p.eps);
  else
    w_update_rows<NTT_MAX_RANK>(red_s, Wn, m, r, R, MP, p.blk, p.eps);
  __syncthreads();
  for (int e = tid; e < m * r; e += blockDim.x) p.W[e] = Wn[e];
  gram_block(Wn, m, r, R, p.G, Gs, p.blk);
  __syncthreads();
  if (p.obj) {
    // <W, P> by rows (two FP64 chains), <G_W, Q> by entries; one reduction of both
    double a0 = 0.0, a1 = 0.0, b = 0.0;
    for (int i = tid; i < m; i += blockDim.x)
      for (int k = 0; k < r; ++k) {
        const double t = (double)Wn[i * r + k] * (double)red_s[i * R + k];
        if (k & 1) a1 += t; else a0 += t;
      }
    for (int kl = tid; kl < r * r; kl += blockDim.x) {
      const int k = kl / r, l = kl - k * r;
      if (p.blk <= 0 || k / p.blk == l / p.blk)
        b += (double)Gs[k * R + l] * (double)red_s[(MP + k) * R + l];
    }
    double A = a0 + a1, B = b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {   // butterfly: every lane ends with the warp sum
      A += __shfl_xor_sync(0xffffffffu, A, o);
      B += __shfl_xor_sync(0xffffffffu, B, o);
    }
    const int nw = blockDim.x / 32;
    if ((tid & 31) == 0) {
      dsh[tid / 32] = A;
      dsh[nw + tid / 32] = B;
    }
    __syncthreads();
    if (tid == 0) {
      double As = 0.0, Bs = 0.0;
      for (int w = 0; w < nw; ++w) {
        As += dsh[w];
        Bs += dsh[nw + w];
      }
      const double f = 0.5 * (*p.xnorm2 - 2.0 * As + Bs);
      p.obj[p.t] = f;
      // stopping test after iteration u = t - t0 + 1 (u a multiple of K, u >= 2K):
      // f_{u-K} - f_u <= tol |f_{u-K}|; the earlier value is this loop's own
      const int u = p.t - p.t0 + 1, K = p.check;
      if (p.stop && p.tol > 0.0 && K > 0 && u % K == 0 && u >= 2 * K) {
        const double f0 = p.obj[p.t - K];
        if (f0 - f <= p.tol * fabs(f0)) *p.stop = u;
      }
    }
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
  p.stop = d.stop;
  p.tol = d.tol;
  p.check = d.check;
  p.t0 = d.loop_t0;
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
