// Column-sharded multiplicative-update NMF: the 1-D column distribution of the
// paper's Section III-B on one GPU per shard.
//
// Every rank holds a contiguous block of columns of X and of H and the whole
// W.  One iteration is
//   1. nmf_mu_shard_pass (this rank):  G = W^T W; the fused pass over the
//      local columns (H update, then [P ; Q] = [X ; H_new] H_new^T of the
//      local columns); the pass partials reduced in a fixed order into FP64;
//   2. the caller's all-reduce (sum) of the (m + r) x r FP64 [P ; Q] over the
//      ranks -- the exchange step of Algorithms 4-6, one message of
//      8 (m + r) r bytes per iteration;
//   3. nmf_mu_shard_update (every rank, replicated): W <- max(0, W o P /
//      (W Q + eps)) and the FP64 objective 1/2 (||X||^2 - 2 <W, P> + <G, Q>).
// The H update of a column needs only W, G and that column, so the shards
// never exchange X or H.
#include "ntt_internal.cuh"

namespace ntt {

namespace {

constexpr int kShardEntries = 32;
constexpr int kShardChunks = kAuxThreads / kShardEntries;   // 8

// pq[e] = sum over the pass CTAs of part[cta][e]: eight FP32 chunks of CTAs,
// then an FP64 pairwise sum of the chunks (a fixed order).
// accumulate: pq[e] += the sum (column chunks of one pass, added in chunk order).
__global__ void __launch_bounds__(kAuxThreads) shard_reduce_kernel(const float* part, int nb, int E, double* pq,
                                                                   int accumulate) {
  __shared__ float chunk[kShardChunks][kShardEntries];
  const int tid = threadIdx.x;
  const int el = tid % kShardEntries, j = tid / kShardEntries;
  const int e = blockIdx.x * kShardEntries + el;
  const int per = (nb + kShardChunks - 1) / kShardChunks;
  const int b0 = j * per, b1 = min(nb, b0 + per);
  float s = 0.0f;
  if (e < E)
    for (int b = b0; b < b1; ++b) s += __ldcg(&part[(size_t)b * E + e]);
  chunk[j][el] = s;
  __syncthreads();
  if (tid < kShardEntries && e < E) {
    double t[kShardChunks];
#pragma unroll
    for (int c = 0; c < kShardChunks; ++c) t[c] = (double)chunk[c][tid];
#pragma unroll
    for (int w = 1; w < kShardChunks; w *= 2)
#pragma unroll
      for (int c = 0; c + w < kShardChunks; c += 2 * w) t[c] += t[c + w];
    pq[e] = accumulate ? pq[e] + t[0] : t[0];
  }
}

// One block: W update from the reduced [P ; Q] (MP + R rows of R, FP64),
// G = W^T W, objective.  Shared memory: P, Q rounded to FP32 as the
// single-GPU combine uses them, W, G.
__global__ void __launch_bounds__(kAuxThreads) shard_update_kernel(const double* pq, int m, int r, int MP, int R,
                                                                   float* W, float* G, float eps, double xnorm2,
                                                                   const double* xn_dev, double* obj) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int E = (MP + R) * R;
  float* red = sm;            // E
  float* Wn = red + E;        // m x r
  float* Gs = Wn + m * r;     // R x R
  __shared__ double dsh[2 * kAuxThreads / 32];
  for (int e = tid; e < E; e += blockDim.x) red[e] = (float)pq[e];
  for (int e = tid; e < m * r; e += blockDim.x) Wn[e] = W[e];
  __syncthreads();
  // W <- max(0, W o P / (W Q + eps)), each row by one thread, the sum over l in order
  for (int i = tid; i < m; i += blockDim.x) {
    float w[NTT_MAX_RANK], wn[NTT_MAX_RANK];
    for (int k = 0; k < r; ++k) w[k] = Wn[i * r + k];
    for (int k = 0; k < r; ++k) {
      float wq = 0.0f;
      for (int l = 0; l < r; ++l) wq = fmaf(w[l], red[(MP + l) * R + k], wq);
      wn[k] = fmaxf(0.0f, __fdiv_rn(w[k] * red[i * R + k], wq + eps));
    }
    for (int k = 0; k < r; ++k) Wn[i * r + k] = wn[k];
  }
  __syncthreads();
  for (int e = tid; e < m * r; e += blockDim.x) W[e] = Wn[e];
  for (int kl = tid; kl < R * R; kl += blockDim.x) {
    const int k = kl / R, l = kl % R;
    float g = 0.0f;
    if (k < r && l < r) {
      float a8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int i = 0;
      for (; i + 8 <= m; i += 8)
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] = fmaf(Wn[(i + u) * r + k], Wn[(i + u) * r + l], a8[u]);
      for (; i < m; ++i) a8[0] = fmaf(Wn[i * r + k], Wn[i * r + l], a8[0]);
      g = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
    }
    G[kl] = g;
    Gs[kl] = g;
  }
  __syncthreads();
  if (!obj) return;
  double a = 0.0, b = 0.0;
  for (int i = tid; i < m; i += blockDim.x)
    for (int k = 0; k < r; ++k) a += (double)Wn[i * r + k] * pq[i * R + k];
  for (int kl = tid; kl < r * r; kl += blockDim.x) {
    const int k = kl / r, l = kl % r;
    b += (double)Gs[k * R + l] * pq[(MP + k) * R + l];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int nw = blockDim.x / 32;
  if ((tid & 31) == 0) {
    dsh[tid / 32] = a;
    dsh[nw + tid / 32] = b;
  }
  __syncthreads();
  if (tid == 0) {
    double As = 0.0, Bs = 0.0;
    for (int w = 0; w < nw; ++w) {
      As += dsh[w];
      Bs += dsh[nw + w];
    }
    *obj = 0.5 * ((xn_dev ? *xn_dev : xnorm2) - 2.0 * As + Bs);
  }
}

}  // namespace

cudaError_t launch_shard_reduce(const float* part, int nb, int E, double* pq, cudaStream_t st, bool accumulate) {
  shard_reduce_kernel<<<(E + kShardEntries - 1) / kShardEntries, kAuxThreads, 0, st>>>(part, nb, E, pq,
                                                                                     accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_shard_update(const double* pq, int m, int r, int MP, int R, float* W, float* G, float eps,
                                double xnorm2, double* obj, cudaStream_t st, const double* xn_dev) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(shard_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const size_t smem = (size_t)((MP + R) * R + m * r + R * R) * sizeof(float);
  shard_update_kernel<<<1, kAuxThreads, smem, st>>>(pq, m, r, MP, R, W, G, eps, xnorm2, xn_dev, obj);
  return cudaGetLastError();
}

}  // namespace ntt
