// Cross-CTA reduction of the pass partials and the W half of the MU iteration.
//
//   [P ; Q] = sum over pass CTAs of their partials            (fixed order)
//   W      <- max(0, W o P / (W Q + eps))                     (Lee-Seung W update)
//   G_W    <- W^T W                                           (Gram, Algorithm 4)
//   f      <- 1/2 (||X||^2 - 2 <W, P> + <G_W, Q>)              (objective, FP64)
//
// The reduction is the single-GPU replacement of the all-reduce of
// Algorithm 4 and the reduce-scatter of Algorithm 5.  Two launches: every
// block of the first reduces 32 entries with 8 partial-chunks per entry (FP32
// within a chunk, FP64 across chunks, fixed order); every block of the second
// updates 32 rows of W and forms their share of G_W and of the objective
// (<G_W, Q> as the sum over rows of W_i Q W_i^T), and the last block to finish
// (ticket counter, no spin) adds the shares in block order and runs the
// stopping test.
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
  float* scratch;   // the W half's per-block partials (the pass partial buffer, consumed by then)
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

// [P ; Q] = sum over the pass CTAs of their partials, 32 entries per block:
// eight chunks of CTAs summed in FP32, the chunks in FP64 pairwise (a fixed
// order), rounded to FP32 into red.
__global__ void __launch_bounds__(kAuxThreads) combine_reduce_kernel(const CombineParams p) {
  __shared__ float chunk[kChunks][kEntriesPerBlock];
  const int tid = threadIdx.x;
  const int E = (p.MP + p.R) * p.R;
  pdl_wait();      // the pass's partials
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the loop's stopping test has fired
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

// The W half, kRowsW rows of W per block:
//   W_i <- max(0, W_i o P_i / (W_i Q + eps))      (the sum over j in index order)
//   G partial = sum over the block's rows of W_i^T W_i   (compensated, rows in order)
//   objective partials  a = <W, P>_rows,  b = sum_i W_i Q W_i^T  (FP64; <G, Q> = sum_i W_i Q W_i^T)
// and in the last block to finish (ticket): G = the partials summed in block
// order, f = 1/2 (||X||^2 - 2 a + b) with a, b summed in block order, the
// stopping test.  blk > 0 keeps Q's and G's diagonal blk x blk blocks only.
// The partials live in the pass partial buffer (consumed by the reduction).
constexpr int kRowsW = 32;
constexpr int kMaxWBlocks = 16;   // 512 rows at most

__global__ void __launch_bounds__(kAuxThreads) combine_w_kernel(const CombineParams p) {
  __shared__ float Qs[NTT_MAX_RANK * NTT_MAX_RANK];
  __shared__ float Pb[kRowsW * NTT_MAX_RANK];
  __shared__ float Wb[kRowsW * NTT_MAX_RANK];
  __shared__ float Wn[kRowsW * NTT_MAX_RANK];
  __shared__ double dsh[2 * kAuxThreads / 32];
  __shared__ double osh[2 * kMaxWBlocks];
  __shared__ int s_last;
  pdl_wait();      // the reduced [P ; Q]
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the loop's stopping test has fired
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = p.m, r = p.r, R = p.R, MP = p.MP, blk = p.blk;
  const int i0 = blockIdx.x * kRowsW;
  const int rows = min(kRowsW, m - i0);
  auto same = [&](int k, int l) { return blk <= 0 || k / blk == l / blk; };
  for (int e = tid; e < r * r; e += nt) {
    const int jj = e / r, k = e % r;
    Qs[jj * R + k] = __ldcg(&p.red[(MP + jj) * R + k]);
  }
  for (int e = tid; e < rows * r; e += nt) {
    const int i = e / r, k = e % r;
    Pb[i * R + k] = __ldcg(&p.red[(i0 + i) * R + k]);
    Wb[i * R + k] = p.W[(i0 + i) * r + k];
  }
  __syncthreads();
  for (int e = tid; e < rows * r; e += nt) {
    const int i = e / r, k = e % r;
    float wq = 0.0f;
    for (int jj = 0; jj < r; ++jj)
      if (same(jj, k)) wq = fmaf(Wb[i * R + jj], Qs[jj * R + k], wq);
    const float w = fmaxf(0.0f, __fdiv_rn(Wb[i * R + k] * Pb[i * R + k], wq + p.eps));
    Wn[i * R + k] = w;
    p.W[(i0 + i) * r + k] = w;
  }
  __syncthreads();
  float* gpart = p.scratch;
  double* opart = reinterpret_cast<double*>(p.scratch + ((gridDim.x * R * R + 1) & ~1));
  // G partial of the block's rows, compensated (exact products by FMA, error-free
  // additions; Ogita, Rump & Oishi 2005): within about an ulp of W_b^T W_b
  for (int kl = tid; kl < R * R; kl += nt) {
    const int k = kl / R, l = kl % R;
    float sum = 0.0f, comp = 0.0f;
    if (k < r && l < r && same(k, l))
      for (int i = 0; i < rows; ++i) {
        const float a = Wn[i * R + k], b = Wn[i * R + l];
        const float pr = __fmul_rn(a, b);
        const float pe = fmaf(a, b, -pr);
        const float t = __fadd_rn(sum, pr);
        const float z = __fsub_rn(t, sum);
        const float q = __fadd_rn(__fsub_rn(sum, __fsub_rn(t, z)), __fsub_rn(pr, z));
        sum = t;
        comp = __fadd_rn(comp, __fadd_rn(q, pe));
      }
    gpart[blockIdx.x * R * R + kl] = __fadd_rn(sum, comp);
  }
  if (p.obj) {
    double a = 0.0, b = 0.0;
    for (int e = tid; e < rows * r; e += nt) {
      const int i = e / r, l = e % r;
      float qw = 0.0f;
      for (int k = 0; k < r; ++k)
        if (same(k, l)) qw = fmaf(Wn[i * R + k], Qs[k * R + l], qw);
      const double w = (double)Wn[i * R + l];
      a += w * (double)Pb[i * R + l];
      b += w * (double)qw;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int nw = nt / 32;
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
      opart[2 * blockIdx.x] = As;
      opart[2 * blockIdx.x + 1] = Bs;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the other blocks' shares: every load of a thread in flight at once, then
  // the sums in block order
  const int nb = (int)gridDim.x;
  for (int i = tid; p.obj && i < 2 * nb; i += nt) osh[i] = __ldcg(&opart[i]);
  for (int kl = tid; kl < R * R; kl += nt) {
    float v[kMaxWBlocks];
#pragma unroll
    for (int b = 0; b < kMaxWBlocks; ++b) v[b] = b < nb ? __ldcg(&gpart[b * R * R + kl]) : 0.0f;
    // compensated sum of the block partials in block order
    float sum = 0.0f, comp = 0.0f;
#pragma unroll
    for (int b = 0; b < kMaxWBlocks; ++b) {
      if (b >= nb) break;
      const float t = __fadd_rn(sum, v[b]);
      const float z = __fsub_rn(t, sum);
      comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(sum, __fsub_rn(t, z)), __fsub_rn(v[b], z)));
      sum = t;
    }
    p.G[kl] = __fadd_rn(sum, comp);
  }
  __syncthreads();
  if (tid == 0) {
    if (p.obj) {
      double As = 0.0, Bs = 0.0;
      for (int b = 0; b < nb; ++b) {
        As += osh[2 * b];
        Bs += osh[2 * b + 1];
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
    *p.ticket = 0u;
  }
}

__global__ void __launch_bounds__(kAuxThreads) gram_kernel(const float* W, int m, int r, int R,
                                                           float* G, int blk) {
  gram_block(W, m, r, R, G, nullptr, blk);
}

}  // namespace

cudaError_t launch_mu_combine(const MuShape& s, const MuDev& d, float eps, int t, cudaStream_t st) {
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
  p.scratch = d.part;
  const int E = s.part_stride();
  const int wblocks = (int)((s.m + kRowsW - 1) / kRowsW);
  if (wblocks > kMaxWBlocks) return cudaErrorInvalidValue;
  // the W half's partials fit the partial buffer the reduction has consumed
  if ((size_t)wblocks * (s.R * s.R + 4) + 2 > (size_t)s.grid * E) return cudaErrorInvalidValue;
  const cudaError_t e =
      launch_pdl(combine_reduce_kernel, dim3((E + kEntriesPerBlock - 1) / kEntriesPerBlock), dim3(kAuxThreads), 0, st, p);
  if (e != cudaSuccess) return e;
  return launch_pdl(combine_w_kernel, dim3(wblocks), dim3(kAuxThreads), 0, st, p);
}

cudaError_t launch_gram(const MuShape& s, const MuDev& d, cudaStream_t st) {
  gram_kernel<<<1, kAuxThreads, 0, st>>>(d.W, (int)s.m, s.r, s.R, d.G, d.blk);
  return cudaGetLastError();
}

}  // namespace ntt
