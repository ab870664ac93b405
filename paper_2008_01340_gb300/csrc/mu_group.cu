// Grouped MU engine: planning, the grouped combine (fixed-order reduction of
// the pass partials, then the W half of the iteration and the Gram W^T W on
// the diagonal rank blocks), and the iteration loop.
//
// Combine, per problem:
//   [P ; Q] = sum over the problem's pass CTAs of their partials   (fixed order)
//   W      <- max(0, W o P / (W Q + eps))      (Q on the diagonal blocks)
//   G_W    <- W^T W                            (diagonal blocks, zero elsewhere)
// Every block reduces 32 entries of one problem with 8 partial chunks per
// entry (FP32 within a chunk, FP64 across chunks); the last block of the
// problem (ticket counter, no waiting) updates W and G_W and resets the ticket.
#include <algorithm>
#include <cstring>

#include "group_engine.cuh"

namespace ntt {

int group_mp_bucket(int m) {
  for (int b = 16; b <= NTT_MAX_ROWS; b *= 2)
    if (m <= b) return b;
  return -1;
}

int group_r_bucket(int re) {
  if (re <= 8) return 8;
  if (re <= 16) return 16;
  if (re <= 32) return 32;
  return -1;
}

int group_tile_cols(int MP, int R) { return std::max(16, std::min(4096 / R, 8192 / MP)); }

cudaError_t launch_gpass(int MP, int R, const GProb* probs, const int* cta_prob, int ncta, float eps,
                         cudaStream_t st) {
  switch (R) {
    case 8: return launch_gpass_r8(MP, probs, cta_prob, ncta, eps, st);
    case 16: return launch_gpass_r16(MP, probs, cta_prob, ncta, eps, st);
    case 32: return launch_gpass_r32(MP, probs, cta_prob, ncta, eps, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

constexpr int kEntries = 32;
constexpr int kChunks = kAuxThreads / kEntries;   // 8

// G = W^T W on the diagonal blocks (R x R, zero elsewhere), W m x re, by one block.
__device__ void group_gram(const float* W, int m, int re, int blk, int R, float* G) {
  for (int kl = threadIdx.x; kl < R * R; kl += blockDim.x) {
    const int k = kl / R, l = kl % R;
    float g = 0.0f;
    if (k < re && l < re && k / blk == l / blk) {
      float a[4] = {0.f, 0.f, 0.f, 0.f};
      int i = 0;
      for (; i + 4 <= m; i += 4)
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = fmaf(__ldcg(&W[(i + u) * re + k]), __ldcg(&W[(i + u) * re + l]), a[u]);
      for (; i < m; ++i) a[0] = fmaf(__ldcg(&W[i * re + k]), __ldcg(&W[i * re + l]), a[0]);
      g = (a[0] + a[1]) + (a[2] + a[3]);
    }
    G[kl] = g;
  }
}

__global__ void __launch_bounds__(kAuxThreads) group_gram_kernel(const GComb* combs) {
  const GComb c = combs[blockIdx.x];
  group_gram(c.W, c.m, c.re, c.blk, c.R, c.G);
}

__global__ void __launch_bounds__(kAuxThreads) group_combine_kernel(const GComb* __restrict__ combs,
                                                                    const int* __restrict__ blk_comb,
                                                                    float eps) {
  __shared__ float chunk[kChunks][kEntries];
  __shared__ int s_last;
  const GComb c = combs[blk_comb[blockIdx.x]];
  const int tid = threadIdx.x;
  const int E = (c.MP + c.R) * c.R;
  {
    const int el = tid % kEntries, j = tid / kEntries;
    const int e = (blockIdx.x - c.blk0) * kEntries + el;
    const int per = (c.S + kChunks - 1) / kChunks;
    const int b0 = j * per, b1 = min(c.S, b0 + per);
    float s = 0.0f;
    if (e < E)
      for (int b = b0; b < b1; ++b) s += __ldcg(&c.part[(size_t)b * E + e]);
    chunk[j][el] = s;
    __syncthreads();
    if (tid < kEntries && e < E) {
      double tot = 0.0;
#pragma unroll
      for (int q = 0; q < kChunks; ++q) tot += (double)chunk[q][tid];
      c.red[e] = (float)tot;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(c.ticket, 1u) == (unsigned)c.nblk - 1u) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // last block of the problem: W update row by row (each row owned by one thread), then the Gram
  const int m = c.m, re = c.re, blk = c.blk, R = c.R, MP = c.MP;
  for (int i = tid; i < m; i += blockDim.x) {
    float w[NTT_MAX_RANK], wn[NTT_MAX_RANK];
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) w[k] = (k < re) ? c.W[i * re + k] : 0.0f;
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) {
      wn[k] = 0.0f;
      if (k < re) {
        const int lo = (k / blk) * blk, hi = min(re, lo + blk);
        float wq = 0.0f;
#pragma unroll
        for (int l = 0; l < NTT_MAX_RANK; ++l)
          if (l >= lo && l < hi) wq = fmaf(w[l], __ldcg(&c.red[(MP + l) * R + k]), wq);
        wn[k] = fmaxf(0.0f, __fdiv_rn(w[k] * __ldcg(&c.red[i * R + k]), wq + eps));
      }
    }
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k)
      if (k < re) c.W[i * re + k] = wn[k];
  }
  __syncthreads();
  group_gram(c.W, m, re, blk, R, c.G);
  if (tid == 0) *c.ticket = 0u;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

ntt_status group_plan(const std::vector<GroupShape>& shapes, int sms, size_t base, GroupPlan* out) {
  GroupPlan& pl = *out;
  pl = GroupPlan();
  const int np = (int)shapes.size();
  pl.probs.resize(np);
  // bucket every problem
  std::vector<std::pair<int, int>> keys;
  for (int p = 0; p < np; ++p) {
    const GroupShape& s = shapes[p];
    if (s.n < 1 || s.m < 1 || s.re < 1 || s.blk < 1 || s.blk > s.re) return NTT_ERR_INVALID_ARG;
    const int MP = group_mp_bucket(s.m), R = group_r_bucket(s.re);
    if (MP < 0 || R < 0) return NTT_ERR_UNSUPPORTED;
    auto& q = pl.probs[p];
    q.n = s.n;
    q.m = s.m;
    q.re = s.re;
    q.blk = s.blk;
    q.MP = MP;
    q.R = R;
    const std::pair<int, int> key(MP, R);
    auto it = std::find(keys.begin(), keys.end(), key);
    if (it == keys.end()) {
      keys.push_back(key);
      q.bucket = (int)keys.size() - 1;
    } else {
      q.bucket = (int)(it - keys.begin());
    }
  }
  // CTAs per problem: every bucket launch aims at about two CTAs per SM, each
  // problem getting CTAs in proportion to its column tiles
  for (int b = 0; b < (int)keys.size(); ++b) {
    GroupPlan::Bucket B;
    B.MP = keys[b].first;
    B.R = keys[b].second;
    B.ncta = 0;
    B.cta_off = pl.total_cta;
    const int T = group_tile_cols(B.MP, B.R);
    int64_t tiles = 0;
    for (auto& q : pl.probs)
      if (q.bucket == b) tiles += (q.n + T - 1) / T;
    const int64_t target = 2LL * std::max(1, sms);
    const int64_t per = std::max<int64_t>(1, (tiles + target - 1) / target);
    for (auto& q : pl.probs) {
      if (q.bucket != b) continue;
      const int64_t nt = (q.n + T - 1) / T;
      q.S = (int)std::min<int64_t>(nt, (nt + per - 1) / per);
      q.cta0 = B.ncta;
      B.ncta += q.S;
    }
    pl.total_cta += B.ncta;
    pl.buckets.push_back(B);
  }
  // scratch: tables, tickets, then per problem G, red, part
  size_t off = base;
  pl.off_tables = off;
  pl.table_bytes = align256((size_t)np * sizeof(GProb)) + align256((size_t)np * sizeof(GComb)) +
                   align256((size_t)pl.total_cta * sizeof(int));
  for (auto& q : pl.probs) {
    const int E = (q.MP + q.R) * q.R;
    q.nblk = (E + kEntries - 1) / kEntries;
    q.blk0 = pl.total_cblk;
    pl.total_cblk += q.nblk;
  }
  pl.table_bytes += align256((size_t)pl.total_cblk * sizeof(int));
  off = align256(off + pl.table_bytes);
  pl.off_tickets = off;
  off = align256(off + (size_t)np * sizeof(unsigned));
  for (auto& q : pl.probs) {
    const size_t E = (size_t)(q.MP + q.R) * q.R;
    q.g_off = off;
    off = align256(off + (size_t)q.R * q.R * 4);
    q.red_off = off;
    off = align256(off + E * 4);
    q.part_off = off;
    off = align256(off + (size_t)q.S * E * 4);
  }
  pl.bytes = off;
  return NTT_OK;
}

ntt_status group_run(const GroupPlan& pl, const GroupPtrs* ptrs, char* scratch, void* host_tables,
                     int iters, float eps, cudaStream_t st) {
  const int np = (int)pl.probs.size();
  if (np == 0) return NTT_OK;
  char* h = reinterpret_cast<char*>(host_tables);
  GProb* hp = reinterpret_cast<GProb*>(h);
  const size_t o_comb = align256((size_t)np * sizeof(GProb));
  GComb* hc = reinterpret_cast<GComb*>(h + o_comb);
  const size_t o_cta = o_comb + align256((size_t)np * sizeof(GComb));
  int* hcta = reinterpret_cast<int*>(h + o_cta);
  const size_t o_cblk = o_cta + align256((size_t)pl.total_cta * sizeof(int));
  int* hcblk = reinterpret_cast<int*>(h + o_cblk);
  unsigned* tickets = reinterpret_cast<unsigned*>(scratch + pl.off_tickets);
  for (int p = 0; p < np; ++p) {
    const auto& q = pl.probs[p];
    const GroupPtrs& g = ptrs[p];
    GProb& a = hp[p];
    std::memset(&a, 0, sizeof(a));
    a.X = g.X;
    a.H = g.H;
    a.W = g.W;
    a.G = reinterpret_cast<const float*>(scratch + q.g_off);
    a.part = reinterpret_cast<float*>(scratch + q.part_off);
    a.n = q.n;
    a.m = q.m;
    a.re = q.re;
    a.blk = q.blk;
    a.S = q.S;
    a.cta0 = q.cta0;
    a.aligned = (q.n % 4 == 0 && reinterpret_cast<uintptr_t>(g.X) % 16 == 0 &&
                 reinterpret_cast<uintptr_t>(g.H) % 16 == 0)
                    ? 1
                    : 0;
    for (int s = 0; s < q.S; ++s) hcta[pl.buckets[q.bucket].cta_off + q.cta0 + s] = p;
    GComb& c = hc[p];
    std::memset(&c, 0, sizeof(c));
    c.part = a.part;
    c.red = reinterpret_cast<float*>(scratch + q.red_off);
    c.W = g.W;
    c.G = reinterpret_cast<float*>(scratch + q.g_off);
    c.ticket = tickets + p;
    c.S = q.S;
    c.MP = q.MP;
    c.R = q.R;
    c.m = q.m;
    c.re = q.re;
    c.blk = q.blk;
    c.blk0 = q.blk0;
    c.nblk = q.nblk;
    for (int b = 0; b < q.nblk; ++b) hcblk[q.blk0 + b] = p;
  }
  char* d = scratch + pl.off_tables;
  if (cudaMemcpyAsync(d, h, pl.table_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(tickets, 0, (size_t)np * sizeof(unsigned), st) != cudaSuccess)
    return NTT_ERR_CUDA;
  const GProb* dp = reinterpret_cast<const GProb*>(d);
  const GComb* dc = reinterpret_cast<const GComb*>(d + o_comb);
  const int* dcta = reinterpret_cast<const int*>(d + o_cta);
  const int* dcblk = reinterpret_cast<const int*>(d + o_cblk);
  group_gram_kernel<<<np, kAuxThreads, 0, st>>>(dc);
  if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  for (int t = 0; t < iters; ++t) {
    for (const auto& B : pl.buckets)
      if (launch_gpass(B.MP, B.R, dp, dcta + B.cta_off, B.ncta, eps, st) != cudaSuccess) return NTT_ERR_CUDA;
    group_combine_kernel<<<pl.total_cblk, kAuxThreads, 0, st>>>(dc, dcblk, eps);
    if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  }
  return NTT_OK;
}

}  // namespace ntt
