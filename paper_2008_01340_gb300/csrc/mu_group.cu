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
#include <tuple>

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

int group_ctas_per_sm(int MP, int R, bool xb) {
  if (xb) return gpass_occupancy_bf16(MP, R);
  switch (R) {
    case 8: return gpass_occupancy_r8(MP);
    case 16: return gpass_occupancy_r16(MP);
    case 32: return gpass_occupancy_r32(MP);
    default: return 1;
  }
}

cudaError_t launch_gpass(int mode, int MP, int R, bool xb, const GProb* probs, const int* cta_prob, int ncta,
                         float eps, cudaStream_t st) {
  if (xb) return mode == 0 ? launch_gpass_bf16(MP, R, probs, cta_prob, ncta, eps, st) : cudaErrorInvalidValue;
  switch (R) {
    case 8: return launch_gpass_r8(mode, MP, probs, cta_prob, ncta, eps, st);
    case 16: return launch_gpass_r16(mode, MP, probs, cta_prob, ncta, eps, st);
    case 32: return launch_gpass_r32(mode, MP, probs, cta_prob, ncta, eps, st);
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

// W <- max(0, W o P / (W Q + eps)) of one problem, Q restricted to its diagonal
// rank blocks; a thread owns whole rows; RM bounds the rank so the loops unroll
// to the padded bucket; the sum over l runs in index order.
template <int RM>
__device__ __forceinline__ void group_w_update(const GComb& c, float eps) {
  const int m = c.m, re = c.re, blk = c.blk, R = c.R, MP = c.MP;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float w[RM], wn[RM];
#pragma unroll
    for (int k = 0; k < RM; ++k) w[k] = (k < re) ? c.W[i * re + k] : 0.0f;
#pragma unroll
    for (int k = 0; k < RM; ++k) {
      wn[k] = 0.0f;
      if (k < re) {
        const int lo = (k / blk) * blk, hi = min(re, lo + blk);
        float wq = 0.0f;
#pragma unroll
        for (int l = 0; l < RM; ++l)
          if (l >= lo && l < hi) wq = fmaf(w[l], __ldcg(&c.red[(MP + l) * R + k]), wq);
        wn[k] = fmaxf(0.0f, __fdiv_rn(w[k] * __ldcg(&c.red[i * R + k]), wq + eps));
      }
    }
#pragma unroll
    for (int k = 0; k < RM; ++k)
      if (k < re) c.W[i * re + k] = wn[k];
  }
}

__global__ void __launch_bounds__(kAuxThreads) group_combine_kernel(const GComb* __restrict__ combs,
                                                                    const int* __restrict__ blk_comb,
                                                                    float eps, int t) {
  __shared__ float chunk[kChunks][kEntries];
  __shared__ double dsh[kAuxThreads];
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
    if (e < E) {
      // batches of eight independent loads, summed in partial order
      constexpr int U = 8;
      for (int bb = b0; bb < b1; bb += U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = bb + u < b1 ? __ldcg(&c.part[(size_t)(bb + u) * E + e]) : 0.0f;
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (bb + u < b1) s += v[u];
      }
    }
    chunk[j][el] = s;
    __syncthreads();
    if (tid < kEntries && e < E) {
      // pairwise FP64 sum of the chunks (fixed order)
      double tq[kChunks];
#pragma unroll
      for (int q = 0; q < kChunks; ++q) tq[q] = (double)chunk[q][tid];
#pragma unroll
      for (int w = 1; w < kChunks; w *= 2)
#pragma unroll
        for (int q = 0; q + w < kChunks; q += 2 * w) tq[q] += tq[q + w];
      c.red[e] = (float)tq[0];
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
  if (R <= 8)
    group_w_update<8>(c, eps);
  else if (R <= 16)
    group_w_update<16>(c, eps);
  else
    group_w_update<NTT_MAX_RANK>(c, eps);
  __syncthreads();
  group_gram(c.W, m, re, blk, R, c.G);
  if (c.obj) {
    // f = 1/2 (||X||^2 - 2 <W, P> + <W^T W, Q>) on the rank blocks, FP64 sums in a fixed order
    __syncthreads();
    // <W, P> by rows (two FP64 chains), <G_W, Q> by entries; one reduction of both
    double a0 = 0.0, a1 = 0.0, b = 0.0;
    for (int i = tid; i < m; i += blockDim.x)
      for (int k = 0; k < re; ++k) {
        const double v = (double)__ldcg(&c.W[i * re + k]) * (double)__ldcg(&c.red[i * R + k]);
        if (k & 1) a1 += v; else a0 += v;
      }
    for (int kl = tid; kl < re * re; kl += blockDim.x) {
      const int k = kl / re, l = kl - k * re;
      if (k / blk == l / blk) b += (double)__ldcg(&c.G[k * R + l]) * (double)__ldcg(&c.red[(MP + k) * R + l]);
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
      c.obj[t] = 0.5 * (*c.xnorm2 - 2.0 * As + Bs);
    }
  }
  if (tid == 0) *c.ticket = 0u;
}

// Tall unfoldings: H <- max(0, H o Y / (G H + eps)) with Y the fixed-order sum
// of the row blocks' partials; one thread per column, G (zero outside the
// diagonal blocks) in shared memory.
constexpr int kTallCols = 256;
__global__ void __launch_bounds__(kTallCols) tall_hupd_kernel(const GTall* __restrict__ talls,
                                                              const int* __restrict__ blk_tall, float eps) {
  __shared__ float Gs[NTT_MAX_RANK * NTT_MAX_RANK];
  const GTall t = talls[blk_tall[blockIdx.x]];
  for (int e = threadIdx.x; e < t.R * t.R; e += blockDim.x) Gs[e] = t.G[e];
  __syncthreads();
  const int64_t c = (int64_t)(blockIdx.x - t.blk0) * kTallCols + threadIdx.x;
  if (c >= t.n) return;
  float h[NTT_MAX_RANK], y[NTT_MAX_RANK];
#pragma unroll
  for (int k = 0; k < NTT_MAX_RANK; ++k) {
    h[k] = k < t.re ? t.H[(int64_t)k * t.n + c] : 0.0f;
    y[k] = 0.0f;
  }
  for (int b = 0; b < t.nb; ++b) {
    const float* Yb = t.Y + (int64_t)b * t.re * t.n;
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k)
      if (k < t.re) y[k] += Yb[(int64_t)k * t.n + c];
  }
#pragma unroll
  for (int k = 0; k < NTT_MAX_RANK; ++k) {
    if (k < t.re) {
      float gh = 0.0f;
#pragma unroll
      for (int l = 0; l < NTT_MAX_RANK; ++l)
        if (l < t.R) gh = fmaf(Gs[k * t.R + l], h[l], gh);
      t.H[(int64_t)k * t.n + c] = fmaxf(0.0f, __fdividef(h[k] * y[k], gh + eps));
    }
  }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int kTallRows = NTT_MAX_ROWS;   // rows per block of a tall unfolding (pass bucket 512)

// CTAs of one problem when its split may not depend on other problems.
int fixed_ctas(int64_t ntiles, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>({ntiles, (int64_t)2 * std::max(1, sms), (ntiles + 7) / 8}));
}

}  // namespace

size_t group_problem_scratch(const GroupShape& sh, int sms) {
  const int R = group_r_bucket(sh.re);
  const bool tall = sh.m > kTallRows;
  const int MP = tall ? kTallRows : group_mp_bucket(sh.m);
  const int qrow0 = tall ? (sh.m + 15) / 16 * 16 : MP;
  const size_t E = (size_t)(qrow0 + R) * R;
  const int T = group_tile_cols(MP, R);
  const int S = fixed_ctas((sh.n + T - 1) / T, sms);
  const int nb = tall ? (sh.m + kTallRows - 1) / kTallRows : 0;
  return align256((size_t)R * R * 4) + align256(E * 4) + align256((size_t)S * E * 4) +
         align256((size_t)nb * sh.re * sh.n * 4);
}

ntt_status group_plan(const std::vector<GroupShape>& shapes, int sms, size_t base, bool fixed_split,
                      bool own_scratch, GroupPlan* out, int split_div) {
  GroupPlan& pl = *out;
  pl = GroupPlan();
  pl.own_scratch = own_scratch;
  const int np = (int)shapes.size();
  pl.probs.resize(np);
  // buckets are (mode, MP, R); mode 0 entries are whole problems, tall
  // problems give one mode-1 and one mode-2 entry per row block
  std::vector<std::tuple<int, int, int, int>> keys;
  auto bucket_of = [&](int mode, int MP, int R, int xb) {
    const auto key = std::make_tuple(mode, MP, R, xb);
    auto it = std::find(keys.begin(), keys.end(), key);
    if (it != keys.end()) return (int)(it - keys.begin());
    keys.push_back(key);
    return (int)keys.size() - 1;
  };
  for (int p = 0; p < np; ++p) {
    const GroupShape& sh = shapes[p];
    if (sh.n < 1 || sh.m < 1 || sh.re < 1 || sh.blk < 1 || sh.blk > sh.re) return NTT_ERR_INVALID_ARG;
    auto& q = pl.probs[p];
    q.n = sh.n;
    q.m = sh.m;
    q.re = sh.re;
    q.blk = sh.blk;
    q.R = group_r_bucket(sh.re);
    if (q.R < 0) return NTT_ERR_UNSUPPORTED;
    q.tall = sh.m > kTallRows ? 1 : 0;
    q.xbf16 = sh.xbf16 ? 1 : 0;
    if (q.xbf16 && (q.tall || !gpass_bf16_supported(group_mp_bucket(sh.m), q.R) || sh.n % 8 != 0))
      return NTT_ERR_UNSUPPORTED;
    if (q.tall) {
      q.nb = (sh.m + kTallRows - 1) / kTallRows;
      q.mb = kTallRows;
      q.qrow0 = (sh.m + 15) / 16 * 16;
      for (int b = 0; b < q.nb; ++b) {
        pl.entries.push_back({p, b, 1, bucket_of(1, kTallRows, q.R, 0), 0});
        pl.entries.push_back({p, b, 2, bucket_of(2, kTallRows, q.R, 0), 0});
      }
    } else {
      q.nb = 1;
      q.mb = sh.m;
      q.qrow0 = group_mp_bucket(sh.m);
      pl.entries.push_back({p, 0, 0, bucket_of(0, q.qrow0, q.R, q.xbf16), 0});
    }
    q.E = (q.qrow0 + q.R) * q.R;
    const int T = group_tile_cols(q.tall ? kTallRows : q.qrow0, q.R);
    q.S = (q.tall || fixed_split) ? fixed_ctas((q.n + T - 1) / T, sms) : 0;
  }
  // split the remaining (fused, not fixed) problems of each mode-0 bucket in
  // proportion to their column tiles
  for (int bk = 0; bk < (int)keys.size(); ++bk) {
    const int mode = std::get<0>(keys[bk]), MP = std::get<1>(keys[bk]), R = std::get<2>(keys[bk]);
    const int xb = std::get<3>(keys[bk]);
    if (mode != 0) continue;
    const int T = group_tile_cols(MP, R);
    std::vector<int> ps;
    for (const auto& e : pl.entries)
      if (e.bucket == bk && !pl.probs[e.p].S) ps.push_back(e.p);
    if (ps.empty()) continue;
    // per-CTA tile count of 1/split_div of one wave's share (4 by default, a
    // quarter): big problems get many CTAs, small ones one CTA each, and CTAs
    // that finish early leave their SM to the rest
    const int64_t wave = (int64_t)std::max(1, sms) * std::max(1, group_ctas_per_sm(MP, R, xb != 0));
    int64_t tiles = 0;
    for (int p : ps) tiles += (pl.probs[p].n + T - 1) / T;
    // one problem alone: equal CTAs, one whole wave; several: a quarter wave's share each
    const int64_t per = ps.size() == 1 ? std::max<int64_t>(1, (tiles + wave - 1) / wave)
                                       : std::max<int64_t>(1, (tiles + split_div * wave - 1) / (split_div * wave));
    for (int p : ps) pl.probs[p].S = (int)(((pl.probs[p].n + T - 1) / T + per - 1) / per);
  }
  // CTA ranges of the entries inside their bucket launches
  for (int bk = 0; bk < (int)keys.size(); ++bk) {
    GroupPlan::Bucket B;
    B.mode = std::get<0>(keys[bk]);
    B.MP = std::get<1>(keys[bk]);
    B.R = std::get<2>(keys[bk]);
    B.xb = std::get<3>(keys[bk]);
    B.ncta = 0;
    B.cta_off = pl.total_cta;
    for (auto& e : pl.entries)
      if (e.bucket == bk) {
        e.cta0 = B.ncta;
        B.ncta += pl.probs[e.p].S;
      }
    pl.total_cta += B.ncta;
    pl.buckets.push_back(B);
  }
  for (auto& q : pl.probs) {
    q.nblk = (q.E + kEntries - 1) / kEntries;
    q.blk0 = pl.total_cblk;
    pl.total_cblk += q.nblk;
    if (q.tall) {
      q.tnblk = (int)((q.n + kTallCols - 1) / kTallCols);
      q.tblk0 = pl.total_tblk;
      pl.total_tblk += q.tnblk;
      ++pl.ntall;
    }
  }
  // tables: GProb per entry, GComb per problem, GTall per tall problem, block maps
  const int ne = (int)pl.entries.size();
  pl.o_prob = 0;
  pl.o_comb = pl.o_prob + align256((size_t)ne * sizeof(GProb));
  pl.o_tall = pl.o_comb + align256((size_t)np * sizeof(GComb));
  pl.o_cta = pl.o_tall + align256((size_t)std::max(1, pl.ntall) * sizeof(GTall));
  pl.o_cblk = pl.o_cta + align256((size_t)pl.total_cta * sizeof(int));
  pl.o_tblk = pl.o_cblk + align256((size_t)pl.total_cblk * sizeof(int));
  pl.table_bytes = pl.o_tblk + align256((size_t)std::max(1, pl.total_tblk) * sizeof(int));
  size_t off = base;
  pl.off_tables = off;
  off = align256(off + pl.table_bytes);
  pl.off_tickets = off;
  off = align256(off + (size_t)np * sizeof(unsigned));
  if (own_scratch)
    for (auto& q : pl.probs) {
      q.g_off = off;
      off = align256(off + (size_t)q.R * q.R * 4);
      q.red_off = off;
      off = align256(off + (size_t)q.E * 4);
      q.part_off = off;
      off = align256(off + (size_t)q.S * q.E * 4);
      q.y_off = off;
      off = align256(off + (size_t)(q.tall ? q.nb : 0) * q.re * q.n * 4);
    }
  pl.bytes = off;
  return NTT_OK;
}

void group_fill_tables(const GroupPlan& pl, const GroupPtrs* ptrs, char* scratch, void* host_tables) {
  const int np = (int)pl.probs.size();
  if (np == 0) return;
  char* h = reinterpret_cast<char*>(host_tables);
  GProb* hp = reinterpret_cast<GProb*>(h + pl.o_prob);
  GComb* hc = reinterpret_cast<GComb*>(h + pl.o_comb);
  GTall* ht = reinterpret_cast<GTall*>(h + pl.o_tall);
  int* hcta = reinterpret_cast<int*>(h + pl.o_cta);
  int* hcblk = reinterpret_cast<int*>(h + pl.o_cblk);
  int* htblk = reinterpret_cast<int*>(h + pl.o_tblk);
  unsigned* tickets = reinterpret_cast<unsigned*>(scratch + pl.off_tickets);
  // per-problem scratch pointers
  std::vector<float*> G(np), red(np), part(np), Y(np);
  for (int p = 0; p < np; ++p) {
    const auto& q = pl.probs[p];
    if (pl.own_scratch) {
      G[p] = reinterpret_cast<float*>(scratch + q.g_off);
      red[p] = reinterpret_cast<float*>(scratch + q.red_off);
      part[p] = reinterpret_cast<float*>(scratch + q.part_off);
      Y[p] = reinterpret_cast<float*>(scratch + q.y_off);
    } else {
      char* s0 = ptrs[p].scratch;
      G[p] = reinterpret_cast<float*>(s0);
      s0 += align256((size_t)q.R * q.R * 4);
      red[p] = reinterpret_cast<float*>(s0);
      s0 += align256((size_t)q.E * 4);
      part[p] = reinterpret_cast<float*>(s0);
      s0 += align256((size_t)q.S * q.E * 4);
      Y[p] = reinterpret_cast<float*>(s0);
    }
  }
  int ti = 0;
  for (int e = 0; e < (int)pl.entries.size(); ++e) {
    const auto& en = pl.entries[e];
    const auto& q = pl.probs[en.p];
    const GroupPtrs& g = ptrs[en.p];
    GProb& a = hp[e];
    std::memset(&a, 0, sizeof(a));
    const int r0 = en.b * q.mb;
    a.X = reinterpret_cast<const char*>(g.X) + (int64_t)r0 * q.n * (q.xbf16 ? 2 : 4);
    a.H = g.H;
    a.W = g.W + (int64_t)r0 * q.re;
    a.G = G[en.p];
    a.part = part[en.p];
    a.Y = Y[en.p] + (int64_t)en.b * q.re * q.n;
    a.n = q.n;
    a.m = q.tall ? std::min(q.mb, q.m - r0) : q.m;
    a.re = q.re;
    a.blk = q.blk;
    a.S = q.S;
    a.cta0 = en.cta0;
    a.aligned = (q.n % 4 == 0 && reinterpret_cast<uintptr_t>(g.X) % 16 == 0 &&
                 reinterpret_cast<uintptr_t>(g.H) % 16 == 0 && reinterpret_cast<uintptr_t>(a.Y) % 16 == 0)
                    ? 1
                    : 0;
    a.prow0 = r0;
    a.qrow0 = q.qrow0;
    a.E = q.E;
    a.hasq = (en.mode == 0 || (en.mode == 2 && en.b == 0)) ? 1 : 0;
    for (int s = 0; s < q.S; ++s) hcta[pl.buckets[en.bucket].cta_off + en.cta0 + s] = e;
  }
  for (int p = 0; p < np; ++p) {
    const auto& q = pl.probs[p];
    GComb& c = hc[p];
    std::memset(&c, 0, sizeof(c));
    c.part = part[p];
    c.red = red[p];
    c.W = ptrs[p].W;
    c.G = G[p];
    c.ticket = tickets + p;
    c.obj = ptrs[p].obj;
    c.xnorm2 = ptrs[p].xnorm2;
    c.S = q.S;
    c.MP = q.qrow0;
    c.R = q.R;
    c.m = q.m;
    c.re = q.re;
    c.blk = q.blk;
    c.blk0 = q.blk0;
    c.nblk = q.nblk;
    for (int b = 0; b < q.nblk; ++b) hcblk[q.blk0 + b] = p;
    if (q.tall) {
      GTall& t = ht[ti];
      t.Y = Y[p];
      t.H = ptrs[p].H;
      t.G = G[p];
      t.n = q.n;
      t.re = q.re;
      t.R = q.R;
      t.nb = q.nb;
      t.blk0 = q.tblk0;
      for (int b = 0; b < q.tnblk; ++b) htblk[q.tblk0 + b] = ti;
      ++ti;
    }
  }
}

ntt_status group_launch(const GroupPlan& pl, char* scratch, const char* d, int iters, float eps,
                        cudaStream_t st, int t0) {
  const int np = (int)pl.probs.size();
  if (np == 0) return NTT_OK;
  unsigned* tickets = reinterpret_cast<unsigned*>(scratch + pl.off_tickets);
  if (launch_zero(tickets, (size_t)np * sizeof(unsigned), st) != cudaSuccess) return NTT_ERR_CUDA;
  const GProb* dp = reinterpret_cast<const GProb*>(d + pl.o_prob);
  const GComb* dc = reinterpret_cast<const GComb*>(d + pl.o_comb);
  const GTall* dt = reinterpret_cast<const GTall*>(d + pl.o_tall);
  const int* dcta = reinterpret_cast<const int*>(d + pl.o_cta);
  const int* dcblk = reinterpret_cast<const int*>(d + pl.o_cblk);
  const int* dtblk = reinterpret_cast<const int*>(d + pl.o_tblk);
  group_gram_kernel<<<np, kAuxThreads, 0, st>>>(dc);
  if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  for (int t = 0; t < iters; ++t) {
    for (int mode = 0; mode <= 2; ++mode) {
      if (mode == 2 && pl.ntall) {
        tall_hupd_kernel<<<pl.total_tblk, kTallCols, 0, st>>>(dt, dtblk, eps);
        if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
      }
      for (const auto& B : pl.buckets)
        if (B.mode == mode && B.ncta > 0 &&
            launch_gpass(B.mode, B.MP, B.R, B.xb != 0, dp, dcta + B.cta_off, B.ncta, eps, st) != cudaSuccess)
          return NTT_ERR_CUDA;
    }
    group_combine_kernel<<<pl.total_cblk, kAuxThreads, 0, st>>>(dc, dcblk, eps, t0 + t);
    if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  }
  return NTT_OK;
}

ntt_status group_run(const GroupPlan& pl, const GroupPtrs* ptrs, char* scratch, void* host_tables,
                     int iters, float eps, cudaStream_t st, int t0) {
  if (pl.probs.empty()) return NTT_OK;
  group_fill_tables(pl, ptrs, scratch, host_tables);
  if (cudaMemcpyAsync(scratch + pl.off_tables, host_tables, pl.table_bytes, cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return NTT_ERR_CUDA;
  return group_launch(pl, scratch, scratch + pl.off_tables, iters, eps, st, t0);
}

}  // namespace ntt
