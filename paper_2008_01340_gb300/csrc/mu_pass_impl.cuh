// Streaming fused pass of one multiplicative-update iteration.
//
// One pass over the columns of X (m x n, row-major) computes, per tile of T
// columns held in shared memory:
//   Y     = W^T X_tile                                  (contraction over m)
//   H_new = max(0, H o Y / (G_W H + eps)),  G_W = W^T W (H update, in place in HBM)
//   P    += X_tile H_new^T,   Q += H_new H_new^T        (contractions over columns)
// The H update of a column only needs that column of X and H plus W and G_W,
// so the exact Lee-Seung order (H first, then W from the new H) needs a single
// read of X per iteration.  These are the paper's W^T X and X H^T products
// (Algorithms 5-6) and the Gram H H^T (Algorithm 4), with their collectives
// replaced by one deterministic cross-CTA reduction of the (P, Q) partials.
//
// Each CTA is persistent over tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// X and H tiles arrive by TMA (cp.async.bulk.tensor.2d) into a ring of
// STAGES buffers signalled by mbarriers, or by cooperative loads when the
// rows of X or H are not 16-byte aligned.  Every mbarrier wait is bounded.
//
// Thread roles (256 threads):
//   phase A  thread = (row split sa, 8-rank block kb, 4-column chunk cq):
//            partial Y over MP/SA rows, then a fixed-order sum over splits.
//   H upd.   thread = (column c, rank slice kg).
//   phase B  thread = (row group g of RB stacked rows, 8-rank block, column
//            group q): the stacked rows are [X_tile ; H_new ; 0] so P and Q
//            come out of one register-blocked outer-product loop.
//
// BCD mode (Algorithm 3, the prox-linear block step): the same pass with the
// H step of block coordinate descent in place of the multiplicative update,
//   H_m   = H + w_h (H - H_prev)                     (extrapolation)
//   H_new = max(0, H_m - (G_W H_m - W^T X) / L_h)    (projected gradient, L_h = ||G_W||_2)
// H and H_prev are the last two accepted iterates and H_new goes to the third
// buffer; the buffer roles rotate on the device (BcdState::rot), so a captured
// graph replays every iteration unchanged.  The init launch (bcd_init) only
// accumulates P = X H^T and Q = H H^T of the current H.
#pragma once

#include "ntt_internal.cuh"

namespace ntt {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
// Row groups of phase B: the fewest (power of two >= 8) that keep <= 5
// stacked rows per thread, capped so that groups x rank blocks <= threads.
__host__ __device__ constexpr int pick_nrg(int ms, int kbb, int nt) {
  int g = 8;
  while ((ms + g - 1) / g > 5 && g * 2 * kbb <= nt) g *= 2;
  return g;
}

template <int MP_, int R_, bool BF16_, bool BCD_ = false>
struct PassCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  static constexpr bool BF16 = BF16_;
  static constexpr bool BCD = BCD_;                // BCD step: a second H tile (H_prev) per stage
  static constexpr int XB = BF16 ? 2 : 4;          // bytes per X element
  static constexpr int NT = kPassThreads;
  static constexpr int T = cmax(16, cmin(cmin(256, 8192 / MP), 4096 / R));
  static constexpr int CH = T / 4;                 // 4-column chunks per tile
  static constexpr int KBA = R / 8;                // 8-rank blocks (phase A)
  static constexpr int SA = NT / (CH * KBA);       // row splits (phase A)
  static constexpr int RPS = MP / SA;              // rows per split
  static constexpr int MS = MP + R;                // stacked rows [X ; H_new]
  static constexpr int KBB = R / 8;                // 8-rank blocks (phase B)
  static constexpr int NRG = pick_nrg(MS, R / 8, NT);  // row groups (phase B)
  static constexpr int RB = (MS + NRG - 1) / NRG;  // rows per group
  static constexpr int MSP = NRG * RB;
  static constexpr int CG = NT / (NRG * KBB);      // column groups (phase B)
  static constexpr bool PAIRB = RB <= 5;           // packed column-pair accumulators
  static constexpr int CPT = T / CG;               // columns per thread per tile
  static constexpr int HKG = cmax(1, NT / T);      // threads per column (H update)
  static constexpr int KPT = cmax(1, R / HKG);     // ranks per thread (H update)
  static constexpr int BR = cmin(MP, 256);         // TMA box rows of X
  static constexpr int NXB = MP / BR;              // X boxes per tile
  static constexpr int XS_BYTES = MP * T * XB;
  static constexpr int HS_BYTES = R * T * 4;
  static constexpr int NHT = BCD ? 2 : 1;          // H tiles per stage
  static constexpr int STAGE_BYTES = (XS_BYTES + NHT * HS_BYTES + 1023) / 1024 * 1024;
  static constexpr int HN_ROWS = MSP - MP;
  static constexpr int HN_BYTES = HN_ROWS * T * 4;
  static constexpr int Y_BYTES = SA * R * T * 4;
  static constexpr int W_BYTES = MP * R * 4;
  static constexpr int G_BYTES = R * R * 4;
  static constexpr int BAR_BYTES = 64;
  static constexpr int HN_BUF = (HN_BYTES + 1023) / 1024 * 1024;   // one H_new buffer
  static constexpr int FIXED = 2 * HN_BUF + Y_BYTES + W_BYTES + G_BYTES + BAR_BYTES + 1024;
  static constexpr int SMEM_CAP = 227 * 1024 - 256;
  static constexpr int STAGES = cmin(4, (SMEM_CAP - FIXED) / STAGE_BYTES);
  static constexpr int SMEM = STAGES * STAGE_BYTES + FIXED;
  static constexpr int RED_BYTES = MSP * R * CG * 4;
  static constexpr uint32_t TX_BYTES = XS_BYTES + NHT * HS_BYTES;

  static_assert(R % 8 == 0 && R <= 32, "rank bucket");
  static_assert(CH * KBA * SA == NT && SA * RPS == MP, "phase A mapping");
  static_assert(NRG * KBB * CG == NT && CPT % 4 == 0 && CPT >= 4, "phase B mapping");
  static_assert(STAGES >= 2 && STAGES <= 4, "pipeline depth");
  static_assert(RED_BYTES <= STAGES * STAGE_BYTES + 2 * HN_BUF + Y_BYTES, "reduction scratch");
  static_assert(SMEM <= SMEM_CAP, "shared memory");
  static_assert(MP % BR == 0 && T <= 256 && R <= 256, "TMA box");
};

template <bool BF16>
struct XLoad;
template <>
struct XLoad<false> {
  using T = float;
  static __device__ __forceinline__ float4 ld4(const float* p) {
    return *reinterpret_cast<const float4*>(p);
  }
  static __device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }
};
template <>
struct XLoad<true> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    float4 f;
    f.x = __uint_as_float(u.x << 16);
    f.y = __uint_as_float(u.x & 0xFFFF0000u);
    f.z = __uint_as_float(u.y << 16);
    f.w = __uint_as_float(u.y & 0xFFFF0000u);
    return f;
  }
  static __device__ __forceinline__ float ldg(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
  }
};

struct PassParams {
  const void* X;       // m x n (FP32 or BF16), used by the cooperative loader
  float* H;            // r x n, updated in place
  const float* W;      // m x r
  const float* G;      // R x R
  float* part;         // grid x (MP+R) x R
  int* status;
  const int* stop;     // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r;
  int ntiles;
  int use_tma;
  float eps;
  // BCD mode
  float* Hb[3];              // the three H buffers (cooperative loader / stores)
  const BcdState* bcd;       // rotation, w_h, L_h
  int64_t ldh;               // row stride of H (n, or more for a column block of a wider H)
  int bcd_init;              // accumulate P, Q of the accepted H only
  double* res_part;          // BCD: per CTA, sum over its tiles of ||x_c - W h_new_c||^2
};


// tmH: the H tile loaded (updated in place in MU mode); tmHp: H_prev (BCD);
// tmHs: the target of the H_new store.  Hld / Hp / Hst: the same buffers for
// the cooperative path.  BCD step parameters come from the state.
template <class C>
__device__ __forceinline__ void mu_pass_body(const CUtensorMap& tmX, const CUtensorMap& tmH,
                                             const CUtensorMap& tmHp, const CUtensorMap& tmHs,
                                             const float* Hld, const float* Hp, float* Hst, float w_h,
                                             float Lh, const PassParams& p) {
  using XT = typename XLoad<C::BF16>::T;
  constexpr int T = C::T, R = C::R, MP = C::MP, NT = C::NT;
  constexpr int HNF = C::HN_BUF / 4;   // floats per H_new buffer

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  float* HnBuf = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES);  // 2 buffers
  float* Ysm = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES + 2 * C::HN_BUF);
  float* Ws = Ysm + C::SA * R * T;
  float* Gs = Ws + MP * R;
  uint64_t* bars = reinterpret_cast<uint64_t*>(Gs + R * R);
  __shared__ int s_err;

  const int tid = threadIdx.x;
  const int m = p.m, r = p.r;
  const int64_t n = p.n;
  const bool tma = p.use_tma != 0;

  if (tid == 0) {
    s_err = 0;
    if (tma) {
      prefetch_tensormap(&tmX);
      prefetch_tensormap(&tmH);
      if constexpr (C::BCD) prefetch_tensormap(&tmHp);
      for (int s = 0; s < C::STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
      fence_mbar_init();
    }
  }
  // W (zero padded to MP x R), G (R x R), zero padding rows of both H_new stacks
  {
    // W loads in batches of eight in flight
    constexpr int NWL = (MP * R + NT - 1) / NT, WB = NWL < 8 ? NWL : 8;
#pragma unroll 1
    for (int u0 = 0; u0 < NWL; u0 += WB) {
      float wv[WB];
#pragma unroll
      for (int u = 0; u < WB; ++u) {
        const int idx = tid + (u0 + u) * NT, i = idx / R, k = idx % R;
        wv[u] = (idx < MP * R && i < m && k < r) ? p.W[i * r + k] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < WB; ++u)
        if (tid + (u0 + u) * NT < MP * R) Ws[tid + (u0 + u) * NT] = wv[u];
    }
  }
  for (int idx = tid; idx < R * R; idx += NT) Gs[idx] = p.G[idx];
  for (int b = 0; b < 2; ++b)
    for (int idx = R * T + tid; idx < C::HN_ROWS * T; idx += NT) HnBuf[b * HNF + idx] = 0.0f;
  __syncthreads();

  auto issue = [&](int stage, int tile) {
    const uint32_t bar = smem_u32(&bars[stage]);
    const uint32_t dst = smem_u32(stage_base + stage * C::STAGE_BYTES);
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
#pragma unroll
    for (int b = 0; b < C::NXB; ++b)
      tma_load_2d(dst + b * C::BR * T * C::XB, &tmX, tile * T, b * C::BR, bar);
    tma_load_2d(dst + C::XS_BYTES, &tmH, tile * T, 0, bar);
    if constexpr (C::BCD) tma_load_2d(dst + C::XS_BYTES + C::HS_BYTES, &tmHp, tile * T, 0, bar);
  };

  int issued = 0;  // tiles issued by thread 0 (TMA mode)
  if (tma && tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile < p.ntiles) {
        issue(s, tile);
        ++issued;
      }
    }
  }

  // phase B accumulators (persistent over tiles): stacked rows gB*RB.., ranks kbB*8..
  const int qB = tid % C::CG;
  const int kbB = (tid / C::CG) % C::KBB;
  const int gB = tid / (C::CG * C::KBB);
  constexpr int NACC = C::PAIRB ? 2 : 1;
  float accB[C::RB][8][NACC];
#pragma unroll
  for (int i = 0; i < C::RB; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int e = 0; e < NACC; ++e) accB[i][k][e] = 0.0f;

  double res_acc = 0.0;   // BCD: this thread's share of the direct residual
  int consumed = 0;
  int cur = 0;  // H_new buffer of this tile
  for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++consumed, cur ^= 1) {
    const int stage = consumed % C::STAGES;
    const XT* Xs = reinterpret_cast<const XT*>(stage_base + stage * C::STAGE_BYTES);
    const float* Hs = reinterpret_cast<const float*>(stage_base + stage * C::STAGE_BYTES +
                                                     C::XS_BYTES);
    float* Hn = HnBuf + cur * HNF;
    const int64_t col0 = (int64_t)tile * T;

    if (tma) {
      if (!mbar_wait_bounded(smem_u32(&bars[stage]), (consumed / C::STAGES) & 1)) s_err = 1;
    } else {
      XT* Xw = const_cast<XT*>(Xs);
      float* Hw = const_cast<float*>(Hs);
      const XT* Xg = reinterpret_cast<const XT*>(p.X);
      for (int idx = tid; idx < MP * T; idx += NT) {
        const int i = idx / T, c = idx % T;
        const int64_t col = col0 + c;
        Xw[idx] = (i < m && col < n) ? Xg[(int64_t)i * n + col] : XT(0.0f);
      }
      for (int idx = tid; idx < R * T; idx += NT) {
        const int k = idx / T, c = idx % T;
        const int64_t col = col0 + c;
        Hw[idx] = (k < r && col < n) ? Hld[(int64_t)k * p.ldh + col] : 0.0f;
        if constexpr (C::BCD) Hw[R * T + idx] = (k < r && col < n) ? Hp[(int64_t)k * p.ldh + col] : 0.0f;
      }
      __syncthreads();
    }

    // ---------------- phase A: partial Y = W^T X over this thread's rows (packed FMA)
    {
      const int cq = tid % C::CH;
      const int kb = (tid / C::CH) % C::KBA;
      const int sa = tid / (C::CH * C::KBA);
      float2 acc[8][2];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k][0] = acc[k][1] = make_float2(0.0f, 0.0f);
      const XT* xp = Xs + (sa * C::RPS) * T + 4 * cq;
      const float* wp = Ws + (sa * C::RPS) * R + kb * 8;
#pragma unroll 4
      for (int ii = 0; ii < C::RPS; ++ii) {
        const float4 x = XLoad<C::BF16>::ld4(xp + ii * T);
        const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
        const float4 w0 = *reinterpret_cast<const float4*>(wp + ii * R);
        const float4 w1 = *reinterpret_cast<const float4*>(wp + ii * R + 4);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float2 wk = make_float2(w[k], w[k]);
          acc[k][0] = __ffma2_rn(wk, x01, acc[k][0]);
          acc[k][1] = __ffma2_rn(wk, x23, acc[k][1]);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *reinterpret_cast<float4*>(Ysm + (sa * R + kb * 8 + k) * T + 4 * cq) =
            make_float4(acc[k][0].x, acc[k][0].y, acc[k][1].x, acc[k][1].y);
    }
    if (tma && tid == 0) bulk_wait_read<1>();  // the store of two tiles ago has read Hn[cur]
    __syncthreads();
    if (s_err) break;

    // ---------------- H update for column c, ranks kg*KPT ..
    if constexpr (C::BCD) {
      // H_m = H + w_h (H - H_prev); H_new = max(0, H_m - (G H_m - Y) / L_h)
      const int c = tid % T;
      const int kg = tid / T;
      if (kg * C::KPT < R) {
        float hm[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          // no extrapolation (first step, after a rejection): H_prev is not read,
          // so a buffer that holds no iterate yet cannot leak into H_m
          const float a = Hs[j * T + c], b = Hs[R * T + j * T + c];
          hm[j] = w_h != 0.0f ? fmaf(w_h, a - b, a) : a;
        }
        const int64_t col = col0 + c;
#pragma unroll
        for (int kk = 0; kk < C::KPT; ++kk) {
          const int k = kg * C::KPT + kk;
          float hn;
          if (p.bcd_init) {
            hn = Hs[k * T + c];
          } else {
            float y = 0.0f;
#pragma unroll
            for (int s2 = 0; s2 < C::SA; ++s2) y += Ysm[(s2 * R + k) * T + c];
            float gh = 0.0f;
#pragma unroll
            for (int j = 0; j < R; j += 4) {
              const float4 g = *reinterpret_cast<const float4*>(Gs + k * R + j);
              gh = fmaf(g.x, hm[j], gh);
              gh = fmaf(g.y, hm[j + 1], gh);
              gh = fmaf(g.z, hm[j + 2], gh);
              gh = fmaf(g.w, hm[j + 3], gh);
            }
            float hk = 0.0f;
#pragma unroll
            for (int j = 0; j < R; ++j)
              if (j == k) hk = hm[j];
            hn = Lh > 0.0f ? fmaxf(0.0f, hk - __fdiv_rn(gh - y, Lh)) : hk;
          }
          Hn[k * T + c] = hn;
          if (!tma && !p.bcd_init && k < r && col < n) Hst[(int64_t)k * p.ldh + col] = hn;
        }
      }
    } else {
      const int c = tid % T;
      const int kg = tid / T;
      if (kg * C::KPT < R) {
        float h[R];
#pragma unroll
        for (int j = 0; j < R; ++j) h[j] = Hs[j * T + c];
        const int64_t col = col0 + c;
        if constexpr (C::HKG == 1) {
          // one thread per column, all ranks: packed G H with G symmetric (row j = column j)
          float2 gh[R / 2];
#pragma unroll
          for (int q = 0; q < R / 2; ++q) gh[q] = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const float2 hj = make_float2(h[j], h[j]);
#pragma unroll
            for (int q = 0; q < R / 4; ++q) {
              const float4 g4 = *reinterpret_cast<const float4*>(Gs + j * R + 4 * q);
              gh[2 * q] = __ffma2_rn(make_float2(g4.x, g4.y), hj, gh[2 * q]);
              gh[2 * q + 1] = __ffma2_rn(make_float2(g4.z, g4.w), hj, gh[2 * q + 1]);
            }
          }
#pragma unroll
          for (int k = 0; k < R; ++k) {
            float y = 0.0f;
#pragma unroll
            for (int s = 0; s < C::SA; ++s) y += Ysm[(s * R + k) * T + c];
            const float den = ((k & 1) ? gh[k / 2].y : gh[k / 2].x) + p.eps;
            const float hn = fmaxf(0.0f, __fdividef(h[k] * y, den));
            Hn[k * T + c] = hn;
            if (!tma && k < r && col < n) Hst[(int64_t)k * p.ldh + col] = hn;
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < C::KPT; ++kk) {
            const int k = kg * C::KPT + kk;
            float y = 0.0f;
#pragma unroll
            for (int s = 0; s < C::SA; ++s) y += Ysm[(s * R + k) * T + c];
            float gh = 0.0f;
#pragma unroll
            for (int j = 0; j < R; j += 4) {
              const float4 g = *reinterpret_cast<const float4*>(Gs + k * R + j);
              gh = fmaf(g.x, h[j], gh);
              gh = fmaf(g.y, h[j + 1], gh);
              gh = fmaf(g.z, h[j + 2], gh);
              gh = fmaf(g.w, h[j + 3], gh);
            }
            float hk = 0.0f;
#pragma unroll
            for (int j = 0; j < R; ++j)
              if (j == k) hk = h[j];
            const float hn = fmaxf(0.0f, __fdividef(hk * y, gh + p.eps));
            Hn[k * T + c] = hn;
            if (!tma && k < r && col < n) Hst[(int64_t)k * p.ldh + col] = hn;
          }
        }
      }
    }
    if (tma) fence_proxy_async_smem();   // H_new visible to the TMA store
    __syncthreads();
    if (tma && tid == 0 && !(C::BCD && p.bcd_init)) {
      tma_store_2d(&tmHs, smem_u32(Hn), (int)col0, 0);
      bulk_commit();
    }
    if constexpr (C::BCD) {
      // direct squared residual of (W, H_new) on this tile: the objective the
      // step's acceptance test needs, without the cancellation of the Gram form
      if (!p.bcd_init) {
        float acc = 0.0f;
        for (int idx = tid; idx < MP * T; idx += NT) {
          const int i = idx / T, c = idx % T;
          float v;
          if constexpr (C::BF16)
            v = __bfloat162float(Xs[i * T + c]);
          else
            v = Xs[i * T + c];
#pragma unroll
          for (int k = 0; k < R; ++k) v = fmaf(-Ws[i * R + k], Hn[k * T + c], v);
          acc = fmaf(v, v, acc);
        }
        res_acc += (double)acc;
      }
    }

    // ---------------- phase B: [P ; Q] += [X_tile ; H_new] H_new^T
    {
#pragma unroll
      for (int cc = 0; cc < C::CPT / 4; ++cc) {
        const int c = 4 * qB + cc * 4 * C::CG;
        float4 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          h[k] = *reinterpret_cast<const float4*>(Hn + (kbB * 8 + k) * T + c);
#pragma unroll
        for (int i = 0; i < C::RB; ++i) {
          const int row = gB * C::RB + i;
          float4 x;
          if (row < MP)
            x = XLoad<C::BF16>::ld4(Xs + row * T + c);
          else
            x = *reinterpret_cast<const float4*>(Hn + (row - MP) * T + c);
          if constexpr (C::PAIRB) {
            const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              float2 a = make_float2(accB[i][k][0], accB[i][k][NACC - 1]);
              a = __ffma2_rn(x01, make_float2(h[k].x, h[k].y), a);
              a = __ffma2_rn(x23, make_float2(h[k].z, h[k].w), a);
              accB[i][k][0] = a.x;
              accB[i][k][NACC - 1] = a.y;
            }
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              float a = accB[i][k][0];
              a = fmaf(x.x, h[k].x, a);
              a = fmaf(x.y, h[k].y, a);
              a = fmaf(x.z, h[k].z, a);
              a = fmaf(x.w, h[k].w, a);
              accB[i][k][0] = a;
            }
          }
        }
      }
    }
    __syncthreads();

    if (tma && tid == 0) {
      const int next = tile + C::STAGES * gridDim.x;
      if (next < p.ntiles) {
        fence_proxy_async_smem();
        issue(stage, next);
        ++issued;
      }
    }
  }

  if (s_err) {
    // Drain copies still in flight (bounded) before the CTA exits.
    if (tma && tid == 0) {
      for (int c = consumed; c < issued; ++c)
        (void)mbar_wait_bounded(smem_u32(&bars[c % C::STAGES]), (c / C::STAGES) & 1);
      bulk_wait<0>();
      atomicExch(p.status, kStatusTimeout);
    }
    return;
  }
  if (tma && tid == 0) bulk_wait<0>();   // H stores complete before smem is reused
  __syncthreads();
  if constexpr (C::BCD) {
    if (!p.bcd_init) {
      // CTA sum of the residual shares: warp butterflies, then warps in order
      __shared__ double s_res[NT / 32];
      double v = res_acc;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) s_res[tid / 32] = v;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += s_res[w];
        p.res_part[blockIdx.x] = t;
      }
    }
  }

  // ---------------- CTA reduction of phase-B accumulators over column groups
  float* red = reinterpret_cast<float*>(smem);
#pragma unroll
  for (int i = 0; i < C::RB; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k)
      red[((gB * C::RB + i) * R + kbB * 8 + k) * C::CG + qB] =
          C::PAIRB ? accB[i][k][0] + accB[i][k][NACC - 1] : accB[i][k][0];
  __syncthreads();
  float* out = p.part + (size_t)blockIdx.x * (C::MS * R);
  for (int e = tid; e < C::MS * R; e += NT) {
    float s = 0.0f;
#pragma unroll 8
    for (int q = 0; q < C::CG; ++q) s += red[e * C::CG + q];
    out[e] = s;
  }
}

template <class C>
__global__ void __launch_bounds__(kPassThreads, 1)
mu_pass_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
               const PassParams p) {
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  mu_pass_body<C>(tmX, tmH, tmH, tmH, p.H, p.H, p.H, 0.0f, 0.0f, p);
}

// BCD step: the buffer roles come from the state the previous combine wrote.
template <class C>
__global__ void __launch_bounds__(kPassThreads, 1)
mu_pass_bcd_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ HMaps3 hm,
                   const PassParams p) {
  const int rot = __ldcg(&p.bcd->rot);
  const int ia = rot, ip = (rot + 2) % 3, in = (rot + 1) % 3;
  const float w_h = p.bcd_init ? 0.0f : __ldcg(&p.bcd->w_h);
  const float Lh = __ldcg(&p.bcd->Lh);
  mu_pass_body<C>(tmX, hm.h[ia], hm.h[ip], hm.h[in], p.Hb[ia], p.Hb[ip], p.Hb[in], w_h, Lh, p);
}

// One BCD pass launch of bucket C.  Hb: the three H buffers (device), maps of
// the same (TMA mode); init: P, Q of the accepted H only.
template <class C>
cudaError_t launch_pass_bcd_cfg(const MuShape& s, const MuDev& d, const CUtensorMap& mx, const HMaps3& mh,
                                float* const* Hb, const BcdState* st_dev, int init, double* res_part,
                                cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_pass_bcd_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  PassParams p;
  p.X = d.X;
  p.H = Hb[0];
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = nullptr;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.ntiles = (int)((s.n + C::T - 1) / C::T);
  p.use_tma = s.tma;
  p.eps = 0.0f;
  p.ldh = s.ldh > 0 ? s.ldh : s.n;
  for (int i = 0; i < 3; ++i) p.Hb[i] = Hb[i];
  p.bcd = st_dev;
  p.bcd_init = init;
  p.res_part = res_part;
  mu_pass_bcd_kernel<C><<<s.grid, kPassThreads, C::SMEM, st>>>(mx, mh, p);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_pass_cfg(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                            const CUtensorMap& mh, cudaStream_t st) {
  static bool attr_set = false;  // per-device attribute; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_pass_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  PassParams p;
  p.X = d.X;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.ntiles = (int)((s.n + C::T - 1) / C::T);
  p.use_tma = s.tma;
  p.eps = eps;
  p.ldh = s.ldh > 0 ? s.ldh : s.n;
  p.Hb[0] = p.Hb[1] = p.Hb[2] = d.H;
  p.bcd = nullptr;
  p.bcd_init = 0;
  p.res_part = nullptr;
  return launch_pdl(mu_pass_kernel<C>, dim3(s.grid), dim3(kPassThreads), C::SMEM, st, mx, mh, p);
}

// Tile width and smem of a (MP, R, BF16) bucket, for host shape decisions.
template <class C>
void pass_cfg_info(int* T, size_t* smem) {
  *T = C::T;
  *smem = C::SMEM;
}

}  // namespace ntt
