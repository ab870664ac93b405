// Fused MU pass on the 5th-generation tensor cores (tcgen05, TMEM accumulators)
// for short unfoldings (m <= 64 rows, rank r <= 16).
//
// Per tile of T = 128 columns of X (m x n, row-major FP32), exactly as the FMA
// pass computes it (H first from W, then the W-side contractions from the new H):
//   Y^T    = X_tile^T W                 phase A: D_A (TMEM, 128 lanes x 16)
//   H_new  = max(0, H o Y / (G_W H + eps))   epilogue, one column per lane
//   [P;Q] += [X_tile ; H_new] H_new^T    phase B: D_B (TMEM), accumulated
// FP32 accuracy from TF32 inputs with the split a = hi + lo (hi = a with the
// low 13 mantissa bits cleared, lo = a - hi exact): a b ~ hi_a hi_b + hi_a lo_b
// + lo_a hi_b, three MMAs per K step; D_B is drained into FP32 registers every
// kFlush tiles so the tensor-core accumulation runs stay short.
//
// Shared-memory layout of a pipeline stage: the X tile arrives by TMA with the
// 128-byte swizzle of 32-byte chunks (the 4-row atom TF32 operands read
// MN-major require) as 4 chunks of 32 columns; chunk c holds rows 0..m-1 of
// those columns followed by R rows of H_new (written by the epilogue with the
// same swizzle), so one chunk buffer is at the same time
//   * the MN-major A operand of phase A (M = columns, K = rows), and
//   * the K-major A operand of phase B (M = stacked rows, K = columns), and
//   * (rows m..m+15) the K-major B operand of phase B (N = ranks).
// A second copy of the chunks holds the lo parts.  Rows of the 128-row M
// extent of phase B past the stack read neighbouring shared memory and only
// feed D_B rows that are never read; columns of N = 16 past r likewise.
#include "ntt_internal.cuh"

namespace ntt {

namespace {

constexpr int kTcThreads = 256;
constexpr int kFlush = 32;

template <int MP_, int R_>
struct TcCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  static constexpr int N2 = 2 * R;                 // MMA N: [hi | lo] columns
  static constexpr int T = 128;                    // columns per tile = M of phase A
  static constexpr int NCH = T / 32;               // 32-column swizzle chunks
  // chunk rows: X_hi [0,MP) | Hn_hi [MP,MP+R) | Hn_lo [MP+R,MP+2R) | X_lo [MP+2R, 2MP+2R)
  static constexpr int ROW_HNH = MP, ROW_HNL = MP + R, ROW_XLO = MP + 2 * R;
  static constexpr int CR = 2 * MP + 2 * R;
  static constexpr int CHUNK = CR * 128;           // bytes per chunk (multiple of 1024)
  static constexpr int XREG = NCH * CHUNK;
  static constexpr int HT = R * T * 4;             // plain tile of the old H
  static constexpr int STAGE = (XREG + HT + 1023) / 1024 * 1024;
  static constexpr int KA = (MP + 31) / 32;        // 128-byte K atoms of the W operands
  static constexpr int WATOM = N2 * 128;           // one K atom of a W operand
  static constexpr int WOP = KA * WATOM;
  static constexpr int HNP = HT;                   // plain H_new buffer (TMA store source)
  static constexpr int KSTEP_A = MP / 8;
  static constexpr int KSTEP_B = T / 8;
  static constexpr int CAP = 227 * 1024 - 1024;
  static constexpr int fixed_bytes() { return 2 * WOP + 2 * HNP + R * R * 4 + 256 + 2 * T * N2 * 4; }
  static constexpr int stages() {
    int s = 4;
    while (s > 3 && s * STAGE + fixed_bytes() + 16384 > CAP) --s;
    return s;
  }
  static constexpr int STAGES = stages();
  static constexpr int OFF_W = STAGES * STAGE;
  static constexpr int OFF_HN = OFF_W + 2 * WOP;
  static constexpr int OFF_G = OFF_HN + 2 * HNP;
  static constexpr int OFF_BAR = OFF_G + R * R * 4;
  static constexpr int OFF_RED = OFF_BAR + 256;    // final D_B row exchange, 128 x N2 floats
  static_assert((5 * 4 + 8) * 8 + 4 <= 256, "barrier area");
  static constexpr int USED = OFF_RED + 128 * N2 * 4;
  // farthest byte any phase-B A descriptor reads: 128 rows from the last chunk
  static constexpr int REACH = (STAGES - 1) * STAGE + (NCH - 1) * CHUNK + 96 + 128 * 128;
  static constexpr int SMEM = (USED > REACH ? USED : REACH) + 1024;
  static constexpr uint32_t TX = NCH * MP * 128 + HT;
  static constexpr int TMEM_COLS = 12 * N2 <= 256 ? 256 : 512;   // D_A 2x2 + D_B 2x4 blocks of N2
  static constexpr uint32_t IDESC_A = idesc_tf32(128, N2, true, false);
  static constexpr uint32_t IDESC_B = idesc_tf32(128, N2, false, false);
  static_assert(CR % 8 == 0 && CR <= 128, "stacked hi/lo rows fit one 128-row MMA");
  static_assert(R == 8 || R == 16, "rank bucket");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(STAGES >= 3, "pipeline depth (phase B lags one tile)");
};

// byte offset of element (row, col) inside a 32-column chunk with the 128-byte
// swizzle of 16-byte chunks (8-row period): used for the W^T operands
__device__ __forceinline__ uint32_t sw128_off(int row, int col) {
  return (uint32_t)(row * 128 + ((((col >> 2) ^ row) & 7) << 4) + ((col & 3) << 2));
}

// same with the 128-byte swizzle of 32-byte chunks (4-row period): X tiles
// and the H_new rows stacked under them
__device__ __forceinline__ uint32_t sw128a32_off(int row, int col) {
  return (uint32_t)(row * 128 + ((((col >> 3) ^ row) & 3) << 5) + ((col & 7) << 2));
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

struct TcParams {
  float* H;
  const float* W;
  const float* G;
  float* part;
  int* status;
  const int* stop;     // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r;
  int ntiles;
  float eps;
};

// Warp roles: warps 0-7 (256 workers) split X into hi/lo and run the
// epilogue (one column per two threads); warp 8 lane 0 (control) issues the
// TMA loads and stores and every MMA.  Hand-offs use mbarriers only:
//   full[s]   TMA -> workers       split[s]  workers -> control (256 arrivals)
//   barA[b]   phase A -> workers   afree[b]  workers -> control (D_A[b] read)
//   epi[s]    workers -> control   barB[s]   phase B done (stage s reusable)
//   hnfree[b] control -> workers (H_new store buffer b read by the TMA)
//   dbfree[b] workers -> control (D_B[b] drained, 128 arrivals)
// Phase B of tile j is issued after phase A of tile j+1 so that the tensor
// pipe runs it while the workers do the epilogue of tile j+1.  D_B alternates
// between two TMEM buffers every kFlush tiles; the workers drain the idle one
// into FP32 registers, which keeps every tensor-core accumulation run short.
template <class C>
__global__ void __launch_bounds__(kTcThreads + 32, 1)
mu_pass_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                  const TcParams p) {
  constexpr int MP = C::MP, R = C::R, T = C::T, N2 = C::N2, S = C::STAGES;
  constexpr int KH = R / 2;          // ranks per worker thread (two threads per column)
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  constexpr int NW = kTcThreads;     // worker threads
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  float* Gs = reinterpret_cast<float*>(smem + C::OFF_G);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5 * S + 8);
  __shared__ int s_err;

  const int tid = threadIdx.x;
  const int warp = tid / 32;
  const int m = p.m, r = p.r;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  auto full = [&](int s) { return bar(s); };
  auto split = [&](int s) { return bar(S + s); };
  auto epi = [&](int s) { return bar(2 * S + s); };
  auto barB = [&](int s) { return bar(3 * S + s); };
  auto barA = [&](int b) { return bar(4 * S + b); };
  auto afree = [&](int b) { return bar(4 * S + 2 + b); };
  auto hnfree = [&](int b) { return bar(4 * S + 4 + b); };
  auto dbfree = [&](int b) { return bar(4 * S + 6 + b); };

  if (tid == 0) {
    s_err = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(split(s), NW);
      mbar_init(epi(s), NW);
      mbar_init(barB(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(barA(b), 1);
      mbar_init(afree(b), NW);
      mbar_init(hnfree(b), 1);
      mbar_init(dbfree(b), 128);
    }
    fence_mbar_init();
  }
  if (warp == 8) {
    tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
    tmem_relinquish();
  }
  // K-major B operands of phase A: W1 = [W_hi ; W_lo] (multiplies X_hi),
  // W2 = [W_hi ; 0] (multiplies X_lo); N2 rows, K = rows of W
  {
    uint8_t* w1 = smem + C::OFF_W;
    uint8_t* w2 = w1 + C::WOP;
    for (int idx = tid; idx < N2 * C::KA * 32; idx += NW + 32) {
      const int n2 = idx / (C::KA * 32);
      const int i = idx % (C::KA * 32);
      const int k = n2 % R;
      const float w = (k < r && i < m) ? p.W[i * r + k] : 0.0f;
      const float hi = tf32_hi(w);
      const uint32_t off = (uint32_t)((i >> 5) * C::WATOM) + sw128_off(n2, i & 31);
      *reinterpret_cast<float*>(w1 + off) = (n2 < R) ? hi : (w - hi);
      *reinterpret_cast<float*>(w2 + off) = (n2 < R) ? hi : 0.0f;
    }
    for (int idx = tid; idx < R * R; idx += NW + 32) Gs[idx] = p.G[idx];
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: D_A[b][chain] (phase A, double-buffered, hi / lo chains) and
  // D_B[pingpong][acc] (phase B, 4 independent accumulators per buffer).
  auto dA = [&](int b, int c) { return tmem + (uint32_t)((2 * b + c) * N2); };
  auto dB = [&](int b, int a) { return tmem + (uint32_t)((4 + 4 * b + a) * N2); };
  auto stage_x = [&](int s) { return sbase + (uint32_t)(s * C::STAGE); };
  // number of tiles of this CTA
  const int count = (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  if (warp == 8) {
    // =================================================================== control
    if ((tid & 31) == 0) {
      int issued = 0, last_a = -1, last_b = -1;
      auto issue = [&](int s, int j) {
        const int tile = (int)blockIdx.x + j * (int)gridDim.x;
        mbar_arrive_expect_tx(full(s), C::TX);
#pragma unroll
        for (int c = 0; c < C::NCH; ++c)
          tma_load_2d(stage_x(s) + c * C::CHUNK, &tmX, tile * T + 32 * c, 0, full(s));
        tma_load_2d(stage_x(s) + C::XREG, &tmH, tile * T, 0, full(s));
      };
      auto wait = [&](uint32_t b, uint32_t ph) {
        if (!mbar_wait_bounded(b, ph)) s_err = 1;
        return s_err == 0;
      };
      for (int j = 0; j < S && j < count; ++j) {
        issue(j, j);
        ++issued;
      }
      // Base descriptors, built once: each MMA adds a compile-time byte offset >> 4
      // to the start-address field (no carry out of its 14 bits: smem < 256 KB).
      const uint64_t dXa = smem_desc(sbase, C::CHUNK, 512, kLayoutSw128Atom32);   // phase A, MN-major
      const uint64_t dXb = smem_desc(sbase, 512, 512, kLayoutSw128Atom32);        // phase B A operand
      const uint64_t dHb = dXb + (uint64_t)((C::ROW_HNH * 128) >> 4);             // phase B B operand
      const uint64_t dW1 = smem_desc(sbase + C::OFF_W, 1024, 1024, kLayoutSw128);
      const uint64_t dW2 = dW1 + (uint64_t)(C::WOP >> 4);
      // phase B of local tile t, the H_new store of t and the refill of t-1's stage
      auto phase_b = [&](int t) -> bool {
        const int st = t % S;
        if (!wait(epi(st), (uint32_t)((t / S) & 1))) return false;
        tc_fence_after();
        const int tile = (int)blockIdx.x + t * (int)gridDim.x;
        tma_store_2d(&tmH, sbase + C::OFF_HN + (t & 1) * C::HNP, tile * T, 0);
        bulk_commit();
        const int g = t / kFlush, db = g & 1;
        const bool fresh = (t % kFlush) == 0;
        if (fresh && g >= 2 && !wait(dbfree(db), (uint32_t)(((g >> 1) - 1) & 1))) return false;
        const uint64_t sof = (uint64_t)((st * C::STAGE) >> 4);
#pragma unroll
        for (int kk = 0; kk < C::KSTEP_B; ++kk) {
          const uint64_t off = sof + (uint64_t)((((kk >> 2) * C::CHUNK + (kk & 3) * 32)) >> 4);
          mma_tf32(dB(db, kk & 3), dXb + off, dHb + off, C::IDESC_B,
                   (fresh && kk < 4) ? 0u : 1u);
        }
        mma_commit(barB(st));
        last_b = t;
        bulk_wait_read<1>();
        if (t >= 1) mbar_arrive(hnfree((t - 1) & 1));
        if (t >= 1) {
          const int next = t - 1 + S;
          if (next < count) {
            if (!wait(barB((t - 1) % S), (uint32_t)(((t - 1) / S) & 1))) return false;
            issue((t - 1) % S, next);
            ++issued;
          }
        }
        return true;
      };
      bool ok = true;
      for (int j = 0; j < count && ok; ++j) {
        const int s = j % S, b = j & 1;
        if (!wait(split(s), (uint32_t)((j / S) & 1))) break;
        if (j >= 2 && !wait(afree(b), (uint32_t)(((j >> 1) - 1) & 1))) break;
        tc_fence_after();
        const uint64_t sof = (uint64_t)((s * C::STAGE) >> 4);
#pragma unroll
        for (int kk = 0; kk < C::KSTEP_A; ++kk) {
          const uint64_t xo = sof + (uint64_t)((kk * 1024) >> 4);
          const uint64_t wo = (uint64_t)((((kk >> 2) * C::WATOM + (kk & 3) * 32)) >> 4);
          mma_tf32(dA(b, 0), dXa + xo, dW1 + wo, C::IDESC_A, kk > 0 ? 1u : 0u);
          mma_tf32(dA(b, 1), dXa + xo + (uint64_t)((C::ROW_XLO * 128) >> 4), dW2 + wo,
                   C::IDESC_A, kk > 0 ? 1u : 0u);
        }
        mma_commit(barA(b));
        last_a = j;
        if (j >= 1) ok = phase_b(j - 1);
      }
      if (ok && s_err == 0 && count > 0) phase_b(count - 1);
      bulk_wait<0>();
      if (count >= 1) mbar_arrive(hnfree((count - 1) & 1));
      if (s_err) {
        // drain every asynchronous operation still in flight (bounded)
        for (int c = 0; c < issued; ++c)
          (void)mbar_wait_bounded(full(c % S), (uint32_t)((c / S) & 1));
        if (last_a >= 0) (void)mbar_wait_bounded(barA(last_a & 1), (uint32_t)((last_a >> 1) & 1));
        if (last_b >= 0)
          (void)mbar_wait_bounded(barB(last_b % S), (uint32_t)((last_b / S) & 1));
        atomicExch(p.status, kStatusTimeout);
      }
    }
    __syncwarp();
  } else {
    // =================================================================== workers
    float accB[N2];
#pragma unroll
    for (int k = 0; k < N2; ++k) accB[k] = 0.0f;
    const int col = tid % T;
    const int kh0 = (tid / T) * KH;
    const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;
    auto drain = [&](int t) {   // threads < 128: add D_B of the group ending at tile t
      if (!mbar_wait_bounded(barB(t % S), (uint32_t)((t / S) & 1))) s_err = 1;
      tc_fence_after();
      const int db = (t / kFlush) & 1;
      float v[16];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int h = 0; h < N2 / 16; ++h) {
          tmem_ld16(dB(db, a) + lane_base + 16 * h, v);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) accB[16 * h + k] += v[k];
        }
      tc_fence_before();
    };
    for (int j = 0; j < count; ++j) {
      if (s_err) break;
      const int s = j % S, b = j & 1;
      if (!mbar_wait_bounded(full(s), (uint32_t)((j / S) & 1))) {
        s_err = 1;
        break;
      }
      // ---- split X into hi (in place) and lo (rows ROW_XLO..), rows 0..MP-1 of every chunk
      {
        uint8_t* xs = smem + s * C::STAGE;
        constexpr int V = C::NCH * MP * 8;
        for (int v = tid; v < V; v += NW) {
          const int c = v / (MP * 8), w = v % (MP * 8);
          const uint32_t off = (uint32_t)(c * C::CHUNK + w * 16);
          float4 x = *reinterpret_cast<float4*>(xs + off);
          float4 hi = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
          *reinterpret_cast<float4*>(xs + off) = hi;
          *reinterpret_cast<float4*>(xs + off + C::ROW_XLO * 128) =
              make_float4(x.x - hi.x, x.y - hi.y, x.z - hi.z, x.w - hi.w);
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(split(s));
      // ---- drain the D_B buffer of the group that ended with tile j-1
      if (j >= kFlush && j % kFlush == 0 && tid < 128) {
        drain(j - 1);
        mbar_arrive(dbfree(((j - 1) / kFlush) & 1));
      }
      // ---- epilogue
      if (!mbar_wait_bounded(barA(b), (uint32_t)((j >> 1) & 1))) {
        s_err = 1;
        break;
      }
      tc_fence_after();
      float ya[KH], yb[KH], yc[KH], yd[KH];
      if constexpr (KH == 4) {
        tmem_ld4(dA(b, 0) + lane_base + kh0, ya);
        tmem_ld4(dA(b, 0) + lane_base + R + kh0, yb);
        tmem_ld4(dA(b, 1) + lane_base + kh0, yc);
        tmem_ld4(dA(b, 1) + lane_base + R + kh0, yd);
      } else {
        tmem_ld8(dA(b, 0) + lane_base + kh0, ya);
        tmem_ld8(dA(b, 0) + lane_base + R + kh0, yb);
        tmem_ld8(dA(b, 1) + lane_base + kh0, yc);
        tmem_ld8(dA(b, 1) + lane_base + R + kh0, yd);
      }
      tmem_wait_ld();
      tc_fence_before();
      mbar_arrive(afree(b));
      const float* Hs = reinterpret_cast<const float*>(smem + s * C::STAGE + C::XREG);
      float h[R];
#pragma unroll
      for (int q = 0; q < R; ++q) h[q] = Hs[q * T + col];
      float hn[KH];
#pragma unroll
      for (int kk = 0; kk < KH; ++kk) {
        const int k = kh0 + kk;
        float gh = 0.0f;
#pragma unroll
        for (int q = 0; q < R; q += 4) {
          const float4 g = *reinterpret_cast<const float4*>(Gs + k * R + q);
          gh = fmaf(g.x, h[q], gh);
          gh = fmaf(g.y, h[q + 1], gh);
          gh = fmaf(g.z, h[q + 2], gh);
          gh = fmaf(g.w, h[q + 3], gh);
        }
        float hk = 0.0f;
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (q == k) hk = h[q];
        const float y = (ya[kk] + yb[kk]) + (yc[kk] + yd[kk]);
        hn[kk] = fmaxf(0.0f, __fdividef(hk * y, gh + p.eps));
      }
      if (j >= 2 && !mbar_wait_bounded(hnfree(b), (uint32_t)(((j >> 1) + 1) & 1))) {
        s_err = 1;
        break;
      }
      float* hnp = reinterpret_cast<float*>(smem + C::OFF_HN + b * C::HNP);
      uint8_t* xs = smem + s * C::STAGE + (col >> 5) * C::CHUNK;
#pragma unroll
      for (int kk = 0; kk < KH; ++kk) {
        const int k = kh0 + kk;
        hnp[k * T + col] = hn[kk];
        const float hi = tf32_hi(hn[kk]);
        *reinterpret_cast<float*>(xs + sw128a32_off(C::ROW_HNH + k, col & 31)) = hi;
        *reinterpret_cast<float*>(xs + sw128a32_off(C::ROW_HNL + k, col & 31)) = hn[kk] - hi;
      }
      fence_proxy_async_smem();
      mbar_arrive(epi(s));
    }
    // final group of D_B
    if (!s_err && count > 0 && tid < 128) drain(count - 1);
    float* red = reinterpret_cast<float*>(smem + C::OFF_RED);
    if (tid < 128)
#pragma unroll
      for (int k = 0; k < N2; ++k) red[tid * N2 + k] = accB[k];
  }
  tc_fence_before();
  __syncthreads();
  if (!s_err && tid < NW) {
    // combine the hi/lo products: P[i] = D[i][k] + D[i][R+k] + D[ROW_XLO+i][k],
    // Q[k'] = D[MP+k'][k] + D[MP+k'][R+k] + D[MP+R+k'][k]
    const float* red = reinterpret_cast<const float*>(smem + C::OFF_RED);
    float* out = p.part + (size_t)blockIdx.x * ((MP + R) * R);
    for (int e = tid; e < (MP + R) * R; e += NW) {
      const int row = e / R, k = e % R;
      const int lo_row = row < MP ? C::ROW_XLO + row : row + R;
      out[e] = red[row * N2 + k] + red[row * N2 + R + k] + red[lo_row * N2 + k];
    }
  }
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <class C>
cudaError_t launch_tc_cfg(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                          const CUtensorMap& mh, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_pass_tc_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcParams p;
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
  p.eps = eps;
  mu_pass_tc_kernel<C><<<s.grid, kTcThreads + 32, C::SMEM, st>>>(mx, mh, p);
  return cudaGetLastError();
}

}  // namespace

bool tc_pass_supported(int MP, int R) { return MP <= 32 && R <= 16; }

cudaError_t launch_mu_pass_tc(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                              const CUtensorMap& mh, cudaStream_t st) {
#define NTT_TC(MPV, RV) \
  if (s.MP == MPV && s.R == RV) return launch_tc_cfg<TcCfg<MPV, RV>>(s, d, eps, mx, mh, st);
  NTT_TC(16, 8)
  NTT_TC(16, 16)
  NTT_TC(32, 8)
  NTT_TC(32, 16)
#undef NTT_TC
  return cudaErrorInvalidValue;
}

}  // namespace ntt
