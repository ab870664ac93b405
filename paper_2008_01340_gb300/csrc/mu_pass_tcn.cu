// Fused MU pass for FP32 X of at most 32 rows on the BF16 tensor cores (the
// split form, stacked): the first unfolding of a tensor whose first mode is
// small (32 x 32^5 for a 32^6 tensor, r_1 = 8), rank buckets 8 and 16.
//
// X is split once per stage into X1 = bf16(X) and X2 = bf16(X - X1) (16
// significand bits).  A tile covers 128 columns; its stage in shared memory is
// one 128-row block of two 64-column atoms (128-byte swizzle):
//   rows 0 .. MP-1          X1 of the tile        (TMA)
//   rows MP .. 2MP-1        X2 of the tile        (TMA)
//   rows 2MP .. 2MP+3R-1    the three BF16 terms of H_new (written by the epilogue)
// Per tile:
//   phase A  D_A (128 cols x 2R) = [X1 ; X2]^T [W1 | W2 ; W1 | W2]   (K = 2MP rows)
//            the sum over X1 and X2 runs in the MMA's K; the two W terms
//            W1 = bf16(W), W2 = bf16(W - W1) are column groups summed in the
//            epilogue (TMEM lane = column: no exchange between threads)
//   epilogue H_new = max(0, H o Y / (G_W H + eps)) on CUDA cores; H_new to HBM
//            and, split into three BF16 terms, into rows 2MP.. of the stage
//   phase B  D_B (128 rows x 3R) += stage block x (H_new rows)^T   (K = 128 cols)
//            lanes i and MP + i hold X1 H_new^T and X2 H_new^T of row i, lanes
//            2MP + t R + k the term rows of Q; all summed when a TMEM run of
//            2048 columns is flushed into the CTA's (MP + R) x R partial block
//
// Warp roles (576 threads): two epilogue groups of eight warps take the even
// and the odd tiles (so two epilogues run at once beside the MMAs of the
// neighbouring tiles); warp 16 lane 0 issues every MMA; warp 17 lane 0 the TMA
// copies.  D_A is double-buffered (one buffer per group); the H_new rows live
// in the tile's own stage.  Hand-offs are mbarriers:
//   full[s]   copies of stage s landed         -> MMA thread
//   empty[s]  phase B of stage s's tile done   -> TMA thread
//   barA[b]   phase A into D_A[b] done         -> epilogue group b
//   epi[b]    epilogue of a tile of group b    -> MMA thread
//   bdone     phase B done (in order)          -> epilogue (TMEM run flushes)
// Every wait is bounded; on expiry the waiting role sets the error flag and
// stops, the others stop at their next wait or check, the MMA thread waits for
// its MMAs and the TMA thread for its copies, TMEM is freed, the partials are
// zeroed and the status word is set.
#include <cstring>

#include "tc_bf16.cuh"

namespace ntt {

namespace {

constexpr int kTnEpi = 256;                      // threads of one epilogue group
constexpr int kTnThreads = 2 * kTnEpi + 64;      // + the MMA warp and the TMA warp

template <int MP_, int R_>
struct TnCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  static constexpr int T = 128;                  // columns per tile (two atoms)
  static constexpr int FLUSH = 2048 / T;         // tiles per TMEM run of D_B
  static constexpr int N2 = 2 * R;               // phase A N: two W terms
  static constexpr int N3 = 3 * R;               // phase B N: three H_new terms
  static constexpr int KH = R / 2;               // ranks per epilogue thread
  static constexpr int HROW = 2 * MP;            // first H_new term row of a stage
  static constexpr int ATOM = 128 * 128;         // bytes of one 128-row atom
  static constexpr int XST = 2 * ATOM;           // one stage
  static constexpr int WOP = N2 * 128;           // W terms: N2 rows of one K atom (K = 2MP <= 64)
  static constexpr int SCR = (2 * MP + N3) * R * 4;   // flush scratch of one group
  static constexpr int BARB = 256;
  static constexpr int FIXED = WOP + R * R * 4 + 2 * SCR + BARB + 1024;
  static constexpr int FIT = (227 * 1024 - FIXED) / XST;
  static constexpr int S = FIT < 6 ? FIT : 6;    // X stages
  static constexpr int OFF_X = 0;
  static constexpr int OFF_W = S * XST;
  static constexpr int OFF_G = OFF_W + WOP;
  static constexpr int OFF_SCR = OFF_G + R * R * 4;
  static constexpr int OFF_BAR = OFF_SCR + 2 * SCR;
  static constexpr int SMEM = OFF_BAR + BARB + 1024;   // + alignment of the 1024-byte atoms
  static constexpr int TMEM_USED = 2 * N2 + N3;
  static constexpr uint32_t TMEM_COLS = TMEM_USED <= 64 ? 64 : 128;
  static constexpr uint32_t IDA = idesc_bf16(128, N2, true, false);
  static constexpr uint32_t IDB = idesc_bf16(128, N3, false, false);
  static constexpr uint32_t TX = 4u * MP * 128u; // X1 and X2, two atoms each
  static_assert((MP == 16 || MP == 32) && (R == 8 || R == 16), "bucket");
  static_assert(HROW + N3 <= 128, "stacked rows fit one M block");
  static_assert(S >= 2 && SMEM <= 227 * 1024, "shared memory");
  static_assert((HROW * 128) % 1024 == 0 && OFF_W % 1024 == 0 && WOP % 1024 == 0, "atom alignment");
  static_assert(TMEM_USED <= 128, "TMEM columns");
};

struct TnParams {
  float* H;          // r x n FP32, updated in place
  const float* W;    // m x r
  const float* G;    // R x R
  float* part;       // grid x (MP + R) x R
  int* status;
  const int* stop;   // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r, ntiles;
  float eps;
};

// Named barrier 1 + g over the 256 threads of epilogue group g, with an OR
// over their predicates (every thread of the group gets the same answer).
__device__ __forceinline__ bool grp_any(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)(pred ? 1u : 0u)), "r"(1 + g)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void grp_sync(int g) { asm volatile("bar.sync %0, 256;" ::"r"(1 + g) : "memory"); }

__device__ __forceinline__ int tn_flag(const int* f) { return *reinterpret_cast<const volatile int*>(f); }

template <int KH>
__device__ __forceinline__ void tn_ld(uint32_t taddr, float* v) {
  if constexpr (KH == 8)
    tmem_ld8(taddr, v);
  else
    tmem_ld4(taddr, v);
}

// tmX1 / tmX2: TMA maps of X1 and X2 (64-column boxes of MP rows, 128-byte
// swizzle; rows past m and columns past n arrive as zeros).
template <class C>
__global__ void __launch_bounds__(kTnThreads, 1) mu_pass_tcn_kernel(const __grid_constant__ CUtensorMap tmX1,
                                                                    const __grid_constant__ CUtensorMap tmX2,
                                                                    const TnParams p) {
  constexpr int MP = C::MP, R = C::R, N2 = C::N2, N3 = C::N3, KH = C::KH, S = C::S;
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  float* Gs = reinterpret_cast<float*>(smem + C::OFF_G);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 24);
  int* s_err = reinterpret_cast<int*>(bars + 25);

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int m = p.m, r = p.r;
  const int64_t n = p.n;
  const int count = (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  auto full = [&](int s) { return bar(s); };
  auto empty = [&](int s) { return bar(6 + s); };
  auto barA = [&](int b) { return bar(12 + b); };
  auto epi = [&](int b) { return bar(14 + b); };
  const uint32_t bdone = bar(16), drain = bar(17);

  // ---- setup: W terms (K-major B operand of phase A: N2 rows, K = X1 rows
  // then X2 rows, both against the same W rows), G, barriers, TMEM, partials
  for (int e = tid; e < N2 * 2 * MP; e += kTnThreads) {
    const int nrow = e / (2 * MP), kk = e % (2 * MP);
    const int t = nrow / R, k = nrow % R, i = kk % MP;
    const float w = (i < m && k < r) ? p.W[i * r + k] : 0.0f;
    const __nv_bfloat16 w1 = __float2bfloat16_rn(w);
    const __nv_bfloat16 wt = t == 0 ? w1 : __float2bfloat16_rn(w - __bfloat162float(w1));
    const uint32_t off = (uint32_t)(nrow * 128 + ((((kk >> 3) & 7) ^ (nrow & 7)) << 4) + ((kk & 7) << 1));
    *reinterpret_cast<__nv_bfloat16*>(smem + C::OFF_W + off) = wt;
  }
  for (int e = tid; e < R * R; e += kTnThreads) Gs[e] = p.G[e];
  float* out = p.part + (size_t)blockIdx.x * ((MP + R) * R);
  for (int e = tid; e < (MP + R) * R; e += kTnThreads) out[e] = 0.0f;
  if (tid == 0) {
    *s_err = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(barA(b), 1);
      mbar_init(epi(b), kTnEpi);
    }
    mbar_init(bdone, 1);
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 16) {
    tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto dA = [&](int b) { return tmem + (uint32_t)(b * N2); };
  const uint32_t dB = tmem + (uint32_t)(2 * N2);
  auto stage_off = [&](int s) { return (uint32_t)(C::OFF_X + s * C::XST); };

  if (warp == 17) {
    // =========================================================== TMA thread
    if (lane == 0) {
      int t = 0;
      for (; t < count; ++t) {
        const int s = t % S;
        if (t >= S && !mbar_wait_bounded(empty(s), (uint32_t)(((t / S) - 1) & 1))) {
          *s_err = 1;
          break;
        }
        if (tn_flag(s_err)) break;
        const int col0 = ((int)blockIdx.x + t * (int)gridDim.x) * C::T;
        const uint32_t dst = sbase + stage_off(s);
        mbar_arrive_expect_tx(full(s), C::TX);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          tma_load_2d(dst + a * C::ATOM, &tmX1, col0 + 64 * a, 0, full(s));
          tma_load_2d(dst + a * C::ATOM + MP * 128, &tmX2, col0 + 64 * a, 0, full(s));
        }
      }
      for (int u = t - S < 0 ? 0 : t - S; u < t; ++u) (void)mbar_wait_bounded(full(u % S), (uint32_t)((u / S) & 1));
    }
  } else if (warp == 16) {
    // =========================================================== MMA thread
    if (lane == 0 && count > 0) {
      const uint64_t dW = smem_desc(sbase + C::OFF_W, 16, 1024, kLayoutSw128);
      bool ok = true;
      auto wait = [&](uint32_t b, uint32_t ph) {
        if (!mbar_wait_bounded(b, ph)) {
          *s_err = 1;
          ok = false;
        }
        return ok;
      };
      // phase A of local tile t (stage s) into D_A[t & 1]: M = the 128 columns
      // (MN-major, LBO = the atom stride), K = the X1 and X2 rows
      auto phase_a = [&](int t, int s) {
        const uint64_t dX = smem_desc(sbase + stage_off(s), C::ATOM, 1024, kLayoutSw128);
#pragma unroll
        for (int kk = 0; kk < 2 * MP / 16; ++kk)
          mma_bf16(dA(t & 1), dX + (uint64_t)((kk * 2048) >> 4), dW + (uint64_t)((kk * 32) >> 4), C::IDA,
                   kk > 0 ? 1u : 0u);
        mma_commit(barA(t & 1));
      };
      // phase B of local tile t: A = the stage's 128 rows, B = its H_new rows, K = the 128 columns
      auto phase_b = [&](int t, int s) {
        const uint32_t xb = sbase + stage_off(s);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint32_t xo = (uint32_t)((kk >> 2) * C::ATOM + (kk & 3) * 32);
          const uint32_t acc = (t % C::FLUSH != 0 || kk > 0) ? 1u : 0u;
          mma_bf16(dB, smem_desc(xb + xo, 16, 1024, kLayoutSw128),
                   smem_desc(xb + xo + C::HROW * 128, 16, 1024, kLayoutSw128), C::IDB, acc);
        }
        mma_commit(empty(s));
        mma_commit(bdone);
      };
      if (wait(full(0), 0u)) {
        tc_fence_after();
        phase_a(0, 0);
      }
      for (int j = 0; ok && j < count; ++j) {
        if (j + 1 < count) {
          // D_A[(j+1) & 1] was read by the epilogue of tile j - 1 (waited for one round earlier)
          if (!wait(full((j + 1) % S), (uint32_t)(((j + 1) / S) & 1))) break;
          tc_fence_after();
          phase_a(j + 1, (j + 1) % S);
        }
        if (!wait(epi(j & 1), (uint32_t)((j >> 1) & 1))) break;
        tc_fence_after();
        phase_b(j, j % S);
        if (tn_flag(s_err)) break;
      }
      // every MMA issued has completed before TMEM is released
      mma_commit(drain);
      (void)mbar_wait_bounded(drain, 0u);
    }
  } else {
    // =========================================================== epilogue
    // group g takes tiles g, g + 2, ...; TMEM lane c = tile column c, ranks kh0 .. kh0 + KH - 1
    const int g = warp / 8, lw = warp % 8;
    const int gtid = tid % kTnEpi;
    const int c = (lw % 4) * 32 + lane;
    const bool hi = lw >= 4;
    const int kh0 = hi ? KH : 0;
    const uint32_t lane_base = (uint32_t)((lw % 4) * 32) << 16;
    float* scr = reinterpret_cast<float*>(smem + C::OFF_SCR + g * C::SCR);
    // old H of a tile's column, all ranks, one tile of the group ahead (registers)
    auto load_h = [&](int tile_, float* hv) {
      const int64_t col_ = (int64_t)tile_ * C::T + c;
#pragma unroll
      for (int l = 0; l < R; ++l) hv[l] = (l < r && col_ < n) ? p.H[(int64_t)l * n + col_] : 0.0f;
    };
    float hnext[R];
    if (g < count) load_h((int)blockIdx.x + g * (int)gridDim.x, hnext);
    // rank bucket 8: the G rows of this thread's ranks in registers
    constexpr bool GREG = R <= 8;
    float gk[GREG ? KH : 1][GREG ? R : 1];
    if constexpr (GREG) {
#pragma unroll
      for (int q = 0; q < KH; ++q)
#pragma unroll
        for (int l = 0; l < R; ++l) gk[q][l] = Gs[(kh0 + q) * R + l];
    }
    // Add the finished TMEM run of D_B into `out`: term sums per lane into the
    // group's scratch, then P = lanes i + MP + i, Q = the three term-row blocks
    auto flush = [&]() {
      float v0[KH], v1[KH], v2[KH];
      tn_ld<KH>(dB + lane_base + kh0, v0);
      tn_ld<KH>(dB + lane_base + R + kh0, v1);
      tn_ld<KH>(dB + lane_base + 2 * R + kh0, v2);
      tmem_wait_ld();
      if (c < C::HROW + N3) {
#pragma unroll
        for (int q = 0; q < KH; ++q) scr[c * R + kh0 + q] = (v0[q] + v1[q]) + v2[q];
      }
      tc_fence_before();
      grp_sync(g);
      for (int e = gtid; e < (MP + R) * R; e += kTnEpi) {
        if (e < MP * R) {
          const int i = e / R, k = e % R;
          out[e] += scr[i * R + k] + scr[(MP + i) * R + k];
        } else {
          const int kl = e - MP * R, k = kl / R, l = kl % R;
          out[e] += (scr[(C::HROW + k) * R + l] + scr[(C::HROW + R + k) * R + l]) + scr[(C::HROW + 2 * R + k) * R + l];
        }
      }
      grp_sync(g);
    };
    bool ok = true;
    for (int j = g; j < count; j += 2) {
      const int s = j % S;
      const int tile = (int)blockIdx.x + j * (int)gridDim.x;
      const int64_t col = (int64_t)tile * C::T + c;
      bool bad = !mbar_wait_bounded(barA(g), (uint32_t)((j >> 1) & 1));
      if (bad) *s_err = 1;
      if (grp_any(g, bad || tn_flag(s_err))) {
        ok = false;
        break;
      }
      tc_fence_after();
      float h[R];
#pragma unroll
      for (int l = 0; l < R; ++l) h[l] = hnext[l];
      if (j + 2 < count) load_h(tile + 2 * (int)gridDim.x, hnext);
      if (j > 0 && j % C::FLUSH == 0) {
        // phase B of tile j - 1 ends a TMEM run (phase B of tile j starts the next);
        // phase A of tile j was issued after phase B of tile j - 2, so the wait is unambiguous
        bad = !mbar_wait_bounded(bdone, (uint32_t)((j - 1) & 1));
        if (bad) *s_err = 1;
        if (grp_any(g, bad)) {
          ok = false;
          break;
        }
        tc_fence_after();
        flush();
      }
      float y[KH];
      {
        float v0[KH], v1[KH];
        tn_ld<KH>(dA(g) + lane_base + kh0, v0);
        tn_ld<KH>(dA(g) + lane_base + R + kh0, v1);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < KH; ++q) y[q] = v0[q] + v1[q];
      }
      tc_fence_before();
      // H update of column c at ranks kh0 + q: all of them first (independent
      // chains), then H_new to HBM and its three BF16 terms into the stage
      float hn[KH];
#pragma unroll
      for (int q = 0; q < KH; ++q) {
        float gh = 0.0f;
        if constexpr (GREG) {
#pragma unroll
          for (int l = 0; l < R; ++l) gh = fmaf(gk[q][l], h[l], gh);
        } else {
          const int k = kh0 + q;
#pragma unroll
          for (int l = 0; l < R; l += 4) {
            const float4 gg = *reinterpret_cast<const float4*>(Gs + k * R + l);
            gh = fmaf(gg.x, h[l], gh);
            gh = fmaf(gg.y, h[l + 1], gh);
            gh = fmaf(gg.z, h[l + 2], gh);
            gh = fmaf(gg.w, h[l + 3], gh);
          }
        }
        const float hk = hi ? h[KH + q] : h[q];
        hn[q] = fmaxf(0.0f, __fdividef(hk * y[q], gh + p.eps));
      }
      uint8_t* st = smem + stage_off(s);
#pragma unroll
      for (int q = 0; q < KH; ++q) {
        const int k = kh0 + q;
        if (k < r && col < n) p.H[(int64_t)k * n + col] = hn[q];
        __nv_bfloat16 t3[3];
        split3(hn[q], t3);
#pragma unroll
        for (int t = 0; t < 3; ++t) *reinterpret_cast<__nv_bfloat16*>(st + swz(C::HROW + t * R + k, c, 128)) = t3[t];
      }
      fence_proxy_async_smem();
      tc_fence_before();
      mbar_arrive(epi(g));
    }
    // the last run (group 0), once every MMA has completed (the drain commit)
    if (g == 0) {
      const bool run = ok && count > 0;
      bool bad = false;
      if (run) bad = !mbar_wait_bounded(drain, 0u);
      if (bad) *s_err = 1;
      if (!grp_any(0, bad || !run)) {
        tc_fence_after();
        flush();
      }
    }
  }
  // ---- teardown
  tc_fence_before();
  __syncthreads();
  if (tn_flag(s_err)) {
    for (int e = tid; e < (MP + R) * R; e += kTnThreads) out[e] = 0.0f;
    if (tid == 0) atomicExch(p.status, kStatusTimeout);
  }
  if (warp == 16) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <class C>
cudaError_t launch_tcn_cfg(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mu_pass_tcn_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TnParams p;
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
  CUtensorMap m1, m2;
  std::memset(&m1, 0, sizeof(m1));
  std::memset(&m2, 0, sizeof(m2));
  if (encode_bf16_atom_map(d.X, s.m, s.n, C::MP, &m1) != NTT_OK ||
      encode_bf16_atom_map(d.X2, s.m, s.n, C::MP, &m2) != NTT_OK)
    return cudaErrorInvalidValue;
  return launch_pdl(mu_pass_tcn_kernel<C>, dim3(s.grid), dim3(kTnThreads), C::SMEM, st, m1, m2, p);
}

}  // namespace

bool tcn_pass_supported(int MP, int R) { return (MP == 16 || MP == 32) && (R == 8 || R == 16); }

cudaError_t launch_mu_pass_tcn(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  if (s.MP == 16 && s.R == 8) return launch_tcn_cfg<TnCfg<16, 8>>(s, d, eps, st);
  if (s.MP == 16 && s.R == 16) return launch_tcn_cfg<TnCfg<16, 16>>(s, d, eps, st);
  if (s.MP == 32 && s.R == 8) return launch_tcn_cfg<TnCfg<32, 8>>(s, d, eps, st);
  if (s.MP == 32 && s.R == 16) return launch_tcn_cfg<TnCfg<32, 16>>(s, d, eps, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
