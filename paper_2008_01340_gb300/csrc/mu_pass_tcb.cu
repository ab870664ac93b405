// Fused MU pass on the tensor cores for BF16 X (the precision form): tcgen05
// kind::f16 MMAs with FP32 accumulation in TMEM, for unfoldings of 16, 32,
// 128 or 256 rows and rank buckets 16 and 32.
//
// X is stored in BF16, so its values are exact BF16 operands.  The FP32
// factors are split into three BF16 terms, a = a1 + a2 + a3 with
// a1 = bf16(a), a2 = bf16(a - a1), a3 = bf16(a - a1 - a2): 3 x 8 significand
// bits hold all 24 of FP32, and every product of a BF16 X value with a term
// is exact in the FP32 accumulator.  Per tile of T = 128 columns:
//   phase A  Y^T (128 cols x 3R) = X_tile^T [W1 | W2 | W3]       (K = rows)
//   epilogue Y = sum of the three column groups; H_new = max(0, H o Y /
//            (G_W H + eps)) on CUDA cores (one column per lane, two threads
//            per column); H_new to HBM and, split in three BF16 terms, into
//            the H_new stack in shared memory
//   phase B  D_B += [X_tile ; Hstack] Hstack^T                    (K = columns)
//            P = sum over the three column groups of the X rows,
//            Q = sum over the nine (row term, column term) blocks
// D_B accumulates in TMEM over runs of 2048 columns; after
// each run its term sums are added, in FP32, into the CTA's (MP + R) x R
// partial block in HBM, which the common combine kernel reduces.  Measured:
// long TMEM runs carry a small accumulation bias -- 12 iterations on
// 256 x 16.8 M differ from the FP32 FMA pass by 4.3e-6 with runs of 128 tiles
// and by 1.4e-6 with runs of 16 (FP32 rounding level), and the first core of
// the 16^6 precision form moves from 3.3e-6 to 6.0e-7 from the FP64 oracle.
//
// Shared memory: the X tile as 64-column atoms of 128-byte rows with the
// 128-byte swizzle of 16-byte chunks (8-row period) -- at the same time the
// MN-major A operand of phase A (LBO = atom stride, SBO = 1024) and the
// K-major A operand of phase B (SBO = 1024); the W terms and the H_new stack
// in the same swizzled K-major form.  Two X stages: the load of tile j+1 is
// issued once phase A of tile j has completed (phase B of tile j-1, issued
// earlier, has then completed too), and overlaps the epilogue and phase B.
// Every wait is bounded; on expiry the kernel sets the status word, drains
// its MMAs and copies, frees its TMEM and returns.

#include "tc_bf16.cuh"

namespace ntt {

namespace {

constexpr int kTbThreads = 256;

template <int MP_, int R_>
struct TbCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  static constexpr int T = 128;                    // tile width in shared memory (MMA M of phase A)
  static constexpr int FLUSH = 2048 / T;           // tiles per TMEM accumulation run of D_B
  static constexpr int N3 = 3 * R;                 // MMA N: three terms of R ranks
  static constexpr int KH = R / 2;                 // ranks per thread in the epilogue
  // Stacked form (MP <= 32): a stage holds 128 rows, X in rows 0..MP-1 and the
  // H_new terms in rows MP..MP+3R-1, so phase B is one 128-row block.
  // Otherwise a stage holds MP rows of X and the H_new stack has its own 128 rows.
  static constexpr bool STACK = MP <= 32;
  static constexpr int SR = STACK ? 128 : MP;      // rows of a stage tile
  static constexpr int XST = SR * T * 2;           // bytes of one stage (two 64-column atoms)
  static constexpr int STAGES = STACK ? 4 : 2;
  static constexpr int HROWS = 128;                // rows of the separate H_new stack
  static constexpr int HNS = STACK ? 0 : HROWS * T * 2;
  static constexpr int HROW0 = STACK ? MP : 0;     // first H_new row in its region
  static constexpr int HSR = STACK ? SR : HROWS;   // rows of the region holding H_new
  static constexpr int KAT = MP < 64 ? 1 : MP / 64;   // 64-row K atoms of the W operand
  static constexpr int WOP = KAT * N3 * 128;
  static constexpr int NMB = STACK ? 0 : MP / 128;    // X-only 128-row M blocks of phase B
  static constexpr int OFF_X = 0;
  static constexpr int OFF_HN = STAGES * XST;
  static constexpr int OFF_W = OFF_HN + HNS;
  static constexpr int OFF_G = OFF_W + WOP;
  static constexpr int OFF_QS = OFF_G + R * R * 4;   // 3R x R scratch of the Q term rows
  static constexpr int OFF_BAR = OFF_QS + 3 * R * R * 4;
  static constexpr int USED = OFF_BAR + 64;
  static constexpr int SMEM = USED + 1024;         // + alignment of the 1024-byte atoms
  static constexpr uint32_t TMEM_COLS = STACK ? 256 : 512;   // D_A (N3) + D_B ((NMB + 1) N3)
  static constexpr uint32_t IDA = idesc_bf16(128, N3, true, false);
  static constexpr uint32_t IDB = idesc_bf16(128, N3, false, false);
  static_assert((MP == 16 || MP == 32 || MP == 128 || MP == 256) && (R == 16 || R == 32), "bucket");
  static_assert(!STACK || MP + 3 * R <= 128, "stacked rows fit one M block");
  static_assert(N3 * (NMB + 2) <= (int)TMEM_COLS, "TMEM columns");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(OFF_HN % 1024 == 0 && OFF_W % 1024 == 0, "atom alignment");
};

struct TbParams {
  const __nv_bfloat16* X;   // m x n BF16, row stride n (n % 8 == 0, 16-byte aligned)
  float* H;                 // r x n FP32, updated in place
  const float* W;           // m x r
  const float* G;           // R x R
  float* part;              // grid x (MP + R) x R
  int* status;
  const int* stop;     // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r, ntiles;
  float eps;
};

template <class C>
__global__ void __launch_bounds__(kTbThreads, 1) mu_pass_tcb_kernel(const TbParams p) {
  constexpr int MP = C::MP, R = C::R, T = C::T, N3 = C::N3, KH = C::KH;
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t sbase = smem_u32(smem);
  float* Gs = reinterpret_cast<float*>(smem + C::OFF_G);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);
  __shared__ int s_err;

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int m = p.m, r = p.r;
  const int64_t n = p.n;
  const uint32_t barA = smem_u32(&bars[0]), barB = smem_u32(&bars[1]);
  const int count = (p.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

  // ---- setup: zero the X stages and the H_new stack, W terms, G, barriers, TMEM
  for (int i = tid; i < (C::OFF_W) / 16; i += kTbThreads)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  // all of a thread's W loads in flight at once, then the splits
  constexpr int NWL = (MP * R + kTbThreads - 1) / kTbThreads;
  float wv[NWL];
#pragma unroll
  for (int u = 0; u < NWL; ++u) {
    const int e = tid + u * kTbThreads, i = e / R, k = e % R;
    wv[u] = (e < MP * R && i < m && k < r) ? p.W[i * r + k] : 0.0f;
  }
#pragma unroll
  for (int u = 0; u < NWL; ++u) {
    const int e = tid + u * kTbThreads;
    if (e >= MP * R) break;
    const int i = e / R, k = e % R;   // W row i (K index), rank k
    const float w = wv[u];
    __nv_bfloat16 t3[3];
    split3(w, t3);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int nrow = t * R + k;
      const uint32_t off = (uint32_t)((i >> 6) * N3 * 128) + nrow * 128 +
                           (((((i & 63) >> 3)) ^ (nrow & 7)) << 4) + ((i & 7) << 1);
      *reinterpret_cast<__nv_bfloat16*>(smem + C::OFF_W + off) = t3[t];
    }
  }
  for (int e = tid; e < R * R; e += kTbThreads) Gs[e] = p.G[e];
  if (tid == 0) {
    s_err = 0;
    mbar_init(barA, 1);
    mbar_init(barB, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t dA = tmem;
  auto dB = [&](int b) { return tmem + (uint32_t)(N3 * (1 + b)); };

  // ---- X tile loader: rows < m, 8 BF16 values per 16-byte copy, zero fill past
  // n; tiles past the CTA's range issue nothing but still commit a group
  auto issue = [&](int stage, int tile, bool valid) {
    uint8_t* dst = smem + C::OFF_X + stage * C::XST;
    const int64_t col0 = (int64_t)tile * T;
    for (int e = tid; valid && e < m * (T / 8); e += kTbThreads) {
      const int row = e / (T / 8), ch = e % (T / 8);
      const int64_t col = col0 + 8 * ch;
      const int64_t left = n - col;
      const int bytes = left >= 8 ? 16 : (left > 0 ? (int)left * 2 : 0);
      const __nv_bfloat16* src = p.X + (int64_t)row * n + (bytes ? col : 0);
      const uint32_t off = swz(row, 8 * ch, C::SR);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + off)), "l"(src),
                   "r"(bytes)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  // descriptors (thread 0 only uses them)
  const uint64_t dW = smem_desc(sbase + C::OFF_W, 16, 1024, kLayoutSw128);
  const uint64_t dH = smem_desc(sbase + C::OFF_HN, 16, 1024, kLayoutSw128);

  // epilogue role: TMEM lane = tile column c, ranks kh0 .. kh0 + KH - 1
  const int c = (warp % 4) * 32 + lane;
  const int kh0 = (warp / 4) * KH;
  const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;

  // this CTA's partial block, accumulated over the TMEM runs
  float* out = p.part + (size_t)blockIdx.x * ((MP + R) * R);
  for (int e = tid; e < (MP + R) * R; e += kTbThreads) out[e] = 0.0f;
  float* qs = reinterpret_cast<float*>(smem + C::OFF_QS);
  // Add the finished TMEM run of D_B: P rows (X blocks) straight into `out`
  // (each entry owned by one thread), Q through the term sums in `qs`.
  auto flush = [&]() {
    for (int b = 0; b <= C::NMB; ++b) {
      const bool qblock = b == C::NMB;
      float acc[KH];
#pragma unroll
      for (int q = 0; q < KH; ++q) acc[q] = 0.0f;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        float v[KH];
        if constexpr (KH == 16)
          tmem_ld16(dB(b) + lane_base + t * R + kh0, v);
        else
          tmem_ld8(dB(b) + lane_base + t * R + kh0, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < KH; ++q) acc[q] += v[q];
      }
      const int row = 32 * (warp % 4) + lane;
      if (!qblock || (C::STACK && row < MP)) {
        float* o = out + (b * 128 + row) * R + kh0;   // P rows (in the stacked block: rows < MP)
#pragma unroll
        for (int q = 0; q < KH; ++q) o[q] += acc[q];
      } else if (row >= C::HROW0 && row < C::HROW0 + 3 * R) {
#pragma unroll
        for (int q = 0; q < KH; ++q) qs[(row - C::HROW0) * R + kh0 + q] = acc[q];
      }
    }
    tc_fence_before();
    __syncthreads();
    for (int e = tid; e < R * R; e += kTbThreads) {
      const int k = e / R, l = e % R;
      out[(MP + k) * R + l] += (qs[k * R + l] + qs[(R + k) * R + l]) + qs[(2 * R + k) * R + l];
    }
    __syncthreads();
  };

  for (int q = 0; q < C::STAGES - 1; ++q) issue(q, (int)blockIdx.x + q * (int)gridDim.x, q < count);
  // old H of a tile's column, all ranks; with rank bucket 16 the next tile's
  // values are loaded one tile ahead (registers), so their latency overlaps
  // the current tile
  constexpr bool PREFETCH_H = R <= 16;
  auto load_h = [&](int tile_, float* hv) {
    const int64_t col_ = (int64_t)tile_ * T + c;
#pragma unroll
    for (int l = 0; l < R; ++l) hv[l] = (l < r && col_ < n) ? p.H[(int64_t)l * n + col_] : 0.0f;
  };
  float hnext[PREFETCH_H ? R : 1];
  if constexpr (PREFETCH_H) {
    if (count > 0) load_h((int)blockIdx.x, hnext);
  }
  int j = 0;
  int a_issued = -1;   // thread 0: the last tile whose phase A it issued
  for (; j < count; ++j) {
    const int s = j % C::STAGES;
    const int tile = (int)blockIdx.x + j * (int)gridDim.x;
    const int64_t col = (int64_t)tile * T + c;
    asm volatile("cp.async.wait_group %0;" ::"n"(C::STAGES - 2) : "memory");
    fence_proxy_async_smem();
    __syncthreads();
    if (s_err) break;
    // ---- phase A
    if (tid == 0) {
      tc_fence_after();
      const uint64_t dXa = smem_desc(sbase + C::OFF_X + s * C::XST, C::SR * 128, 1024, kLayoutSw128);
#pragma unroll
      for (int kk = 0; kk < MP / 16; ++kk)
        mma_bf16(dA, dXa + (uint64_t)((kk * 2048) >> 4),
                 dW + (uint64_t)((((kk >> 2) * N3 * 128) + (kk & 3) * 32) >> 4), C::IDA, kk > 0 ? 1u : 0u);
      mma_commit(barA);
      a_issued = j;
    }
    float h[R];
    if constexpr (PREFETCH_H) {
#pragma unroll
      for (int l = 0; l < R; ++l) h[l] = hnext[l];
      if (j + 1 < count) load_h(tile + (int)gridDim.x, hnext);
    } else {
      load_h(tile, h);   // overlaps the MMAs
    }
    if (!mbar_wait_bounded(barA, (uint32_t)(j & 1))) s_err = 1;
    tc_fence_after();
    __syncthreads();
    if (s_err) break;
    // phase B of tile j-1 is complete: end the TMEM run every FLUSH tiles
    if (j > 0 && j % C::FLUSH == 0) flush();
    // tile j + STAGES - 1 into the stage of tile j - 1, whose readers (phases A
    // and B of tile j - 1) are done.  (Issuing it earlier, after a wait for
    // phase B of tile j - 1 right behind phase A's issue, measured slower: the
    // wait holds back the H loads that otherwise overlap the MMAs.)
    issue((j + C::STAGES - 1) % C::STAGES, tile + (C::STAGES - 1) * (int)gridDim.x, j + C::STAGES - 1 < count);
    // ---- epilogue
    float y[KH];
    {
      float v[KH];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        if constexpr (KH == 16)
          tmem_ld16(dA + lane_base + t * R + kh0, v);
        else
          tmem_ld8(dA + lane_base + t * R + kh0, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < KH; ++q) y[q] = t == 0 ? v[q] : y[q] + v[q];
      }
    }
    tc_fence_before();
    // H update of column c, rank kh0 + q: H_new to HBM and its three BF16
    // terms into the H_new stack
    auto update_rank = [&](int q) {
      const int k = kh0 + q;
      float gh = 0.0f;
#pragma unroll
      for (int l = 0; l < R; l += 4) {
        const float4 g = *reinterpret_cast<const float4*>(Gs + k * R + l);
        gh = fmaf(g.x, h[l], gh);
        gh = fmaf(g.y, h[l + 1], gh);
        gh = fmaf(g.z, h[l + 2], gh);
        gh = fmaf(g.w, h[l + 3], gh);
      }
      const float hk = warp >= 4 ? h[KH + q] : h[q];
      const float hn = fmaxf(0.0f, __fdividef(hk * y[q], gh + p.eps));
      if (k < r && col < n) p.H[(int64_t)k * n + col] = hn;
      __nv_bfloat16 t3[3];
      split3(hn, t3);
#pragma unroll
      for (int t = 0; t < 3; ++t)
        *reinterpret_cast<__nv_bfloat16*>(smem + (C::STACK ? C::OFF_X + s * C::XST : C::OFF_HN) +
                                          swz(C::HROW0 + t * R + k, c, C::HSR)) = t3[t];
    };
#pragma unroll
    for (int q = 0; q < KH; ++q) update_rank(q);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // ---- phase B
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < T / 16; ++kk) {
        const uint32_t xo = (uint32_t)((kk >> 2) * C::SR * 128 + (kk & 3) * 32);
        const uint32_t acc = (j % C::FLUSH != 0 || kk > 0) ? 1u : 0u;
        if constexpr (C::STACK) {
          // one block: A = the stage's 128 rows [X ; H_new terms ; 0], B = its H_new rows
          const uint32_t base = sbase + C::OFF_X + s * C::XST + xo;
          mma_bf16(dB(0), smem_desc(base, 16, 1024, kLayoutSw128),
                   smem_desc(base + C::HROW0 * 128, 16, 1024, kLayoutSw128), C::IDB, acc);
        } else {
          const uint32_t ho = (uint32_t)((kk >> 2) * C::HROWS * 128 + (kk & 3) * 32);
#pragma unroll
          for (int mb = 0; mb < C::NMB; ++mb)
            mma_bf16(dB(mb), smem_desc(sbase + C::OFF_X + s * C::XST + mb * 128 * 128 + xo, 16, 1024, kLayoutSw128),
                     dH + (uint64_t)(ho >> 4), C::IDB, acc);
          mma_bf16(dB(C::NMB), dH + (uint64_t)(ho >> 4), dH + (uint64_t)(ho >> 4), C::IDB, acc);
        }
      }
      mma_commit(barB);
    }
  }
  // ---- drain: the last phase B (or, after a timeout, everything in flight)
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (count > 0 && !s_err) {
    if (!mbar_wait_bounded(barB, (uint32_t)((count - 1) & 1))) s_err = 1;
  }
  if (s_err && tid == 0) {
    // MMAs may still be in flight: phase A of tile j and phase B of tile j - 1 (bounded)
    if (j < count && a_issued == j) (void)mbar_wait_bounded(barA, (uint32_t)(j & 1));
    if (j >= 1) (void)mbar_wait_bounded(barB, (uint32_t)((j - 1) & 1));
  }
  tc_fence_after();
  __syncthreads();
  if (s_err) {
    for (int e = tid; e < (MP + R) * R; e += kTbThreads) out[e] = 0.0f;
    if (tid == 0) atomicExch(p.status, kStatusTimeout);
  } else if (count > 0) {
    flush();   // the last run
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <class C>
cudaError_t launch_tcb_cfg(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mu_pass_tcb_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TbParams p;
  p.X = reinterpret_cast<const __nv_bfloat16*>(d.X);
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
  return launch_pdl(mu_pass_tcb_kernel<C>, dim3(s.grid), dim3(kTbThreads), C::SMEM, st, p);
}

}  // namespace

bool tcb_pass_supported(int MP, int R) {
  return (MP == 16 || MP == 32 || MP == 128 || MP == 256) && (R == 16 || R == 32);
}

cudaError_t launch_mu_pass_tcb(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  if (s.MP == 16 && s.R == 16) return launch_tcb_cfg<TbCfg<16, 16>>(s, d, eps, st);
  if (s.MP == 16 && s.R == 32) return launch_tcb_cfg<TbCfg<16, 32>>(s, d, eps, st);
  if (s.MP == 32 && s.R == 16) return launch_tcb_cfg<TbCfg<32, 16>>(s, d, eps, st);
  if (s.MP == 32 && s.R == 32) return launch_tcb_cfg<TbCfg<32, 32>>(s, d, eps, st);
  // 128/256 rows: the warp-specialised pass of mu_pass_tcs.cu in its BF16 form
  if (s.MP == 128 || s.MP == 256) return launch_mu_pass_tcbx(s, d, eps, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
