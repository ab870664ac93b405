// Fused MU pass for FP32 X on the BF16 tensor cores (the split form), for
// unfoldings of 128 or 256 rows at rank buckets 16 and 32 and of 512 rows at
// rank bucket 16; with BX the same pass for BF16 X (the precision form) at 128
// or 256 rows: X is then an exact operand, a tile covers 128 columns (its two
// atoms), W takes three BF16 terms (24 bits), the H_new stack has one atom per
// column half and Q runs over both, and each TMEM lane is its own column (no
// exchange between threads).
//
// The unfolding is split once per stage into two BF16 matrices X1 = bf16(X)
// and X2 = bf16(X - X1) (16 significand bits of X; the same HBM bytes per
// iteration as FP32 X), stored tile-major as the stages' shared-memory image
// (split_blocked_kernel): a tile covers 64 columns, 8-row groups of X1 and of
// X2 alternate in 1024-byte swizzle atoms, and one contiguous bulk copy moves a
// whole tile (a copy of 128 bytes of every row reached 4.7 TB/s on this read,
// the contiguous tile 6.9).  Per tile:
//   phase A  D_A (128 x 2R) = [X1 | X2]^T [W1 | W2]                 (K = rows)
//            TMEM lane c holds X1^T W of column c, lane 64 + c X2^T W; the
//            two W terms W1 = bf16(W), W2 = bf16(W - W1) (16 significand
//            bits, as for X) are column groups summed in the epilogue
//   epilogue Y = the four parts; H_new = max(0, H o Y / (G_W H + eps)) on
//            CUDA cores; H_new to HBM and, split into three BF16 terms, into
//            the H_new stack (3R rows of one 64-column atom)
//   phase B  D_B += [X1 X2] [Hs Hs]^T over K = both atoms (P = (X1 + X2) H_new^T)
//            and D_Q += Hs Hs^T over one atom; the three term groups of P and
//            the nine term blocks of Q are summed when a TMEM run is flushed
// D_B accumulates over runs of 2048 columns; each finished run is added, in
// FP32, into the CTA's (MP + R) x R partial block, which the common combine
// kernel reduces.
//
// Warp roles (320 threads): warps 0-7 run the epilogue (two TMEM lanes per
// column, each thread a quarter of the ranks of its column); warp 8 lane 0
// issues every MMA; warp 9 lane 0 issues the TMA copies.  D_A and the H_new
// stack are double-buffered, so the epilogue of tile j runs while the tensor
// pipe does phase B of tile j-1 and phase A of tile j+1, and the copies of
// later tiles fill the other X stages (three at 256 rows and rank 16).  At
// 512 rows a stage takes 128 KB and only one fits: phase A of a tile then
// waits for phase B of the previous one (the X of a 512-row unfolding of the
// sizes routed here is resident in L2).
// Hand-offs are mbarriers:
//   full[s]   copies of stage s landed        -> MMA thread
//   empty[s]  phase B of stage s's tile done  -> TMA thread
//   barA[b]   phase A into D_A[b] done        -> epilogue
//   epi[b]    epilogue of a tile of parity b  -> MMA thread (D_A[b] read, stack b written)
//   bdone     phase B done (in order)         -> epilogue (TMEM run flushes)
// Every wait is bounded; on expiry the waiting role sets the error flag and
// stops, the others stop at their next wait or check, the MMA thread waits for
// its MMAs and the TMA thread for its copies, TMEM is freed, the partials are
// zeroed and the status word is set.
#include <cstring>
#include <type_traits>

#include "tc_bf16.cuh"

namespace ntt {

namespace {

constexpr int kTsEpi = 256;                 // epilogue threads (warps 0-7)
constexpr int kTsThreads = kTsEpi + 64;     // + the MMA warp and the TMA warp

template <int MP_, int R_, bool BX_ = false>
struct TsCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  // BX: X itself is BF16 (the precision form): its values are exact operands,
  // a tile's two atoms are 128 consecutive columns, W takes three terms
  static constexpr bool BX = BX_;
  static constexpr int TC = BX ? 128 : 64;      // columns of X per tile
  static constexpr int FLUSH = 2048 / TC;       // tiles per TMEM run of D_B
  static constexpr int N2 = BX ? 3 * R : 2 * R; // phase A N: the W terms
  static constexpr int N3 = 3 * R;              // phase B N: three H_new terms
  static constexpr int KH = R / 2;              // ranks per TMEM lane group (two per column)
  static constexpr int HALF = KH / 2;           // ranks one epilogue thread updates
  static constexpr int XST = MP * 128 * 2;      // one stage: two atoms (X1 and X2, or 128 columns of X)
  // Stage layout.  BF16 form: atom 0 (columns 0..63, MP rows of 128 bytes)
  // then atom 1.  Split form: 1024-byte groups of 8 rows alternating X1, X2
  // (row group g of X1 at 2 g KB, of X2 at 2 g + 1 KB), the image of the
  // tile-major split buffer.  XLBO: offset of the second atom's data (the M
  // step of phase A, the K step past 64 of phase B); XSBO: stride of 8-row groups.
  static constexpr int XLBO = BX ? MP * 128 : 1024;
  static constexpr int XSBO = BX ? 1024 : 2048;
  static constexpr int HATOMS = BX ? 2 : 1;     // atoms of an H_new stack (its tile's columns)
  static constexpr int HS = HATOMS * N3 * 128;  // one H_new stack: 3R rows per atom
  // Split form: two stacks (the epilogue of tile j writes one while phase B of
  // tile j - 1 reads the other).  BF16 form: one (shared memory), written once
  // phase B of the previous tile has completed.
  static constexpr int NSTK = BX ? 1 : 2;
  static constexpr int KAT = MP / 64;           // 64-row K atoms of the W operand
  static constexpr int WOP = KAT * N2 * 128;
  static constexpr int NMB = MP / 128;          // X row blocks of phase B
  static constexpr int BARB = 256;              // mbarriers and the TMEM slot
  static constexpr int FIXED = NSTK * HS + WOP + R * R * 4 + BARB + 1024;
  static constexpr int FIT = (227 * 1024 - FIXED) / XST;
  static constexpr int S = FIT < 6 ? FIT : 6;   // X stages
  static constexpr int BOXR = MP < 256 ? MP : 256; // TMA box rows (two boxes per atom at 512 rows)
  // The stacks come first: the 128-row A operand of the Q MMA reads past a
  // stack's 3R rows into the following shared memory; those rows only reach
  // TMEM lanes >= 3R, which are never read.
  static constexpr int OFF_HN = 0;
  static constexpr int OFF_X = NSTK * HS;
  static constexpr int OFF_W = OFF_X + S * XST;
  static constexpr int OFF_G = OFF_W + WOP;
  static constexpr int OFF_BAR = OFF_G + R * R * 4;
  static constexpr int SMEM = OFF_BAR + BARB + 1024;   // + alignment of the 1024-byte atoms
  static constexpr int TMEM_USED = 2 * N2 + (NMB + 1) * N3;
  static constexpr uint32_t TMEM_COLS = TMEM_USED <= 256 ? 256 : 512;
  static constexpr uint32_t IDA = idesc_bf16(128, N2, true, false);
  static constexpr uint32_t IDB = idesc_bf16(128, N3, false, false);
  static constexpr uint32_t TX = 2u * MP * 128u;   // bytes of one stage's two copies
  static_assert(((MP == 128 || MP == 256) && (R == 16 || R == 32)) || (!BX && MP == 512 && R == 16), "bucket");
  static_assert(S >= 1 && SMEM <= 227 * 1024, "shared memory");
  static_assert(TMEM_USED <= 512, "TMEM columns");
  static_assert(HS % 1024 == 0 && OFF_X % 1024 == 0 && OFF_W % 1024 == 0 && (N2 * 128) % 1024 == 0,
                "atom alignment");
  static_assert(3 * R * R * 4 <= HS && (BX || 64 * (R + 1) * 4 <= HS), "scratch in an H_new stack");
  static_assert(OFF_HN + (NSTK - 1) * HS + (HATOMS - 1) * N3 * 128 + 128 * 128 <= OFF_W,
                "Q operand rows past a stack stay in shared memory");
  static_assert(2 * 6 + 6 <= BARB / 8 - 2, "barrier slots");
};

struct TsParams {
  float* H;          // r x n FP32, updated in place
  const float* W;    // m x r
  const float* G;    // R x R
  float* part;       // grid x (MP + R) x R
  int* status;
  const int* stop;   // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r, ntiles;
  float eps;
  // split form: X1 and X2 stored tile by tile as the stages' shared-memory
  // image (split_blocked_kernel): tile t is XST contiguous bytes at xblk + t XST
  const uint8_t* xblk;
};

// Named barrier 1 over the 256 epilogue threads.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Named barrier 1 with an OR over the epilogue threads' predicates: every
// epilogue thread gets the same answer.
__device__ __forceinline__ bool epi_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, 256, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)(pred ? 1u : 0u))
      : "memory");
  return r != 0;
}

__device__ __forceinline__ int read_flag(const int* f) { return *reinterpret_cast<const volatile int*>(f); }

// KH consecutive FP32 columns of this thread's TMEM lane (no wait).
template <int KH>
__device__ __forceinline__ void tmem_ld_kh(uint32_t taddr, float* v) {
  if constexpr (KH == 16)
    tmem_ld16(taddr, v);
  else
    tmem_ld8(taddr, v);
}

// tmX1: the BF16 form's TMA map of X (64-column boxes of MP rows, 128-byte
// swizzle; rows past m and columns past n arrive as zeros); the split form
// copies p.xblk and takes no map.
template <class C>
__global__ void __launch_bounds__(kTsThreads, 1) mu_pass_tcs_kernel(const __grid_constant__ CUtensorMap tmX1,
                                                                    const TsParams p) {
  constexpr int MP = C::MP, R = C::R, N2 = C::N2, N3 = C::N3, KH = C::KH, HALF = C::HALF, S = C::S;
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

  // ---- setup: W terms (K-major B operand of phase A), G, barriers, TMEM,
  // this CTA's partial block zeroed
  // all of a thread's W loads in flight at once, then the splits
  constexpr int NWL = (MP * R + kTsThreads - 1) / kTsThreads;
  float wv[NWL];
#pragma unroll
  for (int u = 0; u < NWL; ++u) {
    const int e = tid + u * kTsThreads, i = e / R, k = e % R;
    wv[u] = (e < MP * R && i < m && k < r) ? p.W[i * r + k] : 0.0f;
  }
#pragma unroll
  for (int u = 0; u < NWL; ++u) {
    const int e = tid + u * kTsThreads;
    if (e >= MP * R) break;
    const int i = e / R, k = e % R;   // W row i (K index), rank k
    const float w = wv[u];
    __nv_bfloat16 t3[3];
    split3(w, t3);   // the split form takes the first two (16 bits, as its X)
#pragma unroll
    for (int t = 0; t < N2 / R; ++t) {
      const int nrow = t * R + k;
      const uint32_t off = (uint32_t)((i >> 6) * N2 * 128) + nrow * 128 + ((((i & 63) >> 3) ^ (nrow & 7)) << 4) +
                           ((i & 7) << 1);
      *reinterpret_cast<__nv_bfloat16*>(smem + C::OFF_W + off) = t3[t];
    }
  }
  for (int e = tid; e < R * R; e += kTsThreads) Gs[e] = p.G[e];
  float* out = p.part + (size_t)blockIdx.x * ((MP + R) * R);
  for (int e = tid; e < (MP + R) * R; e += kTsThreads) out[e] = 0.0f;
  if (tid == 0) {
    *s_err = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(barA(b), 1);
      mbar_init(epi(b), kTsEpi);
    }
    mbar_init(bdone, 1);
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  if (warp == 8) {
    tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto dA = [&](int b) { return tmem + (uint32_t)(b * N2); };
  auto dB = [&](int blk) { return tmem + (uint32_t)(2 * N2 + blk * N3); };
  auto stack_off = [&](int b) { return (uint32_t)(C::OFF_HN + (C::NSTK == 2 ? b : 0) * C::HS); };

  if (warp == 9) {
    // =========================================================== TMA thread
    if (lane == 0) {
      int t = 0;
      for (; t < count; ++t) {
        const int s = t % S;
        // the stage's previous tile (t - S) has been through phase B
        if (t >= S && !mbar_wait_bounded(empty(s), (uint32_t)(((t / S) - 1) & 1))) {
          *s_err = 1;
          break;
        }
        if (read_flag(s_err)) break;
        const int col0 = ((int)blockIdx.x + t * (int)gridDim.x) * C::TC;
        const uint32_t dst = sbase + C::OFF_X + s * C::XST;
        mbar_arrive_expect_tx(full(s), C::TX);
        if constexpr (C::BX) {
#pragma unroll
          for (int h = 0; h < MP / C::BOXR; ++h) {   // columns col0 .. col0 + 63 and col0 + 64 .. col0 + 127 of X
            tma_load_2d(dst + h * C::BOXR * 128, &tmX1, col0, h * C::BOXR, full(s));
            tma_load_2d(dst + MP * 128 + h * C::BOXR * 128, &tmX1, col0 + 64, h * C::BOXR, full(s));
          }
        } else {   // X1 and X2 of columns col0 .. col0 + 63: one contiguous copy of the tile's image
          bulk_load(dst, p.xblk + (size_t)(col0 / C::TC) * C::XST, C::XST, full(s));
        }
      }
      // every copy issued has landed before the CTA ends (the last one of each stage)
      for (int u = t - S < 0 ? 0 : t - S; u < t; ++u) (void)mbar_wait_bounded(full(u % S), (uint32_t)((u / S) & 1));
    }
  } else if (warp == 8) {
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
      // phase A of local tile t (stage s) into D_A[t & 1]: M = the 128 lanes of
      // [X1 | X2] (MN-major, LBO = the atom stride), K = the rows
      auto phase_a = [&](int t, int s) {
        const uint64_t dX = smem_desc(sbase + C::OFF_X + s * C::XST, C::XLBO, C::XSBO, kLayoutSw128);
#pragma unroll
        for (int kk = 0; kk < MP / 16; ++kk)
          mma_bf16(dA(t & 1), dX + (uint64_t)((kk * 2 * C::XSBO) >> 4),
                   dW + (uint64_t)((((kk >> 2) * N2 * 128) + (kk & 3) * 32) >> 4), C::IDA, kk > 0 ? 1u : 0u);
        mma_commit(barA(t & 1));
      };
      // phase B of local tile t: K = the 64 columns of both atoms; the X2
      // atom's K steps read the same H_new columns; Q over the first atom
      auto phase_b = [&](int t, int s) {
        const uint32_t hb = sbase + stack_off(t & 1);
        const uint32_t xb = sbase + C::OFF_X + s * C::XST;
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const uint32_t xo = (uint32_t)((kk >> 2) * C::XLBO + (kk & 3) * 32);
          const uint32_t acc = (t % C::FLUSH != 0 || kk > 0) ? 1u : 0u;
          // BF16 form: the second atom holds columns 64.., so does the stack's;
          // split form: both atoms are the same columns, Q once
          const uint32_t ha = C::BX ? (uint32_t)((kk >> 2) * N3 * 128) : 0u;
          const uint64_t dh = smem_desc(hb + ha + (kk & 3) * 32, 16, 1024, kLayoutSw128);
#pragma unroll
          for (int mb = 0; mb < C::NMB; ++mb)
            mma_bf16(dB(mb), smem_desc(xb + mb * 16 * C::XSBO + xo, 16, C::XSBO, kLayoutSw128), dh, C::IDB, acc);
          if (C::BX || kk < 4) mma_bf16(dB(C::NMB), dh, dh, C::IDB, acc);
        }
        mma_commit(empty(s));
        mma_commit(bdone);
      };
      if constexpr (S == 1) {
        // one stage: phase A of tile j after phase B of tile j - 1 has freed it
        for (int j = 0; ok && j < count; ++j) {
          if (!wait(full(0), (uint32_t)(j & 1))) break;
          tc_fence_after();
          phase_a(j, 0);
          if (!wait(epi(j & 1), (uint32_t)((j >> 1) & 1))) break;
          tc_fence_after();
          phase_b(j, 0);
          if (read_flag(s_err)) break;
        }
      } else {
        if (wait(full(0), 0u)) {
          tc_fence_after();
          phase_a(0, 0);
        }
        for (int j = 0; ok && j < count; ++j) {
          if (j + 1 < count) {
            // D_A[(j+1) & 1] was read by the epilogue of tile j - 1 (waited for below, one round earlier)
            if (!wait(full((j + 1) % S), (uint32_t)(((j + 1) / S) & 1))) break;
            tc_fence_after();
            phase_a(j + 1, (j + 1) % S);
          }
          if (!wait(epi(j & 1), (uint32_t)((j >> 1) & 1))) break;
          tc_fence_after();
          phase_b(j, j % S);
          if (read_flag(s_err)) break;
        }
      }
      // every MMA issued has completed before TMEM is released
      mma_commit(drain);
      (void)mbar_wait_bounded(drain, 0u);
    }
  } else {
    // =========================================================== epilogue
    // TMEM lane c: split form, the tile column cc = c (its X1 part) or, for
    // c >= 64, the X2 part of column c - 64; BF16 form, column c; lane group
    // kh0 .. kh0 + KH of the ranks
    const int c = (warp % 4) * 32 + lane;
    const int cc = C::BX ? c : c % 64;
    const bool owner = C::BX || c < 64;
    const bool hi = warp >= 4;
    const int kh0 = hi ? KH : 0;
    const uint32_t lane_base = (uint32_t)((warp % 4) * 32) << 16;
    // old H of a tile's column, all ranks; with rank bucket 16 one tile ahead
    // (registers), so the loads' latency overlaps the current tile
    constexpr bool PREFETCH_H = R <= 16 || C::BX;
    auto load_h = [&](int tile_, float* hv) {
      const int64_t col_ = (int64_t)tile_ * C::TC + cc;
#pragma unroll
      for (int l = 0; l < R; ++l) hv[l] = (l < r && col_ < n) ? p.H[(int64_t)l * n + col_] : 0.0f;
    };
    // split form at rank 16: two tiles ahead (the loads wait on DRAM under a
    // full copy stream; one tile of epilogue did not cover them)
    constexpr bool AHEAD2 = !C::BX && R <= 16;
    float hnext[PREFETCH_H ? R : 1], hnext2[AHEAD2 ? R : 1];
    if constexpr (PREFETCH_H) {
      if (count > 0) load_h((int)blockIdx.x, hnext);
      if constexpr (AHEAD2)
        if (count > 1) load_h((int)blockIdx.x + (int)gridDim.x, hnext2);
    }
    // rank bucket 16: the G rows of this thread's ranks in registers (their
    // shared-memory reads otherwise take a large share of the pass's
    // shared-memory bandwidth, which the MMA operands need)
    constexpr bool GREG = !C::BX && R <= 16;
    float gk[GREG ? HALF : 1][GREG ? R : 1];
    if constexpr (GREG) {
      const int kq = kh0 + (owner ? 0 : HALF);
#pragma unroll
      for (int qi = 0; qi < HALF; ++qi)
#pragma unroll
        for (int l = 0; l < R; ++l) gk[qi][l] = Gs[(kq + qi) * R + l];
    }
    // Add the finished TMEM run of D_B: P rows straight into `out` (each
    // entry owned by one thread), Q through its term rows in `qs`.
    auto flush = [&](float* qs) {
      const int row = 32 * (warp % 4) + lane;
#pragma unroll
      for (int blk = 0; blk <= C::NMB; ++blk) {
        float v0[KH], v1[KH], v2[KH];
        tmem_ld_kh<KH>(dB(blk) + lane_base + kh0, v0);
        tmem_ld_kh<KH>(dB(blk) + lane_base + R + kh0, v1);
        tmem_ld_kh<KH>(dB(blk) + lane_base + 2 * R + kh0, v2);
        tmem_wait_ld();
        if (blk < C::NMB) {
          float* o = out + (blk * 128 + row) * R + kh0;
#pragma unroll
          for (int q = 0; q < KH; ++q) o[q] += (v0[q] + v1[q]) + v2[q];
        } else if (row < N3) {
#pragma unroll
          for (int q = 0; q < KH; ++q) qs[row * R + kh0 + q] = (v0[q] + v1[q]) + v2[q];
        }
      }
      tc_fence_before();
      epi_sync();
      for (int e = tid; e < R * R; e += kTsEpi) {
        const int k = e / R, l = e % R;
        out[(MP + k) * R + l] += (qs[k * R + l] + qs[(R + k) * R + l]) + qs[(2 * R + k) * R + l];
      }
      epi_sync();
    };
    bool ok = true;
    for (int j = 0; j < count; ++j) {
      const int b = j & 1;
      const int tile = (int)blockIdx.x + j * (int)gridDim.x;
      const int64_t col = (int64_t)tile * C::TC + cc;
      uint8_t* stk = smem + stack_off(b);
      float* scratch = reinterpret_cast<float*>(stk);   // free until this tile's H_new terms are written
      bool bad = !mbar_wait_bounded(barA(b), (uint32_t)((j >> 1) & 1));
      if (bad) *s_err = 1;
      if (epi_any(bad || read_flag(s_err))) {
        ok = false;
        break;
      }
      tc_fence_after();
      float h[R];
      if constexpr (PREFETCH_H) {
#pragma unroll
        for (int l = 0; l < R; ++l) h[l] = hnext[l];
        if constexpr (AHEAD2) {
#pragma unroll
          for (int l = 0; l < R; ++l) hnext[l] = hnext2[l];
          if (j + 2 < count) load_h(tile + 2 * (int)gridDim.x, hnext2);
        } else {
          if (j + 1 < count) load_h(tile + (int)gridDim.x, hnext);
        }
      } else {
        load_h(tile, h);
      }
      if (j > 0 && j % C::FLUSH == 0) {
        // phase B of tile j - 1 ends a TMEM run (phase B of tile j starts the next)
        bad = !mbar_wait_bounded(bdone, (uint32_t)((j - 1) & 1));
        if (bad) *s_err = 1;
        if (epi_any(bad)) {
          ok = false;
          break;
        }
        tc_fence_after();
        flush(scratch);
      }
      // this lane's part of Y (the W term groups)
      float y[KH];
      {
        float v0[KH], v1[KH];
        tmem_ld_kh<KH>(dA(b) + lane_base + kh0, v0);
        tmem_ld_kh<KH>(dA(b) + lane_base + R + kh0, v1);
        if constexpr (C::BX) {
          float v2[KH];
          tmem_ld_kh<KH>(dA(b) + lane_base + 2 * R + kh0, v2);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < KH; ++q) y[q] = (v0[q] + v1[q]) + v2[q];
        } else {
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < KH; ++q) y[q] = v0[q] + v1[q];
        }
      }
      tc_fence_before();
      if constexpr (C::BX) {
        // H update of column cc at ranks kh0 + q (all of them first), then,
        // once phase B of the previous tile has released the one stack,
        // H_new to HBM and its three BF16 terms into the stack
        float hn[KH];
#pragma unroll
        for (int q = 0; q < KH; ++q) {
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
          const float hk = hi ? h[KH + q] : h[q];
          hn[q] = fmaxf(0.0f, __fdividef(hk * y[q], gh + p.eps));
        }
        if (j > 0) {
          // phase A of tile j was issued after phase B of tile j - 2: unambiguous
          bad = !mbar_wait_bounded(bdone, (uint32_t)((j - 1) & 1));
          if (bad) *s_err = 1;
          if (epi_any(bad)) {
            ok = false;
            break;
          }
        }
#pragma unroll
        for (int q = 0; q < KH; ++q) {
          const int k = kh0 + q;
          if (k < r && col < n) p.H[(int64_t)k * n + col] = hn[q];
          __nv_bfloat16 t3[3];
          split3(hn[q], t3);
#pragma unroll
          for (int t = 0; t < 3; ++t) *reinterpret_cast<__nv_bfloat16*>(stk + swz(t * R + k, cc, N3)) = t3[t];
        }
      } else {
        // Y = X1 part (lane cc) + X2 part (lane 64 + cc): the X1 lane's thread
        // updates the first HALF ranks of the group, the X2 lane's thread the
        // rest; each hands the other its part of the other half (rows of R + 1
        // floats: consecutive columns fall in different banks)
        if (owner) {
#pragma unroll
          for (int q = HALF; q < KH; ++q) scratch[cc * (R + 1) + kh0 + q] = y[q];
        } else {
#pragma unroll
          for (int q = 0; q < HALF; ++q) scratch[cc * (R + 1) + kh0 + q] = y[q];
        }
        epi_sync();
        if (owner) {
#pragma unroll
          for (int q = 0; q < HALF; ++q) y[q] += scratch[cc * (R + 1) + kh0 + q];
        } else {
#pragma unroll
          for (int q = HALF; q < KH; ++q) y[q] += scratch[cc * (R + 1) + kh0 + q];
        }
        epi_sync();   // the exchange area is the stack, written next
        // H update of column cc at this thread's ranks kh0 + Q0 + qi: all of
        // them first (independent chains), then H_new to HBM and its three BF16
        // terms into the stack
        auto update_half = [&](auto q0c) {
          constexpr int Q0 = decltype(q0c)::value;
          float hn[HALF];
#pragma unroll
          for (int qi = 0; qi < HALF; ++qi) {
            const int q = Q0 + qi;
            float gh = 0.0f;
            if constexpr (GREG) {
#pragma unroll
              for (int l = 0; l < R; ++l) gh = fmaf(gk[qi][l], h[l], gh);
            } else {
              const int k = kh0 + q;
#pragma unroll
              for (int l = 0; l < R; l += 4) {
                const float4 g = *reinterpret_cast<const float4*>(Gs + k * R + l);
                gh = fmaf(g.x, h[l], gh);
                gh = fmaf(g.y, h[l + 1], gh);
                gh = fmaf(g.z, h[l + 2], gh);
                gh = fmaf(g.w, h[l + 3], gh);
              }
            }
            const float hk = hi ? h[KH + q] : h[q];
            hn[qi] = fmaxf(0.0f, __fdividef(hk * y[q], gh + p.eps));
          }
#pragma unroll
          for (int qi = 0; qi < HALF; ++qi) {
            const int k = kh0 + Q0 + qi;
            if (k < r && col < n) p.H[(int64_t)k * n + col] = hn[qi];
            __nv_bfloat16 t3[3];
            split3(hn[qi], t3);
#pragma unroll
            for (int t = 0; t < 3; ++t) *reinterpret_cast<__nv_bfloat16*>(stk + swz(t * R + k, cc, N3)) = t3[t];
          }
        };
        if (owner)
          update_half(std::integral_constant<int, 0>{});
        else
          update_half(std::integral_constant<int, HALF>{});
      }
      fence_proxy_async_smem();
      tc_fence_before();
      mbar_arrive(epi(b));
    }
    // the last run, once every MMA has completed (the drain commit; a parity
    // wait on bdone could match an older phase: phase B of the last two tiles
    // may both be outstanding here)
    if (ok && count > 0) {
      const bool bad = !mbar_wait_bounded(drain, 0u);
      if (bad) *s_err = 1;
      if (!epi_any(bad)) {
        tc_fence_after();
        flush(reinterpret_cast<float*>(smem + stack_off(count & 1)));
      }
    }
  }
  // ---- teardown
  tc_fence_before();
  __syncthreads();
  if (read_flag(s_err)) {
    for (int e = tid; e < (MP + R) * R; e += kTsThreads) out[e] = 0.0f;
    if (tid == 0) atomicExch(p.status, kStatusTimeout);
  }
  if (warp == 8) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <class C>
cudaError_t launch_tcs_cfg(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mu_pass_tcs_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TsParams p;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.ntiles = (int)((s.n + C::TC - 1) / C::TC);
  p.eps = eps;
  p.xblk = reinterpret_cast<const uint8_t*>(d.X);
  CUtensorMap m1;
  std::memset(&m1, 0, sizeof(m1));
  if (C::BX && encode_bf16_atom_map(d.X, s.m, s.n, C::BOXR, &m1) != NTT_OK) return cudaErrorInvalidValue;
  if (!C::BX && (reinterpret_cast<uintptr_t>(d.X) & 15)) return cudaErrorInvalidValue;
  return launch_pdl(mu_pass_tcs_kernel<C>, dim3(s.grid), dim3(kTsThreads), C::SMEM, st, m1, p);
}

}  // namespace

// X (m x n FP32) -> the split form's tile-major image: tile t (64 columns),
// 8-row group g, term e (X1 = bf16(X), X2 = bf16(X - X1)) at byte
// ((t MP / 8 + g) 2 + e) 1024; row r8 of the group at r8 128, its 16-byte
// chunk c at (c ^ r8) 16 (the 128-byte swizzle of a 1024-byte-aligned atom).
// Rows past m and columns past n are zeros.
__global__ void split_blocked_kernel(const float* X, uint8_t* out, int64_t m, int64_t n, int MP, int64_t ntiles) {
  const int64_t total = ntiles * MP * 8;   // (tile, row, chunk)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int c = (int)(q & 7);
    const int64_t rowt = q >> 3;
    const int row = (int)(rowt % MP);
    const int64_t t = rowt / MP;
    const int64_t col = t * 64 + c * 8;
    float v[8];
    if (row < m && col + 8 <= n) {
      const float4 a = *reinterpret_cast<const float4*>(X + row * n + col);
      const float4 b = *reinterpret_cast<const float4*>(X + row * n + col + 4);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (row < m && col + j < n) ? X[row * n + col + j] : 0.0f;
    }
    uint32_t t1[4], t2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
      t1[j] = *reinterpret_cast<const uint32_t*>(&h);
      t2[j] = *reinterpret_cast<const uint32_t*>(&l);
    }
    const int g = row >> 3, r8 = row & 7;
    uint8_t* base = out + ((t * (MP / 8) + g) * 2) * 1024 + r8 * 128 + ((c ^ r8) << 4);
    *reinterpret_cast<uint4*>(base) = make_uint4(t1[0], t1[1], t1[2], t1[3]);
    *reinterpret_cast<uint4*>(base + 1024) = make_uint4(t2[0], t2[1], t2[2], t2[3]);
  }
}

size_t split_blocked_bytes(int64_t n, int MP) { return (size_t)((n + 63) / 64) * (size_t)MP * 256; }

// Bytes of the two BF16 terms of an FP32 X: m x n x 4, or for the split
// tensor-core form's tile-major image (128..512 rows) whole 64-column tiles of
// the padded row count.
size_t split_scratch_bytes(int64_t m, int64_t n) {
  int MP = 16;
  while (MP < m) MP *= 2;
  const size_t plain = (size_t)(m * n) * 4;
  return MP >= 128 ? std::max(plain, split_blocked_bytes(n, MP)) : plain;
}

cudaError_t launch_split_blocked(const float* X, void* out, int64_t m, int64_t n, int MP, cudaStream_t st) {
  const int64_t ntiles = (n + 63) / 64;
  const int64_t total = ntiles * MP * 8;
  int64_t grid = (total + kAuxThreads - 1) / kAuxThreads;
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  split_blocked_kernel<<<(unsigned)grid, kAuxThreads, 0, st>>>(X, reinterpret_cast<uint8_t*>(out), m, n, MP, ntiles);
  return cudaGetLastError();
}

bool tcs_pass_supported(int MP, int R) {
  return ((MP == 128 || MP == 256) && (R == 16 || R == 32)) || (MP == 512 && R == 16) || tcn_pass_supported(MP, R);
}

cudaError_t launch_mu_pass_tcs(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  if (s.MP <= 32) return launch_mu_pass_tcn(s, d, eps, st);
  if (s.MP == 128 && s.R == 16) return launch_tcs_cfg<TsCfg<128, 16>>(s, d, eps, st);
  if (s.MP == 128 && s.R == 32) return launch_tcs_cfg<TsCfg<128, 32>>(s, d, eps, st);
  if (s.MP == 256 && s.R == 16) return launch_tcs_cfg<TsCfg<256, 16>>(s, d, eps, st);
  if (s.MP == 256 && s.R == 32) return launch_tcs_cfg<TsCfg<256, 32>>(s, d, eps, st);
  if (s.MP == 512 && s.R == 16) return launch_tcs_cfg<TsCfg<512, 16>>(s, d, eps, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_mu_pass_tcbx(const MuShape& s, const MuDev& d, float eps, cudaStream_t st) {
  if (s.MP == 128 && s.R == 16) return launch_tcs_cfg<TsCfg<128, 16, true>>(s, d, eps, st);
  if (s.MP == 128 && s.R == 32) return launch_tcs_cfg<TsCfg<128, 32, true>>(s, d, eps, st);
  if (s.MP == 256 && s.R == 16) return launch_tcs_cfg<TsCfg<256, 16, true>>(s, d, eps, st);
  if (s.MP == 256 && s.R == 32) return launch_tcs_cfg<TsCfg<256, 32, true>>(s, d, eps, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
