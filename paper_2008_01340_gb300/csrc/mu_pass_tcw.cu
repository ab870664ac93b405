// Fused MU pass for FP32 X of at most 32 rows at rank bucket 8 on warp-level
// BF16 tensor-core MMAs (mma.sync m16n8k16, FP32 accumulation): the first
// unfolding of a tensor whose first mode is small (32 x 32^5 for a 32^6
// tensor, r_1 = 8).  One launch is one MU iteration step of the pass, as in
// the other passes (Algorithms 4-6, the collectives replaced by the combine
// kernel's fixed-order reduction of this kernel's per-CTA partials).
//
// X is split once per MU loop into two BF16 terms, X = X1 + X2 with
// X1 = bf16(X), X2 = bf16(X - X1), stored interleaved by 64-column segments:
// row i of the split matrix is [X1 seg 0 | X2 seg 0 | X1 seg 1 | X2 seg 1 ...],
// so one copy of a segment moves 256 contiguous bytes of every row.  In
// shared memory a stage (64 columns) holds 2 MP lines of 128 bytes, line
// L = 2 i + term, 16-byte chunks XOR L mod 8; the H box is 8 ranks x two
// 32-column halves (line 2 k + half), FP32, same swizzle.
//
// Per 16-column chunk, one warp (g = lane >> 2, t = lane & 3):
//   Y^T (16 cols x 8 ranks) = sum over the 2 MP lines  X_line^T W_row(line)
//        A = the chunk's lines transposed (ldmatrix .trans), B = W1 or W2
//        (bf16(W), bf16(W - bf16(W))) with each row's value on both of its
//        lines: the X1 + X2 sum runs inside the MMA's K
//   H_new = max(0, H o Y / (G_W H + eps)) on CUDA cores (G_W H in FP32) for
//        the lane's two columns g, g + 8 and ranks 2t, 2t + 1; stored to HBM
//        and, in place, into the stage's H box
//   P_line (16 lines x 8) += X_line H_new^T  per 16-line tile, B = the three
//        BF16 terms h1, h2, h3 of H_new (24 significand bits): P of row i is
//        the sum of its lines 2i, 2i + 1 (added once at the end)
//   Q: one MMA with A = [h1 ; h2] (the 16 rows of the MMA), B = h1, one with
//        B = h2, one with A = [h1 ; h3], B = h3; Q = the four blocks
//        h1h1 + h2h1 + h1h2 + h2h2 plus h1h3 and its transpose.
// Each warp streams its own 64-column stages through a ring of TMA copies
// (3-D tensor maps, mbarrier-tracked, bounded waits).
#include "ntt_internal.cuh"

#include <cuda_bf16.h>

namespace ntt {
namespace {

constexpr int kTwWarps = 8;
constexpr int kTwThreads = kTwWarps * 32;
constexpr int kSegCols = 64;          // columns per stage (one 128-byte BF16 line per term)

template <int MP_>
struct TwCfg {
  static constexpr int MP = MP_;
  static constexpr int LINES = 2 * MP;          // X lines per stage: (row, term)
  static constexpr int KSTEPS = LINES / 16;     // Y: K steps of 16 lines
  static constexpr int MTILES = LINES / 16;     // P: 16-line tiles
  static constexpr int XBOX = LINES * 128;
  static constexpr int HBOX = 8 * 2 * 128;      // 8 ranks x two 32-column halves
  static constexpr int STAGE = XBOX + HBOX;
  static constexpr int FIT = 220 * 1024 / kTwWarps / STAGE;
  static constexpr int S = FIT < 6 ? FIT : 6;
  static constexpr int WARP_BYTES = S * STAGE;
  static constexpr int STG_OFF = kTwWarps * WARP_BYTES;   // 1 KB H_new staging tile per warp
  static constexpr int BAR_OFF = STG_OFF + kTwWarps * 1024;
  static constexpr int E = (MP + 8) * 8;        // partial floats per CTA: P rows, then Q rows
  static constexpr int RED_FLOATS = kTwWarps * (E + 64);   // + the transposed Q block
  static constexpr int SMEM = BAR_OFF + kTwWarps * S * 8 + 1024;
  static_assert(MP == 16 || MP == 32, "row bucket");
  static_assert(STAGE % 1024 == 0 && XBOX % 1024 == 0, "swizzle atoms of 1024 bytes");
  static_assert(S >= 2, "pipeline depth");
  static_assert(RED_FLOATS * 4 <= STG_OFF, "reduction scratch");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct TwParams {
  float* H;            // r x n, updated in place
  const float* W;      // m x r
  const float* G;      // 8 x 8 Gram of W, zero padded
  float* part;         // grid x (MP + 8) x 8
  int* status;
  const int* stop;     // nullable stop word: a set word makes the launch a no-op
  int64_t n;
  int m, r;
  int nseg;            // n / 64
  float eps;
};

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// (lo, hi) -> bf16x2 (lo in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

// (x, y) = t1 + t2 + t3 with BF16 pairs t1 = bf16(x, y), t2 = bf16 of the rest, ...
__device__ __forceinline__ void split3_pair(float2 v, uint32_t* t) {
  t[0] = pack_bf16(v.x, v.y);
  const float2 a = unpack_bf16(t[0]);
  const float2 r1 = make_float2(v.x - a.x, v.y - a.y);
  t[1] = pack_bf16(r1.x, r1.y);
  const float2 b = unpack_bf16(t[1]);
  t[2] = pack_bf16(r1.x - b.x, r1.y - b.y);
}

// Compile-time part of the byte offset of H box element (i, c0 + g + 8 h)
// (line 2 i + (c0 >> 5), chunk (A ^ (2 i & 6)) + ((g >> 2) ^ half) with
// A = ((c0 & 31) >> 2) + 2 h); the lane adds ((g >> 2) ^ half) * 16 + (g & 3) * 4.
__device__ __forceinline__ constexpr int h_ct(int i, int c0, int h) {
  return (2 * i + (c0 >> 5)) * 128 + (((((c0 & 31) >> 2) + 2 * h) ^ ((2 * i) & 6)) << 4);
}

template <class C>
__global__ void __launch_bounds__(kTwThreads, 1)
mu_pass_tcw_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                   const TwParams p) {
  constexpr int S = C::S, KS = C::KSTEPS, MT = C::MTILES;
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  uint8_t* wbuf = smem + warp * C::WARP_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF) + warp * S;

  if (lane == 0) {
    if (warp == 0) {
      prefetch_tensormap(&tmX);
      prefetch_tensormap(&tmH);
    }
    for (int s = 0; s < S; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
  }
  // B fragments of W for Y: K step ks covers lines 16 ks .. 16 ks + 15 = rows
  // 8 ks .. 8 ks + 7 (both terms); b0 holds lines 16 ks + 2t, + 2t + 1 (row
  // 8 ks + t twice), b1 lines + 2t + 8, + 2t + 9 (row 8 ks + 4 + t), column g.
  uint32_t bw[KS][2][2];   // [ks][W term][b0, b1]
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = 8 * ks + 4 * h + t;
      const float w = (row < p.m && g < p.r) ? p.W[row * p.r + g] : 0.0f;
      const float w1 = __bfloat162float(__float2bfloat16_rn(w));
      const float w2 = w - w1;
      bw[ks][0][h] = pack_bf16(w1, w1);
      bw[ks][1][h] = pack_bf16(w2, w2);
    }
  // G_W entries (2t, i) and (2t + 1, i), each as a pair for the lane's two columns
  float2 ge[8], go[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float a = p.G[(2 * t) * 8 + i], b = p.G[(2 * t + 1) * 8 + i];
    ge[i] = make_float2(a, a);
    go[i] = make_float2(b, b);
  }
  __syncthreads();

  const int gw = blockIdx.x * kTwWarps + warp;
  const int gstride = gridDim.x * kTwWarps;
  auto issue = [&](int s, int seg) {
    const uint32_t bar = smem_u32(&bars[s]);
    const uint32_t dst = smem_u32(wbuf + s * C::STAGE);
    mbar_arrive_expect_tx(bar, C::STAGE);
    tma_load_3d(dst, &tmX, 0, 2 * seg, 0, bar);
    tma_load_3d(dst + C::XBOX, &tmH, 0, 2 * seg, 0, bar);
  };
  int issued = 0;
  if (lane == 0)
    for (int s = 0; s < S; ++s) {
      const int seg = gw + s * gstride;
      if (seg < p.nseg) {
        issue(s, seg);
        ++issued;
      }
    }

  // MMA accumulators of one stage, and their sums over the stages (FP32
  // additions rounded to nearest).  One MMA accumulation chain over a warp's
  // whole column range (27,000 stages' worth on 32 x 33,554,432) put the
  // stage's Gram-form objective 27% away from its direct FP64 residual; with
  // the per-stage sums the two agree as on the other passes.
  float accP[MT][4], sumP[MT][4];
  float accQa[4], accQb[4], sumQa[4], sumQb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    accQa[i] = accQb[i] = sumQa[i] = sumQb[i] = 0.0f;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) accP[mt][i] = sumP[mt][i] = 0.0f;
  }
  const float eps = p.eps;
  // ldmatrix lane roles: matrix j = lane >> 3, its row i = lane & 7.  The
  // lane's row is line 16 x + li + 8 (lj >> 1) (Y, transposed) or
  // 16 x + li + 8 (lj & 1) (P); line mod 8 = li, so the 16-byte chunk of
  // columns 8 (2 ck) + 8 (lj & 1) (Y) is 2 ck ^ li ^ (lj & 1).
  const int lj = lane >> 3, li = lane & 7;
  const uint32_t ly = (uint32_t)((li + 8 * (lj >> 1)) * 128), lamy = (uint32_t)(li ^ (lj & 1));
  const uint32_t lp = (uint32_t)((li + 8 * (lj & 1)) * 128), lamp = (uint32_t)(li ^ (lj >> 1));
  // H box element (i, c0 + g + 8 h): line 2 i + half (half = c0 >> 5), chunk
  // (A ^ (2 i & 6)) + ((g >> 2) ^ half) with A = ((c0 & 31) >> 2) + 2 h, word
  // g & 3: a compile-time part (h_ct) and the lane's part for half = 0, 1
  const uint32_t hq0 = (uint32_t)(((g >> 2) << 4) + (g & 3) * 4);
  const uint32_t hq1 = (uint32_t)((((g >> 2) ^ 1) << 4) + (g & 3) * 4);
  // the warp's H_new staging tile: word (rank, col) at rank * 32 + (col ^ 8 pi(rank)),
  // pi(k) = (k & 3) ^ (k >> 2): the lane's four stores (ranks 2t + e, columns
  // g + 8 h) and its two B-fragment loads (rank g, columns 2t + 8 h, + 1) each
  // cover the 32 banks once
  float* stw = reinterpret_cast<float*>(smem + C::STG_OFF + warp * 1024);
  auto pi = [](int kk) { return (kk & 3) ^ (kk >> 2); };
  int sto[2][2], ldo[2];
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int h = 0; h < 2; ++h) sto[e][h] = (2 * t + e) * 32 + ((g + 8 * h) ^ (8 * pi(2 * t + e)));
#pragma unroll
  for (int h = 0; h < 2; ++h) ldo[h] = g * 32 + ((2 * t + 8 * h) ^ (8 * pi(g)));
  float* Hr0 = p.H + (int64_t)(2 * t) * p.n;
  float* Hr1 = p.H + (int64_t)(2 * t + 1) * p.n;
  const bool w0 = 2 * t < p.r, w1 = 2 * t + 1 < p.r;

  bool err = false;
  int k = 0;
  for (int seg = gw; seg < p.nseg; seg += gstride, ++k) {
    const int s = k % S;
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((k / S) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      err = true;
      break;
    }
    const uint8_t* xs = wbuf + s * C::STAGE;
    const uint8_t* hs = xs + C::XBOX;
    const uint32_t xs_u = smem_u32(xs);
#pragma unroll
    for (int ck = 0; ck < kSegCols / 16; ++ck) {
      const int c0 = ck * 16;
      // ---- Y^T = X^T W over the 2 MP lines, W1 and W2 in two chains
      float y1[4] = {0.f, 0.f, 0.f, 0.f}, y2[4] = {0.f, 0.f, 0.f, 0.f};
      const uint32_t xy = ((uint32_t)(2 * ck) ^ lamy) << 4;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        uint32_t a[4];
        ldsm_x4_t(xs_u + ks * 2048 + ly + xy, a);
        mma16816(y1, a, bw[ks][0][0], bw[ks][0][1]);
        mma16816(y2, a, bw[ks][1][0], bw[ks][1][1]);
      }
      // ---- H update of (cols ca = c0 + g, cb = c0 + g + 8) x (ranks 2t, 2t + 1)
      const uint8_t* hb = hs + ((c0 >> 5) ? hq1 : hq0);
      float2 hp[8];   // (H[i][ca], H[i][cb])
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        hp[i].x = *reinterpret_cast<const float*>(hb + h_ct(i, c0, 0));
        hp[i].y = *reinterpret_cast<const float*>(hb + h_ct(i, c0, 1));
      }
      float2 gk0 = make_float2(0.f, 0.f), gk1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        gk0 = __ffma2_rn(ge[i], hp[i], gk0);   // (G H)[2t][ca, cb]
        gk1 = __ffma2_rn(go[i], hp[i], gk1);   // (G H)[2t + 1][ca, cb]
      }
      const float2 h0e = t == 0 ? hp[0] : (t == 1 ? hp[2] : (t == 2 ? hp[4] : hp[6]));
      const float2 h0o = t == 0 ? hp[1] : (t == 1 ? hp[3] : (t == 2 ? hp[5] : hp[7]));
      // D layout: y[0] = (col ca, rank 2t), y[1] = (ca, 2t + 1), y[2] = (cb, 2t), y[3] = (cb, 2t + 1)
      const float na0 = fmaxf(0.0f, __fdividef(h0e.x * (y1[0] + y2[0]), gk0.x + eps));
      const float na1 = fmaxf(0.0f, __fdividef(h0o.x * (y1[1] + y2[1]), gk1.x + eps));
      const float nb0 = fmaxf(0.0f, __fdividef(h0e.y * (y1[2] + y2[2]), gk0.y + eps));
      const float nb1 = fmaxf(0.0f, __fdividef(h0o.y * (y1[3] + y2[3]), gk1.y + eps));
      const int64_t gcol = (int64_t)seg * kSegCols + c0 + g;   // n % 64 == 0: in range
      if (w0) {
        Hr0[gcol] = na0;
        Hr0[gcol + 8] = nb0;
      }
      if (w1) {
        Hr1[gcol] = na1;
        Hr1[gcol + 8] = nb1;
      }
      __syncwarp();   // the previous chunk's fragment loads from the tile are done
      stw[sto[0][0]] = na0;
      stw[sto[1][0]] = na1;
      stw[sto[0][1]] = nb0;
      stw[sto[1][1]] = nb1;
      __syncwarp();
      // ---- B fragments of H_new^T (K = the chunk's 16 columns, N = rank g),
      // each split in three BF16 terms
      uint32_t hb0[3], hb1[3];
      split3_pair(*reinterpret_cast<const float2*>(stw + ldo[0]), hb0);
      split3_pair(*reinterpret_cast<const float2*>(stw + ldo[1]), hb1);
      // ---- P_line += X_line H_new^T per 16-line tile
      const uint32_t xp = ((uint32_t)(2 * ck) ^ lamp) << 4;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t a[4];
        ldsm_x4(xs_u + mt * 2048 + lp + xp, a);
#pragma unroll
        for (int h = 0; h < 3; ++h) mma16816(accP[mt], a, hb0[h], hb1[h]);
      }
      // ---- Q blocks
      {
        const uint32_t a12[4] = {hb0[0], hb0[1], hb1[0], hb1[1]};
        const uint32_t a13[4] = {hb0[0], hb0[2], hb1[0], hb1[2]};
        mma16816(accQa, a12, hb0[0], hb1[0]);
        mma16816(accQa, a12, hb0[1], hb1[1]);
        mma16816(accQb, a13, hb0[2], hb1[2]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      sumQa[i] += accQa[i];
      sumQb[i] += accQb[i];
      accQa[i] = accQb[i] = 0.0f;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        sumP[mt][i] += accP[mt][i];
        accP[mt][i] = 0.0f;
      }
    }
    __syncwarp();   // every lane is done with this stage
    if (lane == 0) {
      const int next = seg + S * gstride;
      if (next < p.nseg) {
        fence_proxy_async_smem();
        issue(s, next);
        ++issued;
      }
    }
  }

  if (err && lane == 0) {
    for (int c = k; c < issued; ++c)
      (void)mbar_wait_bounded(smem_u32(&bars[c % S]), (uint32_t)((c / S) & 1));
    atomicExch(p.status, kStatusTimeout);
  }
  __syncthreads();   // every stage buffer is free: reuse it for the reduction

  // per warp: P rows (the two lines of a row summed: lanes g, g ^ 1), the Q
  // block sums and the h1 h3 block (added transposed below)
  float* red = reinterpret_cast<float*>(smem);
  constexpr int E = C::E;
  float* rw = red + warp * (E + 64);
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float v = sumP[mt][q] + __shfl_xor_sync(0xffffffffu, sumP[mt][q], 4);
      // q: (line g or g + 8, rank 2t + (q & 1)); line 16 mt + g + 8 (q >> 1) is row that / 2
      if ((g & 1) == 0) rw[((16 * mt + g + 8 * (q >> 1)) >> 1) * 8 + 2 * t + (q & 1)] = v;
    }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    rw[(C::MP + g) * 8 + 2 * t + q] = sumQa[q] + sumQa[2 + q] + sumQb[q];
    rw[E + g * 8 + 2 * t + q] = sumQb[q];
  }
  __syncthreads();
  float* out = p.part + (size_t)blockIdx.x * E;
  for (int e = tid; e < E; e += kTwThreads) {
    float v = 0.0f;
    if (e < C::MP * 8) {
#pragma unroll
      for (int wi = 0; wi < kTwWarps; ++wi) v += red[wi * (E + 64) + e];
    } else {
      const int kq = (e - C::MP * 8) >> 3, lq = e & 7;
#pragma unroll
      for (int wi = 0; wi < kTwWarps; ++wi)
        v += red[wi * (E + 64) + e] + red[wi * (E + 64) + E + lq * 8 + kq];
    }
    out[e] = v;
  }
}

// X (m x n FP32) -> the interleaved split matrix (m x 2n BF16): row i, 64-column
// segment sg holds bf16(X) of its columns, then bf16(X - bf16(X)).
__global__ void split_x12_kernel(const float* X, __nv_bfloat16* out, int64_t m, int64_t n) {
  const int64_t groups = m * (n / 8);   // 8 columns per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < groups; q += stride) {
    const int64_t row = q / (n / 8), c8 = (q % (n / 8)) * 8;
    const float4 v0 = *reinterpret_cast<const float4*>(X + row * n + c8);
    const float4 v1 = *reinterpret_cast<const float4*>(X + row * n + c8 + 4);
    const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    uint32_t t1[4], t2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      t1[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
      const float2 a = unpack_bf16(t1[j]);
      t2[j] = pack_bf16(v[2 * j] - a.x, v[2 * j + 1] - a.y);
    }
    const int64_t sg = c8 / kSegCols, c = c8 % kSegCols;
    __nv_bfloat16* base = out + row * 2 * n + sg * 2 * kSegCols + c;
    *reinterpret_cast<uint4*>(base) = make_uint4(t1[0], t1[1], t1[2], t1[3]);
    *reinterpret_cast<uint4*>(base + kSegCols) = make_uint4(t2[0], t2[1], t2[2], t2[3]);
  }
}

template <class C>
cudaError_t launch_tcw_cfg(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                           const CUtensorMap& mh, cudaStream_t st) {
  static bool attr_set = false;   // per-function attribute; set once per process
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mu_pass_tcw_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TwParams p;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.nseg = (int)(s.n / kSegCols);
  p.eps = eps;
  return launch_pdl(mu_pass_tcw_kernel<C>, dim3(s.grid), dim3(kTwThreads), C::SMEM, st, mx, mh, p);
}

}  // namespace

bool tcw_pass_supported(int MP, int R, int64_t n) { return (MP == 16 || MP == 32) && R == 8 && n % 64 == 0; }

cudaError_t launch_split_x12(const float* X, __nv_bfloat16* out, int64_t m, int64_t n, cudaStream_t st) {
  if (n % 64 != 0) return cudaErrorInvalidValue;
  const int64_t groups = m * (n / 8);
  int64_t grid = (groups + kAuxThreads - 1) / kAuxThreads;
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  split_x12_kernel<<<(unsigned)grid, kAuxThreads, 0, st>>>(X, out, m, n);
  return cudaGetLastError();
}

cudaError_t launch_mu_pass_tcw(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                               const CUtensorMap& mh, cudaStream_t st) {
  if (s.R != 8 || s.n % 64 != 0) return cudaErrorInvalidValue;
  if (s.MP == 32) return launch_tcw_cfg<TwCfg<32>>(s, d, eps, mx, mh, st);
  if (s.MP == 16) return launch_tcw_cfg<TwCfg<16>>(s, d, eps, mx, mh, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
