// Grouped multiplicative-update pass: one launch advances many independent
// NMF problems by one iteration's H half and the (P, Q) partials of its W half.
//
// Every problem is an NMF X ~ W H with X m x n (row stride n) and re ranks;
// its ranks form diagonal blocks of size blk (blk = re for a single NMF,
// blk = r for g restarts of rank r solved side by side, re = g r), and the
// Gram matrices W^T W and H H^T are kept only on those blocks -- the only
// coupling between the columns of W, so each block is its own NMF.
//
// Per column tile of T columns (the fused single-read scheme of the Lee-Seung
// order, H first, then W from the new H):
//   Y   = W^T X_tile,   GH = G_W H_tile  (G_W restricted to the blocks)
//   H  <- max(0, H o Y / (GH + eps))                      (in place in HBM)
//   P  += X_tile H^T,   Q += H H^T       (Q on the diagonal blocks only)
// P and Q leave the CTA as one partial per CTA; the grouped combine kernel
// sums them in a fixed order and updates W and G_W (mu_group.cu).
//
// Layout in shared memory (floats): a ring of STAGES tiles, each MP rows of X
// then R rows of H with row stride LDX = T + 4 (the 4-float pad puts
// consecutive rows in different bank groups); H_new transposed (T x (R + 4));
// W (MP x R) and G (R x R) zero padded.  Tiles arrive by cp.async (16-byte
// copies when rows are 16-byte aligned, 4-byte copies otherwise) with zero
// fill past n; rows past m and re are never written and stay zero.
//
// Thread roles (256 threads):
//   phase A  thread = (4-rank group, 4-column group, row split): a 4 x 4
//            register tile of Y over its rows and, in split 0, of GH over the
//            rank block(s) of its 4 ranks; split 0 then forms H_new.
//   phase B  thread = (4 x 4 output tile of [P ; Q], column group): P tiles
//            take rows a, a + Ra, a + 2Ra, a + 3Ra (Ra = ceil(m / 4), so a
//            warp's rows are consecutive) and ranks 4b..4b+3; Q tiles are the
//            4 x 4 rank tiles that meet a diagonal block.
#pragma once

#include "group_engine.cuh"

namespace ntt {

__host__ __device__ constexpr int gmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int gmax(int a, int b) { return a > b ? a : b; }

template <int MP_, int R_, bool XB_ = false>
struct GCfg {
  static constexpr int MP = MP_;
  static constexpr int R = R_;
  static constexpr bool XB = XB_;                 // X rows in BF16 (H stays FP32)
  static constexpr int NT = 256;
  static constexpr int T = gmax(16, gmin(4096 / R, 8192 / MP));
  static constexpr int LDX = T + 4;               // H rows (floats)
  // X rows: T + 4 floats, or T + 8 BF16 values; both a 16-byte pad, in float units
  static constexpr int XLD = XB ? T / 2 + 4 : T + 4;
  static constexpr int LDH = R + 4;            // H_new^T row stride
  static constexpr int RQ = R / 4;
  static constexpr int CQ = T / 4;
  static constexpr int NA = RQ * CQ;            // phase-A threads per row split
  static constexpr int SA = NT / NA;            // row splits
  static constexpr int MS = MP + R;
  static constexpr int NTB_MAX = (MP / 4) * RQ + RQ * RQ;
  static constexpr int TPB = (NTB_MAX + NT - 1) / NT;   // phase-B tiles per thread (max)
  static constexpr bool PAIR = TPB <= 2;
  static constexpr int STAGE_FLOATS = MP * XLD + R * LDX;
  static constexpr int HNT_FLOATS = T * LDH;
  static constexpr int W_FLOATS = MP * R;
  static constexpr int G_FLOATS = R * R;
  static constexpr int YP_FLOATS = (SA - 1) * R * T;
  static constexpr int FIXED_BYTES = 4 * (HNT_FLOATS + W_FLOATS + G_FLOATS + YP_FLOATS) + 4 * RQ * RQ + 256;
  static constexpr int SMEM_CAP = 227 * 1024 - 1024;
  // two CTAs per SM (16 warps) when two ring stages fit in half the SM's shared memory
  static constexpr int SMEM_CAP2 = 113 * 1024 - 1024;
  static constexpr bool TWO = FIXED_BYTES + 2 * 4 * STAGE_FLOATS <= SMEM_CAP2;
  static constexpr int MINB = TWO ? 2 : 1;
  static constexpr int STAGES = gmin(3, ((TWO ? SMEM_CAP2 : SMEM_CAP) - FIXED_BYTES) / (4 * STAGE_FLOATS));
  static constexpr int SMEM = 4 * STAGES * STAGE_FLOATS + FIXED_BYTES;
  // end-of-CTA reduction scratch, from the ring on: [P ; Q] (MS x R) + column-group partials
  static constexpr int RED_FLOATS = MS * R + NT * 16;

  static_assert(R % 8 == 0 && R <= 32 && MP % 16 == 0 && T % 8 == 0, "bucket");
  static_assert(NA <= NT && NT % NA == 0 && MP % SA == 0, "phase A mapping");
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(SMEM <= SMEM_CAP, "shared memory");
  // the scratch may run into the H_new buffer, which follows the ring and is free by then
  static_assert(RED_FLOATS <= STAGES * STAGE_FLOATS + HNT_FLOATS, "reduction scratch");
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ float f4c(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Four consecutive X values of row `row` from column c (c % 4 == 0) of a ring
// stage: FP32 rows of XLD floats, or BF16 rows of 2 XLD values widened exactly.
template <class C>
__device__ __forceinline__ float4 ldx4(const float* Xs, int row, int c) {
  if constexpr (C::XB) {
    const uint2 u = *reinterpret_cast<const uint2*>(reinterpret_cast<const char*>(Xs) +
                                                    (size_t)row * C::XLD * 4 + (size_t)c * 2);
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                       __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
  } else {
    return *reinterpret_cast<const float4*>(Xs + row * C::XLD + c);
  }
}

// MODE 0: the fused pass.  MODE 1 (tall unfoldings, one CTA group per row
// block): phase A only, the block's partial Y written to P.Y.  MODE 2: phase B
// only, on the updated H read back from HBM; Q only where P.hasq.
template <class C, int MODE>
__global__ void __launch_bounds__(256, C::MINB)
gpass_kernel(const GProb* __restrict__ probs, const int* __restrict__ cta_prob, float eps) {
  constexpr int T = C::T, R = C::R, MP = C::MP, NT = C::NT, LDX = C::LDX, LDH = C::LDH;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* ring = smem;                                         // STAGES x STAGE_FLOATS
  float* Hnt = ring + C::STAGES * C::STAGE_FLOATS;            // T x LDH
  float* Ws = Hnt + C::HNT_FLOATS;                            // MP x R
  float* Gs = Ws + C::W_FLOATS;                               // R x R
  float* Yp = Gs + C::G_FLOATS;                               // (SA-1) x R x T
  int* qlist = reinterpret_cast<int*>(Yp + C::YP_FLOATS);     // <= RQ*RQ
  __shared__ int s_nq;

  const int tid = threadIdx.x;
  const GProb P = probs[cta_prob[blockIdx.x]];
  const int slot = blockIdx.x - P.cta0;
  const int m = P.m, re = P.re, blk = P.blk;
  const int64_t n = P.n;
  const int ntiles = (int)((n + T - 1) / T);

  // ---- CTA setup: zero the ring, load W and G, list the Q tiles that meet a block
  for (int i = tid; i < C::STAGES * C::STAGE_FLOATS / 4; i += NT)
    reinterpret_cast<float4*>(ring)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < MP * R; e += NT) {
    const int i = e / R, k = e % R;
    Ws[e] = (i < m && k < re) ? P.W[i * re + k] : 0.0f;
  }
  for (int e = tid; e < R * R; e += NT) Gs[e] = P.G[e];
  const int rqe = (re + 3) / 4;   // rank groups in use
  if (tid == 0) {
    int nq = 0;
    if (MODE != 1 && P.hasq)
    for (int a = 0; a < rqe; ++a)
      for (int b = 0; b < rqe; ++b) {
        const int a0 = 4 * a / blk, a1 = (gmin(4 * a + 4, re) - 1) / blk;
        const int b0 = 4 * b / blk, b1 = (gmin(4 * b + 4, re) - 1) / blk;
        if (a0 <= b1 && b0 <= a1) qlist[nq++] = a * C::RQ + b;
      }
    s_nq = nq;
  }
  __syncthreads();

  // ---- tile loader: rows < m of X and < re of H, T columns from col0, zero fill past n
  auto issue = [&](int stage, int tile) {
    float* dstb = ring + stage * C::STAGE_FLOATS;
    const int64_t col0 = (int64_t)tile * T;
    const int rows = m + (MODE == 1 ? 0 : re);
    if constexpr (C::XB) {
      // BF16 X rows (8 values per 16-byte copy; rows 16-byte aligned, checked on the host)
      constexpr int CQB = T / 8;
      for (int e = tid; e < m * CQB; e += NT) {
        const int row = e / CQB, ch = e % CQB;
        const int64_t col = col0 + 8 * ch;
        const int64_t left = n - col;
        const int bytes = left >= 8 ? 16 : (left > 0 ? (int)left * 2 : 0);
        const char* src = reinterpret_cast<const char*>(P.X) + ((int64_t)row * n + (bytes ? col : 0)) * 2;
        cp_async16(smem_u32(reinterpret_cast<char*>(dstb) + (size_t)row * C::XLD * 4 + 16 * ch), src, bytes);
      }
      if constexpr (MODE != 1)
        for (int e = tid; e < re * C::CQ; e += NT) {
          const int k = e / C::CQ, ch = e % C::CQ;
          const int64_t col = col0 + 4 * ch;
          const int64_t left = n - col;
          const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
          const float* src = P.H + (int64_t)k * n;
          cp_async16(smem_u32(dstb + MP * C::XLD + k * LDX + 4 * ch), bytes ? src + col : src, bytes);
        }
    } else if (P.aligned) {
      for (int e = tid; e < rows * C::CQ; e += NT) {
        const int row = e / C::CQ, ch = e % C::CQ;
        const int64_t col = col0 + 4 * ch;
        const int64_t left = n - col;
        const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
        const float* src = row < m ? reinterpret_cast<const float*>(P.X) + (int64_t)row * n
                                   : P.H + (int64_t)(row - m) * n;
        const int srow = row < m ? row : MP + row - m;
        cp_async16(smem_u32(dstb + srow * LDX + 4 * ch), bytes ? src + col : src, bytes);
      }
    } else {
      for (int e = tid; e < rows * T; e += NT) {
        const int row = e / T, c = e % T;
        const int64_t col = col0 + c;
        const int bytes = col < n ? 4 : 0;
        const float* src = row < m ? reinterpret_cast<const float*>(P.X) + (int64_t)row * n
                                   : P.H + (int64_t)(row - m) * n;
        const int srow = row < m ? row : MP + row - m;
        cp_async4(smem_u32(dstb + srow * LDX + c), bytes ? src + col : src, bytes);
      }
    }
  };

  // ---- phase-A role
  const int ua = tid % C::NA, sa = tid / C::NA;
  const int kq = ua % C::RQ, cq = ua / C::RQ;
  const int k0 = 4 * kq, c0 = 4 * cq;
  int glo = 0, ghi = 0;   // rank range of the GH contraction for ranks k0..k0+3
  if (k0 < re) {
    glo = (k0 / blk) * blk;
    ghi = gmin(re, ((gmin(k0 + 3, re - 1) / blk) + 1) * blk);
  }
  // Row splits share the m X rows and the G H rows evenly: splits before the
  // last take q X rows each, the last split the remaining X rows plus all G H
  // rows, and it also sums the others' partial Y (in split order) and forms H_new.
  const bool last = sa == C::SA - 1;
  const int gk = MODE == 0 ? ghi - glo : 0;
  const int qa = (m + gk + C::SA - 1) / C::SA;
  const int ia0 = gmin(m, sa * qa);
  const int ia1 = last ? m : gmin(m, (sa + 1) * qa);

  // ---- phase-B role
  const int ra = (m + 3) / 4;                 // P row groups (strided rows)
  const int np = ra * rqe;
  const int ntb = np + s_nq;
  const int cg = gmax(1, gmin(NT / ntb, C::CQ));   // column groups: chunks q, q + cg, ...
  const int qB = tid / ntb;                   // column group (cg > 1), else 0
  constexpr int NACC = C::PAIR ? 2 : 4;
  float2 accp[C::TPB][4][2];
  float accs[C::PAIR ? 1 : C::TPB][4][4];
#pragma unroll
  for (int t = 0; t < C::TPB; ++t)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      accp[t][i][0] = accp[t][i][1] = make_float2(0.f, 0.f);
      if constexpr (!C::PAIR)
#pragma unroll
        for (int j = 0; j < 4; ++j) accs[t][i][j] = 0.f;
    }
  (void)NACC;

  // ---- pipeline: STAGES - 1 tiles in flight ahead of the one being computed
#pragma unroll 1
  for (int s = 0; s < C::STAGES - 1; ++s) {
    const int tile = slot + s * P.S;
    if (tile < ntiles) issue(s, tile);
    cp_async_commit();
  }
  int it = 0;
#pragma unroll 1
  for (int tile = slot; tile < ntiles; tile += P.S, ++it) {
    {
      const int nt = tile + (C::STAGES - 1) * P.S;
      if (nt < ntiles) issue((it + C::STAGES - 1) % C::STAGES, nt);
      cp_async_commit();
    }
    cp_async_wait<C::STAGES - 1>();
    __syncthreads();
    const float* Xs = ring + (it % C::STAGES) * C::STAGE_FLOATS;
    const float* Hs = Xs + MP * C::XLD;
    const int64_t col0 = (int64_t)tile * T;

    // ---------------- phase A: Y (and GH in the last split) as 4 x 4 register tiles
    if constexpr (MODE == 2) {
      // H already updated in HBM: transpose its tile into H_new^T
      if (last)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          *reinterpret_cast<float4*>(Hnt + (c0 + cc) * LDH + k0) =
              make_float4(Hs[(k0 + 0) * LDX + c0 + cc], Hs[(k0 + 1) * LDX + c0 + cc],
                          Hs[(k0 + 2) * LDX + c0 + cc], Hs[(k0 + 3) * LDX + c0 + cc]);
      __syncthreads();
    } else {
    float2 ay[4][2], ag[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) ay[i][0] = ay[i][1] = ag[i][0] = ag[i][1] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int i = ia0; i < ia1; ++i) {
      const float4 w = *reinterpret_cast<const float4*>(Ws + i * R + k0);
      const float4 x = ldx4<C>(Xs, i, c0);
      const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float wk = f4c(w, kk);
        const float2 ww = make_float2(wk, wk);
        ay[kk][0] = __ffma2_rn(ww, x01, ay[kk][0]);
        ay[kk][1] = __ffma2_rn(ww, x23, ay[kk][1]);
      }
    }
    if (MODE == 0 && last) {
#pragma unroll 4
      for (int l = glo; l < ghi; ++l) {
        const float4 g = *reinterpret_cast<const float4*>(Gs + l * R + k0);
        const float4 h = *reinterpret_cast<const float4*>(Hs + l * LDX + c0);
        const float2 h01 = make_float2(h.x, h.y), h23 = make_float2(h.z, h.w);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const float gk = f4c(g, kk);
          const float2 gg = make_float2(gk, gk);
          ag[kk][0] = __ffma2_rn(gg, h01, ag[kk][0]);
          ag[kk][1] = __ffma2_rn(gg, h23, ag[kk][1]);
        }
      }
    }
    if constexpr (C::SA > 1) {
      if (!last)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          *reinterpret_cast<float4*>(Yp + (sa * R + k0 + kk) * T + c0) =
              make_float4(ay[kk][0].x, ay[kk][0].y, ay[kk][1].x, ay[kk][1].y);
      __syncthreads();
      if (last) {
        // Y = (partial of split 0 + ... + split SA-2) + own partial, in that order
        float4 acc[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) acc[kk] = *reinterpret_cast<const float4*>(Yp + (k0 + kk) * T + c0);
        for (int s2 = 1; s2 < C::SA - 1; ++s2)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const float4 v = *reinterpret_cast<const float4*>(Yp + (s2 * R + k0 + kk) * T + c0);
            acc[kk].x += v.x;
            acc[kk].y += v.y;
            acc[kk].z += v.z;
            acc[kk].w += v.w;
          }
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          ay[kk][0].x += acc[kk].x;
          ay[kk][0].y += acc[kk].y;
          ay[kk][1].x += acc[kk].z;
          ay[kk][1].y += acc[kk].w;
        }
      }
    }
    if (MODE == 1 && last) {
      // partial Y of this row block to HBM, ranks < re, columns < n
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        if (k >= re) break;
        float* dst = P.Y + (int64_t)k * n + col0 + c0;
        const int64_t left = n - (col0 + c0);
        const float y[4] = {ay[kk][0].x, ay[kk][0].y, ay[kk][1].x, ay[kk][1].y};
        if (P.aligned && left >= 4) {
          *reinterpret_cast<float4*>(dst) = make_float4(y[0], y[1], y[2], y[3]);
        } else {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            if (cc < left) dst[cc] = y[cc];
        }
      }
    }
    if (MODE == 0 && last) {
      float hn[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 h = *reinterpret_cast<const float4*>(Hs + (k0 + kk) * LDX + c0);
        const float y[4] = {ay[kk][0].x, ay[kk][0].y, ay[kk][1].x, ay[kk][1].y};
        const float d[4] = {ag[kk][0].x, ag[kk][0].y, ag[kk][1].x, ag[kk][1].y};
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
          hn[kk][cc] = fmaxf(0.0f, __fdividef(f4c(h, cc) * y[cc], d[cc] + eps));
      }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
        *reinterpret_cast<float4*>(Hnt + (c0 + cc) * LDH + k0) =
            make_float4(hn[0][cc], hn[1][cc], hn[2][cc], hn[3][cc]);
      // H_new to HBM, ranks < re, columns < n
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const int k = k0 + kk;
        if (k >= re) break;
        float* dst = P.H + (int64_t)k * n + col0 + c0;
        const int64_t left = n - (col0 + c0);
        if (P.aligned && left >= 4) {
          *reinterpret_cast<float4*>(dst) = make_float4(hn[kk][0], hn[kk][1], hn[kk][2], hn[kk][3]);
        } else {
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            if (cc < left) dst[cc] = hn[kk][cc];
        }
      }
    }
    __syncthreads();
    }

    // ---------------- phase B: [P ; Q] += [X ; H_new] H_new^T on 4 x 4 tiles
    if (MODE != 1 && qB < cg) {
#pragma unroll
      for (int t = 0; t < C::TPB; ++t) {
        const int j = (cg > 1) ? (tid % ntb) : (tid + t * NT);
        if ((cg > 1 && t > 0) || j >= ntb) break;
        const bool isP = j < np;
        int a, b;
        if (isP) {
          a = j / rqe;
          b = j % rqe;
        } else {
          const int q = qlist[j - np];
          a = q / C::RQ;
          b = q % C::RQ;
        }
#pragma unroll 2
        for (int c = 4 * qB; c < T; c += 4 * cg) {
          float4 bv[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) bv[cc] = *reinterpret_cast<const float4*>(Hnt + (c + cc) * LDH + 4 * b);
          float av[4][4];   // av[i][cc]
          if (isP) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 x = ldx4<C>(Xs, a + i * ra, c);
              av[i][0] = x.x;
              av[i][1] = x.y;
              av[i][2] = x.z;
              av[i][3] = x.w;
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const float4 h = *reinterpret_cast<const float4*>(Hnt + (c + cc) * LDH + 4 * a);
              av[0][cc] = h.x;
              av[1][cc] = h.y;
              av[2][cc] = h.z;
              av[3][cc] = h.w;
            }
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              if constexpr (C::PAIR) {
                const float2 aa = make_float2(av[i][cc], av[i][cc]);
                accp[t][i][0] = __ffma2_rn(aa, make_float2(bv[cc].x, bv[cc].y), accp[t][i][0]);
                accp[t][i][1] = __ffma2_rn(aa, make_float2(bv[cc].z, bv[cc].w), accp[t][i][1]);
              } else {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) accs[t][i][jj] = fmaf(av[i][cc], f4c(bv[cc], jj), accs[t][i][jj]);
              }
            }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  __syncthreads();
  if constexpr (MODE == 1) return;

  // ---------------- CTA reduction: [P ; Q] (MS x R) in the ring, column groups in fixed order
  float* F = ring;                  // MS x R
  float* Sg = ring + C::MS * R;     // (tile, column group) x 16
  for (int e = tid; e < C::MS * R; e += NT) F[e] = 0.0f;
  __syncthreads();
  auto tile_val = [&](int t, int i, int jj) -> float {
    if constexpr (C::PAIR) {
      const float2 v = accp[t][i][jj >> 1];
      return (jj & 1) ? v.y : v.x;
    } else {
      return accs[t][i][jj];
    }
  };
  auto tile_entry = [&](int j, int i, int jj) -> int {   // index into F, or -1
    if (j < np) {
      const int a = j / rqe, b = j % rqe;
      const int row = a + i * ra, k = 4 * b + jj;
      return (row < m && k < re) ? row * R + k : -1;
    }
    const int q = qlist[j - np];
    const int a = q / C::RQ, b = q % C::RQ;
    const int k = 4 * a + i, l = 4 * b + jj;
    return (k < re && l < re) ? (MP + k) * R + l : -1;
  };
  if (cg > 1) {
    if (qB < cg) {
      const int j = tid % ntb;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) Sg[(qB * ntb + j) * 16 + i * 4 + jj] = tile_val(0, i, jj);
    }
    __syncthreads();
    for (int j = tid; j < ntb; j += NT)
      for (int v = 0; v < 16; ++v) {
        float s = 0.0f;
        for (int q = 0; q < cg; ++q) s += Sg[(q * ntb + j) * 16 + v];
        const int e = tile_entry(j, v / 4, v % 4);
        if (e >= 0) F[e] = s;
      }
  } else {
#pragma unroll
    for (int t = 0; t < C::TPB; ++t) {
      const int j = tid + t * NT;
      if (j < ntb)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int e = tile_entry(j, i, jj);
            if (e >= 0) F[e] = tile_val(t, i, jj);
          }
    }
  }
  __syncthreads();
  // P rows of this problem (or row block) at rows prow0 + i, Q rows at qrow0 + k
  float* out = P.part + (size_t)slot * P.E;
  for (int e = tid; e < C::MS * R; e += NT) {
    const int row = e / R, k = e % R;
    if (row < MP) {
      if (row < m) out[(int64_t)(P.prow0 + row) * R + k] = F[e];
    } else if (P.hasq) {
      out[(int64_t)(P.qrow0 + row - MP) * R + k] = F[e];
    }
  }
}

// Resident CTAs per SM of one instantiation (1 when the query fails).
template <class C>
int gpass_occupancy_cfg() {
  if (cudaFuncSetAttribute(gpass_kernel<C, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, gpass_kernel<C, 0>, C::NT, C::SMEM) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    return 1;
  }
  return nb;
}

template <class C, int MODE>
cudaError_t launch_gpass_cfg(const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(gpass_kernel<C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  gpass_kernel<C, MODE><<<ncta, C::NT, C::SMEM, st>>>(probs, cta_prob, eps);
  return cudaGetLastError();
}

}  // namespace ntt
