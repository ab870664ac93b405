// Fused MU pass for BF16 X of at most 16 rows at rank bucket 16 on warp-level
// BF16 tensor-core MMAs (mma.sync m16n8k16, FP32 accumulation): the first
// unfolding of the precision form of a tensor whose first mode is 16
// (16 x 16^7 for a 16^8 tensor, r_1 = 16).  Same iteration step as the other
// passes (Algorithms 4-6, the collectives replaced by the combine kernel's
// fixed-order reduction of this kernel's per-CTA partials).
//
// X is an exact BF16 operand.  A stage (64 columns) holds X as 16 lines of
// 128 bytes (one per row, 2-D TMA box, 128-byte swizzle) and H as 16 ranks x
// two 32-column halves (3-D TMA box: 256 contiguous bytes of every H row).
// Per 16-column chunk, one warp (g = lane >> 2, t = lane & 3), ranks in two
// n-tiles of 8 (nt):
//   Y^T (16 cols x 16 ranks) = X^T W     A = X^T (ldmatrix .trans), B = W in
//        three BF16 terms (registers; with two, the 16^6 precision-form test's
//        last core drifted from 4.4e-4 to 6.4e-4 of the oracle's)
//   (G_W H)^T = H^T G_W                  A = H^T of the chunk in three BF16
//        terms (from the H box; its FP32 values are also the lane's own
//        H entries for the update), B = G_W in three terms (registers),
//        the six term products whose orders add to at most 4
//   H_new = max(0, H o Y / (G_W H + eps)) per lane: columns g, g + 8, ranks
//        8 nt + 2t, + 1; stored to HBM, and through a per-warp staging tile
//        into B fragments of H_new^T in three BF16 terms
//   P (16 rows x 16) += X H_new^T        A = X (ldmatrix), 3 terms x 2 n-tiles
//   Q = Qa + Qb + Qb^T with Qa = h1 h1^T + h2 h2^T, Qb = h1 h2^T + h1 h3^T
// MMA accumulators are added into FP32 register sums after every stage.
#include "ntt_internal.cuh"

#include <cuda_bf16.h>

namespace ntt {
namespace {

constexpr int kWbWarps = 8;
constexpr int kWbThreads = kWbWarps * 32;
constexpr int kWbSeg = 64;            // columns per stage
constexpr int kWbMP = 16, kWbR = 16;

struct WbCfg {
  static constexpr int XBOX = kWbMP * 128;          // 16 lines of 64 BF16
  static constexpr int HBOX = kWbR * 2 * 128;       // 16 ranks x two 32-column halves
  static constexpr int STAGE = XBOX + HBOX;
  static constexpr int FIT = 200 * 1024 / kWbWarps / STAGE;
  static constexpr int S = FIT < 6 ? FIT : 6;
  static constexpr int WARP_BYTES = S * STAGE;
  static constexpr int STG_OFF = kWbWarps * WARP_BYTES;       // 2 KB H_new staging tile per warp
  static constexpr int BAR_OFF = STG_OFF + kWbWarps * 2048;
  static constexpr int E = (kWbMP + kWbR) * kWbR;             // partial floats per CTA: P rows, then Q rows
  static constexpr int RED_FLOATS = kWbWarps * (E + kWbR * kWbR);
  static constexpr int SMEM = BAR_OFF + kWbWarps * S * 8 + 1024;
  static_assert(STAGE % 1024 == 0 && XBOX % 1024 == 0, "swizzle atoms of 1024 bytes");
  static_assert(S >= 2, "pipeline depth");
  static_assert(RED_FLOATS * 4 <= STG_OFF, "reduction scratch");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct WbParams {
  float* H;            // r x n, updated in place
  const float* W;      // m x r
  const float* G;      // 16 x 16 Gram of W, zero padded
  float* part;         // grid x 32 x 16
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

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float2 unpack_bf16(uint32_t v) {
  return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

// (x, y) = t1 + t2 + t3 with BF16 pairs
__device__ __forceinline__ void split3_pair(float2 v, uint32_t* t) {
  t[0] = pack_bf16(v.x, v.y);
  const float2 a = unpack_bf16(t[0]);
  const float2 r1 = make_float2(v.x - a.x, v.y - a.y);
  t[1] = pack_bf16(r1.x, r1.y);
  const float2 b = unpack_bf16(t[1]);
  t[2] = pack_bf16(r1.x - b.x, r1.y - b.y);
}

__global__ void __launch_bounds__(kWbThreads, 1)
mu_pass_tcwb_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                    const WbParams p) {
  using C = WbCfg;
  constexpr int S = C::S;
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
  // B fragments.  Y: K = the 16 rows, n-tile nt = ranks 8 nt .. 8 nt + 7; b0
  // holds rows 2t, 2t + 1, b1 rows 2t + 8, 2t + 9 of rank 8 nt + g; W in three
  // terms.  G H: K = the 16 ranks i, B[i][n] = G[i][8 nt + g] (G symmetric),
  // G in three terms.
  uint32_t bw[2][3][2], bg[2][3][2];   // [nt][term][b0, b1]
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    const int k = 8 * nt + g;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i0 = 2 * t + 8 * h;
      float w[2], gg[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        w[e] = (i0 + e < p.m && k < p.r) ? p.W[(i0 + e) * p.r + k] : 0.0f;
        gg[e] = p.G[(i0 + e) * kWbR + k];
      }
      uint32_t tw[3], tg[3];
      split3_pair(make_float2(w[0], w[1]), tw);
      split3_pair(make_float2(gg[0], gg[1]), tg);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        bw[nt][q][h] = tw[q];
        bg[nt][q][h] = tg[q];
      }
    }
  }
  __syncthreads();

  const int gw = blockIdx.x * kWbWarps + warp;
  const int gstride = gridDim.x * kWbWarps;
  auto issue = [&](int s, int seg) {
    const uint32_t bar = smem_u32(&bars[s]);
    const uint32_t dst = smem_u32(wbuf + s * C::STAGE);
    mbar_arrive_expect_tx(bar, C::STAGE);
    tma_load_2d(dst, &tmX, seg * kWbSeg, 0, bar);
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

  float accP[2][4], sumP[2][4], accQa[2][4], accQb[2][4], sumQa[2][4], sumQb[2][4];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) accP[nt][i] = sumP[nt][i] = accQa[nt][i] = accQb[nt][i] = sumQa[nt][i] =
        sumQb[nt][i] = 0.0f;
  const float eps = p.eps;
  // ldmatrix lane roles (as in the 32-row form): the lane's X line (row) is
  // li + 8 (lj >> 1) (Y) or li + 8 (lj & 1) (P), row mod 8 = li
  const int lj = lane >> 3, li = lane & 7;
  const uint32_t ly = (uint32_t)((li + 8 * (lj >> 1)) * 128), lamy = (uint32_t)(li ^ (lj & 1));
  const uint32_t lp = (uint32_t)((li + 8 * (lj & 1)) * 128), lamp = (uint32_t)(li ^ (lj >> 1));
  // H box element (rank, c0 + g + 8 h) with rank = 2t + e + 8 q: line 2 rank +
  // half (half = c0 >> 5), line mod 8 = 4 (t & 1) + 2 e + half; chunk
  // (A ^ (4 (t & 1) + 2 e)) + ((g >> 2) ^ half), A = ((c0 & 31) >> 2) + 2 h
  const uint32_t hl0 = (uint32_t)(4 * t * 128 + ((g >> 2) << 4) + (g & 3) * 4);
  const uint32_t hl1 = (uint32_t)(4 * t * 128 + 128 + (((g >> 2) ^ 1) << 4) + (g & 3) * 4);
  const uint32_t t4 = (uint32_t)(4 * (t & 1));
  // staging tile: word (rank, col) at rank * 32 + (col ^ 8 pi(rank mod 8)), pi(k) = (k & 3) ^ (k >> 2)
  float* stw = reinterpret_cast<float*>(smem + C::STG_OFF + warp * 2048);
  auto pi = [](int kk) { return ((kk & 7) & 3) ^ ((kk & 7) >> 2); };
  int sto[2][2][2], ldo[2][2];   // sto[nt][e][h] (rank 8 nt + 2t + e, col g + 8h); ldo[nt][h]
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 8 * nt + 2 * t + e;
        sto[nt][e][h] = k * 32 + ((g + 8 * h) ^ (8 * pi(k)));
      }
#pragma unroll
    for (int h = 0; h < 2; ++h) ldo[nt][h] = (8 * nt + g) * 32 + ((2 * t + 8 * h) ^ (8 * pi(8 * nt + g)));
  }
  float* Hrow[2][2];
  bool wr[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int k = 8 * nt + 2 * t + e;
      wr[nt][e] = k < p.r;
      Hrow[nt][e] = p.H + (int64_t)k * p.n;
    }

  bool err = false;
  int kst = 0;
  for (int seg = gw; seg < p.nseg; seg += gstride, ++kst) {
    const int s = kst % S;
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((kst / S) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      err = true;
      break;
    }
    const uint8_t* xs = wbuf + s * C::STAGE;
    const uint8_t* hs = xs + C::XBOX;
    const uint32_t xs_u = smem_u32(xs);
#pragma unroll
    for (int ck = 0; ck < kWbSeg / 16; ++ck) {
      const int c0 = ck * 16;
      // ---- Y^T = X^T W
      float y[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      {
        uint32_t a[4];
        ldsm_x4_t(xs_u + ly + ((((uint32_t)(2 * ck)) ^ lamy) << 4), a);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int q = 0; q < 3; ++q) mma16816(y[nt], a, bw[nt][q][0], bw[nt][q][1]);
      }
      // ---- A fragment of H^T: hv[q][h] = (H[2t + 8q][c0 + g + 8h], H[2t + 8q + 1][..])
      float2 hv[2][2];
      {
        const uint8_t* hb = hs + ((c0 >> 5) ? hl1 : hl0);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t A = (uint32_t)(((c0 & 31) >> 2) + 2 * h);
            float v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const uint32_t off = (uint32_t)((2 * e + 16 * q) * 128) + (((A ^ (uint32_t)(2 * e)) ^ t4) << 4);
              v[e] = *reinterpret_cast<const float*>(hb + off);
            }
            hv[q][h] = make_float2(v[0], v[1]);
          }
      }
      // ---- (G H)^T = H^T G: H and G in three terms, the products of order <= 4
      float gh[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      {
        uint32_t ht[2][2][3];   // [q][h][term]
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) split3_pair(hv[q][h], ht[q][h]);
        // A: a0 = (row g, k 2t..) = H^T[c0 + g][2t..] -> hv[0][0]; a1 = rows g + 8 -> hv[0][1];
        // a2 = k 2t + 8.. -> hv[1][0]; a3 -> hv[1][1]
        auto afrag = [&](int term, uint32_t* a) {
          a[0] = ht[0][0][term];
          a[1] = ht[0][1][term];
          a[2] = ht[1][0][term];
          a[3] = ht[1][1][term];
        };
        uint32_t a1[4], a2[4], a3[4];
        afrag(0, a1);
        afrag(1, a2);
        afrag(2, a3);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          mma16816(gh[nt], a1, bg[nt][0][0], bg[nt][0][1]);
          mma16816(gh[nt], a1, bg[nt][1][0], bg[nt][1][1]);
          mma16816(gh[nt], a2, bg[nt][0][0], bg[nt][0][1]);
          mma16816(gh[nt], a1, bg[nt][2][0], bg[nt][2][1]);
          mma16816(gh[nt], a3, bg[nt][0][0], bg[nt][0][1]);
          mma16816(gh[nt], a2, bg[nt][1][0], bg[nt][1][1]);
        }
      }
      // ---- H update: D entry q of n-tile nt is (col c0 + g + 8 (q >> 1), rank 8 nt + 2t + (q & 1));
      // its old H is hv[nt][q >> 1] component (q & 1)
      float hn[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 o = hv[nt][q >> 1];
          const float h0 = (q & 1) ? o.y : o.x;
          hn[nt][q] = fmaxf(0.0f, __fdividef(h0 * y[nt][q], gh[nt][q] + eps));
        }
      const int64_t gcol = (int64_t)seg * kWbSeg + c0 + g;   // n % 64 == 0: in range
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (wr[nt][e]) {
            Hrow[nt][e][gcol] = hn[nt][e];
            Hrow[nt][e][gcol + 8] = hn[nt][2 + e];
          }
      __syncwarp();   // the previous chunk's fragment loads from the tile are done
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          stw[sto[nt][e][0]] = hn[nt][e];
          stw[sto[nt][e][1]] = hn[nt][2 + e];
        }
      __syncwarp();
      // ---- B fragments of H_new^T (K = the chunk's 16 columns, N = rank 8 nt + g), three terms
      uint32_t hb0[2][3], hb1[2][3];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        split3_pair(*reinterpret_cast<const float2*>(stw + ldo[nt][0]), hb0[nt]);
        split3_pair(*reinterpret_cast<const float2*>(stw + ldo[nt][1]), hb1[nt]);
      }
      // ---- P (16 rows x 16) += X H_new^T
      {
        uint32_t a[4];
        ldsm_x4(xs_u + lp + ((((uint32_t)(2 * ck)) ^ lamp) << 4), a);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int h = 0; h < 3; ++h) mma16816(accP[nt], a, hb0[nt][h], hb1[nt][h]);
      }
      // ---- Q: A = H_new term (M = the 16 ranks): a0 = rank g -> hb0[0], a1 = rank 8 + g -> hb0[1],
      // a2 = hb1[0], a3 = hb1[1]
      {
        uint32_t q1[4] = {hb0[0][0], hb0[1][0], hb1[0][0], hb1[1][0]};
        uint32_t q2[4] = {hb0[0][1], hb0[1][1], hb1[0][1], hb1[1][1]};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          mma16816(accQa[nt], q1, hb0[nt][0], hb1[nt][0]);
          mma16816(accQa[nt], q2, hb0[nt][1], hb1[nt][1]);
          mma16816(accQb[nt], q1, hb0[nt][1], hb1[nt][1]);
          mma16816(accQb[nt], q1, hb0[nt][2], hb1[nt][2]);
        }
      }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        sumP[nt][i] += accP[nt][i];
        sumQa[nt][i] += accQa[nt][i];
        sumQb[nt][i] += accQb[nt][i];
        accP[nt][i] = accQa[nt][i] = accQb[nt][i] = 0.0f;
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
    for (int c = kst; c < issued; ++c)
      (void)mbar_wait_bounded(smem_u32(&bars[c % S]), (uint32_t)((c / S) & 1));
    atomicExch(p.status, kStatusTimeout);
  }
  __syncthreads();   // every stage buffer is free: reuse it for the reduction

  // per warp: P (row, rank), Qa + Qb (rank, rank) and Qb (added transposed below)
  float* red = reinterpret_cast<float*>(smem);
  constexpr int E = C::E, QQ = kWbR * kWbR;
  float* rw = red + warp * (E + QQ);
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = g + 8 * (q >> 1), col = 8 * nt + 2 * t + (q & 1);
      rw[row * kWbR + col] = sumP[nt][q];
      rw[(kWbMP + row) * kWbR + col] = sumQa[nt][q] + sumQb[nt][q];
      rw[E + row * kWbR + col] = sumQb[nt][q];
    }
  __syncthreads();
  float* out = p.part + (size_t)blockIdx.x * E;
  for (int e = tid; e < E; e += kWbThreads) {
    float v = 0.0f;
    if (e < kWbMP * kWbR) {
#pragma unroll
      for (int wi = 0; wi < kWbWarps; ++wi) v += red[wi * (E + QQ) + e];
    } else {
      const int kq = (e - kWbMP * kWbR) / kWbR, lq = e % kWbR;
#pragma unroll
      for (int wi = 0; wi < kWbWarps; ++wi)
        v += red[wi * (E + QQ) + e] + red[wi * (E + QQ) + E + lq * kWbR + kq];
    }
    out[e] = v;
  }
}

}  // namespace

bool tcwb_route_ok(int64_t m, int64_t n, int r, int route) {
  if (route == NTT_ROUTE_FMA || route == NTT_ROUTE_GENERIC || route == NTT_ROUTE_TC) return false;
  return m >= 1 && m <= 16 && r > 8 && r <= 16 && n % 64 == 0;
}

cudaError_t launch_mu_pass_tcwb(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                                const CUtensorMap& mh, cudaStream_t st) {
  if (s.MP != 16 || s.R != 16 || s.n % 64 != 0) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(mu_pass_tcwb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WbCfg::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  WbParams p;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.nseg = (int)(s.n / kWbSeg);
  p.eps = eps;
  return launch_pdl(mu_pass_tcwb_kernel, dim3(s.grid), dim3(kWbThreads), WbCfg::SMEM, st, mx, mh, p);
}

}  // namespace ntt
