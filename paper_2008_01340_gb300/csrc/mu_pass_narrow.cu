// Warp-streamed fused MU pass for narrow unfoldings: at most 32 rows, rank
// bucket 8, FP32 X -- the first unfolding of a tensor whose first mode is
// small (32 x 32^5 for a 32^6 tensor, r_1 = 8).
//
// One launch is the same iteration step as the generic pass: per column
//   Y = W^T X,  H_new = max(0, H o Y / (W^T W H + eps)),
//   P += X H_new^T,  Q += H_new H_new^T,
// with one read of X (the MU update of H, then the products the W update
// needs; Algorithms 4-6 with the collectives replaced by the fixed-order
// cross-CTA reduction of the combine kernel, which consumes this kernel's
// partials unchanged: per CTA [MP + 8] x 8 floats, P rows then Q rows).
//
// Organised for shared-memory traffic, which bounds the generic pass on this
// shape (every 128-bit shared load costs four wavefronts, broadcast or not):
//   * each warp streams its own 32-column boxes (128 bytes of every row)
//     through its own TMA ring of mbarrier-tracked stages: no CTA-wide
//     barrier in the main loop;
//   * X and H boxes use the 128-byte swizzle (16-byte chunk index XOR row
//     mod 8), so eight lanes reading one column quad of eight different rows
//     touch eight different bank groups;
//   * lane = (row split sa = lane & 7, column group cq = lane >> 3, CPL
//     columns per group).  A lane keeps W rows sa, sa + 8, ... in registers
//     with its ranks in the order slot i -> rank i ^ sa; the reduce-scatter of
//     Y over the eight row splits is then three shuffle steps (lane xor 4, 2,
//     1) that always keep the low half of the slots, and leaves lane sa with Y
//     of rank sa for its CPL columns;
//   * the H update of (rank sa, CPL columns) reads the eight H rows of those
//     columns from shared memory, stores H_new straight to global memory, and
//     takes H_new of the other ranks from lanes sa ^ i by shuffles, so P and Q
//     accumulate in registers without a second read of X;
//   * packed FP32x2 FMAs pair slots (2j, 2j + 1), so the X value of a column
//     is the one broadcast operand of both Y = W^T X and P = X H_new^T, and
//     the P, Q partials take 2 x (4 RPL + 4) registers; at 168 registers a
//     lane, 12 warps fit on an SM.
#include "ntt_internal.cuh"

namespace ntt {
namespace {

constexpr int kBoxCols = 32;   // one 128-byte swizzle span of FP32

template <int MP_, int NW_, int CPL_>
struct NarrowCfg {
  static constexpr int MP = MP_;
  static constexpr int NW = NW_;                // warps per CTA
  static constexpr int CPL = CPL_;              // columns per lane per step (2 or 4)
  static constexpr int NSTEP = kBoxCols / (4 * CPL);   // steps per box
  static constexpr int kNarrowWarps = NW;
  static constexpr int kNarrowThreads = NW * 32;
  static constexpr int RPL = MP / 8;            // X rows per lane
  static constexpr int XBOX = MP * 128;         // bytes of one X box
  static constexpr int HBOX = 8 * 128;          // bytes of one H box (rank bucket 8)
  static constexpr int STAGE = XBOX + HBOX;
  static constexpr int BUDGET = 220 * 1024;
  static constexpr int FIT = BUDGET / kNarrowWarps / STAGE;
  static constexpr int STAGES = FIT < 8 ? FIT : 8;
  static constexpr int WARP_BYTES = STAGES * STAGE;
  static constexpr int BAR_OFF = kNarrowWarps * WARP_BYTES;
  static constexpr int RED_BYTES = kNarrowWarps * (MP + 8) * 8 * 4;
  static constexpr int SMEM = BAR_OFF + kNarrowWarps * STAGES * 8 + 1024;   // + alignment slack
  static_assert(MP == 16 || MP == 32, "row bucket");
  static_assert(CPL == 2 || CPL == 4, "columns per lane");
  static_assert(STAGE % 1024 == 0, "swizzle atoms of 1024 bytes");
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(RED_BYTES <= BAR_OFF, "reduction scratch");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct NarrowParams {
  float* H;            // r x n, updated in place
  const float* W;      // m x r
  const float* G;      // 8 x 8 Gram of W, zero padded
  float* part;         // grid x (MP + 8) x 8
  int* status;
  const int* stop;     // nullable: the stage's stop word; a set word makes the launch a no-op
  int64_t n;
  int m, r;
  int nbox;            // boxes: ceil(n / 32), or stages of NB segments in the 3-D form
  float eps;
};

// CPL consecutive floats of shared memory (16- or 8-byte aligned) into registers.
template <int N>
__device__ __forceinline__ void lds_cols(const uint8_t* p, float* v) {
  if constexpr (N == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int N>
__device__ __forceinline__ void stg_cols(float* p, const float* v) {
  if constexpr (N == 4)
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int mask) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask));
}

template <class C>
__global__ void __launch_bounds__(C::kNarrowThreads, 1)
mu_pass_narrow_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                      const NarrowParams p) {
  constexpr int RPL = C::RPL, MP = C::MP, S = C::STAGES;
  constexpr int kNarrowWarps = C::kNarrowWarps, kNarrowThreads = C::kNarrowThreads;
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sa = lane & 7, cq = lane >> 3;
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
  // W rows sa + 8 ii and the G row sa, ranks in slot order (slot i -> rank i ^ sa)
  float w[RPL][8], g[8];
#pragma unroll
  for (int ii = 0; ii < RPL; ++ii) {
    const int row = sa + 8 * ii;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = i ^ sa;
      w[ii][i] = (row < p.m && k < p.r) ? p.W[row * p.r + k] : 0.0f;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) g[i] = p.G[sa * 8 + (i ^ sa)];
  __syncthreads();

  const int gw = blockIdx.x * kNarrowWarps + warp;
  const int gstride = gridDim.x * kNarrowWarps;
  auto issue = [&](int s, int box) {
    const uint32_t bar = smem_u32(&bars[s]);
    const uint32_t dst = smem_u32(wbuf + s * C::STAGE);
    mbar_arrive_expect_tx(bar, C::STAGE);
    tma_load_2d(dst, &tmX, box * kBoxCols, 0, bar);
    tma_load_2d(dst + C::XBOX, &tmH, box * kBoxCols, 0, bar);
  };
  int issued = 0;   // boxes whose loads lane 0 issued
  if (lane == 0) {
    for (int s = 0; s < S; ++s) {
      const int box = gw + s * gstride;
      if (box < p.nbox) {
        issue(s, box);
        ++issued;
      }
    }
  }

  // partials of (P[sa + 8 ii][sa ^ 2j], P[sa + 8 ii][sa ^ (2j + 1)]) in accP[ii][j],
  // of (Q[sa][sa ^ 2j], Q[sa][sa ^ (2j + 1)]) in accQ[j]
  constexpr int NA = 4, CPL = C::CPL;
  float2 accP[RPL][NA];
  float2 accQ[NA];
#pragma unroll
  for (int i = 0; i < NA; ++i) {
    accQ[i] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int ii = 0; ii < RPL; ++ii) accP[ii][i] = make_float2(0.0f, 0.0f);
  }

  bool err = false;
  int k = 0;   // boxes consumed by this warp
  for (int box = gw; box < p.nbox; box += gstride, ++k) {
    const int s = k % S;
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((k / S) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      err = true;
      break;
    }
    const uint8_t* xs = wbuf + s * C::STAGE;
    const uint8_t* hs = xs + C::XBOX;
#pragma unroll
    for (int step = 0; step < C::NSTEP; ++step) {
      // this lane's CPL columns: byte offset cb in a 128-byte row, 16-byte chunk cb >> 4
      const int cb = (step * 4 + cq) * CPL * 4;
      const int ch = cb >> 4, cw = cb & 15;
      // X rows sa + 8 ii (row mod 8 = sa: physical chunk ch ^ sa)
      float xr[RPL][CPL];
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii)
        lds_cols<CPL>(xs + (sa + 8 * ii) * 128 + ((ch ^ sa) << 4) + cw, xr[ii]);
      // Y partials in rank pairs: y2[j][c] = (slot 2j, slot 2j + 1) at column c
      float2 y2[4][CPL];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < CPL; ++c) y2[j][c] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const float2 xb = make_float2(xr[ii][c], xr[ii][c]);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            y2[j][c] = __ffma2_rn(make_float2(w[ii][2 * j], w[ii][2 * j + 1]), xb, y2[j][c]);
        }
      // reduce-scatter over the row splits: the partner's upper slots hold the
      // ranks of this lane's lower slots, in the same order
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int c = 0; c < CPL; ++c) y2[t][c] = __fadd2_rn(y2[t][c], shfl_xor2(y2[2 + t][c], 4));
#pragma unroll
      for (int c = 0; c < CPL; ++c) y2[0][c] = __fadd2_rn(y2[0][c], shfl_xor2(y2[1][c], 2));
      float yv[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) yv[c] = y2[0][c].x + __shfl_xor_sync(0xffffffffu, y2[0][c].y, 1);

      // G H for rank sa from H rows sa ^ i (rows < 8: physical chunk ch ^ row)
      // (column pairs, even and odd i in separate chains)
      float h0[CPL];
      float2 ga[CPL / 2], gb[CPL / 2];
#pragma unroll
      for (int t = 0; t < CPL / 2; ++t) ga[t] = gb[t] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = sa ^ i;
        float hv[CPL];
        lds_cols<CPL>(hs + row * 128 + ((ch ^ row) << 4) + cw, hv);
        if (i == 0)
#pragma unroll
          for (int c = 0; c < CPL; ++c) h0[c] = hv[c];
        const float2 gi = make_float2(g[i], g[i]);
#pragma unroll
        for (int t = 0; t < CPL / 2; ++t) {
          if (i & 1)
            gb[t] = __ffma2_rn(gi, make_float2(hv[2 * t], hv[2 * t + 1]), gb[t]);
          else
            ga[t] = __ffma2_rn(gi, make_float2(hv[2 * t], hv[2 * t + 1]), ga[t]);
        }
      }
      float hn[CPL];
#pragma unroll
      for (int t = 0; t < CPL / 2; ++t) {
        const float2 gh = __fadd2_rn(ga[t], gb[t]);
        hn[2 * t] = fmaxf(0.0f, __fdividef(h0[2 * t] * yv[2 * t], gh.x + p.eps));
        hn[2 * t + 1] = fmaxf(0.0f, __fdividef(h0[2 * t + 1] * yv[2 * t + 1], gh.y + p.eps));
      }
      const int64_t col = (int64_t)box * kBoxCols + (cb >> 2);   // n % 4 == 0: whole group in or out
      if (sa < p.r && col < p.n) stg_cols<CPL>(p.H + (int64_t)sa * p.n + col, hn);

      // H_new of ranks sa ^ 2j, sa ^ (2j + 1) from lanes ^ 2j, ^ (2j + 1); P and Q
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 hp[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          hp[c].x = j == 0 ? hn[c] : __shfl_xor_sync(0xffffffffu, hn[c], 2 * j);
          hp[c].y = __shfl_xor_sync(0xffffffffu, hn[c], 2 * j + 1);
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
#pragma unroll
          for (int ii = 0; ii < RPL; ++ii)
            accP[ii][j] = __ffma2_rn(make_float2(xr[ii][c], xr[ii][c]), hp[c], accP[ii][j]);
          accQ[j] = __ffma2_rn(make_float2(hn[c], hn[c]), hp[c], accQ[j]);
        }
      }
    }
    __syncwarp();   // every lane is done with this stage
    if (lane == 0) {
      const int next = box + S * gstride;
      if (next < p.nbox) {
        fence_proxy_async_smem();
        issue(s, next);
        ++issued;
      }
    }
  }

  if (err && lane == 0) {
    // drain this warp's copies still in flight (bounded), then flag the timeout
    for (int c = k; c < issued; ++c)
      (void)mbar_wait_bounded(smem_u32(&bars[c % S]), (uint32_t)((c / S) & 1));
    atomicExch(p.status, kStatusTimeout);
  }
  __syncthreads();   // every stage buffer is free: reuse it for the reduction

  // sum the column-parity halves, then the four column quads of the warp (lanes
  // xor 8, 16), then the eight warps in a fixed order
  float* red = reinterpret_cast<float*>(smem);
  constexpr int E = (MP + 8) * 8;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int ai = i / 2;   // slot i is half (i & 1) of pair i / 2
#pragma unroll
    for (int ii = 0; ii < RPL; ++ii) {
      float v = (i & 1) ? accP[ii][ai].y : accP[ii][ai].x;
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (cq == 0) red[warp * E + (sa + 8 * ii) * 8 + (sa ^ i)] = v;
    }
    float v = (i & 1) ? accQ[ai].y : accQ[ai].x;
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    if (cq == 0) red[warp * E + (MP + sa) * 8 + (sa ^ i)] = v;
  }
  __syncthreads();
  float* out = p.part + (size_t)blockIdx.x * E;
  for (int e = tid; e < E; e += kNarrowThreads) {
    float v = red[e];
#pragma unroll
    for (int wi = 1; wi < kNarrowWarps; ++wi) v += red[wi * E + e];
    out[e] = v;
  }
}

// Second organisation, for 32 rows when n is a multiple of 32: wide copies
// and four row splits x eight column groups.
//   * Copies: a 32-column box moves 128 bytes of every row, and on this
//     access pattern the copy engine reached 5.7 TB/s against 6.9 TB/s when a
//     copy moves 256 contiguous bytes of every row (measured with the loads
//     and the H stores alone).  X and H are therefore described as 3-D
//     tensors (32 columns, n / 32 segments, rows) whose box holds NB = 2
//     adjacent segments of every row; a stage is 64 columns, its lines of 128
//     bytes ordered (row, segment), 16-byte chunks XOR line mod 8.
//   * lane = sb + 4 cq (row split sb = lane & 3, column group cq = lane >> 2),
//     two columns per lane per step, a segment in two steps.  Lane sb keeps W
//     rows sb + 4 ii with its ranks in slot order slot i -> rank i ^ 2 sb, so
//     the reduce-scatter of Y over the four row splits is two shuffle steps
//     (lane xor 2, 1) and leaves lane sb with Y of ranks 2 sb, 2 sb + 1 for
//     its two columns.  Against eight row splits this halves the lanes that
//     share a column: the Y reduce-scatter and the H_new gather take 24
//     shuffles per 16 columns instead of 56, and every H element is read from
//     shared memory four times instead of eight, at the price of twice the W
//     and P registers per lane (8 warps).
//   * Shared-memory reads are 64-bit, 16 lanes per wavefront: the X lines of a
//     half-warp's four rows are 2 (sb + 4 ii) + g, so line mod 8 = 2 sb + g
//     puts the four rows in distinct chunk pairs; H rows are read in the
//     order i ^ sb (line mod 8 = 2 ((i ^ sb) & 3) + g: distinct), the two
//     ranks a lane updates once more by name.
template <int MP_, int NW_>
struct Narrow4Cfg {
  static constexpr int MP = MP_;
  static constexpr int NW = NW_;                // warps per CTA
  static constexpr int kThreads = NW * 32;
  static constexpr int NB = 2;                  // 32-column segments per stage
  static constexpr int NSTEP = kBoxCols / 16;   // steps per segment: 8 column groups x 2 columns
  static constexpr int RPL = MP / 4;            // X rows per lane
  static constexpr int XBOX = MP * NB * 128;
  static constexpr int HBOX = 8 * NB * 128;
  static constexpr int STAGE = XBOX + HBOX;
  static constexpr int BUDGET = 220 * 1024;
  static constexpr int FIT = BUDGET / NW / STAGE;
  static constexpr int STAGES = FIT < 8 ? FIT : 8;
  static constexpr int WARP_BYTES = STAGES * STAGE;
  static constexpr int BAR_OFF = NW * WARP_BYTES;
  static constexpr int RED_BYTES = NW * (MP + 8) * 8 * 4;
  static constexpr int SMEM = BAR_OFF + NW * STAGES * 8 + 1024;
  static_assert(MP == 32, "row bucket: the chunk pairs are distinct for 2 (sb + 4 ii) + g");
  static_assert(STAGE % 1024 == 0 && XBOX % 1024 == 0, "swizzle atoms of 1024 bytes");
  static_assert(STAGES >= 2, "pipeline depth");
  static_assert(RED_BYTES <= BAR_OFF, "reduction scratch");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// X row held in register row ii of lane split sb
__device__ __forceinline__ int n4_row(int sb, int ii) { return sb + 4 * ii; }

template <class C>
__global__ void __launch_bounds__(C::kThreads, 1)
mu_pass_narrow4_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                       const NarrowParams p) {
  constexpr int RPL = C::RPL, MP = C::MP, S = C::STAGES, NW = C::NW;
  pdl_wait();      // the previous kernel's W, G and stop word
  pdl_trigger();
  if (p.stop && __ldcg(p.stop)) return;   // the stage's stopping test has fired
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sb = lane & 3, cq = lane >> 2, s2 = 2 * sb;
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
  // W rows n4_row(sb, ii), ranks in slot order (slot i -> rank i ^ 2 sb);
  // G rows 2 sb, 2 sb + 1 as pairs, columns in H read order (i -> rank i ^ sb)
  float w[RPL][8];
  float2 g2[8];
#pragma unroll
  for (int ii = 0; ii < RPL; ++ii) {
    const int row = n4_row(sb, ii);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = i ^ s2;
      w[ii][i] = (row < p.m && k < p.r) ? p.W[row * p.r + k] : 0.0f;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) g2[i] = make_float2(p.G[s2 * 8 + (i ^ sb)], p.G[(s2 + 1) * 8 + (i ^ sb)]);
  __syncthreads();

  const int gw = blockIdx.x * NW + warp;
  const int gstride = gridDim.x * NW;
  auto issue = [&](int s, int box) {   // box: NB consecutive 32-column segments
    const uint32_t bar = smem_u32(&bars[s]);
    const uint32_t dst = smem_u32(wbuf + s * C::STAGE);
    mbar_arrive_expect_tx(bar, C::STAGE);
    tma_load_3d(dst, &tmX, 0, box * C::NB, 0, bar);
    tma_load_3d(dst + C::XBOX, &tmH, 0, box * C::NB, 0, bar);
  };
  int issued = 0;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) {
      const int box = gw + s * gstride;
      if (box < p.nbox) {
        issue(s, box);
        ++issued;
      }
    }
  }

  // accP[ii][d] = (P[row ii][2 (sb ^ d)], P[row ii][2 (sb ^ d) + 1]);
  // accQ[e][d] = (Q[2 sb + e][2 (sb ^ d)], Q[2 sb + e][2 (sb ^ d) + 1])
  float2 accP[RPL][4];
  float2 accQ[2][4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    accQ[0][d] = accQ[1][d] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int ii = 0; ii < RPL; ++ii) accP[ii][d] = make_float2(0.0f, 0.0f);
  }

  bool err = false;
  int k = 0;
  for (int box = gw; box < p.nbox; box += gstride, ++k) {
    const int s = k % S;
    const bool ok = mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)((k / S) & 1));
    if (!__all_sync(0xffffffffu, ok)) {
      err = true;
      break;
    }
    const uint8_t* xs = wbuf + s * C::STAGE;
    const uint8_t* hs = xs + C::XBOX;
#pragma unroll 1
    for (int g = 0; g < C::NB; ++g)
#pragma unroll
    for (int step = 0; step < C::NSTEP; ++step) {
      // segment g, step within it; this lane's two columns at byte offset cb of
      // the segment's 128-byte lines (line = row * NB + g)
      const int cb = (step * 8 + cq) * 8;
      const int ch = cb >> 4, cw = cb & 15;
      float2 xr[RPL];
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii) {
        const int line = n4_row(sb, ii) * C::NB + g;
        xr[ii] = *reinterpret_cast<const float2*>(xs + line * 128 + ((ch ^ (line & 7)) << 4) + cw);
      }
      // Y partials over this lane's rows: y2[j][c] = (slot 2j, slot 2j + 1) at column c
      float2 y2[4][2];
#pragma unroll
      for (int j = 0; j < 4; ++j) y2[j][0] = y2[j][1] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii) {
        const float2 xa = make_float2(xr[ii].x, xr[ii].x), xb = make_float2(xr[ii].y, xr[ii].y);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 wj = make_float2(w[ii][2 * j], w[ii][2 * j + 1]);
          y2[j][0] = __ffma2_rn(wj, xa, y2[j][0]);
          y2[j][1] = __ffma2_rn(wj, xb, y2[j][1]);
        }
      }
      // reduce-scatter over the row splits: the partner's upper slots hold the
      // ranks of this lane's lower slots, in the same order
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        y2[0][c] = __fadd2_rn(y2[0][c], shfl_xor2(y2[2][c], 2));
        y2[1][c] = __fadd2_rn(y2[1][c], shfl_xor2(y2[3][c], 2));
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) y2[0][c] = __fadd2_rn(y2[0][c], shfl_xor2(y2[1][c], 1));
      // y2[0][c] = (Y[2 sb][c], Y[2 sb + 1][c])

      // G H for ranks 2 sb, 2 sb + 1 from H rows i ^ sb
      auto hline = [&](int rank) {
        const int line = rank * C::NB + g;
        return *reinterpret_cast<const float2*>(hs + line * 128 + ((ch ^ (line & 7)) << 4) + cw);
      };
      float2 h0[2], ga[2], gb[2];
      {
        const float2 ha = hline(s2), hb = hline(s2 + 1);
        h0[0] = make_float2(ha.x, hb.x);
        h0[1] = make_float2(ha.y, hb.y);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) ga[c] = gb[c] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 hv = hline(i ^ sb);
        const float2 ha = make_float2(hv.x, hv.x), hb = make_float2(hv.y, hv.y);
        if (i & 1) {
          gb[0] = __ffma2_rn(g2[i], ha, gb[0]);
          gb[1] = __ffma2_rn(g2[i], hb, gb[1]);
        } else {
          ga[0] = __ffma2_rn(g2[i], ha, ga[0]);
          ga[1] = __ffma2_rn(g2[i], hb, ga[1]);
        }
      }
      // hn[c] = (H_new[2 sb][c], H_new[2 sb + 1][c])
      float2 hn[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float2 gh = __fadd2_rn(ga[c], gb[c]);
        hn[c].x = fmaxf(0.0f, __fdividef(h0[c].x * y2[0][c].x, gh.x + p.eps));
        hn[c].y = fmaxf(0.0f, __fdividef(h0[c].y * y2[0][c].y, gh.y + p.eps));
      }
      const int64_t col = ((int64_t)box * C::NB + g) * kBoxCols + (cb >> 2);   // n % 32 == 0
      if (col < p.n) {
        if (s2 < p.r) *reinterpret_cast<float2*>(p.H + (int64_t)s2 * p.n + col) = make_float2(hn[0].x, hn[1].x);
        if (s2 + 1 < p.r)
          *reinterpret_cast<float2*>(p.H + (int64_t)(s2 + 1) * p.n + col) = make_float2(hn[0].y, hn[1].y);
      }

      // H_new of ranks 2 (sb ^ d), 2 (sb ^ d) + 1 from lane ^ d; P and Q
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        float2 hp[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) hp[c] = d == 0 ? hn[c] : shfl_xor2(hn[c], d);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
          for (int ii = 0; ii < RPL; ++ii) {
            const float xv = c ? xr[ii].y : xr[ii].x;
            accP[ii][d] = __ffma2_rn(make_float2(xv, xv), hp[c], accP[ii][d]);
          }
          accQ[0][d] = __ffma2_rn(make_float2(hn[c].x, hn[c].x), hp[c], accQ[0][d]);
          accQ[1][d] = __ffma2_rn(make_float2(hn[c].y, hn[c].y), hp[c], accQ[1][d]);
        }
      }
    }
    __syncwarp();   // every lane is done with this stage
    if (lane == 0) {
      const int next = box + S * gstride;
      if (next < p.nbox) {
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

  // sum the eight column groups of the warp (lanes xor 4, 8, 16), then the
  // warps in a fixed order
  float* red = reinterpret_cast<float*>(smem);
  constexpr int E = (MP + 8) * 8;
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int kk = 2 * (sb ^ d) + e;
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii) {
        float v = e ? accP[ii][d].y : accP[ii][d].x;
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (cq == 0) red[warp * E + n4_row(sb, ii) * 8 + kk] = v;
      }
#pragma unroll
      for (int e2 = 0; e2 < 2; ++e2) {
        float v = e ? accQ[e2][d].y : accQ[e2][d].x;
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        if (cq == 0) red[warp * E + (MP + s2 + e2) * 8 + kk] = v;
      }
    }
  __syncthreads();
  float* out = p.part + (size_t)blockIdx.x * E;
  for (int e = tid; e < E; e += C::kThreads) {
    float v = red[e];
#pragma unroll
    for (int wi = 1; wi < NW; ++wi) v += red[wi * E + e];
    out[e] = v;
  }
}

template <class C>
cudaError_t launch_narrow4_cfg(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                               const CUtensorMap& mh, cudaStream_t st) {
  static bool attr_set = false;   // per-function attribute; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_pass_narrow4_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  NarrowParams p;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.nbox = (int)((s.n + C::NB * kBoxCols - 1) / (C::NB * kBoxCols));   // stages of NB segments
  p.eps = eps;
  return launch_pdl(mu_pass_narrow4_kernel<C>, dim3(s.grid), dim3(C::kThreads), C::SMEM, st, mx, mh, p);
}

template <class C>
cudaError_t launch_narrow_cfg(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                              const CUtensorMap& mh, cudaStream_t st) {
  static bool attr_set = false;   // per-function attribute; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(mu_pass_narrow_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  NarrowParams p;
  p.H = d.H;
  p.W = d.W;
  p.G = d.G;
  p.part = d.part;
  p.status = d.status;
  p.stop = d.stop;
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.nbox = (int)((s.n + kBoxCols - 1) / kBoxCols);
  p.eps = eps;
  return launch_pdl(mu_pass_narrow_kernel<C>, dim3(s.grid), dim3(C::kNarrowThreads), C::SMEM, st, mx, mh, p);
}

}  // namespace

bool narrow_pass_supported(int MP, int R) { return (MP == 16 || MP == 32) && R == 8; }

cudaError_t launch_mu_pass_narrow(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                                  const CUtensorMap& mh, cudaStream_t st) {
  if (s.R != 8) return cudaErrorInvalidValue;
  // 32 rows: 12 warps x 4 columns per lane (168 registers); measured on
  // 32 x 4,194,304 against 8 warps (0.193 vs 0.213 ms per iteration) and
  // against 2 columns per lane at 12 or 16 warps (0.199, 0.206 ms).
  // 16 rows: 16 warps x 2 columns per lane (128 registers).
  // 32 rows, n a multiple of 32 (s.narrow == 2): the 3-D form with 64-column
  // stages, 4 row splits, 8 warps (248 registers).
  if (s.narrow == 2) return s.MP == 32 ? launch_narrow4_cfg<Narrow4Cfg<32, 8>>(s, d, eps, mx, mh, st)
                                       : cudaErrorInvalidValue;
  if (s.MP == 16) return launch_narrow_cfg<NarrowCfg<16, 16, 2>>(s, d, eps, mx, mh, st);
  if (s.MP == 32) return launch_narrow_cfg<NarrowCfg<32, 12, 4>>(s, d, eps, mx, mh, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
