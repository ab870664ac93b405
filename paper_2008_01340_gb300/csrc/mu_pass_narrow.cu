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
//   * lane = (row split sa = lane & 7, column quad cq = lane >> 3).  A lane
//     keeps W rows sa, sa + 8, ... in registers with its ranks in the order
//     slot i -> rank i ^ sa; the reduce-scatter of Y over the eight row splits
//     is then three shuffle steps (lane xor 4, 2, 1) that always keep the low
//     half of the slots, and leaves lane sa with Y of rank sa for its four
//     columns;
//   * the H update of (rank sa, 4 columns) reads the eight H rows of those
//     columns from shared memory, stores H_new straight to global memory, and
//     takes H_new of the other ranks from lanes sa ^ i by shuffles, so P and Q
//     accumulate in registers without a second read of X.
#include "ntt_internal.cuh"

namespace ntt {
namespace {

constexpr int kNarrowWarps = 8;
constexpr int kNarrowThreads = kNarrowWarps * 32;
constexpr int kBoxCols = 32;   // one 128-byte swizzle span of FP32

template <int MP_>
struct NarrowCfg {
  static constexpr int MP = MP_;
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
  int64_t n;
  int m, r;
  int nbox;            // ceil(n / 32)
  float eps;
};

__device__ __forceinline__ float2 shfl_xor2(float2 v, int mask) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask));
}

template <class C>
__global__ void __launch_bounds__(kNarrowThreads, 1)
mu_pass_narrow_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmH,
                      const NarrowParams p) {
  constexpr int RPL = C::RPL, MP = C::MP, S = C::STAGES;
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

  float2 accP[RPL][8];   // (even, odd column) partials of P[sa + 8 ii][sa ^ i]
  float2 accQ[8];        // partials of Q[sa][sa ^ i]
#pragma unroll
  for (int i = 0; i < 8; ++i) {
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
    for (int half = 0; half < 2; ++half) {
      const int q = 4 * half + cq;   // column quad within the box
      // X rows sa + 8 ii (row mod 8 = sa: physical chunk q ^ sa)
      float4 x[RPL];
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii)
        x[ii] = *reinterpret_cast<const float4*>(xs + (sa + 8 * ii) * 128 + ((q ^ sa) << 4));
      // Y partials over this lane's rows: slot i = rank i ^ sa, columns (0,1) and (2,3)
      float2 y[8][2];
#pragma unroll
      for (int i = 0; i < 8; ++i) y[i][0] = y[i][1] = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int ii = 0; ii < RPL; ++ii) {
        const float2 x01 = make_float2(x[ii].x, x[ii].y), x23 = make_float2(x[ii].z, x[ii].w);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 wi = make_float2(w[ii][i], w[ii][i]);
          y[i][0] = __ffma2_rn(wi, x01, y[i][0]);
          y[i][1] = __ffma2_rn(wi, x23, y[i][1]);
        }
      }
      // reduce-scatter over the row splits: the partner's upper slots hold the
      // ranks of this lane's lower slots, in the same order
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) y[t][h] = __fadd2_rn(y[t][h], shfl_xor2(y[4 + t][h], 4));
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) y[t][h] = __fadd2_rn(y[t][h], shfl_xor2(y[2 + t][h], 2));
#pragma unroll
      for (int h = 0; h < 2; ++h) y[0][h] = __fadd2_rn(y[0][h], shfl_xor2(y[1][h], 1));

      // H rows sa ^ i of the four columns (rows < 8: physical chunk q ^ row)
      float4 h0;
      float2 gh01 = make_float2(0.0f, 0.0f), gh23 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = sa ^ i;
        const float4 hv = *reinterpret_cast<const float4*>(hs + row * 128 + ((q ^ row) << 4));
        if (i == 0) h0 = hv;
        const float2 gi = make_float2(g[i], g[i]);
        gh01 = __ffma2_rn(gi, make_float2(hv.x, hv.y), gh01);
        gh23 = __ffma2_rn(gi, make_float2(hv.z, hv.w), gh23);
      }
      float4 hn;
      hn.x = fmaxf(0.0f, __fdividef(h0.x * y[0][0].x, gh01.x + p.eps));
      hn.y = fmaxf(0.0f, __fdividef(h0.y * y[0][0].y, gh01.y + p.eps));
      hn.z = fmaxf(0.0f, __fdividef(h0.z * y[0][1].x, gh23.x + p.eps));
      hn.w = fmaxf(0.0f, __fdividef(h0.w * y[0][1].y, gh23.y + p.eps));
      const int64_t col = (int64_t)box * kBoxCols + 4 * q;   // n % 4 == 0: whole quad in or out
      if (sa < p.r && col < p.n)
        *reinterpret_cast<float4*>(p.H + (int64_t)sa * p.n + col) = hn;

      // H_new of rank sa ^ i from lane ^ i; P and Q over these four columns
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float4 hq = hn;
        if (i > 0) {
          hq.x = __shfl_xor_sync(0xffffffffu, hn.x, i);
          hq.y = __shfl_xor_sync(0xffffffffu, hn.y, i);
          hq.z = __shfl_xor_sync(0xffffffffu, hn.z, i);
          hq.w = __shfl_xor_sync(0xffffffffu, hn.w, i);
        }
        const float2 q01 = make_float2(hq.x, hq.y), q23 = make_float2(hq.z, hq.w);
#pragma unroll
        for (int ii = 0; ii < RPL; ++ii) {
          accP[ii][i] = __ffma2_rn(make_float2(x[ii].x, x[ii].y), q01, accP[ii][i]);
          accP[ii][i] = __ffma2_rn(make_float2(x[ii].z, x[ii].w), q23, accP[ii][i]);
        }
        accQ[i] = __ffma2_rn(make_float2(hn.x, hn.y), q01, accQ[i]);
        accQ[i] = __ffma2_rn(make_float2(hn.z, hn.w), q23, accQ[i]);
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
#pragma unroll
    for (int ii = 0; ii < RPL; ++ii) {
      float v = accP[ii][i].x + accP[ii][i].y;
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 16);
      if (cq == 0) red[warp * E + (sa + 8 * ii) * 8 + (sa ^ i)] = v;
    }
    float v = accQ[i].x + accQ[i].y;
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
  p.n = s.n;
  p.m = (int)s.m;
  p.r = s.r;
  p.nbox = (int)((s.n + kBoxCols - 1) / kBoxCols);
  p.eps = eps;
  mu_pass_narrow_kernel<C><<<s.grid, kNarrowThreads, C::SMEM, st>>>(mx, mh, p);
  return cudaGetLastError();
}

}  // namespace

bool narrow_pass_supported(int MP, int R) { return (MP == 16 || MP == 32) && R == 8; }

cudaError_t launch_mu_pass_narrow(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                                  const CUtensorMap& mh, cudaStream_t st) {
  if (s.R != 8) return cudaErrorInvalidValue;
  if (s.MP == 16) return launch_narrow_cfg<NarrowCfg<16>>(s, d, eps, mx, mh, st);
  if (s.MP == 32) return launch_narrow_cfg<NarrowCfg<32>>(s, d, eps, mx, mh, st);
  return cudaErrorInvalidValue;
}

}  // namespace ntt
