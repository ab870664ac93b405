// Algorithm 3 (distBCDnmf) on one GPU: block coordinate descent NMF with
// prox-linear block steps, extrapolation and the restart ("correction") test,
// read through the APG-BCD method the paper cites (Xu & Yin 2013):
//
//   W_new = max(0, W_m - (W_m Q - P) / L_w),   L_w = ||Q||_2,  P = X H^T, Q = H H^T
//   H_new = max(0, H_m - (G H_m - W_new^T X) / L_h),  G = W_new^T W_new, L_h = ||G||_2
//   f     = 1/2 ||X - W_new H_new||^2  (the pass's direct residual of each tile
//           it holds, FP64 across tiles: no extra read of X)
//   f >= f_accepted: reject -- the next steps start from the accepted iterate
//   otherwise accept; t' = (1 + sqrt(1 + 4 t^2)) / 2, w = (t - 1) / t',
//   w_W = min(w, delta sqrt(L_w,prev / L_w)), w_H likewise, and
//   W_m = W_new + w_W (W_new - W_acc), H_m = H_new + w_H (H_new - H_acc).
//
// One iteration is one pass over X (the BCD mode of the fused pass: the H step,
// then P and Q of H_new from the same tile) plus one combine launch: the
// fixed-order reduction of the pass partials, then in its last block the
// accept/reject decision, the W extrapolation and W step of the next
// iteration, G and the Lipschitz constants.  H lives in three buffers whose
// roles (accepted, previous accepted, new) rotate through the device state, so
// the launch sequence is fixed and graph-capturable.
//
// Lipschitz constants: the largest eigenvalue of an r x r (r <= 32) symmetric
// positive semi-definite matrix A from 20 normalised squarings in FP32
// (A^(2^20) is the projector onto the top eigenspace up to scale) and the FP64
// Rayleigh quotient of one of its columns; the relative error is below 2e-7
// however close the top eigenvalues are.
#include <cmath>
#include <cstring>

#include "ntt_internal.cuh"

namespace ntt {

#define NTT_DECL_BCD(MP)                                                                                   \
  cudaError_t launch_pass_bcd_f32_m##MP(int R, const MuShape& s, const MuDev& d, const CUtensorMap& mx,    \
                                         const HMaps3& mh, float* const* Hb, const BcdState* st_dev,        \
                                         int init, double* res_part, cudaStream_t st);
NTT_DECL_BCD(16)
NTT_DECL_BCD(32)
NTT_DECL_BCD(64)
NTT_DECL_BCD(128)
NTT_DECL_BCD(256)
NTT_DECL_BCD(512)
#undef NTT_DECL_BCD

#define NTT_TRY_I(expr)              \
  do {                               \
    ntt_status s_ = (expr);          \
    if (s_ != NTT_OK) return s_;     \
  } while (0)

namespace {

constexpr int kEntries = 32;
constexpr int kChunks = kAuxThreads / kEntries;   // 8
constexpr int kSquarings = 20;

struct BcdCombineParams {
  const float* part;   // grid x E partials of [P ; Q] of H_new
  const double* res_part;   // grid: ||X - W_new H_new||^2 over each pass CTA's tiles
  int nb;              // pass CTAs
  int MP, R, m, r;
  float* red;          // E: reduced [P ; Q] (FP32)
  float* pacc;         // E: [P ; Q] of the accepted H
  float* Wn;           // m x r: W_new of this iteration (in), of the next one (out)
  float* Wacc;         // m x r: accepted W (the caller's W)
  float* G;            // R x R: Gram of W_new (in: this iteration's; out: the next one's)
  unsigned* ticket;
  BcdState* st;
  const double* xnorm2;
  double* obj;         // trace (obj[t] = accepted objective after iteration t) or NULL
  int t;
  int init;            // first combine: [P ; Q] of the initial H, no decision
  double delta;
};

// Largest eigenvalue of the r x r block of A (row stride R) in shared memory.
// M0, M1: R x R scratch; red64: >= 8 doubles.  Whole block; returns the value in every thread.
__device__ double lambda_max(const float* A, int r, int R, float* M0, float* M1, double* red64) {
  __shared__ float s_tr;
  __shared__ int s_col;
  const int tid = threadIdx.x;
  if (tid == 0) {
    float tr = 0.0f;
    for (int i = 0; i < r; ++i) tr += A[i * R + i];
    s_tr = tr;
  }
  __syncthreads();
  const float tr0 = s_tr;
  if (!(tr0 > 0.0f)) return 0.0;
  for (int e = tid; e < r * r; e += blockDim.x) M0[e] = A[(e / r) * R + e % r] / tr0;
  __syncthreads();
  float* a = M0;
  float* b = M1;
  for (int it = 0; it < kSquarings; ++it) {
    for (int e = tid; e < r * r; e += blockDim.x) {
      const int i = e / r, j = e % r;
      float s = 0.0f;
      for (int k = 0; k < r; ++k) s = fmaf(a[i * r + k], a[k * r + j], s);
      b[e] = s;
    }
    __syncthreads();
    if (tid == 0) {
      float tr = 0.0f;
      for (int i = 0; i < r; ++i) tr += b[i * r + i];
      s_tr = tr;
    }
    __syncthreads();
    const float tr = s_tr;
    for (int e = tid; e < r * r; e += blockDim.x) b[e] = tr > 0.0f ? b[e] / tr : 0.0f;
    __syncthreads();
    float* t = a;
    a = b;
    b = t;
  }
  if (tid == 0) {
    int best = 0;
    for (int i = 1; i < r; ++i)
      if (a[i * r + i] > a[best * r + best]) best = i;
    s_col = best;
  }
  __syncthreads();
  // Rayleigh quotient of v = column s_col of the projector, in FP64
  if (tid == 0) {
    const int c = s_col;
    double num = 0.0, den = 0.0;
    for (int i = 0; i < r; ++i) {
      const double vi = (double)a[i * r + c];
      double av = 0.0;
      for (int k = 0; k < r; ++k) av += (double)A[i * R + k] * (double)a[k * r + c];
      num += vi * av;
      den += vi * vi;
    }
    red64[0] = den > 0.0 ? num / den : 0.0;
  }
  __syncthreads();
  const double v = red64[0];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kAuxThreads) bcd_combine_kernel(const BcdCombineParams p) {
  extern __shared__ float sm[];
  __shared__ float chunk[kChunks][kEntries];
  __shared__ double dsh[kAuxThreads];
  __shared__ int s_last;
  __shared__ int s_acc;
  __shared__ float s_ww, s_lw;
  const int tid = threadIdx.x;
  const int E = (p.MP + p.R) * p.R;

  // ---- 1. fixed-order reduction of 32 entries per block (FP32 chunks, FP64 across)
  {
    const int el = tid % kEntries, j = tid / kEntries;
    const int e = blockIdx.x * kEntries + el;
    const int per = (p.nb + kChunks - 1) / kChunks;
    const int b0 = j * per, b1 = min(p.nb, b0 + per);
    float s = 0.0f;
    if (e < E)
      for (int bb = b0; bb < b1; ++bb) s += __ldcg(&p.part[(size_t)bb * E + e]);
    chunk[j][el] = s;
    __syncthreads();
    if (tid < kEntries && e < E) {
      double t[kChunks];
#pragma unroll
      for (int c = 0; c < kChunks; ++c) t[c] = (double)chunk[c][tid];
#pragma unroll
      for (int w = 1; w < kChunks; w *= 2)
#pragma unroll
        for (int c = 0; c + w < kChunks; c += 2 * w) t[c] += t[c + w];
      p.red[e] = (float)t[0];
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(p.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---- 2. last block
  const int m = p.m, r = p.r, R = p.R, MP = p.MP;
  float* red_s = sm;                      // E
  float* Ws = red_s + E;                  // m x r: W_new of the next iteration
  float* Gs = Ws + m * r;                 // R x R
  float* M0 = Gs + R * R;                 // r x r scratch (two)
  float* M1 = M0 + R * R;
  BcdState* st = p.st;
  for (int e = tid; e < E; e += blockDim.x) red_s[e] = __ldcg(&p.red[e]);
  for (int e = tid; e < R * R; e += blockDim.x) Gs[e] = __ldcg(&p.G[e]);
  __syncthreads();

  if (p.init) {
    if (tid == 0) {
      st->t = 1.0;
      st->obj = 0.5 * (*p.xnorm2);
      st->Lw_prev = -1.0;
      st->Lh_prev = -1.0;
      st->accepted = 0;
      st->last_ok = 0;
      st->rot = 0;
      st->w_h = 0.0f;
      s_acc = 0;
      s_ww = 0.0f;
    }
    for (int e = tid; e < E; e += blockDim.x) p.pacc[e] = red_s[e];
  } else {
    // objective of (W_new, H_new): 1/2 ||X - W_new H_new||^2 from the pass's
    // direct per-CTA residuals (FP32 within a tile, FP64 across), summed in a
    // fixed order -- the value Algorithm 3's test compares; the expanded Gram
    // form would lose about 1e-7 ||X||^2 to cancellation near convergence
    if (tid < 32) {
      double v = 0.0;
      for (int b2 = tid; b2 < p.nb; b2 += 32) v += __ldcg(&p.res_part[b2]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (tid == 0) dsh[0] = v;
    }
    __syncthreads();
    if (tid == 0) {
      const double f = 0.5 * dsh[0];
      const int acc = f < st->obj ? 1 : 0;
      s_acc = acc;
      if (acc) {
        const double t = st->t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        const double w = (t - 1.0) / tn;
        const double Lw = st->Lw, Lh = (double)st->Lh;
        const double lwp = st->Lw_prev < 0.0 ? Lw : st->Lw_prev;
        const double lhp = st->Lh_prev < 0.0 ? Lh : st->Lh_prev;
        s_ww = Lw > 0.0 ? (float)fmin(w, p.delta * sqrt(lwp / Lw)) : 0.0f;
        st->w_h = Lh > 0.0 ? (float)fmin(w, p.delta * sqrt(lhp / Lh)) : 0.0f;
        st->t = tn;
        st->obj = f;
        st->Lw_prev = Lw;
        st->Lh_prev = Lh;
        st->rot = (st->rot + 1) % 3;
        st->accepted += 1;
      } else {
        s_ww = 0.0f;
        st->w_h = 0.0f;
      }
      st->last_ok = acc;
      if (p.obj) p.obj[p.t] = st->obj;
    }
    __syncthreads();
    if (s_acc) {
      for (int e = tid; e < E; e += blockDim.x) p.pacc[e] = red_s[e];
    } else {
      for (int e = tid; e < E; e += blockDim.x) red_s[e] = __ldcg(&p.pacc[e]);   // back to the accepted P, Q
    }
    __syncthreads();
  }
  // W_m (per row, in place of the accepted W when accepted), then the W step
  // of the next iteration with Q, P of the accepted H: L_w = ||Q||_2
  const double Lw = lambda_max(red_s + MP * R, r, R, M0, M1, dsh);
  if (tid == 0) s_lw = (float)Lw;
  __syncthreads();
  const float lw = s_lw, ww = s_ww;
  const bool accepted = p.init || s_acc;
  for (int i = tid; i < m; i += blockDim.x) {
    float wm[NTT_MAX_RANK];
#pragma unroll
    for (int k = 0; k < NTT_MAX_RANK; ++k) {
      if (k >= r) break;
      const float wa = __ldcg(&p.Wacc[i * r + k]);
      if (accepted && !p.init) {
        const float wn = __ldcg(&p.Wn[i * r + k]);
        wm[k] = fmaf(ww, wn - wa, wn);
        p.Wacc[i * r + k] = wn;
      } else {
        wm[k] = wa;
      }
    }
    for (int k = 0; k < r; ++k) {
      float g = 0.0f;
      for (int l = 0; l < r; ++l) g = fmaf(wm[l], red_s[(MP + l) * R + k], g);
      g -= red_s[i * R + k];
      Ws[i * r + k] = lw > 0.0f ? fmaxf(0.0f, wm[k] - __fdiv_rn(g, lw)) : wm[k];
    }
  }
  __syncthreads();
  for (int e = tid; e < m * r; e += blockDim.x) p.Wn[e] = Ws[e];
  // G = W_new^T W_new (R x R, zero padded) and L_h = ||G||_2
  for (int kl = tid; kl < R * R; kl += blockDim.x) {
    const int k = kl / R, l = kl % R;
    float g = 0.0f;
    if (k < r && l < r) {
      float a8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int i = 0;
      for (; i + 8 <= m; i += 8)
#pragma unroll
        for (int u = 0; u < 8; ++u) a8[u] = fmaf(Ws[(i + u) * r + k], Ws[(i + u) * r + l], a8[u]);
      for (; i < m; ++i) a8[0] = fmaf(Ws[i * r + k], Ws[i * r + l], a8[0]);
      g = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
    }
    Gs[kl] = g;
    p.G[kl] = g;
  }
  __syncthreads();
  const double Lh = lambda_max(Gs, r, R, M0, M1, dsh);
  if (tid == 0) {
    st->Lw = Lw;
    st->Lh = (float)Lh;
    if (p.init) st->init = 1;
    *p.ticket = 0u;
  }
}

// W and H scaled to Frobenius norm sqrt(||X||_F) each (Algorithm 3's normalisation);
// acc = [||X||^2, ||W||^2, ||H||^2].  Also resets the solve's state.
__global__ void bcd_scale_kernel(float* W, int64_t mw, float* H, int64_t mh, const double* xn2, const double* wn2,
                                 const double* hn2, BcdState* st) {
  const double sx = sqrt(sqrt(*xn2));
  const double w2 = *wn2, h2 = *hn2;
  const float fw = w2 > 0.0 ? (float)(sx / sqrt(w2)) : 1.0f;
  const float fh = h2 > 0.0 ? (float)(sx / sqrt(h2)) : 1.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mw; i += stride) W[i] *= fw;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < mh; i += stride) H[i] *= fh;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rot = 0;
    st->w_h = 0.0f;
    st->Lh = 0.0f;
    st->init = 0;
  }
}

// The accepted H into buffer 0 (the caller's H) when it ended in another buffer.
__global__ void bcd_copy_kernel(float* H0, const float* H1, const float* H2, int64_t count, const BcdState* st) {
  const int rot = st->rot;
  if (rot == 0) return;
  const float* src = rot == 1 ? H1 : H2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) H0[i] = src[i];
}

}  // namespace

BcdWs bcd_ws_layout(const MuShape& s) {
  BcdWs w;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = (off + b + 255) / 256 * 256;
    return o;
  };
  w.state = take(sizeof(BcdState));
  w.Wn = take((size_t)s.m * s.r * 4);
  w.pacc = take((size_t)s.part_stride() * 4);
  w.H1 = take((size_t)s.r * s.n * 4);
  w.H2 = take((size_t)s.r * s.n * 4);
  w.norms = take(4 * sizeof(double));
  w.respart = take((size_t)kMaxPassCtas * sizeof(double));
  w.bytes = off;
  return w;
}

ntt_status run_bcd_iters(const MuShape& shp, const MuDev& dev, const BcdWs& L, char* bws, int iters, int t0,
                         cudaStream_t st) {
  MuShape s = shp;
  s.route = NTT_ROUTE_GENERIC;   // the BCD step lives in the generic pass
  mu_finalize_shape(&s, dev.X, dev.H, device_sms());
  float* Hb[3] = {dev.H, reinterpret_cast<float*>(bws + L.H1), reinterpret_cast<float*>(bws + L.H2)};
  // every H buffer must satisfy the TMA alignment rules for the maps to be used
  for (int i = 1; i < 3 && s.tma; ++i)
    if (!mu_tma_ok(s, dev.X, Hb[i])) s.tma = 0;
  CUtensorMap mx;
  HMaps3 mh;
  std::memset(&mx, 0, sizeof(mx));
  std::memset(&mh, 0, sizeof(mh));
  if (s.tma)
    for (int i = 0; i < 3; ++i) {
      CUtensorMap dummy;
      NTT_TRY_I(mu_encode_maps(s, dev.X, Hb[i], i == 0 ? &mx : &dummy, &mh.h[i]));
    }
  BcdState* state = reinterpret_cast<BcdState*>(bws + L.state);
  float* Wn = reinterpret_cast<float*>(bws + L.Wn);
  double* norms = reinterpret_cast<double*>(bws + L.norms);
  double* respart = reinterpret_cast<double*>(bws + L.respart);
  // Algorithm 3's normalisation of the initial factors, the state reset
  NTT_TRY_I(resid_into(dev.X, 0, nullptr, nullptr, s.m, s.n, 0, 0, 1.0, norms, nullptr, dev.part64, dev.ticket + 1, st));
  NTT_TRY_I(resid_into(dev.W, 0, nullptr, nullptr, s.m, s.r, 0, 0, 1.0, norms + 1, nullptr, dev.part64, dev.ticket + 1, st));
  NTT_TRY_I(resid_into(dev.H, 0, nullptr, nullptr, s.r, s.n, 0, 0, 1.0, norms + 2, nullptr, dev.part64, dev.ticket + 1, st));
  bcd_scale_kernel<<<(unsigned)std::min<int64_t>(4 * device_sms(), (s.r * s.n + 255) / 256 + 1), 256, 0, st>>>(
      dev.W, s.m * s.r, dev.H, (int64_t)s.r * s.n, norms, norms + 1, norms + 2, state);
  if (cudaGetLastError() != cudaSuccess) return NTT_ERR_CUDA;
  MuDev d2 = dev;
  d2.G = dev.G;
  if (launch_gram(s, dev, st) != cudaSuccess) return NTT_ERR_CUDA;
  auto pass = [&](int init) -> cudaError_t {
    MuDev dp = dev;
    dp.W = init ? dev.W : Wn;
#define NTT_CASE(MPV) \
  case MPV:           \
    return launch_pass_bcd_f32_m##MPV(s.R, s, dp, mx, mh, Hb, state, init, respart, st);
    switch (s.MP) {
      NTT_CASE(16)
      NTT_CASE(32)
      NTT_CASE(64)
      NTT_CASE(128)
      NTT_CASE(256)
      NTT_CASE(512)
      default:
        return cudaErrorInvalidValue;
    }
#undef NTT_CASE
  };
  const int E = s.part_stride();
  const int blocks = (E + kEntries - 1) / kEntries;
  const size_t smem = (size_t)(E + s.m * s.r + 3 * s.R * s.R) * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(bcd_combine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
        cudaSuccess)
      return NTT_ERR_CUDA;
    attr_set = true;
  }
  auto combine = [&](int init, int t) -> cudaError_t {
    BcdCombineParams c;
    c.part = dev.part;
    c.res_part = respart;
    c.nb = s.grid;
    c.MP = s.MP;
    c.R = s.R;
    c.m = (int)s.m;
    c.r = s.r;
    c.red = dev.red;
    c.pacc = reinterpret_cast<float*>(bws + L.pacc);
    c.Wn = Wn;
    c.Wacc = dev.W;
    c.G = dev.G;
    c.ticket = dev.ticket;
    c.st = state;
    c.xnorm2 = norms;
    c.obj = init ? nullptr : dev.obj;
    c.t = t;
    c.init = init;
    c.delta = kBcdDelta;
    bcd_combine_kernel<<<blocks, kAuxThreads, smem, st>>>(c);
    return cudaGetLastError();
  };
  if (pass(1) != cudaSuccess || combine(1, 0) != cudaSuccess) return NTT_ERR_CUDA;
  for (int t = 0; t < iters; ++t)
    if (pass(0) != cudaSuccess || combine(0, t0 + t) != cudaSuccess) return NTT_ERR_CUDA;
  bcd_copy_kernel<<<(unsigned)std::min<int64_t>(4 * device_sms(), (s.r * s.n + 255) / 256 + 1), 256, 0, st>>>(
      Hb[0], Hb[1], Hb[2], (int64_t)s.r * s.n, state);
  return cudaGetLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // namespace ntt
