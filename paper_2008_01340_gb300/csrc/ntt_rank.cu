// Algorithm 2's rank rule on the device: r_l is the smallest k with
//   sqrt(sigma_{k+1}^2 + ... + sigma_N^2) / sqrt(sigma_1^2 + ... + sigma_N^2) <= eps,
// sigma_i the singular values of the unfolding X_l (m x n), N = min(m, n).
//
// The singular values come from the eigenvalues of the N x N Gram matrix
// (X X^T when m <= n, X^T X otherwise), whose eigenvalues are the sigma_i^2:
//   gram_part_kernel   64 x 64 blocks of the Gram over column (or row) chunks:
//                      FP32 products and sums over runs of 256, added into
//                      FP64 accumulators (X >= 0: no cancellation inside a run)
//   gram_combine_kernel fixed-order FP64 sum of the chunk partials, both
//                      triangles written
//   tridiag_kernel     Householder reduction of the FP64 Gram to a symmetric
//                      tridiagonal matrix (one CTA; the matrix stays in L2)
//   eig_rule_kernel    every eigenvalue by bisection on Sturm counts of the
//                      tridiagonal matrix (FP64), sigma_i = sqrt(max(0, lambda_i))
//                      in non-increasing order, then the tail rule in FP64
// Everything after the Gram runs in FP64; the Gram itself carries the FP32
// rounding of its runs (about 1e-7 relative per entry).
#include <cmath>

#include "ntt_internal.cuh"

namespace ntt {

namespace {

constexpr int kGB = 64;          // Gram block rows
constexpr int kGK = 32;          // reduction indices per tile
constexpr int kGRun = 8;         // tiles per FP32 run (256 indices)
constexpr int kGThreads = 256;   // 16 x 16 threads, 4 x 4 entries each
constexpr int kTriThreads = 1024;
constexpr int kMaxGram = NTT_MAX_ROWS;   // N <= 512

// U(r, k): r < M indexes the Gram, k < K the reduction; U = X (m <= n) or X^T.
struct GramArgs {
  const float* X;
  int64_t m, n;
  int trans;        // 1: U = X^T (M = n, K = m)
  int M;            // Gram size
  int64_t K;        // reduction length
  int nb;           // row blocks of 64
  int S;            // chunks of the reduction
  int64_t chunk;    // reduction indices per chunk (multiple of kGK)
  double* part;     // npairs x S x 64 x 64
};

__device__ __forceinline__ void pair_of(int p, int nb, int* bi, int* bj) {
  int i = 0;
  while (p >= nb - i) {
    p -= nb - i;
    ++i;
  }
  *bi = i;
  *bj = i + p;
}

__global__ void __launch_bounds__(kGThreads) gram_part_kernel(const GramArgs a) {
  __shared__ __align__(16) float ua[kGK][kGB + 4];
  __shared__ __align__(16) float ub[kGK][kGB + 4];
  const int pair = blockIdx.x / a.S, s = blockIdx.x % a.S;
  int bi, bj;
  pair_of(pair, a.nb, &bi, &bj);
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t k0 = (int64_t)s * a.chunk;
  const int64_t k1 = min(a.K, k0 + a.chunk);
  double acc64[4][4];
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc64[i][j] = 0.0, acc[i][j] = 0.0f;
  int run = 0;
  for (int64_t kt = k0; kt < k1; kt += kGK) {
    __syncthreads();
    // tile: U(r, k) for r in the two blocks, k in [kt, kt + 32)
    for (int e = tid; e < kGK * kGB; e += kGThreads) {
      int kk, rr;
      if (a.trans) {   // X rows k, Gram index contiguous: coalesced over rr
        kk = e / kGB;
        rr = e % kGB;
      } else {         // X rows r, reduction index contiguous: coalesced over kk
        rr = e / kGK;
        kk = e % kGK;
      }
      const int64_t k = kt + kk;
      const int ra = bi * kGB + rr, rb = bj * kGB + rr;
      float va = 0.0f, vb = 0.0f;
      if (k < k1) {
        if (a.trans) {
          if (ra < a.M) va = __ldg(&a.X[k * a.n + ra]);
          if (rb < a.M) vb = __ldg(&a.X[k * a.n + rb]);
        } else {
          if (ra < a.M) va = __ldg(&a.X[(int64_t)ra * a.n + k]);
          if (rb < a.M) vb = __ldg(&a.X[(int64_t)rb * a.n + k]);
        }
      }
      ua[kk][rr] = va;
      ub[kk][rr] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 x = *reinterpret_cast<const float4*>(&ua[kk][ty * 4]);
      const float4 y = *reinterpret_cast<const float4*>(&ub[kk][tx * 4]);
      const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], yb[j], acc[i][j]);
    }
    if (++run == kGRun) {
      run = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc64[i][j] += (double)acc[i][j], acc[i][j] = 0.0f;
    }
  }
  double* out = a.part + ((size_t)pair * a.S + s) * (kGB * kGB);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * kGB + tx * 4 + j] = acc64[i][j] + (double)acc[i][j];
}

// G (M x M, FP64) = fixed-order sum of the chunk partials; one block per pair.
__global__ void __launch_bounds__(kGThreads) gram_combine_kernel(const double* part, int S, int nb, int M,
                                                                 double* G) {
  int bi, bj;
  pair_of(blockIdx.x, nb, &bi, &bj);
  const double* p = part + (size_t)blockIdx.x * S * (kGB * kGB);
  for (int e = threadIdx.x; e < kGB * kGB; e += kGThreads) {
    const int r = bi * kGB + e / kGB, c = bj * kGB + e % kGB;
    double v = 0.0;
    for (int s = 0; s < S; ++s) v += p[(size_t)s * (kGB * kGB) + e];
    if (r < M && c < M) {
      G[(size_t)r * M + c] = v;
      G[(size_t)c * M + r] = v;
    }
  }
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];   // same order in every thread
  return t;
}

// Householder reduction A -> Q^T A Q = tridiag(d, e) in place (A: M x M FP64,
// symmetric, both triangles).  Step k reflects rows/columns k+1.. so that
// column k below the subdiagonal vanishes: x = A[k+1:, k], alpha =
// -sign(x_0) ||x||, u = (x - alpha e_1) / ||x - alpha e_1||, p = A22 u,
// q = p - (u^T p) u, A22 <- A22 - 2 (u q^T + q u^T).
__global__ void __launch_bounds__(kTriThreads) tridiag_kernel(double* A, int M, double* d, double* e) {
  __shared__ double u[kMaxGram], q[kMaxGram];
  __shared__ double red[kTriThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kTriThreads / 32;
  for (int k = 0; k + 2 < M; ++k) {
    const int L = M - k - 1;
    double* A22 = A + (size_t)(k + 1) * M + (k + 1);
    // x = A[k+1.., k] (column k = row k by symmetry: contiguous)
    double ss = 0.0;
    for (int i = tid; i < L; i += kTriThreads) {
      const double x = A[(size_t)k * M + k + 1 + i];
      u[i] = x;
      ss += x * x;
    }
    const double nrm2 = block_sum(ss, red);
    const double x0 = u[0];
    __syncthreads();
    if (tid == 0) d[k] = A[(size_t)k * M + k];
    const double tail2 = nrm2 - x0 * x0;
    if (!(tail2 > 0.0)) {            // column already reduced
      if (tid == 0) e[k] = x0;
      __syncthreads();
      continue;
    }
    const double alpha = x0 >= 0.0 ? -sqrt(nrm2) : sqrt(nrm2);
    const double v0 = x0 - alpha;
    const double inv = 1.0 / sqrt(tail2 + v0 * v0);
    if (tid == 0) e[k] = alpha;
    __syncthreads();
    for (int i = tid; i < L; i += kTriThreads) u[i] = (i == 0 ? v0 : u[i]) * inv;
    __syncthreads();
    // p = A22 u: one warp per row, lanes over columns (coalesced)
    for (int i = warp; i < L; i += nw) {
      const double* row = A22 + (size_t)i * M;
      double s = 0.0;
      for (int j = lane; j < L; j += 32) s += row[j] * u[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) q[i] = s;
    }
    __syncthreads();
    double up = 0.0;
    for (int i = tid; i < L; i += kTriThreads) up += u[i] * q[i];
    const double K = block_sum(up, red);
    for (int i = tid; i < L; i += kTriThreads) q[i] -= K * u[i];
    __syncthreads();
    for (int i = warp; i < L; i += nw) {
      double* row = A22 + (size_t)i * M;
      const double ui = u[i], qi = q[i];
      for (int j = lane; j < L; j += 32) row[j] -= 2.0 * (ui * q[j] + qi * u[j]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (M >= 2) {
      d[M - 2] = A[(size_t)(M - 2) * M + (M - 2)];
      e[M - 2] = A[(size_t)(M - 1) * M + (M - 2)];
    }
    d[M - 1] = A[(size_t)(M - 1) * M + (M - 1)];
  }
}

// Number of eigenvalues of tridiag(d, e) below x (Sturm count of T - x I).
__device__ int sturm_below(const double* d, const double* e2, int M, double x, double tiny) {
  int cnt = 0;
  double q = d[0] - x;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < M; ++i) {
    if (fabs(q) < tiny) q = -tiny;
    q = d[i] - x - e2[i - 1] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// sigma (non-increasing) and, when rank_out is set, the tail rule.
__global__ void __launch_bounds__(kTriThreads) eig_rule_kernel(const double* d_in, const double* e_in, int M,
                                                               double eps_rank, int rank_cap, double* sigma,
                                                               int* rank_out) {
  __shared__ double d[kMaxGram], e2[kMaxGram], lam[kMaxGram];
  __shared__ double bounds[2];
  const int tid = threadIdx.x;
  for (int i = tid; i < M; i += kTriThreads) {
    d[i] = d_in[i];
    e2[i] = i + 1 < M ? e_in[i] * e_in[i] : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    // Gershgorin interval of every eigenvalue
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < M; ++i) {
      const double rad = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < M ? sqrt(e2[i]) : 0.0);
      lo = fmin(lo, d[i] - rad);
      hi = fmax(hi, d[i] + rad);
    }
    const double w = fmax(fabs(lo), fabs(hi));
    bounds[0] = lo - 1e-12 * w - 1e-300;
    bounds[1] = hi + 1e-12 * w + 1e-300;
  }
  __syncthreads();
  const double scale = fmax(fabs(bounds[0]), fabs(bounds[1]));
  const double tiny = 1e-300 + 1e-30 * scale;
  // lambda_j (ascending, j = 0..M-1): the point where the count passes j
  for (int j = tid; j < M; j += kTriThreads) {
    double lo = bounds[0], hi = bounds[1];
    for (int it = 0; it < 200 && hi - lo > 2e-16 * scale; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (sturm_below(d, e2, M, mid, tiny) > j)
        hi = mid;
      else
        lo = mid;
    }
    lam[j] = 0.5 * (lo + hi);
  }
  __syncthreads();
  for (int i = tid; i < M; i += kTriThreads) sigma[i] = sqrt(fmax(0.0, lam[M - 1 - i]));
  if (rank_out && tid == 0) {
    // the total is the trace (= the sum of the eigenvalues), exactly 0 for X = 0
    double total = 0.0;
    for (int i = 0; i < M; ++i) total += d[i];
    int k_sel = M;
    if (!(total > 0.0)) {
      k_sel = 1;
    } else {
      // tail after k: the M - k smallest eigenvalues, summed from the smallest up
      double tail = 0.0;
      int k = M;
      // tails[k] for k = M-1 .. 1 is tail + lam of the next larger one
      for (k = M - 1; k >= 1; --k) {
        tail += fmax(0.0, lam[M - 1 - k]);   // sigma_{k+1}^2 (1-based) = lam[M-1-k]
        if (sqrt(tail) / sqrt(total) <= eps_rank) k_sel = k;
        else break;
      }
    }
    if (rank_cap > 0 && k_sel > rank_cap) k_sel = rank_cap;
    *rank_out = k_sel < 1 ? 1 : k_sel;
  }
}

}  // namespace

RankWs rank_ws_layout(int64_t m, int64_t n, int num_sms) {
  RankWs w;
  const int64_t M = m <= n ? m : n;
  const int64_t K = m <= n ? n : m;
  w.M = (int)M;
  w.nb = (int)((M + kGB - 1) / kGB);
  const int npairs = w.nb * (w.nb + 1) / 2;
  // chunks: about two CTAs per SM in total, each at least one tile
  const int64_t tiles = (K + kGK - 1) / kGK;
  int64_t S = ((int64_t)2 * (num_sms > 0 ? num_sms : 152) + npairs - 1) / npairs;
  if (S > tiles) S = tiles;
  if (S < 1) S = 1;
  w.S = (int)S;
  w.chunk = ((tiles + S - 1) / S) * kGK;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = (off + b + 255) / 256 * 256;
    return o;
  };
  w.off_part = take((size_t)npairs * w.S * kGB * kGB * sizeof(double));
  w.off_G = take((size_t)M * M * sizeof(double));
  w.off_d = take((size_t)M * sizeof(double));
  w.off_e = take((size_t)M * sizeof(double));
  w.off_sigma = take((size_t)M * sizeof(double));
  w.off_rank = take(64);
  w.bytes = off;
  return w;
}

cudaError_t launch_rank_select(const float* X, int64_t m, int64_t n, double eps_rank, int rank_cap,
                               const RankWs& w, char* ws, double* sigma_out, int* rank_out, cudaStream_t st) {
  if (w.M < 1 || w.M > kMaxGram) return cudaErrorInvalidValue;
  GramArgs a;
  a.X = X;
  a.m = m;
  a.n = n;
  a.trans = m <= n ? 0 : 1;
  a.M = w.M;
  a.K = m <= n ? n : m;
  a.nb = w.nb;
  a.S = w.S;
  a.chunk = w.chunk;
  a.part = reinterpret_cast<double*>(ws + w.off_part);
  const int npairs = w.nb * (w.nb + 1) / 2;
  gram_part_kernel<<<npairs * w.S, kGThreads, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* G = reinterpret_cast<double*>(ws + w.off_G);
  gram_combine_kernel<<<npairs, kGThreads, 0, st>>>(a.part, w.S, w.nb, w.M, G);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double* d = reinterpret_cast<double*>(ws + w.off_d);
  double* ev = reinterpret_cast<double*>(ws + w.off_e);
  tridiag_kernel<<<1, kTriThreads, 0, st>>>(G, w.M, d, ev);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  double* sigma = sigma_out ? sigma_out : reinterpret_cast<double*>(ws + w.off_sigma);
  eig_rule_kernel<<<1, kTriThreads, 0, st>>>(d, ev, w.M, eps_rank, rank_cap, sigma, rank_out);
  return cudaGetLastError();
}

}  // namespace ntt
