// Internal declarations shared by the CUDA translation units of libntt.
//
// Device helpers: SplitMix64 counter RNG, bounded mbarrier waits, TMA 2-D
// tile loads (cp.async.bulk.tensor), and the launchers of every kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ntt.h"

namespace ntt {

// ---------------------------------------------------------------------------
// Limits and constants
// ---------------------------------------------------------------------------
constexpr int kPassThreads = 256;      // threads of the streaming pass kernel
constexpr int kMaxPassCtas = 1024;     // upper bound of the pass grid
constexpr int kAuxThreads = 256;
constexpr long long kWaitLimitNs = 2000000000LL;   // 2 s bound on every device wait

// Device status word values (a subset of ntt_status).
constexpr int kStatusOk = NTT_OK;
constexpr int kStatusTimeout = NTT_ERR_TIMEOUT;

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014): output i of a generator seeded with s
// is mix64(s + (i+1) * gamma).
// ---------------------------------------------------------------------------
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t splitmix_output(uint64_t seed, uint64_t index) {
  return mix64(seed + (index + 1ULL) * kGamma);
}

// Key of the stream (stage, restart, matrix): output stage*2^20 + restart*2 + matrix.
inline uint64_t stream_key(uint64_t seed, int stage, int restart, int matrix) {
  const uint64_t stream = ((uint64_t)stage << 20) + ((uint64_t)restart << 1) + (uint64_t)matrix;
  return splitmix_output(seed, stream);
}

__device__ __forceinline__ float uniform24(uint64_t key, uint64_t index) {
  return (float)(splitmix_output(key, index) >> 40) * (1.0f / 16777216.0f);
}

// ---------------------------------------------------------------------------
// Shared-memory barriers and TMA (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// Host-side shape decisions for one multiplicative-update NMF
// ---------------------------------------------------------------------------
struct MuShape {
  int64_t m = 0, n = 0;
  int r = 0;
  int MP = 0;        // padded row count (template bucket)
  int R = 0;         // padded rank (8, 16, 32)
  int T = 0;         // tile width in columns
  int grid = 0;      // pass CTAs (= number of partials)
  int bf16 = 0;      // X stored as BF16
  int tma = 0;       // X/H tiles loaded by TMA (else cooperative loads)
  size_t smem = 0;   // dynamic shared memory of the pass kernel
  int part_stride() const { return (MP + R) * R; }
};

// Device pointers of one NMF.
struct MuDev {
  const void* X = nullptr;
  float* W = nullptr;
  float* H = nullptr;
  float* G = nullptr;            // R x R Gram of W, zero padded
  float* part = nullptr;         // grid x (MP+R) x R partials of [X H^T ; H H^T]
  float* red = nullptr;          // (MP+R) x R reduced partials
  unsigned* ticket = nullptr;    // last-block counter of the combine kernel
  double* obj = nullptr;         // objective trace or nullptr
  const double* xnorm2 = nullptr;
  int* status = nullptr;
};

// Pick template bucket, tile width and grid for an m x n x r problem.
ntt_status mu_choose_shape(int64_t m, int64_t n, int r, int bf16, int num_sms, MuShape* out);
// Whether X and H of these pointers can use TMA (alignment rules of the tensor maps).
bool mu_tma_ok(const MuShape& s, const void* X, const float* H);
// Encode the two tensor maps (X: m x n, H: r x n) for a TMA pass.
ntt_status mu_encode_maps(const MuShape& s, const void* X, const float* H, CUtensorMap* mx,
                          CUtensorMap* mh);

// Launchers (enqueue only; return the launch error).
cudaError_t launch_mu_pass(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                           const CUtensorMap& mh, cudaStream_t st);
cudaError_t launch_mu_combine(const MuShape& s, const MuDev& d, float eps, int t, cudaStream_t st);
cudaError_t launch_gram(const MuShape& s, const MuDev& d, cudaStream_t st);

cudaError_t launch_uniform(uint64_t key, int64_t count, float* out, cudaStream_t st);
cudaError_t launch_cast_bf16(const float* in, __nv_bfloat16* out, int64_t count, cudaStream_t st);

// Sum-of-squares / residual / reconstruction over an M x N matrix X (FP32 or
// BF16) against the product L (M x r) * Rm (r x N).
//   mode 0: acc[0] = sum X^2
//   mode 1: acc[0] = sum (X - L Rm)^2, acc[1] = sum X^2
//   mode 2: out = L Rm (no X)
// part64 holds `blocks` doubles, ticket one counter; results go to acc.
// When `rel` is non-null (mode 1), rel[0..2] = sqrt(acc0/acc1), acc0, acc1.
struct ResidArgs {
  const void* X = nullptr;
  int xbf16 = 0;
  const float* L = nullptr;
  const float* Rm = nullptr;
  float* out = nullptr;
  int64_t M = 0, N = 0;
  int r = 0;
  int mode = 0;
  double* part64 = nullptr;
  unsigned* ticket = nullptr;
  double* acc = nullptr;
  double* rel = nullptr;
  double scale = 1.0;   // acc[0] is multiplied by this (e.g. 0.5 for an objective)
};
int resid_blocks(int num_sms);
cudaError_t launch_resid(const ResidArgs& a, int blocks, cudaStream_t st);

// C = A (M x K) * B (K x N), FP32 row-major, K <= 32.
cudaError_t launch_small_mm(const float* A, const float* B, float* C, int64_t M, int K, int64_t N,
                            cudaStream_t st);

// Hand-off: s_k = sum_i W[i,k]; W[:,k] /= s_k and H[k,:] *= s_k where s_k > 0.
cudaError_t launch_handoff(float* W, float* H, int64_t m, int64_t n, int r, float* s_scratch,
                           cudaStream_t st);

// Number of SMs of the current device (cached; 152 when no device).
int device_sms();

}  // namespace ntt
