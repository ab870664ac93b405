// Internal declarations shared by the CUDA translation units of libntt.
//
// Device helpers: SplitMix64 counter RNG, bounded mbarrier waits, TMA 2-D
// tile loads (cp.async.bulk.tensor), and the launchers of every kernel.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// Programmatic dependent launch: a kernel started with launch_pdl may be
// scheduled before the previous kernel of its stream has finished; pdl_wait()
// returns once that kernel has completed and its writes are visible (a no-op
// for a kernel launched the ordinary way), so it comes before any read of
// them.  pdl_trigger() lets the next such kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Untiled bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completion counted on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// TMA tile store (shared -> global) tracked by the issuing thread's bulk group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(src), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most N committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N committed bulk groups are incomplete.
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): TMEM allocation, MMA issue, commit,
// TMEM loads and the shared-memory / instruction descriptors (sm_100 family).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D (TMEM, FP32) [+]= A (smem desc) x B (smem desc), TF32 inputs, one CTA.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  __syncwarp();
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Store 4 consecutive 32-bit columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c,
                                         uint32_t d) {
  __syncwarp();
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Load 4 / 8 / 16 consecutive FP32 columns of this thread's TMEM lane.  The
// loads are warp-collective (.sync.aligned): the warp is re-converged first.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  __syncwarp();
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  __syncwarp();
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor (sm_100 format): start address >> 4 in bits
// 0-13, leading byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45,
// descriptor version 1 at bit 46, base offset 0 (atoms are 1024-byte aligned),
// layout type in bits 61-63: 2 = 128-byte swizzle of 16-byte chunks over 8
// rows, 1 = 128-byte swizzle of 32-byte chunks over 4 rows (the layout TMA
// writes with CU_TENSOR_MAP_SWIZZLE_128B_ATOM_32B; TF32 operands read
// MN-major need it).  In layout 1, MN-major: LBO = stride between 32-element
// MN atoms, SBO = stride between 4-row K groups; K-major: SBO = stride between
// 4-row M/N groups.
constexpr uint32_t kLayoutSw128 = 2;
constexpr uint32_t kLayoutSw128Atom32 = 1;
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)layout << 61;
  return d;
}

// Instruction descriptor of kind::tf32 with FP32 accumulation: D format F32
// (bits 4-5 = 1), A and B format TF32 (bits 7-9, 10-12 = 2), A / B major
// (bit 15 / 16: 0 = K-major, 1 = MN-major), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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
  int grid_cap = 0;  // largest grid any pass may use (sizes the partial buffer)
  int bf16 = 0;      // X stored as BF16
  int tma = 0;       // X/H tiles loaded by TMA (else cooperative loads)
  int tcb = 0;       // BF16-X tensor-core pass (kind::f16, three-term split of the factors)
  int tcs = 0;       // FP32 X split in two BF16 matrices on the same tensor-core pass
  int narrow = 0;    // warp-streamed FMA pass for <= 32 rows, rank bucket 8, FP32 X (2: its 3-D-copy form)
  int tcw = 0;       // warp-level MMA pass: on the interleaved split of FP32 X (17..32 rows, rank bucket 8),
                     // or with bf16 on BF16 X (<= 16 rows, rank bucket 16)
  int route = NTT_ROUTE_AUTO;   // ntt_route restricting the pass choice
  int split_ok = 0;  // scratch for the two BF16 terms of X exists (MuDev::xs)
  int64_t ldh = 0;   // row stride of H when it is a column block of a wider H (generic pass only)
  size_t smem = 0;   // dynamic shared memory of the pass kernel
  int part_stride() const { return (MP + R) * R; }
};

// Device state of a BCD solve (Algorithm 3), written by its combine kernel.
struct BcdState {
  int rot;          // accepted H in buffer rot, previous accepted in (rot + 2) % 3, new in (rot + 1) % 3
  int init;         // 1 once the init combine has run
  float w_h;        // extrapolation weight of the next H step (0 after a rejection)
  float Lh;         // ||W^T W||_2 of the next H step
  double obj;       // last accepted objective 1/2 ||X - W H||^2 (FP64, Gram form)
  double t;         // extrapolation sequence t_k
  double Lw, Lw_prev, Lh_prev;   // Lipschitz constants: current W step, last accepted iteration
  int accepted;     // iterations accepted so far
  int last_ok;      // whether the last iteration was accepted
};

struct HMaps3 {
  CUtensorMap h[3];          // the three H buffers of a BCD solve
};

constexpr double kBcdDelta = 0.9999;   // delta of Algorithm 3's extrapolation weights

// Scratch of a BCD solve (after the nmf_mu_step scratch): state, W_new,
// accepted [P ; Q], the two extra H buffers, norms.
struct BcdWs {
  size_t state = 0, Wn = 0, pacc = 0, H1 = 0, H2 = 0, norms = 0, respart = 0, bytes = 0;
};

// Device pointers of one NMF.
struct MuDev {
  const void* X = nullptr;
  const void* X2 = nullptr;      // split form: X - bf16(X) in BF16 (X then holds bf16(X))
  __nv_bfloat16* xs = nullptr;   // scratch of 2 m n BF16 for the split form, or NULL
  float* W = nullptr;
  float* H = nullptr;
  float* G = nullptr;            // R x R Gram of W, zero padded
  float* part = nullptr;         // grid x (MP+R) x R partials of [X H^T ; H H^T]
  float* red = nullptr;          // (MP+R) x R reduced partials
  unsigned* ticket = nullptr;    // last-block counter of the combine kernel
  double* obj = nullptr;         // objective trace or nullptr
  const double* xnorm2 = nullptr;
  double* part64 = nullptr;      // FP64 partials of the residual kernel (2 * kMaxResidBlocks)
  int* status = nullptr;
  int blk = 0;                   // > 0: independent restarts of rank blk side by side
  // optional stopping test of the loop (the plan's main MU loop of a stage):
  // the combine of iteration t writes t - loop_t0 + 1 to *stop once the
  // objective's relative decrease over `check` iterations is <= tol, and every
  // later pass / combine launch with this stop word returns at entry
  int* stop = nullptr;
  double tol = 0.0;
  int check = 0;
  int loop_t0 = 0;
};

// Pick template bucket, tile width and grid for an m x n x r problem.
ntt_status mu_choose_shape(int64_t m, int64_t n, int r, int bf16, int num_sms, MuShape* out);
// Whether the split tensor-core form may run this FP32 shape under `route`.
bool tcs_route_ok(int64_t m, int64_t n, int r, int route);
// Whether X and H of these pointers can use TMA (alignment rules of the tensor maps).
bool mu_tma_ok(const MuShape& s, const void* X, const float* H);
// Decide TMA / tensor-core pass for these pointers (may change T and grid).
void mu_finalize_shape(MuShape* s, const void* X, const float* H, int num_sms);
// TMA map of a row-major BF16 matrix (rows x cols, 16-byte aligned rows) in
// boxes of 64 columns x box_rows rows with the 128-byte swizzle of 16-byte
// chunks: one box is one 64-column atom of the tensor-core passes' tiles.
ntt_status encode_bf16_atom_map(const void* base, int64_t rows, int64_t cols, int box_rows, CUtensorMap* out);
// Encode the two tensor maps (X: m x n, H: r x n) for a TMA pass.
ntt_status mu_encode_maps(const MuShape& s, const void* X, const float* H, CUtensorMap* mx,
                          CUtensorMap* mh);

// Launchers (enqueue only; return the launch error).
cudaError_t launch_mu_pass(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                           const CUtensorMap& mh, cudaStream_t st);
cudaError_t launch_mu_combine(const MuShape& s, const MuDev& d, float eps, int t, cudaStream_t st);
cudaError_t launch_gram(const MuShape& s, const MuDev& d, cudaStream_t st);
// BF16-X tensor-core pass (tcgen05 kind::f16) for 128 or 256 rows and rank buckets 16, 32.
bool tcb_pass_supported(int MP, int R);
cudaError_t launch_mu_pass_tcb(const MuShape& s, const MuDev& d, float eps, cudaStream_t st);
// FP32 X split in two BF16 matrices (X1 = bf16(X), X2 = bf16(X - X1)) on the
// BF16 tensor-core pass, 64 columns per tile: 128 or 256 rows, rank buckets 16, 32.
bool tcs_pass_supported(int MP, int R);
cudaError_t launch_mu_pass_tcs(const MuShape& s, const MuDev& d, float eps, cudaStream_t st);
// The split form for unfoldings of at most 32 rows (X1, X2 and the H_new terms
// stacked in one 128-row block; 128-column tiles).
bool tcn_pass_supported(int MP, int R);
// The warp-specialised form of mu_pass_tcs.cu for BF16 X at 128/256 rows.
cudaError_t launch_mu_pass_tcbx(const MuShape& s, const MuDev& d, float eps, cudaStream_t st);
cudaError_t launch_mu_pass_tcn(const MuShape& s, const MuDev& d, float eps, cudaStream_t st);
// X1 = bf16(X), X2 = bf16(X - X1) elementwise (round to nearest even).
cudaError_t launch_split_bf16x2(const float* X, __nv_bfloat16* X1, __nv_bfloat16* X2, int64_t count,
                                cudaStream_t st);
// Warp-streamed FMA pass for 16/32-row buckets at rank bucket 8 (FP32 X, TMA-aligned).
bool narrow_pass_supported(int MP, int R);
bool tcw_pass_supported(int MP, int R, int64_t n);
size_t split_blocked_bytes(int64_t n, int MP);
size_t split_scratch_bytes(int64_t m, int64_t n);
cudaError_t launch_split_blocked(const float* X, void* out, int64_t m, int64_t n, int MP, cudaStream_t st);
bool tcw_route_ok(int64_t m, int64_t n, int r, int route);
bool tcwb_route_ok(int64_t m, int64_t n, int r, int route);
ntt_status encode_tcwb_maps(const MuShape& s, const void* X, const float* H, CUtensorMap* mx, CUtensorMap* mh);
cudaError_t launch_mu_pass_tcwb(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                                const CUtensorMap& mh, cudaStream_t st);
cudaError_t launch_split_x12(const float* X, __nv_bfloat16* out, int64_t m, int64_t n, cudaStream_t st);
ntt_status encode_tcw_maps(const MuShape& s, const __nv_bfloat16* X12, const float* H, CUtensorMap* mx,
                           CUtensorMap* mh);
cudaError_t launch_mu_pass_tcw(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                               const CUtensorMap& mh, cudaStream_t st);
cudaError_t launch_mu_pass_narrow(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                                  const CUtensorMap& mh, cudaStream_t st);

cudaError_t launch_uniform(uint64_t key, int64_t count, float* out, cudaStream_t st);
// Zero `bytes` (a multiple of 4) at a 4-byte aligned device address by a
// kernel, so a captured graph holds no memset node.
cudaError_t launch_zero(void* dst, size_t bytes, cudaStream_t st);
// Copy `bytes` (a multiple of 4) from mapped pinned host memory (a device
// pointer of it) to device memory by a kernel, so a captured graph holds no
// memcpy node that could queue behind a large transfer on a copy engine.
cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t st);
// Failure-detection probe: one CTA starts a real bulk copy of `src` (256
// bytes, 16-byte aligned), waits at most limit_ns for an mbarrier that nothing
// arrives at, then drains its copy (bounded by kWaitLimitNs) and sets *status
// to NTT_ERR_TIMEOUT -- the path every kernel takes when a wait gives up.
cudaError_t launch_wait_probe(const void* src, int* status, long long limit_ns, cudaStream_t st);
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

// Algorithm 2's rank rule on the device (ntt_rank.cu): Gram of the unfolding
// on its smaller side (N = min(m, n) <= NTT_MAX_ROWS), FP64 eigenvalues by
// tridiagonalisation and bisection, singular values and the tail rule.
struct RankWs {
  int M = 0, nb = 0, S = 0;
  int64_t chunk = 0;
  size_t off_part = 0, off_G = 0, off_d = 0, off_e = 0, off_sigma = 0, off_rank = 0, bytes = 0;
};
RankWs rank_ws_layout(int64_t m, int64_t n, int num_sms);
// sigma_out (nullable: workspace) receives the N singular values, non-increasing;
// rank_out (nullable) the rule's rank for eps_rank, capped by rank_cap (> 0).
cudaError_t launch_rank_select(const float* X, int64_t m, int64_t n, double eps_rank, int rank_cap,
                               const RankWs& w, char* ws, double* sigma_out, int* rank_out, cudaStream_t st);

// Column-sharded NMF (mu_shard.cu): the fixed-order reduction of one pass's
// partials into FP64 [P ; Q] ((MP + R) x R), and the replicated W half of the
// iteration from the all-reduced [P ; Q].
cudaError_t launch_shard_reduce(const float* part, int nb, int E, double* pq, cudaStream_t st,
                                bool accumulate = false);
// xn_dev (nullable) overrides xnorm2 with a device value.
cudaError_t launch_shard_update(const double* pq, int m, int r, int MP, int R, float* W, float* G, float eps,
                                double xnorm2, double* obj, cudaStream_t st, const double* xn_dev = nullptr);

// Out-of-core MU (ntt_stream.cu): X in host memory streamed in column chunks.
ntt_status stream_ws_size(int64_t m, int64_t n, int r, int64_t chunk_cols, size_t* bytes);
ntt_status stream_mu(int64_t m, int64_t n, int r, const float* X_host, float* W, float* H, int iters, float eps,
                     double* obj_dev, int64_t chunk_cols, void* workspace, cudaStream_t st);

// Number of SMs of the current device (cached; 152 when no device).
int device_sms();

constexpr int kMaxResidBlocks = 4096;
// Enqueue the gram and `iters` (pass, combine) pairs of one NMF (t0 = index of
// the first objective entry).
ntt_status run_mu_iters(const MuShape& shp, const MuDev& dev, float eps, int iters, int t0,
                        cudaStream_t st, int* engine = nullptr);
// Algorithm 3 (BCD): the scratch layout for a shape, and the enqueue of the
// normalisation, the init pass/combine and `iters` (pass, combine) pairs with
// the final H moved into dev.H.  dev.W / dev.H: initial factors in, accepted out.
BcdWs bcd_ws_layout(const MuShape& s);
ntt_status run_bcd_iters(const MuShape& shp, const MuDev& dev, const BcdWs& L, char* bws, int iters, int t0,
                         cudaStream_t st);
// Enqueue one residual / norm pass (see ResidArgs); part64 holds 2 * kMaxResidBlocks doubles.
ntt_status resid_into(const void* X, int xbf16, const float* L, const float* Rm, int64_t M,
                      int64_t N, int r, int mode, double scale, double* acc, double* rel,
                      double* part64, unsigned* ticket, cudaStream_t st);

}  // namespace ntt
