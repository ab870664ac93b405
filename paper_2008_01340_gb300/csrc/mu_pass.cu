// Host side of the fused MU pass: bucket choice, TMA tensor maps, dispatch.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "ntt_internal.cuh"

namespace ntt {

#define NTT_DECL_BUCKET(B, MP)                                                                   \
  cudaError_t launch_pass_##B##_m##MP(int R, const MuShape& s, const MuDev& d, float eps,       \
                                      const CUtensorMap& mx, const CUtensorMap& mh,             \
                                      cudaStream_t st);                                         \
  bool info_pass_##B##_m##MP(int R, int* T, size_t* smem);
NTT_DECL_BUCKET(f32, 16)
NTT_DECL_BUCKET(f32, 32)
NTT_DECL_BUCKET(f32, 64)
NTT_DECL_BUCKET(f32, 128)
NTT_DECL_BUCKET(f32, 256)
NTT_DECL_BUCKET(f32, 512)
NTT_DECL_BUCKET(bf16, 16)
NTT_DECL_BUCKET(bf16, 32)
NTT_DECL_BUCKET(bf16, 64)
NTT_DECL_BUCKET(bf16, 128)
NTT_DECL_BUCKET(bf16, 256)
NTT_DECL_BUCKET(bf16, 512)
#undef NTT_DECL_BUCKET

static bool pass_info(int MP, int R, int bf16, int* T, size_t* smem) {
#define NTT_CASE(MPV)                                                                  \
  case MPV:                                                                            \
    return bf16 ? info_pass_bf16_m##MPV(R, T, smem) : info_pass_f32_m##MPV(R, T, smem);
  switch (MP) {
    NTT_CASE(16)
    NTT_CASE(32)
    NTT_CASE(64)
    NTT_CASE(128)
    NTT_CASE(256)
    NTT_CASE(512)
    default:
      return false;
  }
#undef NTT_CASE
}

int device_sms() {
  static int sms = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      sms = 152;
    cudaGetLastError();
  });
  return sms;
}

ntt_status mu_choose_shape(int64_t m, int64_t n, int r, int bf16, int num_sms, MuShape* out) {
  if (m < 1 || n < 1 || r < 1 || !out) return NTT_ERR_INVALID_ARG;
  if (m > NTT_MAX_ROWS || r > NTT_MAX_RANK) return NTT_ERR_UNSUPPORTED;
  if (n > (int64_t)INT32_MAX - 256) return NTT_ERR_UNSUPPORTED;
  MuShape s;
  s.m = m;
  s.n = n;
  s.r = r;
  s.bf16 = bf16 ? 1 : 0;
  int MP = 16;
  while (MP < m) MP *= 2;
  s.MP = MP;
  s.R = r <= 8 ? 8 : (r <= 16 ? 16 : 32);
  if (!pass_info(s.MP, s.R, s.bf16, &s.T, &s.smem)) return NTT_ERR_UNSUPPORTED;
  const int64_t ntiles = (n + s.T - 1) / s.T;
  int64_t grid = num_sms > 0 ? num_sms : 152;
  if (grid > kMaxPassCtas) grid = kMaxPassCtas;
  if (grid > ntiles) grid = ntiles;
  s.grid = (int)grid;
  int64_t cap = num_sms > 0 ? num_sms : 152;
  if (cap > kMaxPassCtas) cap = kMaxPassCtas;
  if (cap > (n + 15) / 16) cap = (n + 15) / 16;   // every pass tile is >= 16 columns
  s.grid_cap = (int)(cap > grid ? cap : grid);
  s.tma = 0;
  *out = s;
  return NTT_OK;
}

// Which single-problem pass runs an m x n x r problem, by route:
//  - BF16 X with 128 or 256 rows at rank bucket 16 or 32 runs on the BF16
//    tensor-core pass (kind::f16, FP32 accumulation, factors split in three
//    BF16 terms).  Its stacked form for 16 and 32 rows runs only with
//    NTT_ROUTE_TC: on 16 x 268,435,456 (rank 16) it ran 30.8 iterations/s
//    against 52.3 for the grouped FMA pass -- that shape moves 160 B of H per
//    column against 32 B of X, and one CTA per SM with its H loads in the
//    epilogue leaves the latency exposed.  NTT_ROUTE_FMA / _GENERIC keep the
//    packed-FMA pass.
//  - FP32 X with at most 32 rows at rank bucket 8 runs on the warp-streamed
//    pass (mu_pass_narrow.cu) unless the route is NTT_ROUTE_GENERIC.
static bool tcb_enabled(int MP, int route) {
  if (route == NTT_ROUTE_FMA || route == NTT_ROUTE_GENERIC) return false;
  if (MP <= 32) return route == NTT_ROUTE_TC;
  return true;
}

// FP32 X with 128 or 256 rows at rank bucket 16 or 32, or 512 rows at rank
// bucket 16 (n a multiple of 8), runs on the split tensor-core form (X in two
// BF16 matrices) where the caller provides its scratch.
bool tcs_route_ok(int64_t m, int64_t n, int r, int route) {
  if (route == NTT_ROUTE_FMA || route == NTT_ROUTE_GENERIC || route == NTT_ROUTE_GROUPED) return false;
  int MP = 16;
  while (MP < m) MP *= 2;
  const int R = r <= 8 ? 8 : (r <= 16 ? 16 : 32);
  // at most 32 rows (the stacked form) only when asked for: the narrow FMA pass
  // measured faster on the 32-row, rank-8 shape (0.222 vs 0.358 ms per
  // iteration on 32 x 4,194,304)
  if (MP <= 32 && route != NTT_ROUTE_TC) return false;
  return n % 8 == 0 && tcs_pass_supported(MP, R);
}

static bool narrow_enabled(int route) { return route != NTT_ROUTE_GENERIC; }

// FP32 X of 17 to 32 rows at rank bucket 8 (n a multiple of 64) runs on the
// warp-level MMA form (mu_pass_tcw.cu) where the caller provides the scratch of
// its split X, except on the CUDA-core routes and on NTT_ROUTE_TC (which keeps
// the stacked tcgen05 form there).
bool tcw_route_ok(int64_t m, int64_t n, int r, int route) {
  if (route == NTT_ROUTE_FMA || route == NTT_ROUTE_GENERIC || route == NTT_ROUTE_TC) return false;
  return m > 16 && m <= 32 && r >= 1 && r <= 8 && n % 64 == 0;
}

void mu_finalize_shape(MuShape* s, const void* X, const float* H, int num_sms) {
  s->tma = mu_tma_ok(*s, X, H) ? 1 : 0;
  s->tcb = 0;
  s->tcs = 0;
  s->narrow = 0;
  s->tcw = 0;
  if (!s->bf16 && s->tma && s->split_ok && tcs_route_ok(s->m, s->n, s->r, s->route)) {
    s->tcs = 1;
    s->T = s->MP <= 32 ? 128 : 64;   // <= 32 rows: the stacked form's 128-column tiles
    const int64_t ntiles = (s->n + s->T - 1) / s->T;
    int64_t grid = num_sms > 0 ? num_sms : 152;
    if (grid > ntiles) grid = ntiles;
    if (grid > s->grid_cap) grid = s->grid_cap;
    s->grid = (int)grid;
    return;
  }
  if (s->bf16 && s->tma && tcwb_route_ok(s->m, s->n, s->r, s->route)) {
    s->tcw = 1;
    s->T = 512;   // 8 warps x 64-column stages per CTA round
    const int64_t ntiles = (s->n + s->T - 1) / s->T;
    int64_t grid = num_sms > 0 ? num_sms : 152;
    if (grid > ntiles) grid = ntiles;
    if (grid > s->grid_cap) grid = s->grid_cap;
    s->grid = (int)grid;
    return;
  }
  if (s->bf16 && s->tma && s->n % 8 == 0 && tcb_pass_supported(s->MP, s->R) && tcb_enabled(s->MP, s->route)) {
    s->tcb = 1;
    s->T = 128;
    const int64_t ntiles = (s->n + s->T - 1) / s->T;
    int64_t grid = num_sms > 0 ? num_sms : 152;
    if (grid > ntiles) grid = ntiles;
    if (grid > s->grid_cap) grid = s->grid_cap;
    s->grid = (int)grid;
    return;
  }
  if (!s->bf16 && s->tma && s->split_ok && tcw_route_ok(s->m, s->n, s->r, s->route)) {
    s->tcw = 1;
    s->T = 512;   // 8 warps x 64-column stages per CTA round
    const int64_t ntiles = (s->n + s->T - 1) / s->T;
    int64_t grid = num_sms > 0 ? num_sms : 152;
    if (grid > ntiles) grid = ntiles;
    if (grid > s->grid_cap) grid = s->grid_cap;
    s->grid = (int)grid;
    return;
  }
  if (s->tma && !s->bf16 && narrow_pass_supported(s->MP, s->R) && narrow_enabled(s->route)) {
    // 32 rows with n a multiple of 32: the form whose copies move 256 bytes of
    // every row (3-D tensor maps); else 32-column boxes
    s->narrow = (s->MP == 32 && s->n % 32 == 0) ? 2 : 1;
    s->T = s->narrow == 2 ? 512 : 256;   // 8 warps x 64- or 32-column stages per CTA round
    const int64_t ntiles = (s->n + s->T - 1) / s->T;
    int64_t grid = num_sms > 0 ? num_sms : 152;
    if (grid > ntiles) grid = ntiles;
    if (grid > s->grid_cap) grid = s->grid_cap;
    s->grid = (int)grid;
  }
}

bool mu_tma_ok(const MuShape& s, const void* X, const float* H) {
  const int xb = s.bf16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(H) & 15)) return false;
  const int64_t ldh = s.ldh > 0 ? s.ldh : s.n;
  if ((s.n * xb) % 16 != 0 || (ldh * 4) % 16 != 0) return false;
  return true;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

ntt_status encode_bf16_atom_map(const void* base, int64_t rows, int64_t cols, int box_rows, CUtensorMap* out) {
  auto fn = encode_fn();
  if (!fn || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (cols * 2) % 16 != 0) return NTT_ERR_CUDA;
  if (box_rows < 1 || box_rows > 256) return NTT_ERR_INVALID_ARG;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUresult e = fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return e == CUDA_SUCCESS ? NTT_OK : NTT_ERR_CUDA;
}

ntt_status encode_tcwb_maps(const MuShape& s, const void* X, const float* H, CUtensorMap* mx, CUtensorMap* mh) {
  auto fn = encode_fn();
  if (!fn || s.n % 64 != 0) return NTT_ERR_CUDA;
  // X: 64-column boxes of the 16 rows (128-byte swizzle)
  if (encode_bf16_atom_map(X, s.m, s.n, 16, mx) != NTT_OK) return NTT_ERR_CUDA;
  // H: (32 columns, n / 32 halves, ranks), a box of two halves x the 16 rank rows
  cuuint64_t dims[3] = {32, (cuuint64_t)(s.n / 32), (cuuint64_t)s.r};
  cuuint64_t strides[2] = {128, (cuuint64_t)(s.n * 4)};
  cuuint32_t box[3] = {32, 2, 16};
  cuuint32_t es[3] = {1, 1, 1};
  if (fn(mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(H), dims, strides, box, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return NTT_ERR_CUDA;
  return NTT_OK;
}

ntt_status encode_tcw_maps(const MuShape& s, const __nv_bfloat16* X12, const float* H, CUtensorMap* mx,
                           CUtensorMap* mh) {
  auto fn = encode_fn();
  if (!fn || s.n % 64 != 0) return NTT_ERR_CUDA;
  {
    // (64 columns, 2 n / 64 lines, rows): a box of one segment's two terms x all rows
    cuuint64_t dims[3] = {64, (cuuint64_t)(2 * s.n / 64), (cuuint64_t)s.m};
    cuuint64_t strides[2] = {128, (cuuint64_t)(s.n * 4)};
    cuuint32_t box[3] = {64, 2, (cuuint32_t)s.MP};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(X12), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return NTT_ERR_CUDA;
  }
  {
    // (32 columns, n / 32 halves, ranks): a box of two halves x the 8 rank rows
    cuuint64_t dims[3] = {32, (cuuint64_t)(s.n / 32), (cuuint64_t)s.r};
    cuuint64_t strides[2] = {128, (cuuint64_t)(s.n * 4)};
    cuuint32_t box[3] = {32, 2, 8};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(H), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return NTT_ERR_CUDA;
  }
  return NTT_OK;
}

ntt_status mu_encode_maps(const MuShape& s, const void* X, const float* H, CUtensorMap* mx,
                          CUtensorMap* mh) {
  auto fn = encode_fn();
  if (!fn) return NTT_ERR_CUDA;
  const int xb = s.bf16 ? 2 : 4;
  const int br = s.MP < 256 ? s.MP : 256;
  if (s.narrow == 2) {
    // (32 columns, n / 32 segments, rows): a box of 2 segments x all rows
    // moves 256 contiguous bytes of every row; lines ordered (row, segment)
    for (int t = 0; t < 2; ++t) {
      const int64_t rows = t == 0 ? s.m : s.r;
      const int64_t ld = t == 0 ? s.n : (s.ldh > 0 ? s.ldh : s.n);
      cuuint64_t dims[3] = {32, (cuuint64_t)(s.n / 32), (cuuint64_t)rows};
      cuuint64_t strides[2] = {128, (cuuint64_t)(ld * 4)};
      cuuint32_t box[3] = {32, 2, (cuuint32_t)(t == 0 ? br : s.R)};
      cuuint32_t es[3] = {1, 1, 1};
      const CUresult e = fn(t == 0 ? mx : mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            t == 0 ? const_cast<void*>(X) : static_cast<void*>(const_cast<float*>(H)), dims, strides,
                            box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (e != CUDA_SUCCESS) return NTT_ERR_CUDA;
    }
    return NTT_OK;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)s.n, (cuuint64_t)s.m};
    cuuint64_t strides[1] = {(cuuint64_t)(s.n * xb)};
    // narrow pass: 32-column boxes, 128-byte swizzle of 16-byte chunks
    cuuint32_t box[2] = {(cuuint32_t)(s.narrow ? 32 : s.T), (cuuint32_t)br};
    cuuint32_t es[2] = {1, 1};
    CUresult e = fn(mx, s.bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void*>(X), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    s.narrow ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (e != CUDA_SUCCESS) return NTT_ERR_CUDA;
  }
  {
    cuuint64_t dims[2] = {(cuuint64_t)s.n, (cuuint64_t)s.r};
    cuuint64_t strides[1] = {(cuuint64_t)((s.ldh > 0 ? s.ldh : s.n) * 4)};
    cuuint32_t box[2] = {(cuuint32_t)(s.narrow ? 32 : s.T), (cuuint32_t)s.R};
    cuuint32_t es[2] = {1, 1};
    CUresult e = fn(mh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(H), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    s.narrow ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (e != CUDA_SUCCESS) return NTT_ERR_CUDA;
  }
  return NTT_OK;
}

cudaError_t launch_mu_pass(const MuShape& s, const MuDev& d, float eps, const CUtensorMap& mx,
                           const CUtensorMap& mh, cudaStream_t st) {
  if (s.tcs) return launch_mu_pass_tcs(s, d, eps, st);
  if (s.tcw) return s.bf16 ? launch_mu_pass_tcwb(s, d, eps, mx, mh, st) : launch_mu_pass_tcw(s, d, eps, mx, mh, st);
  if (s.tcb) return launch_mu_pass_tcb(s, d, eps, st);
  if (s.narrow) return launch_mu_pass_narrow(s, d, eps, mx, mh, st);
#define NTT_CASE(MPV)                                                       \
  case MPV:                                                                 \
    return s.bf16 ? launch_pass_bf16_m##MPV(s.R, s, d, eps, mx, mh, st)    \
                  : launch_pass_f32_m##MPV(s.R, s, d, eps, mx, mh, st);
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
}

}  // namespace ntt
