// Auxiliary kernels of the nTT path:
//   uniform_kernel   counter-based U[0,1) initialisation of W and H (INIT)
//   cast_bf16_kernel FP32 -> BF16 (round to nearest even) staging of X
//   split_bf16x2_kernel FP32 X -> bf16(X) and bf16(X - bf16(X)) (the split form
//                    of the tensor-core pass)
//   resid_kernel     ||X||^2, ||X - L R||^2 (FP64) or L R written out:
//                    objective at stage end, Eq. (3) and Eq. (2) via the
//                    split-chain product
//   small_mm_kernel  C = A B with K <= 32 (chain products of TT cores)
//   handoff kernels  column L1 normalisation of W folded into H
//   zero / copy      word fills and copies as kernels (graph nodes that use
//                    no copy engine)
#include "ntt_internal.cuh"

namespace ntt {

namespace {

__global__ void uniform_kernel(uint64_t key, int64_t count, float* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = uniform24(key, (uint64_t)i);
}

__global__ void zero_words_kernel(uint32_t* dst, int64_t words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) dst[i] = 0u;
}

__global__ void copy_words_kernel(uint32_t* dst, const uint32_t* src, int64_t words) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) dst[i] = src[i];
}

// One thread: barrier `never` expects an arrival nobody makes; barrier `copy`
// tracks a real 256-byte bulk copy.  The wait on `never` gives up after
// limit_ns, the copy is drained, and the timeout is recorded.
__global__ void wait_probe_kernel(const void* src, int* status, long long limit_ns) {
  __shared__ __align__(128) uint8_t buf[256];
  __shared__ __align__(8) uint64_t bars[2];
  if (threadIdx.x != 0) return;
  const uint32_t never = smem_u32(&bars[0]), copy = smem_u32(&bars[1]);
  mbar_init(never, 1);
  mbar_init(copy, 1);
  fence_mbar_init();
  mbar_arrive_expect_tx(copy, 256);
  bulk_load(smem_u32(buf), src, 256, copy);
  const bool ok = mbar_wait_bounded(never, 0, limit_ns);
  const bool drained = mbar_wait_bounded(copy, 0);   // the copy completes by itself
  if (!ok || !drained) atomicExch(status, kStatusTimeout);
}

__global__ void split_bf16x2_kernel(const float* in, __nv_bfloat16* x1, __nv_bfloat16* x2, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float v = in[i];
    const __nv_bfloat16 a = __float2bfloat16_rn(v);
    x1[i] = a;
    x2[i] = __float2bfloat16_rn(v - __bfloat162float(a));
  }
}

__global__ void cast_bf16_kernel(const float* in, __nv_bfloat16* out, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = count / 4;
  const bool vec = ((reinterpret_cast<uintptr_t>(in) & 15) == 0) &&
                   ((reinterpret_cast<uintptr_t>(out) & 7) == 0);
  if (vec) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = reinterpret_cast<const float4*>(in)[i];
      __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
      __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
      reinterpret_cast<uint2*>(out)[i] = u;
    }
    for (int64_t i = n4 * 4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
      out[i] = __float2bfloat16_rn(in[i]);
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
      out[i] = __float2bfloat16_rn(in[i]);
  }
}

// ---------------------------------------------------------------------------
// Residual / reconstruction over an M x N matrix in tiles of 32 rows x 256
// columns.  Thread = (row group of 8 rows, 4-column chunk).  FP32 partial sums
// over <= 32 squares per tile, FP64 across tiles and threads, per-block FP64
// partials reduced in fixed order by the last block.
// ---------------------------------------------------------------------------
constexpr int kRTileRows = 32;
constexpr int kRTileCols = 256;
constexpr int kRMaxR = NTT_MAX_RANK;

template <bool BF16>
__device__ __forceinline__ float ldx(const void* X, int64_t idx) {
  if constexpr (BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(X)[idx]);
  else
    return __ldcs(reinterpret_cast<const float*>(X) + idx);
}

template <bool BF16, bool VEC>
__device__ __forceinline__ float4 ldx4(const void* X, int64_t idx) {
  if constexpr (BF16) {
    if constexpr (VEC) {
      const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(X) + idx));
      return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                         __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
    } else {
      return make_float4(ldx<true>(X, idx), ldx<true>(X, idx + 1), ldx<true>(X, idx + 2),
                         ldx<true>(X, idx + 3));
    }
  } else {
    if constexpr (VEC)
      return __ldcs(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(X) + idx));
    else
      return make_float4(ldx<false>(X, idx), ldx<false>(X, idx + 1), ldx<false>(X, idx + 2),
                         ldx<false>(X, idx + 3));
  }
}

template <bool BF16, bool VEC>
__global__ void __launch_bounds__(kAuxThreads) resid_kernel(const ResidArgs a) {
  __shared__ float Rs[kRMaxR * kRTileCols];   // r x 256 slice of Rm
  __shared__ float Ls[kRTileRows * kRMaxR];   // 32 x r slice of L
  __shared__ double dsh[kAuxThreads];
  __shared__ double dsh2[kAuxThreads];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int cq = tid % 64;          // 4-column chunk
  const int rg = tid / 64;          // row group: rows rg*8 .. rg*8+7
  const int64_t tiles_c = (a.N + kRTileCols - 1) / kRTileCols;
  const int64_t tiles_r = (a.M + kRTileRows - 1) / kRTileRows;
  const int64_t ntiles = tiles_c * tiles_r;
  const int r = a.r;
  double acc0 = 0.0, acc1 = 0.0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t tr = tile / tiles_c, tc = tile % tiles_c;
    const int64_t row0 = tr * kRTileRows, col0 = tc * kRTileCols;
    if (a.mode != 0) {
      __syncthreads();
      for (int idx = tid; idx < r * kRTileCols; idx += blockDim.x) {
        const int k = idx / kRTileCols, c = idx % kRTileCols;
        const int64_t col = col0 + c;
        Rs[idx] = (col < a.N) ? a.Rm[(int64_t)k * a.N + col] : 0.0f;
      }
      for (int idx = tid; idx < kRTileRows * r; idx += blockDim.x) {
        const int i = idx / r, k = idx % r;
        const int64_t row = row0 + i;
        Ls[i * kRMaxR + k] = (row < a.M) ? a.L[row * r + k] : 0.0f;
      }
      __syncthreads();
    }
    const int64_t col = col0 + 4 * cq;
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 2
    for (int ii = 0; ii < 8; ++ii) {
      const int i = rg * 8 + ii;
      const int64_t row = row0 + i;
      if (row >= a.M || col >= a.N) continue;
      const int64_t base = row * a.N + col;
      const bool full = (col + 3 < a.N);
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.mode != 2) {
        if (full) {
          x = ldx4<BF16, VEC>(a.X, base);
        } else {
          x.x = ldx<BF16>(a.X, base);
          if (col + 1 < a.N) x.y = ldx<BF16>(a.X, base + 1);
          if (col + 2 < a.N) x.z = ldx<BF16>(a.X, base + 2);
        }
      }
      float4 pr = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a.mode != 0) {
        for (int k = 0; k < r; ++k) {
          const float l = Ls[i * kRMaxR + k];
          const float4 rv = *reinterpret_cast<const float4*>(&Rs[k * kRTileCols + 4 * cq]);
          pr.x = fmaf(l, rv.x, pr.x);
          pr.y = fmaf(l, rv.y, pr.y);
          pr.z = fmaf(l, rv.z, pr.z);
          pr.w = fmaf(l, rv.w, pr.w);
        }
      }
      if (a.mode == 2) {
        float* o = a.out + base;
        if (full && VEC) {
          *reinterpret_cast<float4*>(o) = pr;
        } else {
          o[0] = pr.x;
          if (col + 1 < a.N) o[1] = pr.y;
          if (col + 2 < a.N) o[2] = pr.z;
          if (col + 3 < a.N) o[3] = pr.w;
        }
        continue;
      }
      if (a.mode == 1) {
        const float d0 = x.x - pr.x, d1 = x.y - pr.y, d2 = x.z - pr.z, d3 = x.w - pr.w;
        // entries past the last column are zero on both sides
        s0 += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
      }
      s1 += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
    }
    acc0 += (double)s0;
    acc1 += (double)s1;
  }
  if (a.mode == 2) return;

  // block partials (deterministic tree), then the last block reduces them
  dsh[tid] = acc0;
  dsh2[tid] = acc1;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      dsh[tid] += dsh[tid + s];
      dsh2[tid] += dsh2[tid + s];
    }
    __syncthreads();
  }
  if (tid == 0) {
    a.part64[2 * blockIdx.x] = dsh[0];
    a.part64[2 * blockIdx.x + 1] = dsh2[0];
    __threadfence();
    s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) {
      t0 += __ldcg(&a.part64[2 * b]);
      t1 += __ldcg(&a.part64[2 * b + 1]);
    }
    if (a.mode == 0) {
      a.acc[0] = t1 * a.scale;
    } else {
      a.acc[0] = t0 * a.scale;
      a.acc[1] = t1;
      if (a.rel) {
        a.rel[0] = t1 > 0.0 ? sqrt(t0 / t1) : 0.0;
        a.rel[1] = t0;
        a.rel[2] = t1;
      }
    }
    *a.ticket = 0u;
  }
}

__global__ void small_mm_kernel(const float* A, const float* B, float* C, int64_t M, int K,
                                int64_t N) {
  const int64_t total = M * N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int64_t i = idx / N, j = idx % N;
    float s = 0.0f;
    for (int k = 0; k < K; ++k) s = fmaf(A[i * K + k], B[(int64_t)k * N + j], s);
    C[idx] = s;
  }
}

// One block: column L1 norms of W, then W[:, k] /= s_k (s_k > 0).
__global__ void handoff_w_kernel(float* W, int64_t m, int r, float* s_out) {
  __shared__ float s[NTT_MAX_RANK];
  const int tid = threadIdx.x;
  if (tid < r) {
    float acc = 0.0f;
    for (int64_t i = 0; i < m; ++i) acc += W[i * r + tid];
    s[tid] = acc;
    s_out[tid] = acc;
  }
  __syncthreads();
  for (int64_t e = tid; e < m * r; e += blockDim.x) {
    const float sk = s[e % r];
    if (sk > 0.0f) W[e] = __fdiv_rn(W[e], sk);
  }
}

// grid.y = row k of H; 4-wide accesses when rows are 16-byte aligned.
__global__ void handoff_h_kernel(float* H, int64_t n, int r, const float* s) {
  const int k = blockIdx.y;
  const float sk = s[k];
  if (!(sk > 0.0f)) return;
  float* row = H + (int64_t)k * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(H) & 15) == 0) {
    float4* r4 = reinterpret_cast<float4*>(row);
    for (int64_t e = t0; e < n / 4; e += stride) {
      float4 v = r4[e];
      v.x *= sk; v.y *= sk; v.z *= sk; v.w *= sk;
      r4[e] = v;
    }
  } else {
    for (int64_t e = t0; e < n; e += stride) row[e] *= sk;
  }
}

int grid_for(int64_t work, int per_block_items) {
  int64_t b = (work + per_block_items - 1) / per_block_items;
  const int64_t cap = (int64_t)device_sms() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_uniform(uint64_t key, int64_t count, float* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  uniform_kernel<<<grid_for(count, kAuxThreads * 4), kAuxThreads, 0, st>>>(key, count, out);
  return cudaGetLastError();
}

cudaError_t launch_zero(void* dst, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if ((bytes & 3) || (reinterpret_cast<uintptr_t>(dst) & 3)) return cudaErrorInvalidValue;
  const int64_t words = (int64_t)(bytes / 4);
  zero_words_kernel<<<grid_for(words, kAuxThreads * 4), kAuxThreads, 0, st>>>(
      reinterpret_cast<uint32_t*>(dst), words);
  return cudaGetLastError();
}

cudaError_t launch_copy_words(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if ((bytes & 3) || (reinterpret_cast<uintptr_t>(dst) & 3) || (reinterpret_cast<uintptr_t>(src) & 3))
    return cudaErrorInvalidValue;
  const int64_t words = (int64_t)(bytes / 4);
  copy_words_kernel<<<grid_for(words, kAuxThreads * 4), kAuxThreads, 0, st>>>(
      reinterpret_cast<uint32_t*>(dst), reinterpret_cast<const uint32_t*>(src), words);
  return cudaGetLastError();
}

cudaError_t launch_wait_probe(const void* src, int* status, long long limit_ns, cudaStream_t st) {
  if (reinterpret_cast<uintptr_t>(src) & 15) return cudaErrorInvalidValue;
  wait_probe_kernel<<<1, 32, 0, st>>>(src, status, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16x2(const float* X, __nv_bfloat16* X1, __nv_bfloat16* X2, int64_t count,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  split_bf16x2_kernel<<<grid_for(count, kAuxThreads * 4), kAuxThreads, 0, st>>>(X, X1, X2, count);
  return cudaGetLastError();
}

cudaError_t launch_cast_bf16(const float* in, __nv_bfloat16* out, int64_t count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  cast_bf16_kernel<<<grid_for(count / 4 + 1, kAuxThreads * 4), kAuxThreads, 0, st>>>(in, out, count);
  return cudaGetLastError();
}

int resid_blocks(int num_sms) { return (num_sms > 0 ? num_sms : 152) * 4; }

cudaError_t launch_resid(const ResidArgs& a, int blocks, cudaStream_t st) {
  const int xb = a.xbf16 ? 2 : 4;
  bool vec = (a.N % 4 == 0);
  if (a.mode != 2 && (reinterpret_cast<uintptr_t>(a.X) % (4 * xb))) vec = false;
  if (a.mode == 2 && (reinterpret_cast<uintptr_t>(a.out) % 16)) vec = false;
  const int64_t tiles = ((a.M + kRTileRows - 1) / kRTileRows) * ((a.N + kRTileCols - 1) / kRTileCols);
  if (blocks > tiles) blocks = (int)tiles;
  if (blocks < 1) blocks = 1;
  if (a.xbf16) {
    if (vec)
      resid_kernel<true, true><<<blocks, kAuxThreads, 0, st>>>(a);
    else
      resid_kernel<true, false><<<blocks, kAuxThreads, 0, st>>>(a);
  } else {
    if (vec)
      resid_kernel<false, true><<<blocks, kAuxThreads, 0, st>>>(a);
    else
      resid_kernel<false, false><<<blocks, kAuxThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_small_mm(const float* A, const float* B, float* C, int64_t M, int K, int64_t N,
                            cudaStream_t st) {
  small_mm_kernel<<<grid_for(M * N, kAuxThreads * 4), kAuxThreads, 0, st>>>(A, B, C, M, K, N);
  return cudaGetLastError();
}

cudaError_t launch_handoff(float* W, float* H, int64_t m, int64_t n, int r, float* s_scratch,
                           cudaStream_t st) {
  handoff_w_kernel<<<1, kAuxThreads, 0, st>>>(W, m, r, s_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int gx = grid_for(n / 4 + 1, kAuxThreads * 4);
  const int cap = (device_sms() * 8 + r - 1) / r;
  if (gx > cap) gx = cap;
  handoff_h_kernel<<<dim3(gx, r), kAuxThreads, 0, st>>>(H, n, r, s_scratch);
  return cudaGetLastError();
}

}  // namespace ntt
