// Out-of-core multiplicative updates: X stays in host memory and every MU
// iteration streams it to the GPU in column chunks (the analogue of the
// paper's 550 GB synthetic run, whose tensor exceeds device memory; on a
// Grace-Blackwell node host memory is reached over NVLink-C2C).
//
// Per iteration:
//   G = W^T W
//   for each chunk c of columns [c0, c1):
//     copy stream: X[:, c0:c1] (row pitch n in host memory) -> device buffer c % 2
//     compute stream (after that copy): the fused pass over the buffer with
//       H[:, c0:c1] read and written in place (row stride n), then its partials
//       reduced into FP64 and added to [P ; Q] in chunk order
//   W <- max(0, W o P / (W Q + eps)), objective (FP64)
// The copy of chunk c + 1 overlaps the pass over chunk c (two buffers, events
// in both directions).  With a single chunk the data stay resident after the
// first copy.  The stream's rate is bounded by the host-to-device copy rate,
// not by HBM.
#include <cstring>

#include "ntt_internal.cuh"

namespace ntt {

namespace {

__global__ void sum_in_order_kernel(const double* v, int count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += v[i];
    *out = s;
  }
}

struct StreamWs {
  size_t status, tickets, G, red, part, part64, buf[2], pq, xnp, xn, bytes;
  int64_t chunk;
  int nchunks;
};

StreamWs stream_layout(const MuShape& full_chunk, int64_t chunk, int nchunks, int64_t m) {
  StreamWs w;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off = (off + (b ? b : 1) + 255) / 256 * 256;
    return o;
  };
  w.status = take(64);
  w.tickets = take(64);
  w.G = take(NTT_MAX_RANK * NTT_MAX_RANK * 4);
  w.red = take((size_t)full_chunk.part_stride() * 4);
  w.part = take((size_t)full_chunk.grid_cap * full_chunk.part_stride() * 4);
  w.part64 = take(2 * kMaxResidBlocks * sizeof(double));
  w.buf[0] = take((size_t)m * chunk * 4);
  w.buf[1] = nchunks > 1 ? take((size_t)m * chunk * 4) : w.buf[0];
  w.pq = take((size_t)full_chunk.part_stride() * sizeof(double));
  w.xnp = take((size_t)nchunks * sizeof(double));
  w.xn = take(sizeof(double));
  w.bytes = off;
  w.chunk = chunk;
  w.nchunks = nchunks;
  return w;
}

}  // namespace

ntt_status stream_ws_size(int64_t m, int64_t n, int r, int64_t chunk_cols, size_t* bytes) {
  if (m < 1 || n < 1 || r < 1 || chunk_cols < 4 || chunk_cols % 4) return NTT_ERR_INVALID_ARG;
  const int64_t chunk = chunk_cols < n ? chunk_cols : n;
  MuShape s;
  const ntt_status e = mu_choose_shape(m, chunk, r, 0, device_sms(), &s);
  if (e != NTT_OK) return e;
  *bytes = stream_layout(s, chunk, (int)((n + chunk - 1) / chunk), m).bytes;
  return NTT_OK;
}

ntt_status stream_mu(int64_t m, int64_t n, int r, const float* X_host, float* W, float* H, int iters, float eps,
                     double* obj_dev, int64_t chunk_cols, void* workspace, cudaStream_t st) {
  if (chunk_cols < 4 || chunk_cols % 4) return NTT_ERR_INVALID_ARG;
  const int64_t chunk = chunk_cols < n ? chunk_cols : n;
  const int nc = (int)((n + chunk - 1) / chunk);
  MuShape full;
  ntt_status e = mu_choose_shape(m, chunk, r, 0, device_sms(), &full);
  if (e != NTT_OK) return e;
  const StreamWs L = stream_layout(full, chunk, nc, m);
  char* ws = reinterpret_cast<char*>(workspace);
  cudaStream_t cp = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) {
      if (ready[i]) cudaEventDestroy(ready[i]);
      if (freed[i]) cudaEventDestroy(freed[i]);
    }
    if (cp) cudaStreamDestroy(cp);   // released once its queued work has run
  };
#define NTT_STREAM_TRY(expr)        \
  do {                              \
    if ((expr) != cudaSuccess) {    \
      cudaGetLastError();           \
      cleanup();                    \
      return NTT_ERR_CUDA;          \
    }                               \
  } while (0)
  NTT_STREAM_TRY(cudaStreamCreateWithFlags(&cp, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    NTT_STREAM_TRY(cudaEventCreateWithFlags(&ready[i], cudaEventDisableTiming));
    NTT_STREAM_TRY(cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming));
  }
  // the copy stream starts after everything the caller's stream holds
  NTT_STREAM_TRY(cudaEventRecord(freed[0], st));
  NTT_STREAM_TRY(cudaEventRecord(freed[1], st));
  NTT_STREAM_TRY(launch_zero(ws + L.status, L.tickets + 64 - L.status, st));
  MuDev dev;
  dev.W = W;
  dev.G = reinterpret_cast<float*>(ws + L.G);
  dev.part = reinterpret_cast<float*>(ws + L.part);
  dev.red = reinterpret_cast<float*>(ws + L.red);
  dev.ticket = reinterpret_cast<unsigned*>(ws + L.tickets);
  dev.status = reinterpret_cast<int*>(ws + L.status);
  double* pq = reinterpret_cast<double*>(ws + L.pq);
  double* xnp = reinterpret_cast<double*>(ws + L.xnp);
  double* xn = reinterpret_cast<double*>(ws + L.xn);
  for (int t = 0; t < iters; ++t) {
    dev.H = H;
    NTT_STREAM_TRY(launch_gram(full, dev, st));
    for (int c = 0; c < nc; ++c) {
      const int64_t c0 = (int64_t)c * chunk, cols = (c0 + chunk <= n) ? chunk : n - c0;
      const int b = nc == 1 ? 0 : (int)(((int64_t)t * nc + c) & 1);
      float* buf = reinterpret_cast<float*>(ws + L.buf[b]);
      if (nc > 1 || t == 0) {
        NTT_STREAM_TRY(cudaStreamWaitEvent(cp, freed[b], 0));
        NTT_STREAM_TRY(cudaMemcpy2DAsync(buf, (size_t)cols * 4, X_host + c0, (size_t)n * 4, (size_t)cols * 4,
                                         (size_t)m, cudaMemcpyHostToDevice, cp));
        NTT_STREAM_TRY(cudaEventRecord(ready[b], cp));
        NTT_STREAM_TRY(cudaStreamWaitEvent(st, ready[b], 0));
      }
      MuShape s;
      if (mu_choose_shape(m, cols, r, 0, device_sms(), &s) != NTT_OK) {
        cleanup();
        return NTT_ERR_UNSUPPORTED;
      }
      s.route = NTT_ROUTE_GENERIC;   // the stride-aware pass; the copy rate bounds the loop
      s.ldh = n;
      MuDev d = dev;
      d.X = buf;
      d.H = H + c0;
      mu_finalize_shape(&s, buf, d.H, device_sms());
      CUtensorMap mx, mh;
      std::memset(&mx, 0, sizeof(mx));
      std::memset(&mh, 0, sizeof(mh));
      if (s.tma && mu_encode_maps(s, buf, d.H, &mx, &mh) != NTT_OK) {
        cleanup();
        return NTT_ERR_CUDA;
      }
      NTT_STREAM_TRY(launch_mu_pass(s, d, eps, mx, mh, st));
      NTT_STREAM_TRY(launch_shard_reduce(d.part, s.grid, s.part_stride(), pq, st, c > 0));
      if (t == 0 && obj_dev) {
        if (resid_into(buf, 0, nullptr, nullptr, m, cols, 0, 0, 1.0, xnp + c, nullptr,
                       reinterpret_cast<double*>(ws + L.part64), dev.ticket + 1, st) != NTT_OK) {
          cleanup();
          return NTT_ERR_CUDA;
        }
      }
      NTT_STREAM_TRY(cudaEventRecord(freed[b], st));
    }
    if (t == 0 && obj_dev) {
      sum_in_order_kernel<<<1, 32, 0, st>>>(xnp, nc, xn);
      NTT_STREAM_TRY(cudaGetLastError());
    }
    NTT_STREAM_TRY(launch_shard_update(pq, (int)m, r, full.MP, full.R, W, dev.G, eps, 0.0,
                                       obj_dev ? obj_dev + t : nullptr, st, xn));
  }
#undef NTT_STREAM_TRY
  cleanup();
  return NTT_OK;
}

}  // namespace ntt
