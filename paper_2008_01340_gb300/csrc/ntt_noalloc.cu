// nmf_mu_step_noalloc: the multiplicative-update NMF entry point for callers
// that cannot allocate device memory.
//
// Some callers have no way to call cudaMalloc: code loaded as a plugin into a
// host process whose own runtime owns every device allocation, or a tight
// control loop that must not take the implicit device synchronisation and the
// failure modes of an allocation call.  This entry point takes no workspace
// argument.  Its scratch (status word, tickets, Gram matrix, reduction buffers
// and the per-CTA partials of the pass kernel) lives in one file-scope device
// array of kNoAllocScratchBytes, which every GPU that loads this library holds
// until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents; the call clears the words that must start at zero (status and
// tickets) and overwrites everything else before reading it.  Calls whose
// device work overlaps (two streams, or two host threads) race on the array:
// serialise them.
#include <mutex>

#include "ntt_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a stand-in; the real address is looked up once per
// device, with that device current, and cached.
ntt_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return NTT_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return NTT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return NTT_OK;
}

}  // namespace

extern "C" {

ntt_status nmf_mu_step_noalloc(int64_t m, int64_t n, int r, const void* X, ntt_dtype x_dtype,
                               float* W, float* H, int iters, float eps_mu, double* obj_dev,
                               void* stream) {
  if (!X || !W || !H || iters < 0 || !(eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  size_t need = 0;
  ntt_status s = nmf_mu_workspace_size(m, n, r, x_dtype, &need);
  if (s != NTT_OK) return s;
  if (need > kNoAllocScratchBytes) return NTT_ERR_OOM;   // shape needs more scratch than the array holds
  void* ws = nullptr;
  s = noalloc_scratch(&ws);
  if (s != NTT_OK) return s;
  return nmf_mu_step(m, n, r, X, x_dtype, W, H, iters, eps_mu, obj_dev, ws, stream);
}

}  // extern "C"
