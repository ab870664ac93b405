// nmf_mu_many: many independent NMFs advanced together by the grouped engine
// (one pass launch per shape bucket and one combine launch per iteration for
// all of them).  Every problem's CTA split -- and so the order of every one of
// its reductions -- depends on its own shape only, so a problem gives the same
// bits alone or among others.
#include <vector>

#include "group_engine.cuh"

using namespace ntt;

namespace {

ntt_status many_shapes(int count, const int64_t* m, const int64_t* n, const int* r,
                       std::vector<GroupShape>* out) {
  if (count < 1 || !m || !n || !r) return NTT_ERR_INVALID_ARG;
  out->clear();
  for (int i = 0; i < count; ++i) {
    if (m[i] < 1 || n[i] < 1 || r[i] < 1) return NTT_ERR_INVALID_ARG;
    if (r[i] > NTT_MAX_RANK || m[i] > NTT_MAX_TALL_ROWS || n[i] > ((int64_t)1 << 40)) return NTT_ERR_UNSUPPORTED;
    GroupShape s;
    s.n = n[i];
    s.m = (int)m[i];
    s.re = r[i];
    s.blk = r[i];
    out->push_back(s);
  }
  return NTT_OK;
}

}  // namespace

extern "C" {

ntt_status nmf_mu_many_workspace_size(int count, const int64_t* m, const int64_t* n, const int* r,
                                      size_t* bytes) {
  if (!bytes) return NTT_ERR_INVALID_ARG;
  std::vector<GroupShape> shapes;
  ntt_status s = many_shapes(count, m, n, r, &shapes);
  if (s != NTT_OK) return s;
  GroupPlan pl;
  s = group_plan(shapes, device_sms(), 0, true, true, &pl);
  if (s != NTT_OK) return s;
  *bytes = pl.bytes;
  return NTT_OK;
}

ntt_status nmf_mu_many(int count, const int64_t* m, const int64_t* n, const int* r, const float* const* X,
                       float* const* W, float* const* H, int iters, float eps_mu, void* ws, void* stream) {
  if (!X || !W || !H || !ws || iters < 0 || !(eps_mu >= 0.0f)) return NTT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return NTT_ERR_INVALID_ARG;
  std::vector<GroupShape> shapes;
  ntt_status s = many_shapes(count, m, n, r, &shapes);
  if (s != NTT_OK) return s;
  std::vector<GroupPtrs> ptrs(count);
  for (int i = 0; i < count; ++i) {
    if (!X[i] || !W[i] || !H[i]) return NTT_ERR_INVALID_ARG;
    ptrs[i].X = X[i];
    ptrs[i].W = W[i];
    ptrs[i].H = H[i];
    ptrs[i].scratch = nullptr;
  }
  GroupPlan pl;
  s = group_plan(shapes, device_sms(), 0, true, true, &pl);
  if (s != NTT_OK) return s;
  if (iters == 0) return NTT_OK;
  // pageable host tables: the copy is staged before cudaMemcpyAsync returns
  std::vector<char> tables(pl.table_bytes);
  return group_run(pl, ptrs.data(), reinterpret_cast<char*>(ws), tables.data(), iters, eps_mu,
                   reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
