// Grouped pass instantiations with BF16 X rows (fused mode; heights up to 256,
// rank buckets 16 and 32), used by the precision form of the plan.
#include "mu_group.cuh"

namespace ntt {

bool gpass_bf16_supported(int MP, int R) { return MP >= 16 && MP <= 256 && (R == 16 || R == 32); }

#define NTT_GB_CASES(F)                                                                       \
  F(16, 16) F(32, 16) F(64, 16) F(128, 16) F(256, 16) F(16, 32) F(32, 32) F(64, 32) F(128, 32) \
  F(256, 32)

int gpass_occupancy_bf16(int MP, int R) {
#define NTT_GB_OCC(M, RR) \
  if (MP == M && R == RR) return gpass_occupancy_cfg<GCfg<M, RR, true>>();
  NTT_GB_CASES(NTT_GB_OCC)
#undef NTT_GB_OCC
  return 1;
}

cudaError_t launch_gpass_bf16(int MP, int R, const GProb* probs, const int* cta_prob, int ncta, float eps,
                              cudaStream_t st) {
#define NTT_GB_LAUNCH(M, RR) \
  if (MP == M && R == RR) return launch_gpass_cfg<GCfg<M, RR, true>, 0>(probs, cta_prob, ncta, eps, st);
  NTT_GB_CASES(NTT_GB_LAUNCH)
#undef NTT_GB_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace ntt
