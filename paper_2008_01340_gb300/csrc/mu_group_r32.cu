// Grouped pass instantiations for rank bucket R = 32.
#include "mu_group.cuh"

namespace ntt {

cudaError_t launch_gpass_r32(int mode, int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st) {
  if (mode == 1 && MP == 512) return launch_gpass_cfg<GCfg<512, 32>, 1>(probs, cta_prob, ncta, eps, st);
  if (mode == 2 && MP == 512) return launch_gpass_cfg<GCfg<512, 32>, 2>(probs, cta_prob, ncta, eps, st);
  if (mode != 0) return cudaErrorInvalidValue;
  switch (MP) {
    case 16: return launch_gpass_cfg<GCfg<16, 32>, 0>(probs, cta_prob, ncta, eps, st);
    case 32: return launch_gpass_cfg<GCfg<32, 32>, 0>(probs, cta_prob, ncta, eps, st);
    case 64: return launch_gpass_cfg<GCfg<64, 32>, 0>(probs, cta_prob, ncta, eps, st);
    case 128: return launch_gpass_cfg<GCfg<128, 32>, 0>(probs, cta_prob, ncta, eps, st);
    case 256: return launch_gpass_cfg<GCfg<256, 32>, 0>(probs, cta_prob, ncta, eps, st);
    case 512: return launch_gpass_cfg<GCfg<512, 32>, 0>(probs, cta_prob, ncta, eps, st);
    default: return cudaErrorInvalidValue;
  }
}

int gpass_occupancy_r32(int MP) {
  switch (MP) {
    case 16: return gpass_occupancy_cfg<GCfg<16, 32>>();
    case 32: return gpass_occupancy_cfg<GCfg<32, 32>>();
    case 64: return gpass_occupancy_cfg<GCfg<64, 32>>();
    case 128: return gpass_occupancy_cfg<GCfg<128, 32>>();
    case 256: return gpass_occupancy_cfg<GCfg<256, 32>>();
    case 512: return gpass_occupancy_cfg<GCfg<512, 32>>();
    default: return 1;
  }
}

}  // namespace ntt
