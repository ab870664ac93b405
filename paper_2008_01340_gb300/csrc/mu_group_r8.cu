// Grouped pass instantiations for rank bucket R = 8.
#include "mu_group.cuh"

namespace ntt {

cudaError_t launch_gpass_r8(int mode, int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st) {
  if (mode == 1 && MP == 512) return launch_gpass_cfg<GCfg<512, 8>, 1>(probs, cta_prob, ncta, eps, st);
  if (mode == 2 && MP == 512) return launch_gpass_cfg<GCfg<512, 8>, 2>(probs, cta_prob, ncta, eps, st);
  if (mode != 0) return cudaErrorInvalidValue;
  switch (MP) {
    case 16: return launch_gpass_cfg<GCfg<16, 8>, 0>(probs, cta_prob, ncta, eps, st);
    case 32: return launch_gpass_cfg<GCfg<32, 8>, 0>(probs, cta_prob, ncta, eps, st);
    case 64: return launch_gpass_cfg<GCfg<64, 8>, 0>(probs, cta_prob, ncta, eps, st);
    case 128: return launch_gpass_cfg<GCfg<128, 8>, 0>(probs, cta_prob, ncta, eps, st);
    case 256: return launch_gpass_cfg<GCfg<256, 8>, 0>(probs, cta_prob, ncta, eps, st);
    case 512: return launch_gpass_cfg<GCfg<512, 8>, 0>(probs, cta_prob, ncta, eps, st);
    default: return cudaErrorInvalidValue;
  }
}

int gpass_occupancy_r8(int MP) {
  switch (MP) {
    case 16: return gpass_occupancy_cfg<GCfg<16, 8>>();
    case 32: return gpass_occupancy_cfg<GCfg<32, 8>>();
    case 64: return gpass_occupancy_cfg<GCfg<64, 8>>();
    case 128: return gpass_occupancy_cfg<GCfg<128, 8>>();
    case 256: return gpass_occupancy_cfg<GCfg<256, 8>>();
    case 512: return gpass_occupancy_cfg<GCfg<512, 8>>();
    default: return 1;
  }
}

}  // namespace ntt
