// Grouped pass instantiations for rank bucket R = 16.
#include "mu_group.cuh"

namespace ntt {

cudaError_t launch_gpass_r16(int MP, const GProb* probs, const int* cta_prob, int ncta, float eps,
                             cudaStream_t st) {
  switch (MP) {
    case 16: return launch_gpass_cfg<GCfg<16, 16>>(probs, cta_prob, ncta, eps, st);
    case 32: return launch_gpass_cfg<GCfg<32, 16>>(probs, cta_prob, ncta, eps, st);
    case 64: return launch_gpass_cfg<GCfg<64, 16>>(probs, cta_prob, ncta, eps, st);
    case 128: return launch_gpass_cfg<GCfg<128, 16>>(probs, cta_prob, ncta, eps, st);
    case 256: return launch_gpass_cfg<GCfg<256, 16>>(probs, cta_prob, ncta, eps, st);
    case 512: return launch_gpass_cfg<GCfg<512, 16>>(probs, cta_prob, ncta, eps, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ntt
