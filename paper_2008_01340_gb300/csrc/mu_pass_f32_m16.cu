// Instantiations of the fused MU pass (and its BCD step) for X in f32, padded rows MP = 16.
#include "mu_pass_impl.cuh"

namespace ntt {

cudaError_t launch_pass_f32_m16(int R, const MuShape& s, const MuDev& d, float eps,
                                   const CUtensorMap& mx, const CUtensorMap& mh, cudaStream_t st) {
  switch (R) {
    case 8: return launch_pass_cfg<PassCfg<16, 8, false>>(s, d, eps, mx, mh, st);
    case 16: return launch_pass_cfg<PassCfg<16, 16, false>>(s, d, eps, mx, mh, st);
    case 32: return launch_pass_cfg<PassCfg<16, 32, false>>(s, d, eps, mx, mh, st);
    default: return cudaErrorInvalidValue;
  }
}

bool info_pass_f32_m16(int R, int* T, size_t* smem) {
  switch (R) {
    case 8: pass_cfg_info<PassCfg<16, 8, false>>(T, smem); return true;
    case 16: pass_cfg_info<PassCfg<16, 16, false>>(T, smem); return true;
    case 32: pass_cfg_info<PassCfg<16, 32, false>>(T, smem); return true;
    default: return false;
  }
}

cudaError_t launch_pass_bcd_f32_m16(int R, const MuShape& s, const MuDev& d, const CUtensorMap& mx,
                                     const HMaps3& mh, float* const* Hb, const BcdState* st_dev, int init,
                                     double* res_part, cudaStream_t st) {
  switch (R) {
    case 8: return launch_pass_bcd_cfg<PassCfg<16, 8, false, true>>(s, d, mx, mh, Hb, st_dev, init, res_part, st);
    case 16: return launch_pass_bcd_cfg<PassCfg<16, 16, false, true>>(s, d, mx, mh, Hb, st_dev, init, res_part, st);
    case 32: return launch_pass_bcd_cfg<PassCfg<16, 32, false, true>>(s, d, mx, mh, Hb, st_dev, init, res_part, st);
    default: return cudaErrorInvalidValue;
  }
}

bool info_pass_bcd_f32_m16(int R, int* T, size_t* smem) {
  switch (R) {
    case 8: pass_cfg_info<PassCfg<16, 8, false, true>>(T, smem); return true;
    case 16: pass_cfg_info<PassCfg<16, 16, false, true>>(T, smem); return true;
    case 32: pass_cfg_info<PassCfg<16, 32, false, true>>(T, smem); return true;
    default: return false;
  }
}

}  // namespace ntt
