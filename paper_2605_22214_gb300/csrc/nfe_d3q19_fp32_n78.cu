// D3Q19 time-step kernels, N = 7, 8, fp32 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp32_n78(int N) {
    if (N == 7) return ops_fused3d_one<7, float, float>(NFE_FP32); if (N == 8) return ops_fused3d_one<8, float, float>(NFE_FP32);
    return nullptr;
}
}  // namespace nfe
