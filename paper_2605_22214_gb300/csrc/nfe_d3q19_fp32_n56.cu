// D3Q19 time-step kernels, N = 5, 6, fp32 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp32_n56(int N) {
    if (N == 5) return ops_fused3d_one<5, float, float>(NFE_FP32); if (N == 6) return ops_fused3d_one<6, float, float>(NFE_FP32);
    return nullptr;
}
}  // namespace nfe
