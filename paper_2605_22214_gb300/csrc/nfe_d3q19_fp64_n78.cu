// D3Q19 time-step kernels, N = 7, 8, fp64 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp64_n78(int N) {
    if (N == 7) return ops_fused3d_one<7, double, double>(NFE_FP64); if (N == 8) return ops_fused3d_one<8, double, double>(NFE_FP64);
    return nullptr;
}
}  // namespace nfe
