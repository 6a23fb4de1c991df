// D3Q19 time-step kernels, N = 4, fp64 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp64_n4(int N) {
    if (N == 4) return ops_fused3d_one<4, double, double>(NFE_FP64);
    return nullptr;
}
}  // namespace nfe
