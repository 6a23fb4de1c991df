// D3Q19 time-step kernels, N = 5 .. 8, fp32 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp32_hi(int N) { return ops_fused3d_hi<float, float>(N, NFE_FP32); }
}  // namespace nfe
