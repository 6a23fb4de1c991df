// D3Q19 time-step kernels, N = 5 .. 8, f16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_f16_hi(int N) { return ops_fused3d_hi<float, __half>(N, NFE_FP32_F16STORE); }
}  // namespace nfe
