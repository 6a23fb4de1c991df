// D3Q19 time-step kernels, N = 5 .. 8, bf16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_hi(int N) { return ops_fused3d_hi<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE); }
}  // namespace nfe
