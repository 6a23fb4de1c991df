// D3Q19 time-step kernels, N = 2 .. 8, bf16 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16(int N) { return ops_for_n<LD3Q19, float, __nv_bfloat16>(N, NFE_FP32_BF16STORE); }
}  // namespace nfe
