// D3Q19 time-step kernels, N = 2 .. 4, bf16 storage/arithmetic variant (fused z-marching
// step, two tile shapes), and the dispatch over N.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_hi(int N);
const Ops *ops_d3q19_bf16(int N) { return N <= 4 ? ops_fused3d_lo<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE) : ops_d3q19_bf16_hi(N); }
}  // namespace nfe
