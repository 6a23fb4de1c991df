// D3Q19 time-step kernels, N = 2 .. 4, f16 storage/arithmetic variant (fused z-marching
// step, two tile shapes), and the dispatch over N.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_f16_hi(int N);
const Ops *ops_d3q19_f16(int N) { return N <= 4 ? ops_fused3d_lo<float, __half>(N, NFE_FP32_F16STORE) : ops_d3q19_f16_hi(N); }
}  // namespace nfe
