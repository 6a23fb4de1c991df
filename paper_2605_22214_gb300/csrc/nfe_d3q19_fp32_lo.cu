// D3Q19 time-step kernels, N = 2 .. 4, fp32 storage/arithmetic variant (fused z-marching
// step, two tile shapes), and the dispatch over N.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp32_hi(int N);
const Ops *ops_d3q19_fp32(int N) { return N <= 4 ? ops_fused3d_lo<float, float>(N, NFE_FP32) : ops_d3q19_fp32_hi(N); }
}  // namespace nfe
