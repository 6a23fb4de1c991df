// D3Q19 time-step kernels, N = 2 .. 4, fp64 storage/arithmetic variant (fused z-marching
// step, two tile shapes), and the dispatch over N.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp64_hi(int N);
const Ops *ops_d3q19_fp64(int N) { return N <= 4 ? ops_fused3d_lo<double, double>(N, NFE_FP64) : ops_d3q19_fp64_hi(N); }
}  // namespace nfe
