// D3Q19 time-step kernels, N = 5 .. 8, fp64 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp64_hi(int N) { return ops_fused3d_hi<double, double>(N, NFE_FP64); }
}  // namespace nfe
