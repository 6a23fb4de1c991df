// D3Q19 time-step kernels, N = 2 .. 8, fp64 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d3q19_fp64(int N) { return ops_for_n<LD3Q19, double, double>(N, NFE_FP64); }
}  // namespace nfe
