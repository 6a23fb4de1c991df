// D2Q9 time-step kernels, N = 2 .. 4, fp64 storage/arithmetic variant (the fused
// single-kernel step: three tile shapes, the stored-g and geometry forms), and the dispatch
// over N.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp64_hi(int N);
const Ops *ops_d2q9_fp64(int N) { return N <= 4 ? ops_fused2d_lo<double, double>(N, NFE_FP64) : ops_d2q9_fp64_hi(N); }
}  // namespace nfe
