// D2Q9 time-step kernels, N = 2 .. 4, bf16 storage/arithmetic variant (the fused
// single-kernel step: three tile shapes, the stored-g and geometry forms), and the dispatch
// over N.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_bf16_hi(int N);
const Ops *ops_d2q9_bf16(int N) { return N <= 4 ? ops_fused2d_lo<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE) : ops_d2q9_bf16_hi(N); }
}  // namespace nfe
