// D2Q9 time-step kernels, N = 2 .. 4, bf16 storage/arithmetic variant (the fused
// single-kernel step: three tile shapes, the stored-g and geometry forms), and the dispatch
// over N.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_bf16_n56(int N);
const Ops *ops_d2q9_bf16_n78(int N);
const Ops *ops_d2q9_bf16(int N) {
    if (N <= 4) return ops_fused2d_lo<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE);
    return N <= 6 ? ops_d2q9_bf16_n56(N) : ops_d2q9_bf16_n78(N);
}
}  // namespace nfe
