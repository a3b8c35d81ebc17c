// dslash_bf16.cu -- hop kernels with __nv_bfloat16 spinor and link storage
// (the inner-solver kinds only).
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_bf16(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_inner_t<__nv_bfloat16>(kind, a, coef, st);
}
}  // namespace eofa
