// dslash_f16.cu -- hop kernels with __half spinor and link storage (the
// inner-solver kinds only).
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f16(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_inner_t<__half>(kind, a, coef, st);
}
}  // namespace eofa
