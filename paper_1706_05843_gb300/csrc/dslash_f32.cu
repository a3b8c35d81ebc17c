// dslash_f32.cu -- hop kernels with float spinor and link storage.
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f32(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_hop_t<float>(kind, a, coef, st);
}
}  // namespace eofa
