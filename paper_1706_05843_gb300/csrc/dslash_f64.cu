// dslash_f64.cu -- hop kernels with double spinor and link storage.
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f64(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_hop_t<double>(kind, a, coef, st);
}
}  // namespace eofa
