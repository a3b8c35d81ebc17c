// dslash_f32_outer.cu -- the outer-solver hop kernels (reconstruction,
// source, full operator, site-local D~ products) with float storage.
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f32_outer(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_outer_t<float>(kind, a, coef, st);
}
}  // namespace eofa
