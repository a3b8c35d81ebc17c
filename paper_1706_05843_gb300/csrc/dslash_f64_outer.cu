// dslash_f64_outer.cu -- the outer-solver hop kernels (reconstruction,
// source, full operator, site-local D~ products) with double storage.
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f64_outer(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return launch_outer_t<double>(kind, a, coef, st);
}
}  // namespace eofa
