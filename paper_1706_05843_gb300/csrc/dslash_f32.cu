// dslash_f32.cu -- hop kernels with float spinor and link storage: the
// inner-solver kinds here, the outer-solver kinds in dslash_f32_outer.cu.
#include "blas.h"
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f32(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return kind <= KIND_OE_SCHUR_DAG ? launch_inner_t<float>(kind, a, coef, st)
                                     : launch_hop_f32_outer(kind, a, coef, st);
}
}  // namespace eofa
