// dslash_f64.cu -- hop kernels with double spinor and link storage: the
// inner-solver kinds here, the outer-solver kinds in dslash_f64_outer.cu.
#include "blas.h"
#include "dslash_launch.cuh"

namespace eofa {
cudaError_t launch_hop_f64(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    return kind <= KIND_OE_SCHUR_DAG ? launch_inner_t<double>(kind, a, coef, st)
                                     : launch_hop_f64_outer(kind, a, coef, st);
}
}  // namespace eofa
