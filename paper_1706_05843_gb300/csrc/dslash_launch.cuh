// dslash_launch.cuh -- host-side dispatch of hop_kernel over (Ls, kind, tile
// variant) for one storage type.  Included once per storage type by
// dslash_<prec>.cu so the four precisions compile as separate translation
// units.  The four kinds of the inner CG (the Schur complement and its
// adjoint) exist in two tile variants for the autotuner; the others in one.
#pragma once

#include "dslash.cuh"

namespace eofa {

template <typename S, int LS, int K, int VAR>
static cudaError_t launch_one(const HopArgs& a, const SCoef<typename Traits<S>::R>& c,
                              cudaStream_t st) {
    constexpr int NT = Tile<LS, VAR>::NT;
    constexpr int NS = Tile<LS, VAR>::NS;
    const size_t smem = hop_smem_bytes<S, LS, K, VAR>();
    static bool attr_done = false;  // per instantiation; set before first launch
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(hop_kernel<S, LS, K, VAR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int grid = (a.g.Vh + NS - 1) / NS;
    if (grid == 0) return cudaSuccess;
    hop_kernel<S, LS, K, VAR><<<grid, NT, smem, st>>>(a, c);
    return cudaGetLastError();
}

template <typename S, int LS, int K>
static cudaError_t launch_var(const HopArgs& a, const SCoef<typename Traits<S>::R>& c, cudaStream_t st) {
    return a.tile_var == 1 ? launch_one<S, LS, K, 1>(a, c, st) : launch_one<S, LS, K, 0>(a, c, st);
}

template <typename S, int LS>
static cudaError_t launch_ls(int kind, const HopArgs& a, const SCoef<typename Traits<S>::R>& c,
                             cudaStream_t st) {
    constexpr bool LOWP = sizeof(S) == 2;
    switch (kind) {
        case KIND_EO_MINV: return launch_var<S, LS, KIND_EO_MINV>(a, c, st);
        case KIND_OE_SCHUR: return launch_var<S, LS, KIND_OE_SCHUR>(a, c, st);
        case KIND_EO_MINV_DAG: return launch_var<S, LS, KIND_EO_MINV_DAG>(a, c, st);
        case KIND_OE_SCHUR_DAG: return launch_var<S, LS, KIND_OE_SCHUR_DAG>(a, c, st);
        default: break;
    }
    if constexpr (!LOWP) {
        switch (kind) {
            case KIND_RECON: return launch_one<S, LS, KIND_RECON, 0>(a, c, st);
            case KIND_SRC: return launch_one<S, LS, KIND_SRC, 0>(a, c, st);
            case KIND_FULL: return launch_one<S, LS, KIND_FULL, 0>(a, c, st);
            case KIND_FULL_DAG: return launch_one<S, LS, KIND_FULL_DAG, 0>(a, c, st);
            case KIND_LOC_DTMINV: return launch_one<S, LS, KIND_LOC_DTMINV, 0>(a, c, st);
            case KIND_LOC_DT: return launch_one<S, LS, KIND_LOC_DT, 0>(a, c, st);
            case KIND_LOC_DTINV: return launch_one<S, LS, KIND_LOC_DTINV, 0>(a, c, st);
            default: break;
        }
    }
    return cudaErrorNotSupported;
}

template <typename S>
static cudaError_t launch_hop_t(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    typedef typename Traits<S>::R R;
    const SCoef<R>& c = *reinterpret_cast<const SCoef<R>*>(coef);
    switch (a.g.Ls) {
        case 4: return launch_ls<S, 4>(kind, a, c, st);
        case 8: return launch_ls<S, 8>(kind, a, c, st);
        case 12: return launch_ls<S, 12>(kind, a, c, st);
        case 16: return launch_ls<S, 16>(kind, a, c, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace eofa
