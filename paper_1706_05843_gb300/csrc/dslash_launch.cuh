// dslash_launch.cuh -- host-side dispatch of hop_kernel over (Ls, kind, tile
// variant) for one storage type.  Included by dslash_<prec>.cu (the four
// kinds of the inner CG: the Schur complement and its adjoint) and by
// dslash_<prec>_outer.cu (the FP64/FP32 outer-solver kinds), so the kernel
// instantiations compile as separate translation units.  The inner kinds
// exist in every tile variant the autotuner times (two CTA shapes, and for
// FP32 arithmetic each with and without a register cap); the others in
// the default variant only.
#pragma once

#include <atomic>
#include <mutex>

#include "dslash.cuh"

namespace eofa {

// devices a process may use the hop kernels on
constexpr int kHopMaxDevices = 64;

template <typename S, int LS, int K, int VAR>
static cudaError_t launch_one(const HopArgs& a, const SCoef<typename Traits<S>::R>& c,
                              cudaStream_t st) {
    constexpr int NS = Tile<LS, VAR>::NS;
    constexpr int NT = Tile<LS, VAR>::NT;
    const size_t smem = hop_smem_bytes<S, LS, K, VAR>();
    static_assert(hop_smem_bytes<S, LS, K, VAR>() <= 232448, "tile exceeds the 227 KB of shared memory per CTA");
    constexpr bool RCAP = (VAR & 2) != 0;
    // per instantiation and device, before its first launch there: the
    // shared-memory limit (an attribute of the current device) and the
    // number of CTAs one SM holds (the persistent grid is that many per SM)
    static std::atomic<int> resident_of[kHopMaxDevices];
    static std::mutex setup_mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kHopMaxDevices) return cudaErrorInvalidDevice;
    int resident = resident_of[dev].load(std::memory_order_acquire);
    if (resident == 0) {
        std::lock_guard<std::mutex> lock(setup_mu);
        resident = resident_of[dev].load(std::memory_order_relaxed);
        if (resident == 0) {
            // the one-time set-up must not run inside a stream capture (the
            // drivers launch every kernel once before they capture it)
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
                return cudaErrorStreamCaptureUnsupported;
            if constexpr (RCAP) {
                e = cudaFuncSetAttribute(hop_kernel_rc<S, LS, K, VAR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, hop_kernel_rc<S, LS, K, VAR>,
                                                                      NT, smem);
            } else {
                e = cudaFuncSetAttribute(hop_kernel<S, LS, K, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
                if (e == cudaSuccess)
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, hop_kernel<S, LS, K, VAR>, NT,
                                                                      smem);
            }
            if (e != cudaSuccess) return e;
            if (resident < 1) resident = 1;
            resident_of[dev].store(resident, std::memory_order_release);
        }
    }
    const long nblk = ((long)a.g.Vh + NS - 1) / NS;
    if (nblk == 0) return cudaSuccess;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long>(nblk, (long)resident * sms);
    if constexpr (RCAP) hop_kernel_rc<S, LS, K, VAR><<<grid, NT, smem, st>>>(a, c);
    else hop_kernel<S, LS, K, VAR><<<grid, NT, smem, st>>>(a, c);
    return cudaGetLastError();
}

template <typename S, int LS, int K>
static cudaError_t launch_var(const HopArgs& a, const SCoef<typename Traits<S>::R>& c, cudaStream_t st) {
    if constexpr (kTileVariants<S> == 4) {
        switch (a.tile_var) {
            case 1: return launch_one<S, LS, K, 1>(a, c, st);
            case 2: return launch_one<S, LS, K, 2>(a, c, st);
            case 3: return launch_one<S, LS, K, 3>(a, c, st);
            default: return launch_one<S, LS, K, 0>(a, c, st);
        }
    } else {
        return (a.tile_var & 1) ? launch_one<S, LS, K, 1>(a, c, st) : launch_one<S, LS, K, 0>(a, c, st);
    }
}

template <typename S, int LS>
static cudaError_t launch_inner_ls(int kind, const HopArgs& a, const SCoef<typename Traits<S>::R>& c,
                                   cudaStream_t st) {
    switch (kind) {
        case KIND_EO_MINV: return launch_var<S, LS, KIND_EO_MINV>(a, c, st);
        case KIND_OE_SCHUR: return launch_var<S, LS, KIND_OE_SCHUR>(a, c, st);
        case KIND_EO_MINV_DAG: return launch_var<S, LS, KIND_EO_MINV_DAG>(a, c, st);
        case KIND_OE_SCHUR_DAG: return launch_var<S, LS, KIND_OE_SCHUR_DAG>(a, c, st);
        default: return cudaErrorNotSupported;
    }
}

template <typename S, int LS>
static cudaError_t launch_outer_ls(int kind, const HopArgs& a, const SCoef<typename Traits<S>::R>& c,
                                   cudaStream_t st) {
    switch (kind) {
        case KIND_RECON: return launch_one<S, LS, KIND_RECON, 0>(a, c, st);
        case KIND_SRC: return launch_one<S, LS, KIND_SRC, 0>(a, c, st);
        case KIND_FULL: return launch_one<S, LS, KIND_FULL, 0>(a, c, st);
        case KIND_FULL_DAG: return launch_one<S, LS, KIND_FULL_DAG, 0>(a, c, st);
        case KIND_LOC_DTMINV: return launch_one<S, LS, KIND_LOC_DTMINV, 0>(a, c, st);
        case KIND_LOC_DT: return launch_one<S, LS, KIND_LOC_DT, 0>(a, c, st);
        case KIND_LOC_DTINV: return launch_one<S, LS, KIND_LOC_DTINV, 0>(a, c, st);
        case KIND_D_EO: return launch_one<S, LS, KIND_D_EO, 0>(a, c, st);
        case KIND_D_OE: return launch_one<S, LS, KIND_D_OE, 0>(a, c, st);
        case KIND_D_EO_DAG: return launch_one<S, LS, KIND_D_EO_DAG, 0>(a, c, st);
        case KIND_D_OE_DAG: return launch_one<S, LS, KIND_D_OE_DAG, 0>(a, c, st);
        default: return cudaErrorNotSupported;
    }
}

// kinds 0..3 (every storage type)
template <typename S>
static cudaError_t launch_inner_t(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    typedef typename Traits<S>::R R;
    const SCoef<R>& c = *reinterpret_cast<const SCoef<R>*>(coef);
    switch (a.g.Ls) {
        case 4: return launch_inner_ls<S, 4>(kind, a, c, st);
        case 8: return launch_inner_ls<S, 8>(kind, a, c, st);
        case 12: return launch_inner_ls<S, 12>(kind, a, c, st);
        case 16: return launch_inner_ls<S, 16>(kind, a, c, st);
        default: return cudaErrorNotSupported;
    }
}

// kinds 4..14 (FP64 and FP32 storage)
template <typename S>
static cudaError_t launch_outer_t(int kind, const HopArgs& a, const void* coef, cudaStream_t st) {
    typedef typename Traits<S>::R R;
    const SCoef<R>& c = *reinterpret_cast<const SCoef<R>*>(coef);
    switch (a.g.Ls) {
        case 4: return launch_outer_ls<S, 4>(kind, a, c, st);
        case 8: return launch_outer_ls<S, 8>(kind, a, c, st);
        case 12: return launch_outer_ls<S, 12>(kind, a, c, st);
        case 16: return launch_outer_ls<S, 16>(kind, a, c, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace eofa
