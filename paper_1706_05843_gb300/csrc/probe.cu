// probe.cu -- measured FMA throughput of the current device (a measurement
// utility for the rooflines of the arithmetic-bound kernels; see
// eofa_measure_fma in eofa.h).
//
// Every thread runs kChains independent FMA chains for kIters steps, so
// the FMA pipe is never waiting on a dependency; the grid is resident CTAs
// per SM times the SM count.  The chains' sum is stored only when a runtime
// flag the host never sets is on, which keeps the arithmetic live.
#include <cuda_runtime.h>

#include <algorithm>

#include "eofa.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma(T a, T b, int store, T* out) {
    T v[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) v[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) v[i] = fma(v[i], a, b);
    }
    if (store) {
        T s = 0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += v[i];
        out[blockIdx.x * kThreads + threadIdx.x] = s;
    }
}

template <typename T>
eofa_status measure(int reps, double* tflops, cudaStream_t st) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma<T>, kThreads, 0) != cudaSuccess)
        return EOFA_ERR_CUDA;
    const int grid = std::max(1, occ) * sms;
    // a multiplier just below one and a small addend keep the values finite
    const T a = (T)0.999999, b = (T)1e-6;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return EOFA_ERR_CUDA;
    }
    eofa_status s = EOFA_OK;
    k_fma<T><<<grid, kThreads, 0, st>>>(a, b, 0, nullptr);  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps && s == EOFA_OK; ++r) {
        cudaEventRecord(e0, st);
        k_fma<T><<<grid, kThreads, 0, st>>>(a, b, 0, nullptr);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = EOFA_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    if (s == EOFA_OK && cudaGetLastError() != cudaSuccess) s = EOFA_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != EOFA_OK) return s;
    const double fmas = (double)grid * kThreads * kChains * kIters;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return EOFA_OK;
}

}  // namespace

extern "C" eofa_status eofa_measure_fma(int prec, int reps, double* tflops, void* stream) {
    if (!tflops || reps < 1) return EOFA_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == EOFA_F64) return measure<double>(reps, tflops, st);
    if (prec == EOFA_F32) return measure<float>(reps, tflops, st);
    return EOFA_ERR_ARG;
}
