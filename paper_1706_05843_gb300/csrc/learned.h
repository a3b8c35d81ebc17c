// learned.h -- internal interface of the learned preconditioner (learned.cu).
//
// The network: three 4D convolutions with 3^4 kernels over the full lattice,
// periodic in all directions, applied to every s-slice independently (the
// slices are the batch), real channels 24 -> 32 -> 32 -> 24 (the 12 complex
// spin-colour components of a spinor), no biases, LeakyReLU(0.1) after the
// first two layers.  Weights and activations in BF16, accumulation in FP32
// on the tensor cores.
//
// Public weight layout (FP32, the three layers one after another):
//   W_l[tap][co][ci], tap = ((dt*3 + dz)*3 + dy)*3 + dx with offsets d - 1,
//   (ci, co) = (24, 32), (32, 32), (32, 24).
// y[x, co] = sum_tap sum_ci W[tap][co][ci] in[x + off(tap), ci].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace eofa {

typedef __nv_bfloat16 bf16;

constexpr int kNetLayers = 3;
constexpr int kNetCin[3] = {24, 32, 32};
constexpr int kNetCout[3] = {32, 32, 24};
constexpr long kNetLayerW[3] = {81L * 32 * 24, 81L * 32 * 32, 81L * 24 * 32};
constexpr long kNetWeights = 81L * 32 * 24 + 81L * 32 * 32 + 81L * 24 * 32;  // 207360
constexpr float kLeaky = 0.1f;
constexpr int kCP = 32;  // padded channel count in device activations

struct ConvGeom {
    int X, Y, Z, T;
    int V;      // sites per slice
    int S;      // slices
};

// device copies of one network
struct NetDev {
    float* Wm = nullptr;          // master FP32, public layout
    bf16* Wf[3] = {};             // forward operands [81][32 co][32 ci], zero padded
    bf16* Wb[3] = {};             // backward-data operands [81][32 ci][32 co], taps mirrored
};

// activations [S][V][32] BF16; out [S][V][32] FP32 (channels >= 24 are zero)
cudaError_t net_convert(const NetDev& n, cudaStream_t st);
cudaError_t net_forward(const NetDev& n, const ConvGeom& g, const bf16* a0, bf16* a1, bf16* a2, float* out,
                        cudaStream_t st);
// gradients: dout [S][V][32] FP32 -> dW (FP32 public layout, accumulated), din [S][V][32] FP32 or NULL;
// work buffers d1, d2 [S][V][32] BF16 and dob [S][V][32] BF16.
cudaError_t net_backward(const NetDev& n, const ConvGeom& g, const bf16* a0, const bf16* a1, const bf16* a2,
                         const float* dout, float* dW, float* din, bf16* dob, bf16* d1, bf16* d2,
                         cudaStream_t st);
// after a synchronisation: *fault = 1 (and the flag cleared) when a
// convolution gave up on a bounded wait and skipped its output since the
// last call; the results computed meanwhile are not valid
cudaError_t net_fault(int* fault);
// FP32 [S][V][24] <-> BF16/FP32 [S][V][32]
cudaError_t pack_act(const float* in24, bf16* a32, long rows, cudaStream_t st);
cudaError_t unpack_out(const float* out32, float* out24, long rows, cudaStream_t st);
cudaError_t pad_f32(const float* in24, float* out32, long rows, cudaStream_t st);
// Adam on the FP32 master weights
cudaError_t adam_step(float* w, const float* g, float* m, float* v, long n, float lr, float b1, float b2,
                      float eps, int t, cudaStream_t st);

}  // namespace eofa
