// blas.h -- internal interface between the host driver (eofa.cu) and the
// kernels of blas.cu and dslash_<prec>.cu.  Not part of the public ABI.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace eofa {

struct VecRef {
    void* d;    // chunk array of one parity
    float* n;   // FP16 per-site scales (NULL otherwise)
};

struct HopArgs;

// precision codes: 0 F64, 1 F32, 2 F16, 3 BF16 (the eofa_prec values)
cudaError_t launch_hop_f64(int kind, const HopArgs& a, const void* coef, cudaStream_t st);
cudaError_t launch_hop_f32(int kind, const HopArgs& a, const void* coef, cudaStream_t st);
cudaError_t launch_hop_f16(int kind, const HopArgs& a, const void* coef, cudaStream_t st);
cudaError_t launch_hop_bf16(int kind, const HopArgs& a, const void* coef, cudaStream_t st);
// kinds >= 4 (FP64 and FP32 storage only)
cudaError_t launch_hop_f64_outer(int kind, const HopArgs& a, const void* coef, cudaStream_t st);
cudaError_t launch_hop_f32_outer(int kind, const HopArgs& a, const void* coef, cudaStream_t st);

cudaError_t scal_init(DevScal* sc, double target_rr, int max_iters, unsigned long long timeout_ns,
                      cudaStream_t st);
cudaError_t while_cond(cudaGraphConditionalHandle h, DevScal* sc, cudaStream_t st);
// device-driven defect correction of a batched solve (blas.cu)
cudaError_t outer_begin(DevScal* sc, double tol, double floor_tol, int maxit, int maxouter,
                        unsigned long long timeout_ns, int fin, int x_zero, int body_cap, cudaStream_t st);
cudaError_t outer_gate(DevScal* sc, cudaStream_t st);
cudaError_t outer_decide_dev(DevScal* sc, int first, cudaStream_t st);
cudaError_t outer_cond(cudaGraphConditionalHandle h, const ScalList& L, cudaStream_t st);
// r -= alpha q with |r|^2 (rd: FIN_RR); returns at once when *done
cudaError_t blas_cg_r(int prec, VecRef q, VecRef r, long n5, int Ls, Reduce rd, const int* done,
                      cudaStream_t st);
// x += alpha p; p = z + beta p unless done (rd: FIN_STOP on the same scalars)
cudaError_t blas_cg_px(int prec, int xprec, VecRef x, VecRef p, VecRef z, long n5, int Ls, Reduce rd,
                       cudaStream_t st);
// skip (may be NULL): the kernel returns at once while *skip is nonzero
cudaError_t blas_copy(int dprec, VecRef dst, int sprec, VecRef src, long n5, int Ls, double scale,
                      int inv_sqrt_slot, Reduce rd, cudaStream_t st, const int* skip = nullptr);
cudaError_t blas_acc(VecRef x, int eprec, VecRef e, long n5, int Ls, const DevScal* sc, int slot,
                     cudaStream_t st, const int* skip = nullptr);
cudaError_t blas_sub(VecRef r, VecRef b, VecRef q, long n5, int Ls, Reduce rd, cudaStream_t st,
                     const int* skip = nullptr);
cudaError_t blas_zero(int prec, VecRef v, long n5, int Ls, cudaStream_t st, const int* skip = nullptr);
cudaError_t layout_import(VecRef dst, const double* src, const Geom& g, int par, int g5r5, cudaStream_t st);
cudaError_t layout_export(double* dst, VecRef src, const Geom& g, int par, int g5r5, cudaStream_t st);
cudaError_t gauge_import(const double* U, const Geom& g, void* const links[4][2], int* bad, cudaStream_t st);
// [U; conj(U)] for a G-parity context (n complex entries of U)
cudaError_t gparity_gauge(const double* U, double* out, long n, cudaStream_t st);
int blas_max_grid(long n5);

// learned preconditioner support (FP32 odd-parity fields <-> network activations)
cudaError_t embed_odd(VecRef f, __nv_bfloat16* act, const Geom& g, int sl, double scale, const DevScal* sc,
                      int slot, cudaStream_t st);
cudaError_t extract_odd(const float* out32, VecRef f, const Geom& g, cudaStream_t st);
cudaError_t cdot(VecRef a, VecRef b, long n5, int Ls, Reduce rr, Reduce ri, cudaStream_t st);
cudaError_t caxpby(VecRef y, VecRef x, long n5, int Ls, float ar, float ai, float b, cudaStream_t st);
cudaError_t slice_norm(VecRef f, long vh, int Ls, int sl, Reduce rd, cudaStream_t st);
cudaError_t loss_grad(const float* out, const __nv_bfloat16* e, const float* w, float* dout, const Geom& g, int B,
                      Reduce rd, cudaStream_t st);

// EOFA action and heatbath (action.cu); canonical complex128 fields
constexpr int kMultiMax = 8;       // vectors of one multi-dot or combination
constexpr int kMultiBlocks = 1024; // fixed first-stage grid of the multi-dot
struct OmegaW {
    double w[LSMAX];  // Omega_pm as weights over s (App. A)
};
struct VecSet {
    const double2* v[kMultiMax];
    double2 c[kMultiMax];  // coefficients of combine
    int n;
};
// out5 = Omega P_chi xi4 (om.w[s] times the chi half of xi4)
cudaError_t omega_in(double* out5, const double* xi4, const OmegaW& om, int chi, long V, int Ls, cudaStream_t st);
// out4 = a base4 + coef P_chi Omega^dag psi5 (psi5 NULL: out4 = a base4)
cudaError_t omega_out(double* out4, const double* base4, double a, const double* psi5, const OmegaW& om, int chi,
                      double coef, long V, int Ls, cudaStream_t st);
// out[j] = <v_j, w> for j < set.n (n complex elements; partial holds
// kMultiBlocks * kMultiMax complex values)
cudaError_t multidot(const VecSet& set, const double* w, long n, double* partial, double* out, cudaStream_t st);
// out[0] = sum over links of ||F_mu(x)||^2, out[1] = the largest one (n
// links of 9 complex entries; partial holds kMultiBlocks complex values)
cudaError_t force_norm_sums(const double* F, long nlinks, double* partial, double* out, cudaStream_t st);
// out = sum_j set.c[j] set.v[j]
cudaError_t combine(double* out, const VecSet& set, long n, cudaStream_t st);
// EOFA force F[lex][mu] (3x3 complex, anti-Hermitian traceless) from the
// canonical chi_1, chi_2 and the context's FP64 two-row links
cudaError_t eofa_force_links(const double* chi1, const double* chi2, const void* const links64[2], double* F,
                             const Geom& g, double k, cudaStream_t st);
// G-parity: F = Fs[flavour 1] + conj(Fs[flavour 2]), n = complex entries of F
cudaError_t force_fold(const double* Fs, double* F, long n, cudaStream_t st);

}  // namespace eofa
