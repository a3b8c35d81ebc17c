// action.cu -- kernels of the EOFA action operator and heatbath
// (Eqs. eofa_action, eofa_heatbath): the maps between the caller's 4D field
// and the 5D sources and solutions of the H-form solves (Omega_pm P_pm and
// its adjoint, App. A), and the multi-vector inner products and linear
// combinations of the chronological initial guess (Sec. V.B).  Fields are in
// the caller's canonical complex128 layout ([t][z][y][x][s][spin][colour]
// for 5D, the same without s for 4D); gamma_5 = diag(1, 1, -1, -1), so
// P_+ keeps spins 0, 1 and P_- spins 2, 3.  Memory-bound and small next to
// the solves: one thread per complex element, grid-stride loops.
#include "blas.h"

namespace eofa {

namespace {

constexpr int AT = 256;  // threads per block

inline int grid_of(long n, int cap) { return (int)std::max<long>(1, std::min<long>((n + AT - 1) / AT, cap)); }

__device__ __forceinline__ bool keeps(int chi, int e) { return chi > 0 ? e < 6 : e >= 6; }

}  // namespace

// out(x, s) = om[s] (P_chi xi)(x)
__global__ void __launch_bounds__(AT) k_omega_in(double2* __restrict__ out, const double2* __restrict__ xi,
                                                 const __grid_constant__ OmegaW om, int chi, long V, int Ls) {
    const long n = V * Ls * 12;
    for (long i = blockIdx.x * (long)AT + threadIdx.x; i < n; i += (long)gridDim.x * AT) {
        const int e = (int)(i % 12);
        const long xs = i / 12;
        const int s = (int)(xs % Ls);
        const long x = xs / Ls;
        double2 v = make_double2(0.0, 0.0);
        if (keeps(chi, e)) {
            const double2 a = xi[x * 12 + e];
            v = make_double2(om.w[s] * a.x, om.w[s] * a.y);
        }
        out[i] = v;
    }
}

// out(x) = a base(x) + coef P_chi sum_s om[s] psi(x, s)   (no sum when psi is NULL;
// out may be base: every element is read before it is written by the same thread)
__global__ void __launch_bounds__(AT) k_omega_out(double2* out, const double2* base, double a,
                                                  const double2* __restrict__ psi,
                                                  const __grid_constant__ OmegaW om, int chi, double coef, long V,
                                                  int Ls) {
    const long n = V * 12;
    for (long i = blockIdx.x * (long)AT + threadIdx.x; i < n; i += (long)gridDim.x * AT) {
        const int e = (int)(i % 12);
        const long x = i / 12;
        const double2 b = base[i];
        double2 r = make_double2(a * b.x, a * b.y);
        if (psi && keeps(chi, e)) {
            double sr = 0.0, si = 0.0;
            const double2* p = psi + x * Ls * 12 + e;
            for (int s = 0; s < Ls; ++s) {
                const double2 v = p[s * 12];
                sr = fma(om.w[s], v.x, sr);
                si = fma(om.w[s], v.y, si);
            }
            r.x = fma(coef, sr, r.x);
            r.y = fma(coef, si, r.y);
        }
        out[i] = r;
    }
}

// partial[b][j] = sum over block b's elements of conj(v_j) w, j < set.n
__global__ void __launch_bounds__(AT) k_multidot(const __grid_constant__ VecSet set, const double2* __restrict__ w,
                                                 long n, double2* __restrict__ partial) {
    __shared__ double red[AT / 32][2 * kMultiMax];
    double acc[2 * kMultiMax];
#pragma unroll
    for (int j = 0; j < 2 * kMultiMax; ++j) acc[j] = 0.0;
    for (long i = blockIdx.x * (long)AT + threadIdx.x; i < n; i += (long)gridDim.x * AT) {
        const double2 b = w[i];
#pragma unroll
        for (int j = 0; j < kMultiMax; ++j) {
            if (j < set.n) {
                const double2 a = set.v[j][i];
                acc[2 * j] = fma(a.x, b.x, fma(a.y, b.y, acc[2 * j]));
                acc[2 * j + 1] = fma(a.x, b.y, fma(-a.y, b.x, acc[2 * j + 1]));
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 2 * kMultiMax; ++j) {
        double v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMultiMax) {
        double v = 0.0;
        for (int k = 0; k < AT / 32; ++k) v += red[k][threadIdx.x];
        double* pp = reinterpret_cast<double*>(partial + (long)blockIdx.x * kMultiMax);
        pp[threadIdx.x] = v;
    }
}

// out[j] = sum_b partial[b][j], in block order (deterministic)
__global__ void k_multidot_sum(const double2* __restrict__ partial, int nblk, int nv, double2* __restrict__ out) {
    const int j = threadIdx.x;
    if (j >= nv) return;
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < nblk; ++b) {
        const double2 v = partial[(long)b * kMultiMax + j];
        sr += v.x;
        si += v.y;
    }
    out[j] = make_double2(sr, si);
}

// out = sum_j c_j v_j (complex c_j)
// out may be one of the v_j: each element is read before the same thread writes it
__global__ void __launch_bounds__(AT) k_combine(double2* out, const __grid_constant__ VecSet set, long n) {
    for (long i = blockIdx.x * (long)AT + threadIdx.x; i < n; i += (long)gridDim.x * AT) {
        double r = 0.0, m = 0.0;
#pragma unroll
        for (int j = 0; j < kMultiMax; ++j) {
            if (j < set.n) {
                const double2 a = set.v[j][i];
                const double2 c = set.c[j];
                r = fma(c.x, a.x, fma(-c.y, a.y, r));
                m = fma(c.x, a.y, fma(c.y, a.x, m));
            }
        }
        out[i] = make_double2(r, m);
    }
}

cudaError_t omega_in(double* out5, const double* xi4, const OmegaW& om, int chi, long V, int Ls,
                     cudaStream_t st) {
    k_omega_in<<<grid_of(V * Ls * 12, 1 << 16), AT, 0, st>>>((double2*)out5, (const double2*)xi4, om, chi, V, Ls);
    return cudaGetLastError();
}

cudaError_t omega_out(double* out4, const double* base4, double a, const double* psi5, const OmegaW& om, int chi,
                      double coef, long V, int Ls, cudaStream_t st) {
    k_omega_out<<<grid_of(V * 12, 1 << 16), AT, 0, st>>>((double2*)out4, (const double2*)base4, a,
                                                         (const double2*)psi5, om, chi, coef, V, Ls);
    return cudaGetLastError();
}

int multidot_blocks(long n) { return grid_of(n, kMultiBlocks); }

cudaError_t multidot(const VecSet& set, const double* w, long n, double* partial, double* out, cudaStream_t st) {
    const int nb = multidot_blocks(n);
    k_multidot<<<nb, AT, 0, st>>>(set, (const double2*)w, n, (double2*)partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_multidot_sum<<<1, 32, 0, st>>>((const double2*)partial, nb, set.n, (double2*)out);
    return cudaGetLastError();
}

cudaError_t combine(double* out, const VecSet& set, long n, cudaStream_t st) {
    k_combine<<<grid_of(n, 1 << 16), AT, 0, st>>>((double2*)out, set, n);
    return cudaGetLastError();
}

}  // namespace eofa
