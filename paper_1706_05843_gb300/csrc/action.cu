// action.cu -- kernels of the EOFA action operator and heatbath
// (Eqs. eofa_action, eofa_heatbath): the maps between the caller's 4D field
// and the 5D sources and solutions of the H-form solves (Omega_pm P_pm and
// its adjoint, App. A), and the multi-vector inner products and linear
// combinations of the chronological initial guess (Sec. V.B), and the
// pseudofermion force's spin-traced bilinear (Sec. III.C).  Fields are in
// the caller's canonical complex128 layout ([t][z][y][x][s][spin][colour]
// for 5D, the same without s for 4D); gamma_5 = diag(1, 1, -1, -1), so
// P_+ keeps spins 0, 1 and P_- spins 2, 3.  Small next to the solves: one
// thread per complex element (per link for the force), grid-stride loops.
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

// ---------------------------------------------------------------------------
// EOFA pseudofermion force (Sec. III.C, Eq. eofa_force)
// ---------------------------------------------------------------------------
// gamma_mu in the chiral basis has one entry per row:
// (gamma_mu psi)_alpha = c_{mu,alpha} psi_{perm(mu,alpha)}, c in {+-1, +-i}:
//   gamma_1: (-i psi3, -i psi2, i psi1, i psi0)   gamma_2: (-psi3, psi2, psi1, -psi0)
//   gamma_3: (-i psi2, i psi3, i psi0, -i psi1)   gamma_4: (psi2, psi3, psi0, psi1)
__device__ __forceinline__ double2 gamma_row(int mu, int al, double2 v0, double2 v1, double2 v2, double2 v3) {
    const int src = mu < 2 ? 3 - al : al ^ 2;
    const double2 v = src == 0 ? v0 : src == 1 ? v1 : src == 2 ? v2 : v3;
    const double s03 = (al == 0 || al == 3) ? -1.0 : 1.0;
    double cr, ci;
    if (mu == 0) cr = 0.0, ci = al < 2 ? -1.0 : 1.0;
    else if (mu == 1) cr = s03, ci = 0.0;
    else if (mu == 2) cr = 0.0, ci = s03;
    else cr = 1.0, ci = 0.0;
    return make_double2(cr * v.x - ci * v.y, cr * v.y + ci * v.x);
}

// M[k][i] += sum_alpha ((1 + sg gamma_mu) b)_{alpha k} conj((gamma_5 a)_{alpha i})
// for one s: the spin trace of (1 + sg gamma_mu) b a^dag gamma_5 as a colour matrix
__device__ __forceinline__ void spin_trace(double2 (&M)[3][3], int mu, double sg, const double2* __restrict__ b,
                                           const double2* __restrict__ a) {
    double2 av[4][3];
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double2 v = a[al * 3 + i];
            av[al][i] = al < 2 ? v : make_double2(-v.x, -v.y);  // gamma_5 = diag(1, 1, -1, -1)
        }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 b0 = b[k], b1 = b[3 + k], b2 = b[6 + k], b3 = b[9 + k];
#pragma unroll
        for (int al = 0; al < 4; ++al) {
            const double2 bb = al == 0 ? b0 : al == 1 ? b1 : al == 2 ? b2 : b3;
            const double2 g = gamma_row(mu, al, b0, b1, b2, b3);
            const double pr = bb.x + sg * g.x, pi = bb.y + sg * g.y;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double2 c = av[al][i];  // p * conj(c)
                M[k][i].x = fma(pr, c.x, fma(pi, c.y, M[k][i].x));
                M[k][i].y = fma(pi, c.x, fma(-pr, c.y, M[k][i].y));
            }
        }
    }
}

// One thread per link (x, mu), mu fastest.  For chi_1 (sign +) and chi_2
// (sign -): M1 = sum_s Tr_spin[(1 - gamma_mu) chi(x+mu, s) (g5 R5 chi)(x, s)^dag],
// M2 = sum_s Tr_spin[(1 + gamma_mu) chi(x, s) (g5 R5 chi)(x+mu, s)^dag],
// with (g5 R5 chi)(x, s) = g5 chi(x, Ls-1-s); then
// Y = -k/2 phase sum_f sign_f (U M1 - M2 U^dag), so that d^a S = Tr(T^a Y), and
// F = sum_a T^a d^a S = -(1/2) [Y_A - Tr(Y_A)/3], Y_A = (Y - Y^dag)/2, for
// T^a = i lambda_a / 2.
__global__ void __launch_bounds__(AT) k_force(const double2* __restrict__ chi1, const double2* __restrict__ chi2,
                                              const double* __restrict__ l0, const double* __restrict__ l1,
                                              double2* __restrict__ F, Geom g, double k) {
    const long t = blockIdx.x * (long)AT + threadIdx.x;
    const long V = 2L * g.Vh;
    if (t >= 4 * V) return;
    const long lex = t >> 2;
    const int mu = (int)(t & 3);
    int c[4];
    {
        long r = lex;
        c[0] = (int)(r % g.X); r /= g.X;
        c[1] = (int)(r % g.Y); r /= g.Y;
        c[2] = (int)(r % g.Z);
        c[3] = (int)(r / g.Z);  // t + f Tp (flavour f of a G-parity context)
    }
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int f = c[3] >= g.Tp ? 1 : 0;
    c[3] -= f * g.Tp;
    const int ext = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.Tp;
    const int cm = mu == 0 ? c[0] : mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    const long stride = mu == 0 ? 1L : mu == 1 ? (long)g.X : mu == 2 ? (long)g.X * g.Y : (long)g.X * g.Y * g.Z;
    const bool cross = cm + 1 == ext;
    long nlex = cross ? lex - (long)(ext - 1) * stride : lex + stride;
    bool neg = cross && ((g.apmask >> mu) & 1);
    if (cross && ((g.gpmask >> mu) & 1)) {
        // G-parity: psi_1(x + L) = psi_2(x), psi_2(x + L) = -psi_1(x)
        nlex += (long)(1 - 2 * f) * g.Tp * g.X * g.Y * g.Z;
        neg = neg != (f == 1);
    }
    const double phase = neg ? -1.0 : 1.0;
    const double* l = (par ? l1 : l0) + ((lex >> 1) * 4 + mu) * 12;
    double2 U[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        U[0][j] = make_double2(l[2 * j], l[2 * j + 1]);
        U[1][j] = make_double2(l[6 + 2 * j], l[6 + 2 * j + 1]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // row 2 = conj(row 0 x row 1)
        const int p = (j + 1) % 3, q = (j + 2) % 3;
        const double re = (U[0][p].x * U[1][q].x - U[0][p].y * U[1][q].y) -
                          (U[0][q].x * U[1][p].x - U[0][q].y * U[1][p].y);
        const double im = (U[0][p].x * U[1][q].y + U[0][p].y * U[1][q].x) -
                          (U[0][q].x * U[1][p].y + U[0][q].y * U[1][p].x);
        U[2][j] = make_double2(re, -im);
    }
    const int Ls = g.Ls;
    double2 Y[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Y[a][b] = make_double2(0.0, 0.0);
    for (int f = 0; f < 2; ++f) {
        const double2* chi = f ? chi2 : chi1;
        const double2* cx = chi + lex * Ls * 12;
        const double2* cn = chi + nlex * Ls * 12;
        double2 M1[3][3], M2[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) M1[a][b] = M2[a][b] = make_double2(0.0, 0.0);
        for (int s = 0; s < Ls; ++s) {
            const int sb = Ls - 1 - s;
            spin_trace(M1, mu, -1.0, cn + s * 12, cx + sb * 12);
            spin_trace(M2, mu, +1.0, cx + s * 12, cn + sb * 12);
        }
        const double sgn = f ? -1.0 : 1.0;
        // Y += sgn (U M1 - M2 U^dag)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double re = 0.0, im = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    re += U[a][j].x * M1[j][b].x - U[a][j].y * M1[j][b].y;
                    im += U[a][j].x * M1[j][b].y + U[a][j].y * M1[j][b].x;
                    // M2[a][j] conj(U[b][j])
                    re -= M2[a][j].x * U[b][j].x + M2[a][j].y * U[b][j].y;
                    im -= M2[a][j].y * U[b][j].x - M2[a][j].x * U[b][j].y;
                }
                Y[a][b].x += sgn * re;
                Y[a][b].y += sgn * im;
            }
    }
    const double w = -0.5 * k * phase;
    // F = -(1/2) [Y_A - Tr(Y_A)/3], Y_A = (Y - Y^dag)/2; Y scaled by w
    const double trI = w * (Y[0][0].y + Y[1][1].y + Y[2][2].y) / 3.0;  // Im Tr(Y_A) / 3
    double2* out = F + t * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double re = 0.5 * w * (Y[a][b].x - Y[b][a].x);
            double im = 0.5 * w * (Y[a][b].y + Y[b][a].y);
            if (a == b) im -= trI;
            out[a * 3 + b] = make_double2(-0.5 * re, -0.5 * im);
        }
}

// G-parity: the force on the physical link U_mu(x) is the stacked lattice's
// force on flavour 1's copy plus the conjugate of that on flavour 2's copy
// (flavour 2 carries conj(U), and conj(exp(s T^a) U) = exp(s conj(T^a)) conj(U))
__global__ void __launch_bounds__(AT) k_force_fold(const double2* __restrict__ Fs, double2* __restrict__ F,
                                                   long n) {
    const long i = blockIdx.x * (long)AT + threadIdx.x;
    if (i >= n) return;
    const double2 a = Fs[i], b = Fs[n + i];
    F[i] = make_double2(a.x + b.x, a.y - b.y);
}

cudaError_t force_fold(const double* Fs, double* F, long n, cudaStream_t st) {
    k_force_fold<<<(int)((n + AT - 1) / AT), AT, 0, st>>>((const double2*)Fs, (double2*)F, n);
    return cudaGetLastError();
}

cudaError_t eofa_force_links(const double* chi1, const double* chi2, const void* const links64[2], double* F,
                             const Geom& g, double k, cudaStream_t st) {
    const long n = 8L * g.Vh;
    k_force<<<(int)((n + AT - 1) / AT), AT, 0, st>>>((const double2*)chi1, (const double2*)chi2,
                                                     (const double*)links64[0], (const double*)links64[1],
                                                     (double2*)F, g, k);
    return cudaGetLastError();
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

// Sec. VI force norms: per link ||F_mu(x)||^2 = 2 sum_ij |F_ij|^2 (the sum of
// the squared generator components for Tr T^a T^b = -delta^ab / 2);
// partial[b] = (sum, max) over block b's links, then one block combines them
// in block order (deterministic)
__global__ void __launch_bounds__(AT) k_force_norms(const double2* __restrict__ F, long nlinks,
                                                    double2* __restrict__ partial) {
    __shared__ double rs[AT / 32], rm[AT / 32];
    double sum = 0.0, mx = 0.0;
    for (long l = blockIdx.x * (long)AT + threadIdx.x; l < nlinks; l += (long)gridDim.x * AT) {
        double n2 = 0.0;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const double2 v = F[l * 9 + e];
            n2 = fma(v.x, v.x, fma(v.y, v.y, n2));
        }
        n2 *= 2.0;
        sum += n2;
        mx = fmax(mx, n2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) {
        rs[wid] = sum;
        rm[wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < AT / 32; ++k) {
            a += rs[k];
            b = fmax(b, rm[k]);
        }
        partial[blockIdx.x] = make_double2(a, b);
    }
}

__global__ void k_force_norms_sum(const double2* __restrict__ partial, int nblk, double2* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblk; ++k) {
        a += partial[k].x;
        b = fmax(b, partial[k].y);
    }
    *out = make_double2(a, b);
}

cudaError_t force_norm_sums(const double* F, long nlinks, double* partial, double* out, cudaStream_t st) {
    const int nb = multidot_blocks(nlinks);
    k_force_norms<<<nb, AT, 0, st>>>((const double2*)F, nlinks, (double2*)partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_force_norms_sum<<<1, 1, 0, st>>>((const double2*)partial, nb, (double2*)out);
    return cudaGetLastError();
}

cudaError_t combine(double* out, const VecSet& set, long n, cudaStream_t st) {
    k_combine<<<grid_of(n, 1 << 16), AT, 0, st>>>((double2*)out, set, n);
    return cudaGetLastError();
}

}  // namespace eofa
