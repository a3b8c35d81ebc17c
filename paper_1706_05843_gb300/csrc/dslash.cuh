// dslash.cuh -- the fused 4D Wilson hop + fifth-dimension kernel.
//
// One CTA owns NS output 4D sites of one checkerboard parity and all Ls
// slices of them; thread (i, s) owns 5D site (x_i, s).  Three phases:
//
//  1. hop:   h(x, s) = sum_mu [ (1 - g gamma_mu) U_mu(x) chi(x+mu, s)
//                             + (1 + g gamma_mu) U_mu(x-mu)^dag chi(x-mu, s) ]
//            with g = +1 (D_h) or -1 (gamma_5 D_h gamma_5 = the hop of D^dag),
//            chi = psi, or chi = D~ psi / b5 built on the fly from the
//            neighbour's slices s-1 (P+ half) and s+1 (P- half) -- the
//            "L acts first" order of Eq. (Ddwf).  Spin projection to half
//            spinors, two-row links rebuilt in registers; h goes to shared
//            memory.  An optional site-local input y is staged beside it.
//  2. fifth dimension: each thread takes complex columns (x_i, spin, colour)
//            and applies an O(Ls) program: the cyclic bidiagonal
//            A = alpha + gamma L (the site-diagonal block of D_DWF, App. B),
//            its transpose, its inverse by a closed-form corner plus a
//            first-order recurrence, the rank-one EOFA shift u (x) v
//            (Eqs. Mooee_shift_p/m) and its Sherman-Morrison inverse
//            (Eq. sherman_morrison_mobius_inv), D~ = b5 + c5 L and D~^T.
//            The site-local kinds (M y + h: L reaches one neighbouring
//            slice, the shift one fixed slice) skip this phase: thread
//            (i, s) reads those slices of y itself and keeps h in registers.
//  3. store: thread (i, s) writes its spinor back (coalesced 16-byte
//            chunks) and contributes |out|^2 to a deterministic reduction.
//
// The kernel kinds below are the even-odd blocks of K (App. B):
//   K_ee = K_oo = M (site-local), K_eo = K_oe = -1/2 D_h D~.
#pragma once

#include "common.cuh"

namespace eofa {

enum Kind {
    KIND_EO_MINV = 0,      // out = -1/2 D~ M^-1 D_h D~ in            (Schur step 1)
    KIND_OE_SCHUR = 1,     // out = M y + 1/2 D_h in                  (Schur step 2; in = D~ t)
    KIND_EO_MINV_DAG = 2,  // out = -1/2 M^-T D~^T g5 D_h g5 in       (Schur^dag step 1)
    KIND_OE_SCHUR_DAG = 3, // out = M^T y + 1/2 D~^T g5 D_h g5 in     (Schur^dag step 2)
    KIND_RECON = 4,        // out = M^-1 (y + 1/2 D_h D~ in)          (even reconstruction)
    KIND_SRC = 5,          // out = y + 1/2 D_h in                    (even-odd source)
    KIND_FULL = 6,         // out = M y - 1/2 D_h D~ in               (K, one parity)
    KIND_FULL_DAG = 7,     // out = M^T y - 1/2 D~^T g5 D_h g5 in     (K^dag, one parity)
    KIND_LOC_DTMINV = 8,   // out = D~ M^-1 y
    KIND_LOC_DT = 9,       // out = D~ y
    KIND_LOC_DTINV = 10,   // out = D~^-1 y
    // even-odd on Eq. (non_hermit_sys) without the Cayley form (App. B):
    // A = D_EOFA + beta g5 R5 Delta P, A_ee = A_oo dense in s, A_eo = -1/2 D_h
    KIND_D_EO = 11,        // out = -1/2 A_ee^-1 D_h in
    KIND_D_OE = 12,        // out = A_oo y + 1/2 D_h in
    KIND_D_EO_DAG = 13,    // out = -1/2 A_ee^-T g5 D_h g5 in
    KIND_D_OE_DAG = 14,    // out = A_oo^T y + 1/2 g5 D_h g5 in
    NKIND = 15
};

template <int K> struct KindTraits {
    static constexpr bool DENSE = K >= KIND_D_EO && K <= KIND_D_OE_DAG;
    static constexpr bool HOP = K <= KIND_FULL_DAG || DENSE;
    static constexpr bool DAG = K == KIND_EO_MINV_DAG || K == KIND_OE_SCHUR_DAG || K == KIND_FULL_DAG ||
                                K == KIND_D_EO_DAG || K == KIND_D_OE_DAG;
    static constexpr bool PRE = K == KIND_EO_MINV || K == KIND_RECON || K == KIND_FULL;
    static constexpr bool HASY = !(K == KIND_EO_MINV || K == KIND_EO_MINV_DAG || K == KIND_D_EO || K == KIND_D_EO_DAG);
    // site-local kinds: the fifth-dimension part reaches only slices s-1, s+1
    // and the fixed slice of the rank-one shift, so each thread finishes its
    // own 5D site without the shared-memory column phase
    static constexpr bool PTW = K == KIND_OE_SCHUR || K == KIND_SRC || K == KIND_FULL;
};

struct HopArgs {
    Geom g;
    int out_par;
    int tile_var;                            // CTA tile variant (autotuner)
    const void* in;  const float* in_nrm;    // hop input, parity 1 - out_par
    const void* y;   const float* y_nrm;     // site-local input, parity out_par
    void* out;       float* out_nrm;         // output, parity out_par
    const void* lk_out;                      // links of parity out_par
    const void* lk_in;                       // links of parity 1 - out_par
    Reduce rd;                               // rd.fin == FIN_NONE: no reduction
    const int* done;                         // early exit when *done != 0 (may be NULL)
    // dense kinds: the Ls x Ls s-space matrix of each chirality in compute
    // precision, [chirality][row][col] in mirrored coordinates
    // (A_ee^-1 for the EO kinds, A_oo for the OE kinds)
    const void* dense;
};

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct C2 { R re, im; };

template <typename R>
__device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ C2<R> cmulc(C2<R> a, C2<R> b) {  // conj(a) * b
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// ---------------------------------------------------------------------------
// one hopping direction: acc += (1 + SG gamma_MU) W chi, W = U or U^dag
// u: 18 reals, rows 0..2 of the link (row 2 rebuilt; the boundary sign of the
// hop folded in).
// ---------------------------------------------------------------------------
template <typename R, int MU, int SG, bool ADJ>
__device__ __forceinline__ void hop_dir(R* __restrict__ acc, const R* __restrict__ p,
                                        const R* __restrict__ u) {
    // spin projection: h = psi_up + SG B psi_dn, B = -i sigma_k (k = 1..3) or 1
    R h[12];
    constexpr R s = (R)SG;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R p0r = p[0 * 6 + 2 * c], p0i = p[0 * 6 + 2 * c + 1];
        const R p1r = p[1 * 6 + 2 * c], p1i = p[1 * 6 + 2 * c + 1];
        const R p2r = p[2 * 6 + 2 * c], p2i = p[2 * 6 + 2 * c + 1];
        const R p3r = p[3 * 6 + 2 * c], p3i = p[3 * 6 + 2 * c + 1];
        R h0r, h0i, h1r, h1i;
        if constexpr (MU == 0) {        // B psi_dn = (-i psi3, -i psi2)
            h0r = p0r + s * p3i; h0i = p0i - s * p3r;
            h1r = p1r + s * p2i; h1i = p1i - s * p2r;
        } else if constexpr (MU == 1) { // B psi_dn = (-psi3, psi2)
            h0r = p0r - s * p3r; h0i = p0i - s * p3i;
            h1r = p1r + s * p2r; h1i = p1i + s * p2i;
        } else if constexpr (MU == 2) { // B psi_dn = (-i psi2, i psi3)
            h0r = p0r + s * p2i; h0i = p0i - s * p2r;
            h1r = p1r - s * p3i; h1i = p1i + s * p3r;
        } else {                        // B psi_dn = psi_dn
            h0r = p0r + s * p2r; h0i = p0i + s * p2i;
            h1r = p1r + s * p3r; h1i = p1i + s * p3i;
        }
        h[2 * c] = h0r; h[2 * c + 1] = h0i;
        h[6 + 2 * c] = h1r; h[6 + 2 * c + 1] = h1i;
    }
    // colour: w = W h for both half-spinor components
    R w[12];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // complex multiply-accumulate as plain FMA chains (4 per term)
            R re = (R)0, im = (R)0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R hr = h[sp * 6 + 2 * b], hi = h[sp * 6 + 2 * b + 1];
                if constexpr (!ADJ) {       // U_ab h_b
                    const R ur = u[(a * 3 + b) * 2], ui = u[(a * 3 + b) * 2 + 1];
                    if (b == 0) { re = ur * hr; im = ur * hi; }
                    else { re = fma(ur, hr, re); im = fma(ur, hi, im); }
                    re = fma(-ui, hi, re);
                    im = fma(ui, hr, im);
                } else {                    // conj(U_ba) h_b
                    const R ur = u[(b * 3 + a) * 2], ui = u[(b * 3 + a) * 2 + 1];
                    if (b == 0) { re = ur * hr; im = ur * hi; }
                    else { re = fma(ur, hr, re); im = fma(ur, hi, im); }
                    re = fma(ui, hi, re);
                    im = fma(-ui, hr, im);
                }
            }
            w[sp * 6 + 2 * a] = re;
            w[sp * 6 + 2 * a + 1] = im;
        }
    }
    // reconstruct: upper += w, lower += SG B^dag w
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R w0r = w[2 * c], w0i = w[2 * c + 1];
        const R w1r = w[6 + 2 * c], w1i = w[6 + 2 * c + 1];
        acc[0 * 6 + 2 * c] += w0r; acc[0 * 6 + 2 * c + 1] += w0i;
        acc[1 * 6 + 2 * c] += w1r; acc[1 * 6 + 2 * c + 1] += w1i;
        if constexpr (MU == 0) {        // B^dag w = (i w1, i w0)
            acc[2 * 6 + 2 * c] -= s * w1i; acc[2 * 6 + 2 * c + 1] += s * w1r;
            acc[3 * 6 + 2 * c] -= s * w0i; acc[3 * 6 + 2 * c + 1] += s * w0r;
        } else if constexpr (MU == 1) { // B^dag w = (w1, -w0)
            acc[2 * 6 + 2 * c] += s * w1r; acc[2 * 6 + 2 * c + 1] += s * w1i;
            acc[3 * 6 + 2 * c] -= s * w0r; acc[3 * 6 + 2 * c + 1] -= s * w0i;
        } else if constexpr (MU == 2) { // B^dag w = (i w0, -i w1)
            acc[2 * 6 + 2 * c] -= s * w0i; acc[2 * 6 + 2 * c + 1] += s * w0r;
            acc[3 * 6 + 2 * c] += s * w1i; acc[3 * 6 + 2 * c + 1] -= s * w1r;
        } else {                        // B^dag w = w
            acc[2 * 6 + 2 * c] += s * w0r; acc[2 * 6 + 2 * c + 1] += s * w0i;
            acc[3 * 6 + 2 * c] += s * w1r; acc[3 * 6 + 2 * c + 1] += s * w1i;
        }
    }
}

template <typename R>
__device__ __forceinline__ void rebuild_row2(R* u) {
    // row2 = conj(row0 x row1)
    C2<R> a0 = {u[0], u[1]}, a1 = {u[2], u[3]}, a2 = {u[4], u[5]};
    C2<R> b0 = {u[6], u[7]}, b1 = {u[8], u[9]}, b2 = {u[10], u[11]};
    C2<R> c0 = cmul(a1, b2), d0 = cmul(a2, b1);
    C2<R> c1 = cmul(a2, b0), d1 = cmul(a0, b2);
    C2<R> c2 = cmul(a0, b1), d2 = cmul(a1, b0);
    u[12] = c0.re - d0.re; u[13] = -(c0.im - d0.im);
    u[14] = c1.re - d1.re; u[15] = -(c1.im - d1.im);
    u[16] = c2.re - d2.re; u[17] = -(c2.im - d2.im);
}

// ---------------------------------------------------------------------------
// fifth-dimension column operators (mirrored coordinates: always L+ / L-)
// ---------------------------------------------------------------------------
// (a + g L+) v,  L+: v_s <- v_{s-1}, v_0 <- -m v_{Ls-1}
template <typename R, int LS>
__device__ __forceinline__ void op_fwd(C2<R>* v, R a, R g, R mg) {
    C2<R> last = v[LS - 1];
#pragma unroll
    for (int s = LS - 1; s >= 1; --s) {
        v[s].re = a * v[s].re + g * v[s - 1].re;
        v[s].im = a * v[s].im + g * v[s - 1].im;
    }
    v[0].re = a * v[0].re - mg * last.re;
    v[0].im = a * v[0].im - mg * last.im;
}
// (a + g L-) v = (a + g L+^T) v
template <typename R, int LS>
__device__ __forceinline__ void op_fwdT(C2<R>* v, R a, R g, R mg) {
    C2<R> first = v[0];
#pragma unroll
    for (int s = 0; s < LS - 1; ++s) {
        v[s].re = a * v[s].re + g * v[s + 1].re;
        v[s].im = a * v[s].im + g * v[s + 1].im;
    }
    v[LS - 1].re = a * v[LS - 1].re - mg * first.re;
    v[LS - 1].im = a * v[LS - 1].im - mg * first.im;
}
// solve (a + g L+) t = v in place: t_{Ls-1} = sum_j w_j v_{Ls-1-j},
// t_0 = v_0/a + m z t_{Ls-1}, t_s = v_s/a - z t_{s-1}.
template <typename R, int LS>
__device__ __forceinline__ void op_inv(C2<R>* v, R ia, R z, R mz, const R* w) {
    C2<R> tl = {0, 0};
#pragma unroll
    for (int j = 0; j < LS; ++j) {
        tl.re += w[j] * v[LS - 1 - j].re;
        tl.im += w[j] * v[LS - 1 - j].im;
    }
    v[0].re = ia * v[0].re + mz * tl.re;
    v[0].im = ia * v[0].im + mz * tl.im;
#pragma unroll
    for (int s = 1; s < LS - 1; ++s) {
        v[s].re = ia * v[s].re - z * v[s - 1].re;
        v[s].im = ia * v[s].im - z * v[s - 1].im;
    }
    v[LS - 1] = tl;
}
// solve (a + g L-) t = v in place (the mirror image of op_inv)
template <typename R, int LS>
__device__ __forceinline__ void op_invT(C2<R>* v, R ia, R z, R mz, const R* w) {
    C2<R> t0 = {0, 0};
#pragma unroll
    for (int j = 0; j < LS; ++j) {
        t0.re += w[j] * v[j].re;
        t0.im += w[j] * v[j].im;
    }
    v[LS - 1].re = ia * v[LS - 1].re + mz * t0.re;
    v[LS - 1].im = ia * v[LS - 1].im + mz * t0.im;
#pragma unroll
    for (int s = LS - 2; s >= 1; --s) {
        v[s].re = ia * v[s].re - z * v[s + 1].re;
        v[s].im = ia * v[s].im - z * v[s + 1].im;
    }
    v[0] = t0;
}

// M = A + pm beta u (x) v  on the shift chirality
template <typename R, int LS>
__device__ __forceinline__ void op_M(C2<R>* v, const SCoef<R>& c, bool sh) {
    C2<R> vl = v[LS - 1];
    op_fwd<R, LS>(v, c.alpha, c.gamma, c.m * c.gamma);
    if (sh) {
#pragma unroll
        for (int s = 0; s < LS; ++s) {
            R f = c.sbk * c.um[s];
            v[s].re += f * vl.re;
            v[s].im += f * vl.im;
        }
    }
}
template <typename R, int LS>
__device__ __forceinline__ void op_MT(C2<R>* v, const SCoef<R>& c, bool sh) {
    C2<R> d = {0, 0};
    if (sh) {
#pragma unroll
        for (int s = 0; s < LS; ++s) {
            d.re += c.um[s] * v[s].re;
            d.im += c.um[s] * v[s].im;
        }
    }
    op_fwdT<R, LS>(v, c.alpha, c.gamma, c.m * c.gamma);
    if (sh) {
        v[LS - 1].re += c.sbk * d.re;
        v[LS - 1].im += c.sbk * d.im;
    }
}
// Sherman-Morrison: M^-1 v = A^-1 v - (pm beta k (A^-1 v)_{j*} / den) x
template <typename R, int LS>
__device__ __forceinline__ void op_Minv(C2<R>* v, const SCoef<R>& c, bool sh) {
    op_inv<R, LS>(v, c.ia, c.za, c.mza, c.wa);
    if (sh) {
        C2<R> t = {c.sbk_den * v[LS - 1].re, c.sbk_den * v[LS - 1].im};
#pragma unroll
        for (int s = 0; s < LS; ++s) {
            v[s].re -= c.xm[s] * t.re;
            v[s].im -= c.xm[s] * t.im;
        }
    }
}
// M^-T v = A^-T v - (pm beta (u . A^-T v) / den) y
template <typename R, int LS>
__device__ __forceinline__ void op_MinvT(C2<R>* v, const SCoef<R>& c, bool sh) {
    op_invT<R, LS>(v, c.ia, c.za, c.mza, c.wa);
    if (sh) {
        C2<R> d = {0, 0};
#pragma unroll
        for (int s = 0; s < LS; ++s) {
            d.re += c.um[s] * v[s].re;
            d.im += c.um[s] * v[s].im;
        }
        d.re *= c.sb_den;
        d.im *= c.sb_den;
#pragma unroll
        for (int s = 0; s < LS; ++s) {
            v[s].re -= c.ym[s] * d.re;
            v[s].im -= c.ym[s] * d.im;
        }
    }
}

// ---------------------------------------------------------------------------
// shared-memory staging of the 5D tile
// ---------------------------------------------------------------------------
// A tile row holds the 24 reals of one 5D site.  The P- half (spins 2, 3) of
// slice s is stored in row Ls-1-s, so a column of either chirality reads its
// mirrored coordinate (the one in which both L's are L+) in row order.
template <typename R> struct ShStride;
template <> struct ShStride<float> { static constexpr int V = 28; };   // 112 B rows: conflict-free float4
template <> struct ShStride<double> { static constexpr int V = 26; };  // 208 B rows: conflict-free double2

// rows of one 4D site, padded so that the 12 columns of consecutive sites
// land on consecutive (re, im) bank pairs of a 128-byte line
template <typename R, int LS> struct SiteStride {
    static constexpr int MOD = 128 / (int)sizeof(R);
    static constexpr int WANT = 24 % MOD;
    static constexpr int V = LS * ShStride<R>::V + ((WANT - (LS * ShStride<R>::V) % MOD) + MOD) % MOD;
};

template <typename R> struct Pair;
template <> struct Pair<float> { typedef float2 T; };
template <> struct Pair<double> { typedef double2 T; };
template <typename R> struct Quad;
template <> struct Quad<float> { typedef float4 T; static constexpr int N = 4; };
template <> struct Quad<double> { typedef double2 T; static constexpr int N = 2; };

template <typename R>
__device__ __forceinline__ C2<R> ld_pair(const R* p) {
    const typename Pair<R>::T q = *reinterpret_cast<const typename Pair<R>::T*>(p);
    return {q.x, q.y};
}
template <typename R>
__device__ __forceinline__ void st_pair(R* p, const C2<R>& v) {
    typename Pair<R>::T q;
    q.x = v.re;
    q.y = v.im;
    *reinterpret_cast<typename Pair<R>::T*>(p) = q;
}
// 12 reals (one chirality half of a row) as 16-byte vectors
template <typename R>
__device__ __forceinline__ void st_half(R* p, const R* v) {
    typedef typename Quad<R>::T Q;
    constexpr int N = Quad<R>::N;
#pragma unroll
    for (int i = 0; i < 12 / N; ++i) {
        Q q;
        if constexpr (N == 4) q = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        else q = make_double2(v[2 * i], v[2 * i + 1]);
        reinterpret_cast<Q*>(p)[i] = q;
    }
}
template <typename R>
__device__ __forceinline__ void ld_half(const R* p, R* v) {
    typedef typename Quad<R>::T Q;
    constexpr int N = Quad<R>::N;
#pragma unroll
    for (int i = 0; i < 12 / N; ++i) {
        const Q q = reinterpret_cast<const Q*>(p)[i];
        if constexpr (N == 4) {
            v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
        } else {
            v[2 * i] = q.x; v[2 * i + 1] = q.y;
        }
    }
}

// Column access of a shared tile: one complex per row, rows ST reals apart.
template <typename R, int LS, int ST>
__device__ __forceinline__ void col_load(const R* p, C2<R>* v) {
#pragma unroll
    for (int k = 0; k < LS; ++k) v[k] = ld_pair(p + k * ST);
}
template <typename R, int LS, int ST>
__device__ __forceinline__ void col_store(R* p, const C2<R>* v) {
#pragma unroll
    for (int k = 0; k < LS; ++k) st_pair(p + k * ST, v[k]);
}

// The fifth-dimension program of one (site, spin, colour) column, in the
// mirrored coordinate.  hcol: the hop result (overwritten with the output),
// ycol: the local input; consecutive slices are ST reals apart.
template <typename R, int LS, int KIND, int ST>
__device__ __forceinline__ void column_program(R* hcol, const R* ycol, const SCoef<R>& cf, bool shv,
                                               R hb, const R* mat) {
    typedef KindTraits<KIND> KT;
    C2<R> v[LS];
    if constexpr (KT::DENSE) {
        // dense s-space matrix (row-major in mirrored coordinates) times the
        // column, or its transpose for the adjoint kinds
        constexpr bool TR = KT::DAG;
        constexpr bool EO = (KIND == KIND_D_EO || KIND == KIND_D_EO_DAG);
        col_load<R, LS, ST>(EO ? hcol : ycol, v);
        C2<R> w[LS];
#pragma unroll
        for (int k = 0; k < LS; ++k) {
            R re = (R)0, im = (R)0;
#pragma unroll
            for (int j = 0; j < LS; ++j) {
                const R a = TR ? mat[j * LS + k] : mat[k * LS + j];
                re = fma(a, v[j].re, re);
                im = fma(a, v[j].im, im);
            }
            w[k] = {re, im};
        }
        if constexpr (EO) {
#pragma unroll
            for (int k = 0; k < LS; ++k) v[k] = {(R)(-0.5) * w[k].re, (R)(-0.5) * w[k].im};
        } else {
            C2<R> h[LS];
            col_load<R, LS, ST>(hcol, h);
#pragma unroll
            for (int k = 0; k < LS; ++k) v[k] = {w[k].re + (R)0.5 * h[k].re, w[k].im + (R)0.5 * h[k].im};
        }
    } else if constexpr (KIND == KIND_EO_MINV) {
        col_load<R, LS, ST>(hcol, v);
        op_Minv<R, LS>(v, cf, shv);
        op_fwd<R, LS>(v, cf.b5, cf.c5, cf.m * cf.c5);
        const R f = (R)(-0.5) * hb;
#pragma unroll
        for (int k = 0; k < LS; ++k) { v[k].re *= f; v[k].im *= f; }
    } else if constexpr (KIND == KIND_EO_MINV_DAG) {
        col_load<R, LS, ST>(hcol, v);
        op_fwdT<R, LS>(v, cf.b5, cf.c5, cf.m * cf.c5);
        op_MinvT<R, LS>(v, cf, shv);
#pragma unroll
        for (int k = 0; k < LS; ++k) { v[k].re *= (R)-0.5; v[k].im *= (R)-0.5; }
    } else {
        col_load<R, LS, ST>(ycol, v);
        if constexpr (KIND == KIND_OE_SCHUR || KIND == KIND_FULL) op_M<R, LS>(v, cf, shv);
        if constexpr (KIND == KIND_OE_SCHUR_DAG || KIND == KIND_FULL_DAG) op_MT<R, LS>(v, cf, shv);
        if constexpr (KT::HOP) {
            C2<R> w[LS];
            col_load<R, LS, ST>(hcol, w);
            if constexpr (KIND == KIND_OE_SCHUR_DAG || KIND == KIND_FULL_DAG)
                op_fwdT<R, LS>(w, cf.b5, cf.c5, cf.m * cf.c5);
            const R f = ((KIND == KIND_FULL || KIND == KIND_FULL_DAG) ? (R)-0.5 : (R)0.5) * hb;
#pragma unroll
            for (int k = 0; k < LS; ++k) {
                v[k].re += f * w[k].re;
                v[k].im += f * w[k].im;
            }
        }
        if constexpr (KIND == KIND_RECON) op_Minv<R, LS>(v, cf, shv);
        if constexpr (KIND == KIND_LOC_DTMINV) {
            op_Minv<R, LS>(v, cf, shv);
            op_fwd<R, LS>(v, cf.b5, cf.c5, cf.m * cf.c5);
        }
        if constexpr (KIND == KIND_LOC_DT) op_fwd<R, LS>(v, cf.b5, cf.c5, cf.m * cf.c5);
        if constexpr (KIND == KIND_LOC_DTINV) op_inv<R, LS>(v, cf.ib, cf.zb, cf.mzb, cf.wb);
    }
    col_store<R, LS, ST>(hcol, v);
}

// v <- M v for the 5D site (xcb, s) of field y, v = y(xcb, s) on entry: the
// P+ half takes slice s-1, the P- half slice s+1 (antiperiodic through -m),
// and the shift chirality the rank-one term sbk u_k y(last) of Eq. (Mooee_shift)
// with k the mirrored index and "last" slice Ls-1 (P+) or 0 (P-).
template <typename S, typename R, int LS>
__device__ __forceinline__ void site_M(const void* __restrict__ y, const float* __restrict__ ynrm, long xcb,
                                       int s, const SCoef<R>& cf, R* v) {
    R q[12];
    {
        const int sm = (s == 0) ? LS - 1 : s - 1;
        const R gu = (s == 0) ? -cf.m * cf.gamma : cf.gamma;
        load_half<S, R>(y, ynrm, xcb, sm, LS, 0, q);
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = cf.alpha * v[i] + gu * q[i];
    }
    {
        const int sp = (s == LS - 1) ? 0 : s + 1;
        const R gd = (s == LS - 1) ? -cf.m * cf.gamma : cf.gamma;
        load_half<S, R>(y, ynrm, xcb, sp, LS, 1, q);
#pragma unroll
        for (int i = 0; i < 12; ++i) v[12 + i] = cf.alpha * v[12 + i] + gd * q[i];
    }
    if (cf.has_shift) {
        const int cs = cf.cs;
        load_half<S, R>(y, ynrm, xcb, cs == 0 ? LS - 1 : 0, LS, cs, q);
        const R f = cf.sbk * cf.um[cs == 0 ? s : LS - 1 - s];
        if (cs == 0) {
#pragma unroll
            for (int i = 0; i < 12; ++i) v[i] += f * q[i];
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) v[12 + i] += f * q[i];
        }
    }
}

// The adjoint site-local kinds (M^T y + f D~^T h) need slice s+1 (P+) and
// s-1 (P-) of both y and h, and on the shift chirality the column sum
// d = sum_k u_k y_k.  When Ls is a power of two the Ls threads of a 4D site
// are one aligned lane group of a warp, and these come from warp shuffles;
// otherwise (Ls = 12) the kind goes through the column phase.
template <int K, int LS> struct ShflTail {
    static constexpr bool ON = (K == KIND_OE_SCHUR_DAG || K == KIND_FULL_DAG) && LS <= 32 && (LS & (LS - 1)) == 0;
    static constexpr bool COLS = !KindTraits<K>::PTW && !ON;
};

// o = M^T v + f (b5 + c5 L^T) h for lane s of a group of LS lanes: L^T takes
// P+ from slice s+1 and P- from slice s-1, each with -m across the wall;
// the rank-one part of M^T adds sbk (sum_k u_k v_k) to the last mirrored
// slice of the shift chirality.  Every lane of the warp must call this.
template <typename R, int LS>
__device__ __forceinline__ void site_MT_dtT(int s, const SCoef<R>& cf, const R* v, const R* h, R f, R* o) {
    constexpr unsigned FULL = 0xffffffffu;
    const int up = (s + 1) & (LS - 1), dn = (s - 1) & (LS - 1);
    const R wu = (s == LS - 1) ? -cf.m : (R)1;
    const R wd = (s == 0) ? -cf.m : (R)1;
    const R fb = f * cf.b5, fc = f * cf.c5;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        const R yn = wu * __shfl_sync(FULL, v[i], up, LS);
        const R hn = wu * __shfl_sync(FULL, h[i], up, LS);
        o[i] = cf.alpha * v[i] + cf.gamma * yn + fb * h[i] + fc * hn;
    }
#pragma unroll
    for (int i = 12; i < 24; ++i) {
        const R yn = wd * __shfl_sync(FULL, v[i], dn, LS);
        const R hn = wd * __shfl_sync(FULL, h[i], dn, LS);
        o[i] = cf.alpha * v[i] + cf.gamma * yn + fb * h[i] + fc * hn;
    }
    if (cf.has_shift) {
        const int cs = cf.cs;
        const R u = cf.um[cs == 0 ? s : LS - 1 - s];
        const bool last = s == (cs == 0 ? LS - 1 : 0);
        R d[12];
        if (cs == 0) {
#pragma unroll
            for (int i = 0; i < 12; ++i) d[i] = u * v[i];
        } else {
#pragma unroll
            for (int i = 0; i < 12; ++i) d[i] = u * v[12 + i];
        }
#pragma unroll
        for (int off = LS / 2; off > 0; off >>= 1) {
#pragma unroll
            for (int i = 0; i < 12; ++i) d[i] += __shfl_xor_sync(FULL, d[i], off, LS);
        }
        if (last) {
            if (cs == 0) {
#pragma unroll
                for (int i = 0; i < 12; ++i) o[i] += cf.sbk * d[i];
            } else {
#pragma unroll
                for (int i = 0; i < 12; ++i) o[12 + i] += cf.sbk * d[i];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------

// one staged link: 18 reals padded to a multiple of 16 bytes
template <typename R> struct LinkStride;
template <> struct LinkStride<float> { static constexpr int V = 20; };
template <> struct LinkStride<double> { static constexpr int V = 18; };

// a staged link as 16-byte shared-memory accesses (18 reals; the float
// stride of 20 keeps every link 16-byte aligned)
template <typename R>
__device__ __forceinline__ void ld_link(const R* __restrict__ src, R* u) {
    if constexpr (sizeof(R) == 4) {
        const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 t = q[i];
            u[4 * i] = t.x; u[4 * i + 1] = t.y; u[4 * i + 2] = t.z; u[4 * i + 3] = t.w;
        }
        const float2 t = reinterpret_cast<const float2*>(src)[8];
        u[16] = t.x; u[17] = t.y;
    } else {
        const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double2 t = q[i];
            u[2 * i] = t.x; u[2 * i + 1] = t.y;
        }
    }
}
template <typename R>
__device__ __forceinline__ void st_link(R* __restrict__ dst, const R* u) {
    if constexpr (sizeof(R) == 4) {
        float4* q = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = make_float4(u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3]);
        reinterpret_cast<float2*>(dst)[8] = make_float2(u[16], u[17]);
    } else {
        double2* q = reinterpret_cast<double2*>(dst);
#pragma unroll
        for (int i = 0; i < 9; ++i) q[i] = make_double2(u[2 * i], u[2 * i + 1]);
    }
}

// CTA tile: NS 4D sites x Ls slices, one thread per 5D site.  Bit 0 of the
// variant picks the shape: 0 the default, 1 twice the sites (half for
// Ls = 12).  Bit 1 caps the registers at about 72 per thread (one more
// resident CTA of 128 threads than the compiler's own choice of 80, a few
// spilled values) and applies to FP32 arithmetic only.  The autotuner
// times the variants for the inner-solver kinds.
template <int LS, int VAR = 0> struct Tile {
    static constexpr int NS0 = (LS >= 16) ? 8 : (LS == 12 ? 16 : 128 / LS);
    static constexpr int NS = (VAR & 1) == 0 ? NS0 : (LS == 12 ? NS0 / 2 : NS0 * 2);
    static constexpr int NT = NS * LS;
};

template <typename S> constexpr int kTileVariants = sizeof(typename Traits<S>::R) == 4 ? 4 : 2;

// the register-capped variants ask for this many resident CTAs per SM
template <int LS, int VAR> struct MinBlocksCap {
    static constexpr int V = 65536 / (72 * Tile<LS, VAR>::NT);
};

// sites per CTA of a tile variant (for reports)
inline int tile_sites(int Ls, int var) {
    const bool alt = var & 1;
    switch (Ls) {
        case 4: return alt ? Tile<4, 1>::NS : Tile<4, 0>::NS;
        case 8: return alt ? Tile<8, 1>::NS : Tile<8, 0>::NS;
        case 12: return alt ? Tile<12, 1>::NS : Tile<12, 0>::NS;
        case 16: return alt ? Tile<16, 1>::NS : Tile<16, 0>::NS;
        default: return 0;
    }
}

// raw link records (rows 0 and 1 in storage precision) are staged with
// cp.async, 16-byte pieces (8-byte for 16-bit storage)
template <typename S> struct LinkRaw {
    static constexpr int BYTES = 12 * (int)sizeof(S);
    // storage = compute precision: the record lands in rows 0-1 of its
    // staged link and row 2 is rebuilt in place; 16-bit storage needs a
    // separate raw buffer
    static constexpr bool SEP = sizeof(S) != sizeof(typename Traits<S>::R);
    static constexpr int PAD = SEP ? (BYTES + 15) / 16 * 16 : 0;
};

__device__ __forceinline__ void stage_cp16(void* dst, const void* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void stage_cp8(void* dst, const void* src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void stage_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// one staged raw link record -> 12 reals of compute precision
template <typename S, typename R>
__device__ __forceinline__ void link_from_raw(const unsigned char* raw, R* u) {
    if constexpr (sizeof(S) == 8) {
        const double2* p = reinterpret_cast<const double2*>(raw);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double2 t = p[c];
            u[2 * c] = t.x;
            u[2 * c + 1] = t.y;
        }
    } else if constexpr (sizeof(S) == 4) {
        const float4* p = reinterpret_cast<const float4*>(raw);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 t = p[c];
            u[4 * c] = t.x;
            u[4 * c + 1] = t.y;
            u[4 * c + 2] = t.z;
            u[4 * c + 3] = t.w;
        }
    } else {
        const uint2* p = reinterpret_cast<const uint2*>(raw);
#pragma unroll
        for (int c = 0; c < 3; ++c) unpack4(p[c], (const S*)nullptr, u + 4 * c);
    }
}

// Persistent CTAs: a CTA walks the site blocks blockIdx.x, +gridDim.x, ...
// While it works on one block, the links and neighbour indices of its next
// block are already on their way (cp.async into a second staging buffer),
// so the link latency is off the critical path, and the norm reduction runs
// once per CTA instead of once per block.
template <typename S, int LS, int KIND, int VAR>
__device__ __forceinline__ void hop_body(const HopArgs& a, const SCoef<typename Traits<S>::R>& cf) {
    typedef typename Traits<S>::R R;
    typedef KindTraits<KIND> KT;
    constexpr int NS = Tile<LS, VAR>::NS;
    constexpr int NT = Tile<LS, VAR>::NT;
    constexpr int ST = ShStride<R>::V;
    constexpr int SS = SiteStride<R, LS>::V;
    constexpr int LK = LinkStride<R>::V;
    constexpr int NL = NS * 8;  // staged links (and neighbour indices) per block
    constexpr int RAWB = LinkRaw<S>::PAD;

    if (a.done && *a.done) return;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool SHF = ShflTail<KIND, LS>::ON;
    constexpr bool COLS = ShflTail<KIND, LS>::COLS;  // column phase and its tile buffers
    R* sh = reinterpret_cast<R*>(smem_raw);          // [NS][SS] hop result
    R* sy = sh + (COLS ? NS * SS : 0);                // [NS][SS] local input
    R* smat = sy + ((KT::HASY && COLS) ? NS * SS : 0);  // [2][LS][LS] dense kinds' s-matrices
    R* sl = smat + (KT::DENSE ? 2 * LS * LS : 0);       // [2][NL][LK] links, row 2 rebuilt
    unsigned char* sraw = reinterpret_cast<unsigned char*>(sl + (KT::HOP ? 2 * NL * LK : 0));  // [2][NL][RAWB]
    unsigned* snb = reinterpret_cast<unsigned*>(sraw + (KT::HOP ? 2 * NL * RAWB : 0));        // [2][NL]

    const Geom& g = a.g;
    const int tid = threadIdx.x;
    const int il = tid / LS;
    const int s = tid - il * LS;
    const int rp = il * SS + s * ST;                  // row of the P+ half
    const int rm = il * SS + (LS - 1 - s) * ST + 12;  // row of the P- half
    const long nblk = ((long)g.Vh + NS - 1) / NS;

    // ---------------- phase 0: links and neighbours, once per 4D site ---
    // The 8 links of each site (4 forward from this parity, 4 backward from
    // the neighbours) and the 8 neighbour indices (bit 31: the hop carries a
    // factor -1, from an antiperiodic or a G-parity boundary) for all Ls
    // slices of the site.  Issue: indices and
    // cp.async of the raw records; finish: the third row rebuilt.
    auto stage_issue = [&](long blk, int b) {
        for (int j = tid; j < NL; j += NT) {
            const int jl = j >> 3, d = j & 7, mu = d & 3;
            const long jcb = blk * NS + jl;
            if (jcb < g.Vh) {
                int rem = (int)jcb;
                const int xh = rem % g.Xh; rem /= g.Xh;
                const int y = rem % g.Y; rem /= g.Y;
                const int z = rem % g.Z;
                const int tf = rem / g.Z;  // t + f Tp for flavour f (G-parity), else t
                const int x = 2 * xh + ((a.out_par + y + z + tf) & 1);
                const int f = tf >= g.Tp ? 1 : 0;
                // step in direction mu (forward for d < 4), periodic wrap
                const int c = mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : tf - f * g.Tp;
                const int e = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.Tp;
                const bool cross = (d < 4) ? (c + 1 == e) : (c == 0);
                const int n = (d < 4) ? (cross ? 0 : c + 1) : (cross ? e - 1 : c - 1);
                long ncb = ((((long)(mu == 3 ? n + f * g.Tp : tf) * g.Z + (mu == 2 ? n : z)) * g.Y +
                             (mu == 1 ? n : y)) * g.X + (mu == 0 ? n : x)) >> 1;
                bool neg = cross && ((g.apmask >> mu) & 1);
                if (cross && ((g.gpmask >> mu) & 1)) {
                    // G-parity boundary: psi_1(x + L) = psi_2(x), psi_2(x + L) = -psi_1(x);
                    // the other flavour is half the stacked lattice away
                    ncb += f ? -(long)(g.Vh / 2) : (long)(g.Vh / 2);
                    neg = neg != ((d < 4) ? f == 1 : f == 0);
                }
                const unsigned edge = neg ? 0x80000000u : 0u;
                snb[b * NL + j] = (unsigned)ncb | edge;
                const long site = (d < 4) ? jcb : ncb;
                const unsigned char* src = reinterpret_cast<const unsigned char*>(d < 4 ? a.lk_out : a.lk_in) +
                                           (site * 4 + mu) * LinkRaw<S>::BYTES;
                unsigned char* dst = LinkRaw<S>::SEP ? sraw + (b * NL + j) * RAWB
                                                     : reinterpret_cast<unsigned char*>(sl + (b * NL + j) * LK);
                if constexpr (sizeof(S) >= 4) {
#pragma unroll
                    for (int c = 0; c < LinkRaw<S>::BYTES / 16; ++c) stage_cp16(dst + 16 * c, src + 16 * c);
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) stage_cp8(dst + 8 * c, src + 8 * c);
                }
            }
        }
        stage_commit();
    };
    auto stage_finish = [&](long blk, int b) {
        stage_wait();  // this thread's own copies
        for (int j = tid; j < NL; j += NT) {
            if (blk * NS + (j >> 3) < g.Vh) {
                R u[18];
                R* dl = sl + (b * NL + j) * LK;
                if constexpr (LinkRaw<S>::SEP) link_from_raw<S, R>(sraw + (b * NL + j) * RAWB, u);
                else link_from_raw<S, R>(reinterpret_cast<const unsigned char*>(dl), u);
                rebuild_row2(u);
                // the factor -1 of an antiperiodic or G-parity boundary hop
                // rides on the staged link; the branch is uniform over the grid
                if ((g.gpmask | g.apmask) && (snb[b * NL + j] >> 31)) {
#pragma unroll
                    for (int i = 0; i < 18; ++i) u[i] = -u[i];
                }
                st_link(dl, u);
            }
        }
    };

    long blk = blockIdx.x;
    if constexpr (KT::DENSE) {  // published by the barrier after the first links
        const R* gm = reinterpret_cast<const R*>(a.dense);
        for (int i = tid; i < 2 * LS * LS; i += NT) smat[i] = gm[i];
    }
    if constexpr (KT::HOP) {
        if (blk < nblk) {
            stage_issue(blk, 0);
            stage_finish(blk, 0);
        }
        __syncthreads();
    }

    R nn = (R)0;
    for (int it = 0; blk < nblk; ++it, blk += gridDim.x) {
        const int cur = it & 1;
        const long nxt = blk + gridDim.x;
        if constexpr (KT::HOP) {
            if (nxt < nblk) stage_issue(nxt, cur ^ 1);
        }
        const R* slc = sl + cur * NL * LK;
        const unsigned* snc = snb + cur * NL;
        const long xcb = blk * NS + il;
        const bool valid = xcb < g.Vh;

        // ---------------- phase 1: hop and staging ----------------------
        R o[24];    // the output spinor of this thread's 5D site
        R acc[24];  // its hop result (zero for padding sites)
#pragma unroll
        for (int i = 0; i < 24; ++i) acc[i] = (R)0;
        if (valid) {
            if constexpr (KT::HOP) {
                constexpr int FS = KT::DAG ? +1 : -1;  // forward projector 1 + FS gamma
                // hop k = 2 mu + dir (dir 0 forward, 1 backward)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int mu = k >> 1, dir = k & 1;
                    const long ncb = (long)(snc[il * 8 + dir * 4 + mu] & 0x7fffffffu);
                    R p[24];
                    load_sp<S, R>(a.in, a.in_nrm, ncb, s, LS, p);
                    if constexpr (KT::PRE) {
                        // chi = psi + (c5/b5) L psi (the b5 factor is applied in phase 2)
                        R q[12];
                        const int sm = (s == 0) ? LS - 1 : s - 1;
                        const R fu = (s == 0) ? -cf.mzb : cf.zb;
                        load_half<S, R>(a.in, a.in_nrm, ncb, sm, LS, 0, q);
#pragma unroll
                        for (int i = 0; i < 12; ++i) p[i] += fu * q[i];
                        const int sp = (s == LS - 1) ? 0 : s + 1;
                        const R fd = (s == LS - 1) ? -cf.mzb : cf.zb;
                        load_half<S, R>(a.in, a.in_nrm, ncb, sp, LS, 1, q);
#pragma unroll
                        for (int i = 0; i < 12; ++i) p[12 + i] += fd * q[i];
                    }
                    R u[18];
                    ld_link(slc + (il * 8 + dir * 4 + mu) * LK, u);
                    // every boundary sign rides on the staged link
                    if (dir == 0) {
                        if (mu == 0) hop_dir<R, 0, FS, false>(acc, p, u);
                        if (mu == 1) hop_dir<R, 1, FS, false>(acc, p, u);
                        if (mu == 2) hop_dir<R, 2, FS, false>(acc, p, u);
                        if (mu == 3) hop_dir<R, 3, FS, false>(acc, p, u);
                    } else {
                        if (mu == 0) hop_dir<R, 0, -FS, true>(acc, p, u);
                        if (mu == 1) hop_dir<R, 1, -FS, true>(acc, p, u);
                        if (mu == 2) hop_dir<R, 2, -FS, true>(acc, p, u);
                        if (mu == 3) hop_dir<R, 3, -FS, true>(acc, p, u);
                    }
                }
                if constexpr (KT::PTW) {
                    // out = [M] y + f h, finished in registers
                    const R f = ((KIND == KIND_FULL) ? (R)-0.5 : (R)0.5) * (KT::PRE ? cf.b5 : (R)1);
                    R v[24];
                    load_sp<S, R>(a.y, a.y_nrm, xcb, s, LS, v);
                    if constexpr (KIND != KIND_SRC) site_M<S, R, LS>(a.y, a.y_nrm, xcb, s, cf, v);
#pragma unroll
                    for (int i = 0; i < 24; ++i) o[i] = v[i] + f * acc[i];
                } else if constexpr (COLS) {
                    st_half(sh + rp, acc);
                    st_half(sh + rm, acc + 12);
                }
            }
            if constexpr (KT::HASY && COLS) {
                R v[24];
                load_sp<S, R>(a.y, a.y_nrm, xcb, s, LS, v);
                st_half(sy + rp, v);
                st_half(sy + rm, v + 12);
            }
        }
        if constexpr (SHF) {
            // out = M^T y + f D~^T h with the slice neighbours from the site's lanes
            R v[24];
            if (valid) {
                load_sp<S, R>(a.y, a.y_nrm, xcb, s, LS, v);
            } else {
#pragma unroll
                for (int i = 0; i < 24; ++i) v[i] = (R)0;
            }
            const R f = (KIND == KIND_FULL_DAG) ? (R)-0.5 : (R)0.5;
            site_MT_dtT<R, LS>(s, cf, v, acc, f, o);
        }

        // ---------------- phase 2: fifth-dimension program --------------
        if constexpr (COLS) {
            __syncthreads();
            const R hb = KT::PRE ? cf.b5 : (R)1;  // the b5 of the on-the-fly D~
            for (int col = tid; col < NS * 12; col += NT) {
                const int ci = col / 12;
                const int cc = col - ci * 12;     // spin * 3 + colour
                const bool shv = cf.has_shift && ((cc >= 6 ? 1 : 0) == cf.cs);
                column_program<R, LS, KIND, ST>(sh + ci * SS + 2 * cc, sy + ci * SS + 2 * cc, cf, shv, hb,
                                                smat + (cc >= 6 ? LS * LS : 0));
            }
            __syncthreads();
        }

        // ---------------- phase 3: store ----------------------------------
        if (valid) {
            if constexpr (COLS) {
                ld_half(sh + rp, o);
                ld_half(sh + rm, o + 12);
            }
            store_sp<S, R>(a.out, a.out_nrm, xcb, s, LS, o);
            if (a.rd.fin != FIN_NONE) {
#pragma unroll
                for (int i = 0; i < 24; ++i) nn += o[i] * o[i];
            }
        }

        if constexpr (KT::HOP) {
            if (nxt < nblk) stage_finish(nxt, cur ^ 1);
        }
        __syncthreads();  // next block's links in place; this block's tiles free
    }
    if (a.rd.fin != FIN_NONE) block_reduce_finalize<NT>(nn, a.rd);
}

// the kernel with the compiler's own register choice (variants 0, 1) ...
template <typename S, int LS, int KIND, int VAR = 0>
__global__ void __launch_bounds__(Tile<LS, VAR>::NT) hop_kernel(const HopArgs a, const SCoef<typename Traits<S>::R> cf) {
    hop_body<S, LS, KIND, VAR>(a, cf);
}

// ... and with capped registers (variants 2, 3; FP32 arithmetic)
template <typename S, int LS, int KIND, int VAR>
__global__ void __launch_bounds__(Tile<LS, VAR>::NT, MinBlocksCap<LS, VAR>::V)
    hop_kernel_rc(const HopArgs a, const SCoef<typename Traits<S>::R> cf) {
    hop_body<S, LS, KIND, VAR>(a, cf);
}

template <typename S, int LS, int K, int VAR = 0>
constexpr size_t hop_smem_bytes() {
    typedef typename Traits<S>::R R;
    constexpr size_t bufs = ShflTail<K, LS>::COLS ? (1 + (KindTraits<K>::HASY ? 1 : 0)) : 0;
    constexpr size_t NL = (size_t)Tile<LS, VAR>::NS * 8;
    return bufs * (size_t)Tile<LS, VAR>::NS * SiteStride<R, LS>::V * sizeof(R) +
           (KindTraits<K>::DENSE ? 2 * (size_t)LS * LS * sizeof(R) : 0) +
           (KindTraits<K>::HOP ? 2 * NL * (LinkStride<R>::V * sizeof(R) + LinkRaw<S>::PAD + sizeof(unsigned)) : 0);
}

}  // namespace eofa
