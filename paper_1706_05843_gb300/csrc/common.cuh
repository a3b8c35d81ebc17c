// common.cuh -- internal types of the GB300 EOFA library: lattice geometry,
// fifth-dimension coefficients, storage traits for FP64/FP32/FP16/BF16
// spinors and two-row links, and the deterministic block/grid reduction used
// by every kernel that produces a norm.
//
// Internal (device) layouts, per checkerboard parity p (sites with
// (x+y+z+t) % 2 == p, numbered xcb = lexicographic index / 2):
//   spinor  chunk[(xcb * NC + c) * Ls + s]   16-byte chunks, NC = 12 (FP64),
//           6 (FP32), 3 (FP16/BF16); the 24 reals of a spinor are ordered
//           [spin][colour][re, im], so the upper (P+) half is reals 0..11.
//           FP16 adds one float scale per 5D site: norm[xcb * Ls + s].
//   links   [xcb][mu][row 0..1][col][re, im]: 12 reals per link, the third
//           row rebuilt as conj(row0 x row1).
// Consecutive threads of a warp take consecutive s of one 4D site, so every
// chunk load of a warp reads contiguous 16-byte runs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eofa {

constexpr int LSMAX = 32;

struct Geom {
    int X, Y, Z, T;
    int Xh;      // X / 2
    int Vh;      // 4D sites per parity
    int Ls;
    int apmask;  // bit mu set: hops across the mu boundary carry a factor -1
    // G-parity (Sec. I): bit mu set for a G-parity direction.  The two
    // flavours are stacked along t (T = 2 Tp, flavour f at t + f Tp); a hop
    // across a G-parity boundary changes flavour, psi_1(x + L) = psi_2(x),
    // psi_2(x + L) = -psi_1(x); flavour 2 carries the conjugate links.
    int gpmask;
    int Tp;      // physical time extent (T without G-parity)
};

// Fifth-dimension coefficients of one context, in compute precision R.
// All s-space operators are written in "mirrored" coordinates: a column of
// chirality minus is read with s -> Ls-1-s, which maps L- onto L+, so the
// same code serves both chiralities.  um/xm/ym are the Sherman-Morrison
// vectors of the shift chirality in that chirality's coordinates.
template <typename R>
struct SCoef {
    R alpha, gamma;   // site-diagonal block A = alpha + gamma L
    R b5, c5, m;      // D~ = b5 + c5 L, L with mass m (= m1)
    R ia, za, mza;    // 1/alpha, gamma/alpha, m * gamma/alpha
    R ib, zb, mzb;    // 1/b5, c5/b5, m * c5/b5
    R sbk;            // pm * beta * k
    R sbk_den;        // pm * beta * k / (1 + pm beta k x_{j*})
    R sb_den;         // pm * beta / (1 + pm beta k x_{j*})
    int cs;           // chirality index of the shift: 0 (+) or 1 (-)
    int has_shift;    // beta != 0
    R wa[LSMAX];      // (-za)^j / (alpha (1 + m za^Ls)), cyclic inverse of A
    R wb[LSMAX];      // (-zb)^j / (b5 (1 + m zb^Ls)), cyclic inverse of D~
    R um[LSMAX];      // u of the shift (App. B)
    R xm[LSMAX];      // x = A^-1 u
    R ym[LSMAX];      // y = A^-T (k e_{j*})
};

// ---------------------------------------------------------------------------
// device scalars of the Krylov solvers
// ---------------------------------------------------------------------------
struct DevScal {
    double qq, zz, rr, alpha, beta;
    double target_rr;
    double store[6];
    int iters;
    int done;
    int nonfinite;
    int max_iters;                 // device-driven loops stop here
    unsigned long long t0_ns;      // %globaltimer at the start of the solve
    unsigned long long timeout_ns; // 0: none
    int timed_out;
    int stop;                      // the CG update of x and p has run after done was set
    // device-driven defect correction of a batched solve (one graph launch):
    // every flag below is read by the kernels of one phase, which return at
    // once while it is nonzero
    int o_fin;           // the outer loop of this system has ended (status in o_status)
    int o_status;        // eofa_status of the ended outer loop
    int o_skip_copy;     // first residual is the source itself (no initial guess) unless set
    int o_skip_res;      // first residual is b~o - S x_o (initial guess) unless set
    int o_skip_step;     // no outer step (accumulate, FP64 residual, decide) in this chunk
    int o_skip_restart;  // no inner restart in this chunk
    int outer, total;    // outer steps taken, inner iterations summed over them
    int maxouter, maxit;
    int o_body;          // chunks run (system 0 of a batch counts for the batch)
    int o_body_cap;      // safety bound on the chunks (never reached by a sound solve)
    double tol, floor_tol, rel;
    unsigned long long o_t0_ns, o_timeout_ns;
};

// the device scalars of up to 32 systems (one batched graph)
struct ScalList {
    DevScal* s[32];
    int n;
};

enum Fin { FIN_NONE = 0, FIN_STORE = 1, FIN_ALPHA = 2, FIN_BETA = 3, FIN_RR = 4, FIN_ZZ = 5, FIN_STOP = 6 };

struct Reduce {
    double* partials;   // one per block
    unsigned* counter;  // ticket, zero between launches
    DevScal* scal;
    int fin;
    int slot;
};

// ---------------------------------------------------------------------------
// storage traits
// ---------------------------------------------------------------------------
template <typename S> struct Traits;
template <> struct Traits<double> {
    typedef double R;
    static constexpr int NC = 12;
    static constexpr bool NORM = false;
    static constexpr int BYTES = 8;
};
template <> struct Traits<float> {
    typedef float R;
    static constexpr int NC = 6;
    static constexpr bool NORM = false;
    static constexpr int BYTES = 4;
};
template <> struct Traits<__half> {
    typedef float R;
    static constexpr int NC = 3;
    static constexpr bool NORM = true;
    static constexpr int BYTES = 2;
};
template <> struct Traits<__nv_bfloat16> {
    typedef float R;
    static constexpr int NC = 3;
    static constexpr bool NORM = false;
    static constexpr int BYTES = 2;
};

// 8 sixteen-bit values <-> 8 floats
__device__ __forceinline__ void unpack8(const uint4 q, const __half*, float* v) {
    const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __half22float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void unpack8(const uint4 q, const __nv_bfloat16*, float* v) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void unpack4(const uint2 q, const __half*, float* v) {
    const __half2* h = reinterpret_cast<const __half2*>(&q);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float2 f = __half22float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void unpack4(const uint2 q, const __nv_bfloat16*, float* v) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float2 f = __bfloat1622float2(h[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float* v, const __half*) {
    uint4 q;
    __half2* h = reinterpret_cast<__half2*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    return q;
}
__device__ __forceinline__ uint4 pack8(const float* v, const __nv_bfloat16*) {
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    return q;
}
__device__ __forceinline__ uint2 pack4(const float* v, const __half*) {
    uint2 q;
    __half2* h = reinterpret_cast<__half2*>(&q);
    h[0] = __floats2half2_rn(v[0], v[1]);
    h[1] = __floats2half2_rn(v[2], v[3]);
    return q;
}
__device__ __forceinline__ uint2 pack4(const float* v, const __nv_bfloat16*) {
    uint2 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
    h[0] = __floats2bfloat162_rn(v[0], v[1]);
    h[1] = __floats2bfloat162_rn(v[2], v[3]);
    return q;
}

// ---------------------------------------------------------------------------
// spinor access.  base points at the parity's chunk array; the 24 reals of a
// spinor are in the logical order [spin][colour][re, im] in every precision.
// ---------------------------------------------------------------------------
template <typename S, typename R>
__device__ __forceinline__ void load_raw(const void* __restrict__ base, const float* __restrict__ nrm,
                                         long xcb, int s, int Ls, R* v) {
    if constexpr (sizeof(S) == 8) {
        const double2* p = reinterpret_cast<const double2*>(base) + xcb * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 t = p[c * Ls];
            v[2 * c] = t.x;
            v[2 * c + 1] = t.y;
        }
    } else if constexpr (sizeof(S) == 4) {
        const float4* p = reinterpret_cast<const float4*>(base) + xcb * 6 * Ls + s;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float4 t = p[c * Ls];
            v[4 * c] = t.x;
            v[4 * c + 1] = t.y;
            v[4 * c + 2] = t.z;
            v[4 * c + 3] = t.w;
        }
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(base) + xcb * 3 * Ls + s;
#pragma unroll
        for (int c = 0; c < 3; ++c) unpack8(p[c * Ls], (const S*)nullptr, v + 8 * c);
        if constexpr (Traits<S>::NORM) {
            float n = nrm[xcb * Ls + s];
#pragma unroll
            for (int i = 0; i < 24; ++i) v[i] *= n;
        }
    }
}

// load the upper (hi = 0, reals 0..11) or lower (hi = 1, reals 12..23) half
template <typename S, typename R>
__device__ __forceinline__ void load_half(const void* __restrict__ base, const float* __restrict__ nrm,
                                          long xcb, int s, int Ls, int hi, R* v) {
    if constexpr (sizeof(S) == 8) {
        const double2* p = reinterpret_cast<const double2*>(base) + (xcb * 12 + 6 * hi) * Ls + s;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double2 t = p[c * Ls];
            v[2 * c] = t.x;
            v[2 * c + 1] = t.y;
        }
    } else if constexpr (sizeof(S) == 4) {
        const float4* p = reinterpret_cast<const float4*>(base) + (xcb * 6 + 3 * hi) * Ls + s;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 t = p[c * Ls];
            v[4 * c] = t.x;
            v[4 * c + 1] = t.y;
            v[4 * c + 2] = t.z;
            v[4 * c + 3] = t.w;
        }
    } else {
        // reals 0..7 | 8..15 | 16..23 in chunks 0, 1, 2; chunk 1 is split.
        const uint4* p = reinterpret_cast<const uint4*>(base) + xcb * 3 * Ls + s;
        const uint2* mid = reinterpret_cast<const uint2*>(p + Ls);  // chunk 1 as two halves
        if (hi == 0) {
            unpack8(p[0], (const S*)nullptr, v);
            unpack4(mid[0], (const S*)nullptr, v + 8);
        } else {
            unpack4(mid[1], (const S*)nullptr, v);
            unpack8(p[2 * Ls], (const S*)nullptr, v + 4);
        }
        if constexpr (Traits<S>::NORM) {
            float n = nrm[xcb * Ls + s];
#pragma unroll
            for (int i = 0; i < 12; ++i) v[i] *= n;
        }
    }
}

template <typename S, typename R>
__device__ __forceinline__ void store_raw(void* __restrict__ base, float* __restrict__ nrm, long xcb,
                                          int s, int Ls, const R* v) {
    if constexpr (sizeof(S) == 8) {
        double2* p = reinterpret_cast<double2*>(base) + xcb * 12 * Ls + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) p[c * Ls] = make_double2(v[2 * c], v[2 * c + 1]);
    } else if constexpr (sizeof(S) == 4) {
        float4* p = reinterpret_cast<float4*>(base) + xcb * 6 * Ls + s;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            p[c * Ls] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
        uint4* p = reinterpret_cast<uint4*>(base) + xcb * 3 * Ls + s;
        float w[24];
        if constexpr (Traits<S>::NORM) {
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < 24; ++i) mx = fmaxf(mx, fabsf((float)v[i]));
            float inv = mx > 0.f ? 1.0f / mx : 0.f;
#pragma unroll
            for (int i = 0; i < 24; ++i) w[i] = (float)v[i] * inv;
            nrm[xcb * Ls + s] = mx;
        } else {
#pragma unroll
            for (int i = 0; i < 24; ++i) w[i] = (float)v[i];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c * Ls] = pack8(w + 8 * c, (const S*)nullptr);
    }
}

template <typename S, typename R>
__device__ __forceinline__ void load_sp(const void* __restrict__ base, const float* __restrict__ nrm,
                                        long xcb, int s, int Ls, R* v) {
    load_raw<S, R>(base, nrm, xcb, s, Ls, v);
}

template <typename S, typename R>
__device__ __forceinline__ void store_sp(void* __restrict__ base, float* __restrict__ nrm, long xcb,
                                         int s, int Ls, const R* v) {
    store_raw<S, R>(base, nrm, xcb, s, Ls, v);
}

// ---------------------------------------------------------------------------
// links: 12 reals per link (rows 0 and 1)
// ---------------------------------------------------------------------------
template <typename S, typename R>
__device__ __forceinline__ void load_link(const void* __restrict__ base, long xcb, int mu, R* u) {
    const long l = xcb * 4 + mu;
    if constexpr (sizeof(S) == 8) {
        const double2* p = reinterpret_cast<const double2*>(base) + l * 6;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double2 t = p[c];
            u[2 * c] = t.x;
            u[2 * c + 1] = t.y;
        }
    } else if constexpr (sizeof(S) == 4) {
        const float4* p = reinterpret_cast<const float4*>(base) + l * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 t = p[c];
            u[4 * c] = t.x;
            u[4 * c + 1] = t.y;
            u[4 * c + 2] = t.z;
            u[4 * c + 3] = t.w;
        }
    } else {
        const uint2* p = reinterpret_cast<const uint2*>(base) + l * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) unpack4(p[c], (const S*)nullptr, u + 4 * c);
    }
}

// ---------------------------------------------------------------------------
// deterministic block + grid reduction with a last-block finalisation.
// Every thread of the block must call it (it synchronises).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize(const Reduce& rd, double total) {
    DevScal* sc = rd.scal;
    if (!isfinite(total)) sc->nonfinite = 1;
    switch (rd.fin) {
        case FIN_STORE: sc->store[rd.slot] = total; break;
        case FIN_ALPHA:
            sc->qq = total;
            sc->alpha = (total > 0.0) ? sc->zz / total : 0.0;
            break;
        case FIN_BETA:
            sc->beta = (sc->zz > 0.0) ? total / sc->zz : 0.0;
            sc->zz = total;
            break;
        case FIN_ZZ: sc->zz = total; break;
        case FIN_STOP: sc->stop = sc->done; break;
        case FIN_RR:
            sc->rr = total;
            sc->iters += 1;
            if (!(total > sc->target_rr) || !isfinite(total)) sc->done = 1;
            break;
        default: break;
    }
}

// The per-thread value and the warp-level sum are kept in the kernel's
// compute precision R (FP32 kernels must not touch GB300's slow FP64 pipe
// per element); warp sums are combined in FP64.
template <int NT, typename R>
__device__ __forceinline__ void block_reduce_finalize(R v, const Reduce& rd) {
    __shared__ double red_ws[NT / 32];
    __shared__ int red_last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red_ws[w] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += red_ws[i];
        rd.partials[blockIdx.x] = s;
        __threadfence();
        unsigned t = atomicAdd(rd.counter, 1u);
        red_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (red_last) {
        __threadfence();
        double s = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += NT) s += __ldcg(rd.partials + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) red_ws[w] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
#pragma unroll
            for (int i = 0; i < NT / 32; ++i) tot += red_ws[i];
            finalize(rd, tot);
            *rd.counter = 0u;
        }
    }
}

}  // namespace eofa
