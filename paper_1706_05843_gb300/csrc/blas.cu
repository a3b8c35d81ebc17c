// blas.cu -- Krylov vector updates with fused deterministic reductions,
// precision conversions, and the layout import/export kernels between the
// caller's canonical complex128 fields and the internal even-odd blocked
// layout.  One thread per 5D site (xcb, s) of a half lattice.
#include <algorithm>

#include "blas.h"
#include "eofa.h"
#include "learned.h"

namespace eofa {

constexpr int BT = 256;  // threads per block of every kernel in this file

static inline int grid_for(long n) { return (int)((n + BT - 1) / BT); }

// grid of the grid-stride CG kernels: at most 4 blocks of BT threads per SM
// (fewer partial sums for the last block to finalise)
static int grid_capped(long n) {
    static const int cap = [] {  // initialised once, thread-safe
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            return 4 * sms;
        return 1 << 30;
    }();
    return std::max(1, std::min(grid_for(n), cap));
}

// ---------------------------------------------------------------------------
// scalars
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_scal_init(DevScal* sc, double target_rr, int max_iters, unsigned long long timeout_ns) {
    sc->qq = sc->zz = sc->rr = sc->alpha = sc->beta = 0.0;
    sc->target_rr = target_rr;
    sc->iters = 0;
    sc->done = 0;
    sc->stop = 0;
    sc->nonfinite = 0;
    sc->max_iters = max_iters;
    sc->timeout_ns = timeout_ns;
    sc->timed_out = 0;
    sc->t0_ns = globaltimer_ns();
}

cudaError_t scal_init(DevScal* sc, double target_rr, int max_iters, unsigned long long timeout_ns,
                      cudaStream_t st) {
    k_scal_init<<<1, 1, 0, st>>>(sc, target_rr, max_iters, timeout_ns);
    return cudaGetLastError();
}

// Condition of the device-driven CG loop (a WHILE node of a CUDA graph):
// run the body again unless converged, non-finite, at the iteration cap or
// past the deadline.  Every exit is bounded by max_iters.
__global__ void k_while_cond(cudaGraphConditionalHandle h, DevScal* sc) {
    int go = !sc->done && !sc->nonfinite && sc->iters < sc->max_iters;
    if (go && sc->timeout_ns && globaltimer_ns() - sc->t0_ns > sc->timeout_ns) {
        sc->timed_out = 1;
        go = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

cudaError_t while_cond(cudaGraphConditionalHandle h, DevScal* sc, cudaStream_t st) {
    k_while_cond<<<1, 1, 0, st>>>(h, sc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// device-driven defect correction of a batched solve: each system runs the
// outer FP64 loop on its own scalars.  In every chunk of the batch graph the
// running systems take kChunk CG iterations; the gate then turns a system
// whose inner solve has ended to its outer step (accumulate the correction,
// FP64 residual, decide), which ends its outer loop or restarts the inner
// CGNR at once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool past_deadline(const DevScal* sc) {
    return sc->o_timeout_ns && globaltimer_ns() - sc->o_t0_ns > sc->o_timeout_ns;
}

__device__ __forceinline__ void outer_end(DevScal* sc, int status) {
    sc->o_fin = 1;
    sc->o_status = status;
    sc->o_skip_restart = 1;
    sc->done = 1;
    sc->stop = 1;
}

__global__ void k_outer_begin(DevScal* sc, double tol, double floor_tol, int maxit, int maxouter,
                              unsigned long long timeout_ns, int fin, int x_zero, int body_cap) {
    sc->tol = tol;
    sc->floor_tol = floor_tol;
    sc->maxit = maxit;
    sc->maxouter = maxouter;
    sc->o_t0_ns = globaltimer_ns();
    sc->o_timeout_ns = timeout_ns;
    sc->o_body = 0;
    sc->o_body_cap = body_cap;
    sc->outer = sc->total = 0;
    sc->rel = fin ? 0.0 : 1.0;
    sc->o_fin = fin;
    sc->o_status = EOFA_OK;
    sc->o_skip_copy = fin || !x_zero;
    sc->o_skip_res = fin || x_zero;
    sc->o_skip_step = 1;
    sc->o_skip_restart = 1;
    sc->done = sc->stop = 1;
    sc->iters = 0;
    sc->nonfinite = 0;
    sc->timed_out = 0;
    sc->timeout_ns = 0;
}

cudaError_t outer_begin(DevScal* sc, double tol, double floor_tol, int maxit, int maxouter,
                        unsigned long long timeout_ns, int fin, int x_zero, int body_cap, cudaStream_t st) {
    k_outer_begin<<<1, 1, 0, st>>>(sc, tol, floor_tol, maxit, maxouter, timeout_ns, fin, x_zero, body_cap);
    return cudaGetLastError();
}

// After a chunk: a running system whose inner solve has ended (done,
// non-finite, out of iterations, or past the deadline) takes its outer step
// in this chunk; its CG kernels return at once from here on.
__global__ void k_outer_gate(DevScal* sc) {
    sc->o_skip_step = 1;
    if (sc->o_fin) return;
    const bool timed = past_deadline(sc);
    if (!(sc->done || sc->nonfinite || sc->iters >= sc->max_iters || timed)) return;
    sc->total += sc->iters;
    sc->outer += 1;
    sc->done = sc->stop = 1;
    if (sc->nonfinite) {
        outer_end(sc, EOFA_ERR_NONFINITE);
        return;
    }
    sc->o_skip_step = 0;
}

cudaError_t outer_gate(DevScal* sc, cudaStream_t st) {
    k_outer_gate<<<1, 1, 0, st>>>(sc);
    return cudaGetLastError();
}

// After an FP64 residual |r|^2 = store[0] (|b|^2 = store[1] + store[2]):
// end the outer loop (non-finite, converged, iteration caps, deadline, in
// that order) or restart the inner CGNR on r / |r| with the target
// max(floor, tol |b| / |r|) and the iterations left.  first: the residual of
// the loop's start (taken whether or not a step ran).
__global__ void k_outer_decide(DevScal* sc, int first) {
    if (sc->o_fin || (!first && sc->o_skip_step)) {
        sc->o_skip_restart = 1;
        return;
    }
    const double rr = sc->store[0], bb = sc->store[1] + sc->store[2];
    if (!isfinite(rr)) {
        outer_end(sc, EOFA_ERR_NONFINITE);
        return;
    }
    const double rel = sqrt(rr / bb);
    sc->rel = rel;
    if (!(rel > sc->tol)) {
        outer_end(sc, EOFA_OK);
        return;
    }
    if (sc->outer >= sc->maxouter || sc->total >= sc->maxit) {
        outer_end(sc, EOFA_ERR_NOT_CONVERGED);
        return;
    }
    if (past_deadline(sc)) {
        outer_end(sc, EOFA_ERR_TIMEOUT);
        return;
    }
    const double t = fmax(sc->tol / rel, sc->floor_tol);
    sc->target_rr = t * t;
    sc->qq = sc->zz = sc->rr = sc->alpha = sc->beta = 0.0;
    sc->iters = 0;
    sc->nonfinite = 0;
    sc->max_iters = sc->maxit - sc->total;
    sc->done = sc->stop = 0;
    sc->o_skip_restart = 0;
}

cudaError_t outer_decide_dev(DevScal* sc, int first, cudaStream_t st) {
    k_outer_decide<<<1, 1, 0, st>>>(sc, first);
    return cudaGetLastError();
}

// Condition of the batch graph's WHILE node: another chunk while any
// system's outer loop runs.  The chunk count of system 0 is bounded; a batch
// that reaches the bound ends its running systems as not converged.
__global__ void k_outer_cond(cudaGraphConditionalHandle h, ScalList L) {
    DevScal* s0 = L.s[0];
    int go = 0;
    for (int i = 0; i < L.n; ++i)
        if (!L.s[i]->o_fin) go = 1;
    s0->o_body += 1;
    if (go && s0->o_body >= s0->o_body_cap) {
        for (int i = 0; i < L.n; ++i)
            if (!L.s[i]->o_fin) outer_end(L.s[i], EOFA_ERR_NOT_CONVERGED);
        go = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

cudaError_t outer_cond(cudaGraphConditionalHandle h, const ScalList& L, cudaStream_t st) {
    k_outer_cond<<<1, 1, 0, st>>>(h, L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CG updates
// ---------------------------------------------------------------------------
// r -= alpha q and |r|^2 (FIN_RR: convergence test and iteration count)
template <typename S>
__global__ void __launch_bounds__(BT) k_cg_r(VecRef q, VecRef r, long n5, int Ls, Reduce rd, const int* done) {
    typedef typename Traits<S>::R R;
    if (*done) return;
    const R al = (R)rd.scal->alpha;
    R nn = (R)0;
    for (long t = (long)blockIdx.x * BT + threadIdx.x; t < n5; t += (long)gridDim.x * BT) {
        const long xcb = t / Ls;
        const int s = (int)(t - xcb * Ls);
        R qv[24], rv[24];
        load_sp<S, R>(q.d, q.n, xcb, s, Ls, qv);
        load_sp<S, R>(r.d, r.n, xcb, s, Ls, rv);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            rv[i] -= al * qv[i];
            nn += rv[i] * rv[i];
        }
        store_sp<S, R>(r.d, r.n, xcb, s, Ls, rv);
    }
    block_reduce_finalize<BT>(nn, rd);
}

// x += alpha p, then p = z + beta p, sharing the read of p.  The update of
// x belongs to the iteration whose residual update ran, so it still runs in
// the iteration that set the done flag; the last block then sets stop
// (FIN_STOP), which ends this kernel in the iterations that follow.
template <typename S, typename SX>
__global__ void __launch_bounds__(BT) k_cg_px(VecRef x, VecRef p, VecRef z, long n5, int Ls, Reduce rd) {
    typedef typename Traits<S>::R R;
    typedef typename Traits<SX>::R RX;
    const DevScal* sc = rd.scal;
    if (sc->stop) return;
    for (long t = (long)blockIdx.x * BT + threadIdx.x; t < n5; t += (long)gridDim.x * BT) {
        const long xcb = t / Ls;
        const int s = (int)(t - xcb * Ls);
        const double al = sc->alpha;
        R pv[24];
        RX xv[24];
        load_sp<S, R>(p.d, p.n, xcb, s, Ls, pv);
        load_sp<SX, RX>(x.d, x.n, xcb, s, Ls, xv);
#pragma unroll
        for (int i = 0; i < 24; ++i) xv[i] += (RX)al * (RX)pv[i];
        store_sp<SX, RX>(x.d, x.n, xcb, s, Ls, xv);
        if (!sc->done) {
            const R be = (R)sc->beta;
            R zv[24];
            load_sp<S, R>(z.d, z.n, xcb, s, Ls, zv);
#pragma unroll
            for (int i = 0; i < 24; ++i) pv[i] = zv[i] + be * pv[i];
            store_sp<S, R>(p.d, p.n, xcb, s, Ls, pv);
        }
    }
    block_reduce_finalize<BT>((R)0, rd);
}

// dst = a * src (types may differ); optional |dst|^2 reduction.
// Scale: a = scale, or 1/sqrt(store[slot]) when inv_sqrt_slot >= 0.
template <typename SD, typename SS>
__global__ void __launch_bounds__(BT) k_copy(VecRef dst, VecRef src, long n5, int Ls, double scale,
                                             int inv_sqrt_slot, Reduce rd, const int* skip) {
    typedef typename Traits<SD>::R RD;
    typedef typename Traits<SS>::R RS;
    if (skip && *skip) return;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    RD nn = (RD)0;
    if (t < n5) {
        const long xcb = t / Ls;
        const int s = (int)(t - xcb * Ls);
        double a = scale;
        if (inv_sqrt_slot >= 0) {
            double v = rd.scal->store[inv_sqrt_slot];
            a = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
        }
        RS sv[24];
        RD dv[24];
        load_sp<SS, RS>(src.d, src.n, xcb, s, Ls, sv);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            dv[i] = (RD)((double)sv[i] * a);
            nn += dv[i] * dv[i];
        }
        store_sp<SD, RD>(dst.d, dst.n, xcb, s, Ls, dv);
    }
    if (rd.fin != FIN_NONE) block_reduce_finalize<BT>(nn, rd);
}

// x (FP64) += sqrt(store[slot]) * e  (defect-correction update)
template <typename SE>
__global__ void __launch_bounds__(BT) k_acc(VecRef x, VecRef e, long n5, int Ls, const DevScal* sc,
                                            int slot, const int* skip) {
    typedef typename Traits<SE>::R RE;
    if (skip && *skip) return;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    if (t >= n5) return;
    const long xcb = t / Ls;
    const int s = (int)(t - xcb * Ls);
    const double a = sqrt(sc->store[slot]);
    double xv[24];
    RE ev[24];
    load_sp<double, double>(x.d, nullptr, xcb, s, Ls, xv);
    load_sp<SE, RE>(e.d, e.n, xcb, s, Ls, ev);
#pragma unroll
    for (int i = 0; i < 24; ++i) xv[i] += a * (double)ev[i];
    store_sp<double, double>(x.d, nullptr, xcb, s, Ls, xv);
}

// r = b - q (FP64), |r|^2 reduced
__global__ void __launch_bounds__(BT) k_sub(VecRef r, VecRef b, VecRef q, long n5, int Ls, Reduce rd,
                                            const int* skip) {
    if (skip && *skip) return;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    double nn = 0.0;
    if (t < n5) {
        const long xcb = t / Ls;
        const int s = (int)(t - xcb * Ls);
        double bv[24], qv[24];
        load_sp<double, double>(b.d, nullptr, xcb, s, Ls, bv);
        load_sp<double, double>(q.d, nullptr, xcb, s, Ls, qv);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            bv[i] -= qv[i];
            nn += bv[i] * bv[i];
        }
        store_sp<double, double>(r.d, nullptr, xcb, s, Ls, bv);
    }
    block_reduce_finalize<BT>(nn, rd);
}

template <typename S>
__global__ void __launch_bounds__(BT) k_zero(VecRef v, long n5, int Ls, const int* skip) {
    typedef typename Traits<S>::R R;
    if (skip && *skip) return;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    if (t >= n5) return;
    const long xcb = t / Ls;
    const int s = (int)(t - xcb * Ls);
    R z[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) z[i] = (R)0;
    store_sp<S, R>(v.d, v.n, xcb, s, Ls, z);
}

// ---------------------------------------------------------------------------
// layout conversion: canonical complex128 <-> internal FP64, one parity
// ---------------------------------------------------------------------------
__device__ __forceinline__ long lex_of(const Geom& g, long xcb, int par) {
    int rem = (int)xcb;
    const int xh = rem % g.Xh; rem /= g.Xh;
    const int y = rem % g.Y; rem /= g.Y;
    const int z = rem % g.Z;
    const int t = rem / g.Z;
    const int x = 2 * xh + ((par + y + z + t) & 1);
    return (((long)t * g.Z + z) * g.Y + y) * g.X + x;
}

// g5r5: read slice Ls-1-s and flip the sign of spins 2, 3 (gamma_5 R_5)
__global__ void __launch_bounds__(BT) k_import(VecRef dst, const double* __restrict__ src, Geom g, int par,
                                               int g5r5) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    const long n5 = (long)g.Vh * g.Ls;
    if (t >= n5) return;
    const long xcb = t / g.Ls;
    const int s = (int)(t - xcb * g.Ls);
    const long lex = lex_of(g, xcb, par);
    const int ss = g5r5 ? g.Ls - 1 - s : s;
    const double2* p = reinterpret_cast<const double2*>(src) + (lex * g.Ls + ss) * 12;
    double v[24];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        double2 q = p[c];
        const double f = (g5r5 && c >= 6) ? -1.0 : 1.0;
        v[2 * c] = f * q.x;
        v[2 * c + 1] = f * q.y;
    }
    store_sp<double, double>(dst.d, nullptr, xcb, s, g.Ls, v);
}

__global__ void __launch_bounds__(BT) k_export(double* __restrict__ dst, VecRef src, Geom g, int par,
                                               int g5r5) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    const long n5 = (long)g.Vh * g.Ls;
    if (t >= n5) return;
    const long xcb = t / g.Ls;
    const int s = (int)(t - xcb * g.Ls);
    const long lex = lex_of(g, xcb, par);
    double v[24];
    load_sp<double, double>(src.d, nullptr, xcb, s, g.Ls, v);
    const int ss = g5r5 ? g.Ls - 1 - s : s;
    double2* p = reinterpret_cast<double2*>(dst) + (lex * g.Ls + ss) * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const double f = (g5r5 && c >= 6) ? -1.0 : 1.0;
        p[c] = make_double2(f * v[2 * c], f * v[2 * c + 1]);
    }
}

// gauge: canonical U[lex][mu][3][3] complex128 -> two-row links per parity in
// all four storage precisions; flags links that are not SU(3) to 1e-10.
__global__ void __launch_bounds__(BT) k_gauge(const double* __restrict__ U, Geom g, void* l64_0, void* l64_1,
                                              void* l32_0, void* l32_1, void* l16_0, void* l16_1, void* lb_0,
                                              void* lb_1, int* bad) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    const long V = 2L * g.Vh;
    if (t >= V * 4) return;
    const long lex = t >> 2;
    const int mu = (int)(t & 3);
    int rem = (int)lex;
    const int x = rem % g.X; rem /= g.X;
    const int y = rem % g.Y; rem /= g.Y;
    const int z = rem % g.Z;
    const int tt = rem / g.Z;
    const int par = (x + y + z + tt) & 1;
    const long xcb = lex >> 1;
    const double* u = U + (lex * 4 + mu) * 18;
    // SU(3) check: rows orthonormal and row2 = conj(row0 x row1)
    double dev = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double re = 0, im = 0;
            for (int k = 0; k < 3; ++k) {
                const double ar = u[(a * 3 + k) * 2], ai = u[(a * 3 + k) * 2 + 1];
                const double br = u[(b * 3 + k) * 2], bi = u[(b * 3 + k) * 2 + 1];
                re += ar * br + ai * bi;
                im += ai * br - ar * bi;
            }
            dev = fmax(dev, fabs(re - (a == b ? 1.0 : 0.0)));
            dev = fmax(dev, fabs(im));
        }
    {
        const double* r0 = u;
        const double* r1 = u + 6;
        const double* r2 = u + 12;
        for (int j = 0; j < 3; ++j) {
            const int k = (j + 1) % 3, l = (j + 2) % 3;
            const double cr = (r0[2 * k] * r1[2 * l] - r0[2 * k + 1] * r1[2 * l + 1]) -
                              (r0[2 * l] * r1[2 * k] - r0[2 * l + 1] * r1[2 * k + 1]);
            const double ci = (r0[2 * k] * r1[2 * l + 1] + r0[2 * k + 1] * r1[2 * l]) -
                              (r0[2 * l] * r1[2 * k + 1] + r0[2 * l + 1] * r1[2 * k]);
            dev = fmax(dev, fabs(r2[2 * j] - cr));
            dev = fmax(dev, fabs(r2[2 * j + 1] + ci));
        }
    }
    if (!(dev <= 1e-10)) atomicOr(bad, 1);
    const long off = (xcb * 4 + mu) * 12;
    double* d64 = reinterpret_cast<double*>(par ? l64_1 : l64_0) + off;
    float* d32 = reinterpret_cast<float*>(par ? l32_1 : l32_0) + off;
    __half* d16 = reinterpret_cast<__half*>(par ? l16_1 : l16_0) + off;
    __nv_bfloat16* db = reinterpret_cast<__nv_bfloat16*>(par ? lb_1 : lb_0) + off;
    for (int i = 0; i < 12; ++i) {
        d64[i] = u[i];
        d32[i] = (float)u[i];
        d16[i] = __double2half(u[i]);
        db[i] = __double2bfloat16(u[i]);
    }
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
template <typename F>
static cudaError_t dispatch_prec(int prec, F&& f) {
    switch (prec) {
        case 0: return f((double*)nullptr);
        case 1: return f((float*)nullptr);
        case 2: return f((__half*)nullptr);
        case 3: return f((__nv_bfloat16*)nullptr);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t blas_cg_r(int prec, VecRef q, VecRef r, long n5, int Ls, Reduce rd, const int* done,
                      cudaStream_t st) {
    return dispatch_prec(prec, [&](auto* tag) -> cudaError_t {
        typedef std::remove_pointer_t<decltype(tag)> S;
        k_cg_r<S><<<grid_capped(n5), BT, 0, st>>>(q, r, n5, Ls, rd, done);
        return cudaGetLastError();
    });
}

cudaError_t blas_cg_px(int prec, int xprec, VecRef x, VecRef p, VecRef z, long n5, int Ls, Reduce rd,
                       cudaStream_t st) {
    return dispatch_prec(prec, [&](auto* tag) -> cudaError_t {
        typedef std::remove_pointer_t<decltype(tag)> S;
        if (xprec == 0) k_cg_px<S, double><<<grid_capped(n5), BT, 0, st>>>(x, p, z, n5, Ls, rd);
        else k_cg_px<S, float><<<grid_capped(n5), BT, 0, st>>>(x, p, z, n5, Ls, rd);
        return cudaGetLastError();
    });
}

cudaError_t blas_copy(int dprec, VecRef dst, int sprec, VecRef src, long n5, int Ls, double scale,
                      int inv_sqrt_slot, Reduce rd, cudaStream_t st, const int* skip) {
    return dispatch_prec(dprec, [&](auto* dtag) -> cudaError_t {
        typedef std::remove_pointer_t<decltype(dtag)> SD;
        return dispatch_prec(sprec, [&](auto* stag) -> cudaError_t {
            typedef std::remove_pointer_t<decltype(stag)> SS;
            k_copy<SD, SS><<<grid_for(n5), BT, 0, st>>>(dst, src, n5, Ls, scale, inv_sqrt_slot, rd, skip);
            return cudaGetLastError();
        });
    });
}

cudaError_t blas_acc(VecRef x, int eprec, VecRef e, long n5, int Ls, const DevScal* sc, int slot,
                     cudaStream_t st, const int* skip) {
    return dispatch_prec(eprec, [&](auto* tag) -> cudaError_t {
        typedef std::remove_pointer_t<decltype(tag)> SE;
        k_acc<SE><<<grid_for(n5), BT, 0, st>>>(x, e, n5, Ls, sc, slot, skip);
        return cudaGetLastError();
    });
}

cudaError_t blas_sub(VecRef r, VecRef b, VecRef q, long n5, int Ls, Reduce rd, cudaStream_t st,
                     const int* skip) {
    k_sub<<<grid_for(n5), BT, 0, st>>>(r, b, q, n5, Ls, rd, skip);
    return cudaGetLastError();
}

cudaError_t blas_zero(int prec, VecRef v, long n5, int Ls, cudaStream_t st, const int* skip) {
    return dispatch_prec(prec, [&](auto* tag) -> cudaError_t {
        typedef std::remove_pointer_t<decltype(tag)> S;
        k_zero<S><<<grid_for(n5), BT, 0, st>>>(v, n5, Ls, skip);
        return cudaGetLastError();
    });
}

cudaError_t layout_import(VecRef dst, const double* src, const Geom& g, int par, int g5r5, cudaStream_t st) {
    k_import<<<grid_for((long)g.Vh * g.Ls), BT, 0, st>>>(dst, src, g, par, g5r5);
    return cudaGetLastError();
}

cudaError_t layout_export(double* dst, VecRef src, const Geom& g, int par, int g5r5, cudaStream_t st) {
    k_export<<<grid_for((long)g.Vh * g.Ls), BT, 0, st>>>(dst, src, g, par, g5r5);
    return cudaGetLastError();
}

cudaError_t gauge_import(const double* U, const Geom& g, void* const links[4][2], int* bad, cudaStream_t st) {
    k_gauge<<<grid_for(2L * g.Vh * 4), BT, 0, st>>>(U, g, links[0][0], links[0][1], links[1][0], links[1][1],
                                                    links[2][0], links[2][1], links[3][0], links[3][1], bad);
    return cudaGetLastError();
}

// G-parity: the flavour-stacked gauge field [U; U*] (flavour 2 carries the
// conjugate links) from the physical U, n = complex entries of U
__global__ void __launch_bounds__(BT) k_gparity_gauge(const double2* __restrict__ U, double2* __restrict__ out,
                                                      long n) {
    const long i = (long)blockIdx.x * BT + threadIdx.x;
    if (i >= n) return;
    const double2 u = U[i];
    out[i] = u;
    out[n + i] = make_double2(u.x, -u.y);
}

cudaError_t gparity_gauge(const double* U, double* out, long n, cudaStream_t st) {
    k_gparity_gauge<<<grid_for(n), BT, 0, st>>>((const double2*)U, (double2*)out, n);
    return cudaGetLastError();
}

int blas_max_grid(long n5) { return grid_for(n5); }

// ===========================================================================
// learned preconditioner support: layout bridges and complex BLAS (FP32)
// ===========================================================================

// odd-parity FP32 field (even-odd layout) -> activations [Ls][V][32] BF16 on
// the full lattice, zero on even sites; slice sl only when sl >= 0 (then the
// output is one [V][32] slice), scaled by scale (or 1/sqrt(store[slot]) when
// slot >= 0)
__global__ void __launch_bounds__(BT) k_embed_odd(VecRef f, bf16* __restrict__ act, Geom g, int sl,
                                                  double scale, const DevScal* sc, int slot) {
    const long V = 2L * g.Vh;
    const int ns = sl >= 0 ? 1 : g.Ls;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    if (t >= V * ns) return;
    const int s = sl >= 0 ? sl : (int)(t / V);
    const long lex = t % V;
    int rem = (int)lex;
    const int x = rem % g.X; rem /= g.X;
    const int y = rem % g.Y; rem /= g.Y;
    const int z = rem % g.Z;
    const int tt = rem / g.Z;
    bf16* dst = act + t * kCP;
    float v[24];
    if ((x + y + z + tt) & 1) {
        load_sp<float, float>(f.d, f.n, lex >> 1, s, g.Ls, v);
        float a = (float)scale;
        if (slot >= 0) {
            const double q = sc->store[slot];
            a = q > 0.0 ? (float)(1.0 / sqrt(q)) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] *= a;
    } else {
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < 24; i += 2)
        *reinterpret_cast<__nv_bfloat162*>(dst + i) = __floats2bfloat162_rn(v[i], v[i + 1]);
#pragma unroll
    for (int i = 24; i < 32; i += 2)
        *reinterpret_cast<__nv_bfloat162*>(dst + i) = __floats2bfloat162_rn(0.f, 0.f);
}

// network output [Ls][V][32] FP32 -> odd-parity FP32 field
__global__ void __launch_bounds__(BT) k_extract_odd(const float* __restrict__ out32, VecRef f, Geom g) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    const long n5 = (long)g.Vh * g.Ls;
    if (t >= n5) return;
    const long xcb = t / g.Ls;
    const int s = (int)(t - xcb * g.Ls);
    const long lex = lex_of(g, xcb, 1);
    const float* src = out32 + ((long)s * 2 * g.Vh + lex) * kCP;
    float v[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) v[i] = src[i];
    store_sp<float, float>(f.d, f.n, xcb, s, g.Ls, v);
}

// <a, b> = sum conj(a) b over an FP32 field: real part into rr, imaginary into ri
__global__ void __launch_bounds__(BT) k_cdot(VecRef a, VecRef b, long n5, int Ls, Reduce rr, Reduce ri) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    float re = 0.f, im = 0.f;
    if (t < n5) {
        const long xcb = t / Ls;
        const int s = (int)(t - xcb * Ls);
        float av[24], bv[24];
        load_sp<float, float>(a.d, a.n, xcb, s, Ls, av);
        load_sp<float, float>(b.d, b.n, xcb, s, Ls, bv);
#pragma unroll
        for (int i = 0; i < 24; i += 2) {
            re += av[i] * bv[i] + av[i + 1] * bv[i + 1];
            im += av[i] * bv[i + 1] - av[i + 1] * bv[i];
        }
    }
    block_reduce_finalize<BT>(re, rr);
    __syncthreads();
    block_reduce_finalize<BT>(im, ri);
}

// y = a x + b y with complex a = (ar, ai) and real b (FP32 fields)
__global__ void __launch_bounds__(BT) k_caxpby(VecRef y, VecRef x, long n5, int Ls, float ar, float ai, float b) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    if (t >= n5) return;
    const long xcb = t / Ls;
    const int s = (int)(t - xcb * Ls);
    float xv[24], yv[24];
    load_sp<float, float>(x.d, x.n, xcb, s, Ls, xv);
    load_sp<float, float>(y.d, y.n, xcb, s, Ls, yv);
#pragma unroll
    for (int i = 0; i < 24; i += 2) {
        const float r = ar * xv[i] - ai * xv[i + 1] + b * yv[i];
        const float m = ar * xv[i + 1] + ai * xv[i] + b * yv[i + 1];
        yv[i] = r;
        yv[i + 1] = m;
    }
    store_sp<float, float>(y.d, y.n, xcb, s, Ls, yv);
}

// |slice sl of an FP32 field|^2 (one s-slice of the odd sites)
__global__ void __launch_bounds__(BT) k_slice_norm(VecRef f, long vh, int Ls, int sl, Reduce rd) {
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    float nn = 0.f;
    if (t < vh) {
        float v[24];
        load_sp<float, float>(f.d, f.n, t, sl, Ls, v);
#pragma unroll
        for (int i = 0; i < 24; ++i) nn += v[i] * v[i];
    }
    block_reduce_finalize<BT>(nn, rd);
}

// training loss: out [B][V][32] FP32, target e [B][V][32] BF16, inverse
// norms w[B]; on odd sites, channels < 24:  dout = 2/B w (out - e),
// loss = 1/B sum w |out - e|^2 (reduced into rd)
__global__ void __launch_bounds__(BT) k_loss_grad(const float* __restrict__ out, const bf16* __restrict__ e,
                                                  const float* __restrict__ w, float* __restrict__ dout, Geom g,
                                                  int B, Reduce rd) {
    const long V = 2L * g.Vh;
    const long t = (long)blockIdx.x * BT + threadIdx.x;
    float l = 0.f;
    if (t < V * B) {
        const int b = (int)(t / V);
        const long lex = t % V;
        int rem = (int)lex;
        const int x = rem % g.X; rem /= g.X;
        const int y = rem % g.Y; rem /= g.Y;
        const int z = rem % g.Z;
        const int tt = rem / g.Z;
        const bool odd = (x + y + z + tt) & 1;
        const float wb = w[b];
        for (int c = 0; c < kCP; ++c) {
            float d = 0.f;
            if (odd && c < 24) {
                const float diff = out[t * kCP + c] - __bfloat162float(e[t * kCP + c]);
                l += wb * diff * diff;
                d = 2.f * wb * diff / (float)B;
            }
            dout[t * kCP + c] = d;
        }
        l /= (float)B;
    }
    block_reduce_finalize<BT>(l, rd);
}

cudaError_t embed_odd(VecRef f, bf16* act, const Geom& g, int sl, double scale, const DevScal* sc, int slot,
                      cudaStream_t st) {
    const long n = 2L * g.Vh * (sl >= 0 ? 1 : g.Ls);
    k_embed_odd<<<grid_for(n), BT, 0, st>>>(f, act, g, sl, scale, sc, slot);
    return cudaGetLastError();
}

cudaError_t extract_odd(const float* out32, VecRef f, const Geom& g, cudaStream_t st) {
    k_extract_odd<<<grid_for((long)g.Vh * g.Ls), BT, 0, st>>>(out32, f, g);
    return cudaGetLastError();
}

cudaError_t cdot(VecRef a, VecRef b, long n5, int Ls, Reduce rr, Reduce ri, cudaStream_t st) {
    k_cdot<<<grid_for(n5), BT, 0, st>>>(a, b, n5, Ls, rr, ri);
    return cudaGetLastError();
}

cudaError_t caxpby(VecRef y, VecRef x, long n5, int Ls, float ar, float ai, float b, cudaStream_t st) {
    k_caxpby<<<grid_for(n5), BT, 0, st>>>(y, x, n5, Ls, ar, ai, b);
    return cudaGetLastError();
}

cudaError_t slice_norm(VecRef f, long vh, int Ls, int sl, Reduce rd, cudaStream_t st) {
    k_slice_norm<<<grid_for(vh), BT, 0, st>>>(f, vh, Ls, sl, rd);
    return cudaGetLastError();
}

cudaError_t loss_grad(const float* out, const bf16* e, const float* w, float* dout, const Geom& g, int B, Reduce rd,
                      cudaStream_t st) {
    k_loss_grad<<<grid_for(2L * g.Vh * B), BT, 0, st>>>(out, e, w, dout, g, B, rd);
    return cudaGetLastError();
}

}  // namespace eofa
