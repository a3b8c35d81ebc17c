// eofa.cu -- host driver and C ABI of the GB300 EOFA solver (see eofa.h).
//
// Solve path (App. B of arXiv:1706.05843):
//   b   = g5 R5 phi (H form) or b (K form), imported into the even-odd layout
//   b~o = b_o - K_oe K_ee^-1 b_e                       even-odd source
//   CGNR on S = K_oo - K_oe K_ee^-1 K_eo:  S^dag S x_o = S^dag b~o
//     inside a restarted defect-correction loop (Sec. V.A): the FP64 outer
//     loop forms r = b~o - S x_o, the inner CGNR solves S e = r/|r| in the
//     requested storage precision, x_o += |r| e
//   x_e = K_ee^-1 (b_e - K_eo x_o)                     reconstruction
//   psi = D~(m1) psi'                                  undo the Cayley form
//   true residual ||b - K psi'|| / ||b|| in FP64
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "blas.h"
#include "dslash.cuh"
#include "eofa.h"
#include "learned.h"

using namespace eofa;

namespace {

struct Inner {
    bool ready = false;
    VecRef r{}, p{}, q{}, z{}, t{}, x{};
};

}  // namespace

struct eofa_ctx {
    eofa_params p;
    Geom g;
    long n5 = 0;
    SCoef<double> c64;
    SCoef<float> c32;
    void* links[4][2] = {};
    VecRef b[2]{}, x[2]{}, t[2]{}, ro{}, bto{}, qo{};
    Inner inner[4];
    double* partials = nullptr;
    unsigned* counter = nullptr;
    DevScal* scal = nullptr;
    DevScal* h_scal = nullptr;  // pinned
    int* d_flag = nullptr;
    std::vector<void*> allocs;
    std::string err;
    // hop-kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> evs;
    int ev_used = 0;
    // graph-path timing sample: events around the four hops of the first
    // iteration of every chunk of the captured CG loop, per precision
    cudaEvent_t gev[4][8] = {};
    double hop_ms = 0.0;
    int hop_launches = 0;
    double hop_bytes = 0.0;
    std::vector<double> ev_bytes;
    long launches = 0;  // kernels launched since the last reset
    int gcr_steps = 0, gcr_fallbacks = 0;  // learned-preconditioner statistics of the current solve
    double net_ms = 0.0;                   // device time of the network applications
    cudaEvent_t nev[2] = {};               // events around one network application
    // autotuned CTA tile variant of the four inner-solver hop kinds, per precision
    bool tuned[4] = {};
    int tile[4][4] = {};
    float tune_ms[4][4][4] = {};  // [prec][kind][variant] tuner's time per launch (0: not timed)
    // device-driven CG loops, one per inner method and precision
    cudaStream_t cap = nullptr;
    cudaGraphExec_t cg_exec[2][4] = {};
    cudaGraphExec_t cg_first[2][4] = {};  // the first CG iteration, with timing events
    // inner operator of the current solve (opts.method): 0 Cayley form,
    // 1 dense even-odd on the unpreconditioned system; the dense s-space
    // matrices of method 1, [F64, F32][A_ee^-1, A_oo] -> [chirality][Ls][Ls]
    int method = 0;
    bool dense_ready = false;
    void* dense[2][2] = {};
    // learned preconditioner: weights, activations of all Ls slices on the
    // full lattice, flexible-GCR vectors (FP32, odd parity), second
    // reduction buffers for complex inner products
    bool net_ready = false;
    NetDev net;
    bf16* act[3] = {};
    float* out32 = nullptr;
    VecRef gx{}, gr{}, gz[4]{}, gw[4]{};
    double* partials2 = nullptr;
    unsigned* counter2 = nullptr;
    // EOFA action and heatbath: canonical complex128 5D work fields,
    // allocated on first use; multi-dot partial sums and results
    std::vector<double*> act5;
    double* mdot = nullptr;
    unsigned long long uid = 0;  // identity of the context for the kept batch graphs
    // host-buffer solves: the solution's copy to page-locked host memory runs
    // on this stream while the true residual is computed
    cudaStream_t side = nullptr;
    cudaEvent_t xev[2] = {};
    bool exported = false;  // the current solve has written its solution
};

namespace {

const int kWidth[4] = {8, 4, 2, 2};

eofa_status fail(eofa_ctx* c, eofa_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

eofa_status cuda_fail(eofa_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (c) c->err = m;
    return e == cudaErrorMemoryAllocation ? EOFA_ERR_OOM : EOFA_ERR_CUDA;
}

#define CK(call, where)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);   \
    } while (0)

// CK for calls that launch exactly one kernel
#define CKL(call, where)                                         \
    do {                                                         \
        CK(call, where);                                         \
        ++c->launches;                                           \
    } while (0)

eofa_status dalloc(eofa_ctx* c, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(c, e, "cudaMalloc");
    }
    c->allocs.push_back(*p);
    return EOFA_OK;
}

eofa_status vec_alloc(eofa_ctx* c, int prec, VecRef* v) {
    eofa_status s = dalloc(c, &v->d, (size_t)c->n5 * 24 * kWidth[prec]);
    if (s != EOFA_OK) return s;
    v->n = nullptr;
    if (prec == EOFA_F16) {
        void* n = nullptr;
        s = dalloc(c, &n, (size_t)c->n5 * sizeof(float));
        if (s != EOFA_OK) return s;
        v->n = (float*)n;
    }
    return EOFA_OK;
}

// ---------------------------------------------------------------------------
// fifth-dimension coefficients (host, FP64)
// ---------------------------------------------------------------------------
// solve (a + g L+) t = v, L+ with mass m (mirrored coordinates)
void host_inv(int Ls, double a, double g, double m, const double* v, double* t) {
    const double z = g / a;
    const double den = a * (1.0 + m * std::pow(z, Ls));
    double tl = 0.0, w = 1.0;
    for (int j = 0; j < Ls; ++j) {
        tl += w * v[Ls - 1 - j] / den;
        w *= -z;
    }
    t[0] = v[0] / a + m * z * tl;
    for (int s = 1; s < Ls - 1; ++s) t[s] = v[s] / a - z * t[s - 1];
    t[Ls - 1] = tl;
}
// solve (a + g L-) t = v
void host_invT(int Ls, double a, double g, double m, const double* v, double* t) {
    double vr[LSMAX] = {}, tr[LSMAX] = {};
    for (int s = 0; s < Ls; ++s) vr[s] = v[Ls - 1 - s];
    host_inv(Ls, a, g, m, vr, tr);
    for (int s = 0; s < Ls; ++s) t[s] = tr[Ls - 1 - s];
}

template <typename R>
void cast_coef(const SCoef<double>& d, SCoef<R>& r) {
    r.alpha = (R)d.alpha; r.gamma = (R)d.gamma; r.b5 = (R)d.b5; r.c5 = (R)d.c5; r.m = (R)d.m;
    r.ia = (R)d.ia; r.za = (R)d.za; r.mza = (R)d.mza;
    r.ib = (R)d.ib; r.zb = (R)d.zb; r.mzb = (R)d.mzb;
    r.sbk = (R)d.sbk; r.sbk_den = (R)d.sbk_den; r.sb_den = (R)d.sb_den;
    r.cs = d.cs; r.has_shift = d.has_shift;
    for (int i = 0; i < LSMAX; ++i) {
        r.wa[i] = (R)d.wa[i]; r.wb[i] = (R)d.wb[i];
        r.um[i] = (R)d.um[i]; r.xm[i] = (R)d.xm[i]; r.ym[i] = (R)d.ym[i];
    }
}

// App. B: A = (D_DWF)_ee = alpha + gamma L(m1), alpha = b5 (4 - M5) + 1,
// gamma = c5 (4 - M5) - 1; the shift u_pm (x) v_pm with the closed forms of
// u_pm (mass m1) and v_pm = k(m2, m3) e_{Ls-1 | 0}; Sherman-Morrison vectors
// x = A^-1 u (the tridiagonal-algorithm step of App. B) and y = A^-T v.
// Context-free and free of heap allocation: also used by the entry point
// that allocates nothing.  On failure *why names the reason.
eofa_status coef_from_params(const eofa_params& p, SCoef<double>& k, const char** why) {
    const int Ls = p.Ls;
    std::memset(&k, 0, sizeof(k));
    const double b5 = p.b, c5 = p.c, m = p.m1;
    if (b5 == 0.0) return *why = "b (b5) must be non-zero", EOFA_ERR_UNSUPPORTED;
    const double alpha = b5 * (4.0 - p.M5) + 1.0;
    const double gamma = c5 * (4.0 - p.M5) - 1.0;
    if (alpha == 0.0) return *why = "b5 (4 - M5) + 1 = 0", EOFA_ERR_SINGULAR;
    const double za = gamma / alpha, zb = c5 / b5;
    if (std::fabs(za) >= 1.0 || std::fabs(zb) >= 1.0)
        return *why = "fifth-dimension recurrences need |(c5(4-M5)-1)/(b5(4-M5)+1)| < 1 and |c5/b5| < 1", EOFA_ERR_UNSUPPORTED;
    const double ca = 1.0 + m * std::pow(za, Ls), cb = 1.0 + m * std::pow(zb, Ls);
    if (std::fabs(ca) < 1e-14 || std::fabs(cb) < 1e-14)
        return *why = "cyclic fifth-dimension block is singular", EOFA_ERR_SINGULAR;
    auto N = [&](double mm) { return std::pow(b5, Ls) + mm * std::pow(c5, Ls); };
    if (N(p.m1) == 0.0 || N(p.m2) == 0.0 || N(p.m3) == 0.0)
        return *why = "N(m) = b5^Ls + m c5^Ls vanishes", EOFA_ERR_SINGULAR;
    k.alpha = alpha; k.gamma = gamma; k.b5 = b5; k.c5 = c5; k.m = m;
    k.ia = 1.0 / alpha; k.za = za; k.mza = m * za;
    k.ib = 1.0 / b5; k.zb = zb; k.mzb = m * zb;
    double wa = 1.0, wb = 1.0;
    for (int j = 0; j < Ls; ++j) {
        k.wa[j] = wa / (alpha * ca);
        k.wb[j] = wb / (b5 * cb);
        wa *= -za;
        wb *= -zb;
    }
    // k(m2, m3) = 2c (m3 - m2) (c+d)^{2Ls} / (N(m2) N(m3)), 2c = b5 + c5
    const double kk = (b5 + c5) * (p.m3 - p.m2) * std::pow(b5, 2 * Ls) / (N(p.m2) * N(p.m3));
    const double N1 = N(p.m1);
    double u[LSMAX];
    for (int s = 0; s < Ls; ++s) {
        if (p.pm > 0)
            u[s] = ((s & 1) ? -1.0 : 1.0) * std::pow(c5, s) / std::pow(b5, Ls + s + 1) * N1;
        else
            u[s] = ((s & 1) ? 1.0 : -1.0) * std::pow(c5, Ls - 1 - s) / std::pow(b5, 2 * Ls - s) * N1;
    }
    k.cs = p.pm > 0 ? 0 : 1;
    for (int s = 0; s < Ls; ++s) k.um[s] = (k.cs == 0) ? u[s] : u[Ls - 1 - s];
    host_inv(Ls, alpha, gamma, m, k.um, k.xm);
    double e[LSMAX] = {};
    e[Ls - 1] = kk;
    host_invT(Ls, alpha, gamma, m, e, k.ym);
    k.has_shift = p.beta != 0.0;
    const double sb = p.pm * p.beta;
    const double den = 1.0 + sb * kk * k.xm[Ls - 1];
    if (k.has_shift && std::fabs(den) < 1e-14)
        return *why = "Sherman-Morrison denominator 1 + pm beta <v, A^-1 u> ~ 0", EOFA_ERR_SINGULAR;
    k.sbk = sb * kk;
    k.sbk_den = k.has_shift ? sb * kk / den : 0.0;
    k.sb_den = k.has_shift ? sb / den : 0.0;
    return EOFA_OK;
}

eofa_status build_coef(eofa_ctx* c) {
    const char* why = "";
    eofa_status s = coef_from_params(c->p, c->c64, &why);
    if (s != EOFA_OK) return fail(c, s, why);
    cast_coef(c->c64, c->c32);
    return EOFA_OK;
}

// ---------------------------------------------------------------------------
// kernel helpers
// ---------------------------------------------------------------------------
Reduce red(eofa_ctx* c, int fin, int slot = 0) {
    Reduce r;
    r.partials = c->partials;
    r.counter = c->counter;
    r.scal = c->scal;
    r.fin = fin;
    r.slot = slot;
    return r;
}

double hop_bytes_of(const eofa_ctx* c, int prec, int with_local) {
    const double w = kWidth[prec];
    double per5 = (48.0 + (with_local ? 24.0 : 0.0)) * w;
    if (prec == EOFA_F16) per5 += 4.0 * (2 + (with_local ? 1 : 0));
    return c->n5 * per5 + (double)c->g.Vh * 8.0 * 12.0 * w;
}

eofa_status hop(eofa_ctx* c, int prec, int kind, int out_par, VecRef in, VecRef y, VecRef out, Reduce rd,
                const int* done, cudaStream_t st, bool timed = false) {
    HopArgs a;
    std::memset(&a, 0, sizeof(a));
    a.g = c->g;
    a.out_par = out_par;
    a.in = in.d; a.in_nrm = in.n;
    a.y = y.d; a.y_nrm = y.n;
    a.out = out.d; a.out_nrm = out.n;
    a.lk_out = c->links[prec][out_par];
    a.lk_in = c->links[prec][1 - out_par];
    a.rd = rd;
    a.tile_var = (kind <= KIND_OE_SCHUR_DAG && c->tuned[prec]) ? c->tile[prec][kind] : 0;
    a.done = done;
    if (kind >= KIND_D_EO && kind <= KIND_D_OE_DAG && prec <= EOFA_F32)
        a.dense = c->dense[prec][(kind == KIND_D_OE || kind == KIND_D_OE_DAG) ? 1 : 0];
    const void* coef = prec == EOFA_F64 ? (const void*)&c->c64 : (const void*)&c->c32;
    const bool tm = timed && c->timing;
    if (tm) {
        if (c->ev_used + 2 > (int)c->evs.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e), "cudaEventCreate");
                c->evs.push_back(e);
            }
        }
        CK(cudaEventRecord(c->evs[c->ev_used], st), "cudaEventRecord");
    }
    cudaError_t e;
    switch (prec) {
        case EOFA_F64: e = launch_hop_f64(kind, a, coef, st); break;
        case EOFA_F32: e = launch_hop_f32(kind, a, coef, st); break;
        case EOFA_F16: e = launch_hop_f16(kind, a, coef, st); break;
        default: e = launch_hop_bf16(kind, a, coef, st); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "hop kernel launch");
    ++c->launches;
    if (tm) {
        CK(cudaEventRecord(c->evs[c->ev_used + 1], st), "cudaEventRecord");
        const bool wl = kind == KIND_OE_SCHUR || kind == KIND_OE_SCHUR_DAG;
        if ((int)c->ev_bytes.size() < c->ev_used / 2 + 1) c->ev_bytes.resize(c->ev_used / 2 + 1);
        c->ev_bytes[c->ev_used / 2] = hop_bytes_of(c, prec, wl);
        c->ev_used += 2;
    }
    return EOFA_OK;
}

// after a stream synchronisation: fold the recorded hop timings into the totals
eofa_status drain_timers(eofa_ctx* c) {
    for (int i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->evs[i], c->evs[i + 1]), "cudaEventElapsedTime");
        c->hop_ms += ms;
        c->hop_launches += 1;
        c->hop_bytes += c->ev_bytes[i / 2];
    }
    c->ev_used = 0;
    return EOFA_OK;
}

eofa_status read_scal(eofa_ctx* c, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->h_scal, c->scal, sizeof(DevScal), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return drain_timers(c);
}

eofa_status ensure_inner(eofa_ctx* c, int P) {
    Inner& in = c->inner[P];
    if (in.ready) return EOFA_OK;
    eofa_status s;
    if ((s = vec_alloc(c, P, &in.r)) || (s = vec_alloc(c, P, &in.p)) || (s = vec_alloc(c, P, &in.q)) ||
        (s = vec_alloc(c, P, &in.z)) || (s = vec_alloc(c, P, &in.t)) ||
        (s = vec_alloc(c, P == EOFA_F64 ? EOFA_F64 : EOFA_F32, &in.x)))
        return s;
    in.ready = true;
    return EOFA_OK;
}

// ---------------------------------------------------------------------------
// autotuner: for each of the four inner-solver hop kinds of a precision,
// time both CTA tile variants on this context's buffers and keep the faster.
// Choices are cached per (precision, Ls, lattice) for every context of the
// process; tuning happens before any CG graph is captured.
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;
struct TuneChoice {
    int variant = 0;
    float ms[4] = {0.f, 0.f, 0.f, 0.f};  // per launch of each variant (0: not timed)
};
std::map<std::array<long, 5>, TuneChoice> g_tune_cache;  // (prec, Ls, X*Y, Z*T, kind) -> choice

eofa_status autotune(eofa_ctx* c, int P, cudaStream_t st) {
    if (c->tuned[P]) return EOFA_OK;
    // EOFA_TILE_VARIANT=v fixes every inner-solver hop kind to variant v
    // (reproducible profiles); variants FP64 arithmetic lacks fall back to
    // v & 1.  The kernels are still launched once here, before any graph
    // capture needs them.
    int forced = -1;
    if (const char* fv = std::getenv("EOFA_TILE_VARIANT")) {
        const int v = std::atoi(fv);
        if (v >= 0 && v <= 3) forced = (P == EOFA_F64) ? (v & 1) : v;
    }
    const Geom& g = c->g;
    bool all = forced < 0;
    if (forced < 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (int k = 0; k < 4; ++k) {
            auto it = g_tune_cache.find({P, g.Ls, (long)g.X * g.Y, (long)g.Z * g.T, k});
            if (it == g_tune_cache.end()) {
                all = false;
            } else {
                c->tile[P][k] = it->second.variant;
                for (int v = 0; v < 4; ++v) c->tune_ms[P][k][v] = it->second.ms[v];
            }
        }
    }
    if (all) {
        c->tuned[P] = true;
        return EOFA_OK;
    }
    // operands: the inner vectors of P, or the context's FP64 work vectors
    VecRef odd_a, even_t, odd_b;
    if (P == EOFA_F64) {
        odd_a = c->x[1]; even_t = c->t[0]; odd_b = c->qo;
    } else {
        odd_a = c->inner[P].p; even_t = c->inner[P].t; odd_b = c->inner[P].q;
    }
    const size_t bytes = (size_t)c->n5 * 24 * kWidth[P];
    for (VecRef v : {odd_a, even_t, odd_b}) {
        CK(cudaMemsetAsync(v.d, 0, bytes, st), "memset");
        if (v.n) CK(cudaMemsetAsync(v.n, 0, sizeof(float) * c->n5, st), "memset");
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const VecRef none{};
    eofa_status s = EOFA_OK;
    for (int k = 0; k < 4 && s == EOFA_OK; ++k) {
        const bool even_out = (k == KIND_EO_MINV || k == KIND_EO_MINV_DAG);
        const int nvar = (P == EOFA_F64) ? 2 : 4;  // register-capped variants for FP32 arithmetic
        float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
        // three interleaved rounds; each variant keeps its fastest round
        for (int round = 0; round < (forced < 0 ? 3 : 1) && s == EOFA_OK; ++round) {
            for (int v = 0; v < nvar && s == EOFA_OK; ++v) {
                if (forced >= 0 && v != forced) continue;
                c->tuned[P] = true;
                c->tile[P][k] = v;
                auto launch = [&]() {
                    return even_out ? hop(c, P, k, 0, odd_a, none, even_t, red(c, FIN_NONE), nullptr, st)
                                    : hop(c, P, k, 1, even_t, odd_a, odd_b, red(c, FIN_NONE), nullptr, st);
                };
                if ((s = launch())) {  // warm-up; a variant the device cannot launch is skipped
                    if (v == 0 || forced >= 0) break;
                    cudaGetLastError();
                    c->err.clear();
                    s = EOFA_OK;
                    continue;
                }
                if (forced >= 0) continue;  // fixed variant: launched once, no timing
                cudaEventRecord(e0, st);
                for (int r = 0; r < 3 && s == EOFA_OK; ++r) s = launch();
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best[v] = std::min(best[v], ms);
            }
        }
        int best_v = 0;
        for (int v = 1; v < nvar; ++v)
            if (best[v] < best[best_v]) best_v = v;
        c->tile[P][k] = forced >= 0 ? forced : best_v;
        for (int v = 0; v < 4; ++v) c->tune_ms[P][k][v] = (forced < 0 && best[v] < 1e29f) ? best[v] / 3.f : 0.f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->launches = 0;
    if (s != EOFA_OK) {
        c->tuned[P] = false;
        return s;
    }
    c->tuned[P] = true;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int k = 0; k < 4; ++k) {
        TuneChoice& tc = g_tune_cache[{P, g.Ls, (long)g.X * g.Y, (long)g.Z * g.T, k}];
        tc.variant = c->tile[P][k];
        for (int v = 0; v < 4; ++v) tc.ms[v] = c->tune_ms[P][k][v];
    }
    return EOFA_OK;
}

typedef std::chrono::steady_clock Clock;

double since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

// Inner CGNR on the Schur complement in storage precision P, unit source in
// inner.r, solution in inner.x; stops at |r|^2 <= tol^2 (source norm 1).
// one CGNR iteration on the Schur complement (6 launches); every kernel
// returns at once when the device flag scal->done is set
// One CGNR iteration on the Schur complement (6 launches; every kernel
// returns at once when scal->done is set): q = S p (|q|^2 -> alpha),
// r -= alpha q (|r|^2: convergence), z = S^dag r (|z|^2 -> beta), then
// x += alpha p, p = z + beta p.
// ev (may be NULL): 8 events recorded around the four hop launches.
eofa_status cg_iteration(eofa_ctx* c, int P, cudaStream_t st, bool timed, cudaEvent_t* ev = nullptr) {
    Inner& in = c->inner[P];
    const int xp = P == EOFA_F64 ? EOFA_F64 : EOFA_F32;
    const int* done = &c->scal->done;
    const VecRef none{};
    const bool dn = c->method == 1;  // the four Schur halves of the chosen inner operator
    const int k0 = dn ? KIND_D_EO : KIND_EO_MINV, k1 = dn ? KIND_D_OE : KIND_OE_SCHUR;
    const int k2 = dn ? KIND_D_EO_DAG : KIND_EO_MINV_DAG, k3 = dn ? KIND_D_OE_DAG : KIND_OE_SCHUR_DAG;
    eofa_status s;
    auto mark = [&](int i) -> eofa_status {
        // External: under stream capture this becomes an event record node
        // (a plain record would only mark a capture dependency)
        if (ev) CK(cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
        return EOFA_OK;
    };
    if ((s = mark(0)) || (s = hop(c, P, k0, 0, in.p, none, in.t, red(c, FIN_NONE), done, st, timed)) ||
        (s = mark(1)))
        return s;
    if ((s = mark(2)) || (s = hop(c, P, k1, 1, in.t, in.p, in.q, red(c, FIN_ALPHA), done, st, timed)) ||
        (s = mark(3)))
        return s;
    CKL(blas_cg_r(P, in.q, in.r, c->n5, c->g.Ls, red(c, FIN_RR), done, st), "cg_r");
    if ((s = mark(4)) || (s = hop(c, P, k2, 0, in.r, none, in.t, red(c, FIN_NONE), done, st, timed)) ||
        (s = mark(5)))
        return s;
    if ((s = mark(6)) || (s = hop(c, P, k3, 1, in.t, in.r, in.z, red(c, FIN_BETA), done, st, timed)) ||
        (s = mark(7)))
        return s;
    CKL(blas_cg_px(P, xp, in.x, in.p, in.z, c->n5, c->g.Ls, red(c, FIN_STOP), st), "cg_px");
    return EOFA_OK;
}

// Start of an inner CGNR from x = 0 on the source in inner.r (scal already
// initialised): z = S^dag r (|z|^2 -> zz), p = z.  skip (may be NULL): every
// kernel returns at once while *skip is nonzero.
eofa_status cg_start(eofa_ctx* c, int P, const int* skip, cudaStream_t st) {
    Inner& in = c->inner[P];
    const int xp = P == EOFA_F64 ? EOFA_F64 : EOFA_F32;
    const VecRef none{};
    eofa_status s;
    const bool dn = c->method == 1;
    CKL(blas_zero(xp, in.x, c->n5, c->g.Ls, st, skip), "blas_zero");
    if ((s = hop(c, P, dn ? KIND_D_EO_DAG : KIND_EO_MINV_DAG, 0, in.r, none, in.t, red(c, FIN_NONE), skip, st)))
        return s;
    if ((s = hop(c, P, dn ? KIND_D_OE_DAG : KIND_OE_SCHUR_DAG, 1, in.t, in.r, in.z, red(c, FIN_ZZ), skip, st)))
        return s;
    CKL(blas_copy(P, in.p, P, in.z, c->n5, c->g.Ls, 1.0, -1, red(c, FIN_NONE), st, skip), "blas_copy");
    return EOFA_OK;
}

// After a graph-path inner solve: the four hop launches of its first
// iteration (their own small graph, with events; an iteration that always
// runs) are added to the timing totals.
eofa_status fold_graph_sample(eofa_ctx* c, int P) {
    for (int j = 0; j < 4; ++j) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->gev[P][2 * j], c->gev[P][2 * j + 1]), "cudaEventElapsedTime");
        c->hop_ms += ms;
        c->hop_launches += 1;
        c->hop_bytes += hop_bytes_of(c, P, j == 1 || j == 3);
    }
    return EOFA_OK;
}

constexpr int kChunk = 16;  // iterations per graph body / per host check

// Capture the CG loop of precision P once: a graph whose only node is a
// conditional WHILE; its body holds kChunk iterations and the condition
// kernel.  All pointers it bakes in belong to the context, so the graph is
// replayed by every later solve.
eofa_status build_cg_graph(eofa_ctx* c, int P) {
    if (c->cg_exec[c->method][P]) return EOFA_OK;
    if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    for (int i = 0; i < 8; ++i)
        if (!c->gev[P][i]) CK(cudaEventCreate(&c->gev[P][i]), "cudaEventCreate");
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0), "cudaGraphCreate");
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    // (the params union has no default constructor: zeroed raw storage)
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e, "conditional graph node");
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e, "cudaStreamBeginCaptureToGraph");
    }
    const long launches0 = c->launches;
    eofa_status s = EOFA_OK;
    for (int i = 0; i < kChunk && s == EOFA_OK; ++i) s = cg_iteration(c, P, c->cap, false);
    if (s == EOFA_OK) {
        e = while_cond(h, c->scal, c->cap);
        if (e != cudaSuccess) s = cuda_fail(c, e, "while_cond");
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap, &captured);
    c->launches = launches0;
    if (s == EOFA_OK && e2 != cudaSuccess) s = cuda_fail(c, e2, "cudaStreamEndCapture");
    if (s == EOFA_OK) {
        e = cudaGraphInstantiate(&c->cg_exec[c->method][P], g, 0);
        if (e != cudaSuccess) {
            c->cg_exec[c->method][P] = nullptr;
            s = cuda_fail(c, e, "cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(g);
    if (s != EOFA_OK) return s;
    // the first iteration of every inner solve runs as its own small graph
    // with events around its four hop launches: the timing sample
    cudaGraph_t g1 = nullptr;
    e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
    s = cg_iteration(c, P, c->cap, false, c->gev[P]);
    e2 = cudaStreamEndCapture(c->cap, &g1);
    c->launches = launches0;
    if (s == EOFA_OK && e2 != cudaSuccess) s = cuda_fail(c, e2, "cudaStreamEndCapture");
    if (s == EOFA_OK) {
        e = cudaGraphInstantiate(&c->cg_first[c->method][P], g1, 0);
        if (e != cudaSuccess) {
            c->cg_first[c->method][P] = nullptr;
            s = cuda_fail(c, e, "cudaGraphInstantiate");
        }
    }
    if (g1) cudaGraphDestroy(g1);
    if (s != EOFA_OK && c->cg_exec[c->method][P]) {
        cudaGraphExecDestroy(c->cg_exec[c->method][P]);
        c->cg_exec[c->method][P] = nullptr;
    }
    return s;
}

// Inner CGNR on the Schur complement in storage precision P, unit source in
// inner.r, solution in inner.x; stops at |r|^2 <= tol^2 (source norm 1).
// Without kernel timing the loop runs on the device (one graph launch, no
// host round trip); with timing it is driven from the host, with CUDA events
// around every hop kernel.
eofa_status run_cgnr(eofa_ctx* c, int P, double tol, int maxit, int* iters, double* rr_out, cudaStream_t st,
                     Clock::time_point t0, long timeout_ms) {
    eofa_status s;
    double left_ms = 0.0;
    if (timeout_ms > 0) {
        left_ms = (double)timeout_ms - since(t0) * 1e3;
        if (left_ms <= 0.0) return fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms");
    }
    CKL(scal_init(c->scal, tol * tol, maxit, (unsigned long long)(left_ms * 1e6), st), "scal_init");
    if ((s = cg_start(c, P, nullptr, st))) return s;
    *iters = 0;
    if (!c->timing) {
        if ((s = build_cg_graph(c, P))) return s;
        CK(cudaGraphLaunch(c->cg_first[c->method][P], st), "cudaGraphLaunch");
        CK(cudaGraphLaunch(c->cg_exec[c->method][P], st), "cudaGraphLaunch");
        if ((s = read_scal(c, st))) return s;
        const DevScal& h = *c->h_scal;
        *iters = h.iters;
        *rr_out = h.rr;
        if ((s = fold_graph_sample(c, P))) return s;
        c->launches += 6 + (long)(6 * kChunk + 1) * std::max(1, (h.iters - 1 + kChunk - 1) / kChunk);
        if (h.nonfinite) return fail(c, EOFA_ERR_NONFINITE, "NaN or Inf in the inner CG reductions");
        if (h.done) return EOFA_OK;
        if (h.timed_out) return fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms");
        return EOFA_ERR_NOT_CONVERGED;
    }
    for (;;) {
        for (int i = 0; i < kChunk; ++i)
            if ((s = cg_iteration(c, P, st, true))) return s;
        if ((s = read_scal(c, st))) return s;
        const DevScal& h = *c->h_scal;
        *iters = h.iters;
        *rr_out = h.rr;
        if (h.nonfinite) return fail(c, EOFA_ERR_NONFINITE, "NaN or Inf in the inner CG reductions");
        if (h.done) return EOFA_OK;
        if (h.iters >= maxit) return EOFA_ERR_NOT_CONVERGED;
        if (timeout_ms > 0 && since(t0) * 1e3 > (double)timeout_ms)
            return fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms");
    }
}

// flexible GCR with the learned preconditioner (defined with the learned
// preconditioner below): same contract as run_cgnr for P = FP32
eofa_status run_fgcr(eofa_ctx* c, double tol, int maxit, int* iters, cudaStream_t st, Clock::time_point t0,
                     long timeout_ms);

// Inner targets of the defect correction, per storage precision: the
// smallest that the inner CG still reaches reliably; 2e-6 lets two FP32
// inner solves reach 1e-10 (measured on the 16^3x32, Ls=16 workload:
// 2 outer steps at 2e-6 against 3 at 1e-5, same total inner iterations).
double default_inner_tol(int P) {
    switch (P) {
        case EOFA_F32: return 2e-6;
        case EOFA_F16: return 1e-3;
        case EOFA_BF16: return 1e-2;
        default: return 0.0;
    }
}

// State of one solve between its phases (shared by the single and the
// batched drivers).
struct SolveState {
    Clock::time_point t0;
    int P = 0, xp = 0, H = 1, maxit = 0, maxouter = 0;
    double bb = 0.0, rel = 1.0;
    int total = 0, outer = 0;
    eofa_status result = EOFA_ERR_NOT_CONVERGED;
    bool finished = false;
    bool x_zero = false;  // odd solution still zero: the outer residual is the source itself
};

eofa_status enqueue_read(eofa_ctx* c, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->h_scal, c->scal, sizeof(DevScal), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    return EOFA_OK;
}

// Phase 1: options, b = g5 R5 phi (H form) or b (K form) with |b|^2 into
// store[1] + store[2], the odd part of the initial guess, the even-odd
// source b~o = b_o + 1/2 D_h D~ M^-1 b_e.  Ends with a read-back enqueued.
// Dense Ls x Ls inverse by Gauss-Jordan elimination with partial pivoting
// (row-major, n <= 32); false when singular.
bool dense_inverse(int n, const double* a, double* inv) {
    double m[32][64];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) m[i][j] = j < n ? a[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (std::fabs(m[i][col]) > std::fabs(m[piv][col])) piv = i;
        if (!(std::fabs(m[piv][col]) > 1e-300)) return false;
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) std::swap(m[piv][j], m[col][j]);
        const double d = 1.0 / m[col][col];
        for (int j = 0; j < 2 * n; ++j) m[col][j] *= d;
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            const double f = m[i][col];
            if (f != 0.0)
                for (int j = 0; j < 2 * n; ++j) m[i][j] -= f * m[col][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = m[i][n + j];
    return true;
}

// The s-space blocks of the unpreconditioned even-odd scheme (App. B):
// the site-diagonal block of Eq. (non_hermit_sys) on chirality chi is
// A_chi = K_chi D~^-1, with K_chi = alpha + gamma L+ (+ the rank-one shift on
// the shift chirality) the site-diagonal block of the Cayley form and
// D~ = b5 + c5 L+ (mirrored coordinates, L+ with -m1 across the wall): the
// Cayley identity K = A D~ restricted to one site.  A_ee^-1 = D~ K_chi^-1
// and A_oo = K_chi D~^-1 are formed densely at set-up (FP64), as the dense
// scheme does, and the four dense kinds are launched once here, before any
// graph capture needs them.
eofa_status ensure_dense(eofa_ctx* c, cudaStream_t st) {
    if (c->dense_ready) return EOFA_OK;
    const int n = c->g.Ls;
    const SCoef<double>& k = c->c64;
    std::vector<double> dt(n * n, 0.0), kc(n * n), dti(n * n), kci(n * n);
    std::vector<double> host[2];  // [A_ee^-1, A_oo] as [chi][n][n]
    host[0].assign(2 * n * n, 0.0);
    host[1].assign(2 * n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        dt[i * n + i] = k.b5;
        if (i > 0) dt[i * n + i - 1] = k.c5;
    }
    dt[0 * n + n - 1] = -k.m * k.c5;
    if (!dense_inverse(n, dt.data(), dti.data())) return fail(c, EOFA_ERR_SINGULAR, "D~ is singular");
    for (int chi = 0; chi < 2; ++chi) {
        std::fill(kc.begin(), kc.end(), 0.0);
        for (int i = 0; i < n; ++i) {
            kc[i * n + i] = k.alpha;
            if (i > 0) kc[i * n + i - 1] = k.gamma;
        }
        kc[0 * n + n - 1] = -k.m * k.gamma;
        if (k.has_shift && chi == k.cs)
            for (int i = 0; i < n; ++i) kc[i * n + n - 1] += k.sbk * k.um[i];
        if (!dense_inverse(n, kc.data(), kci.data()))
            return fail(c, EOFA_ERR_SINGULAR, "site-diagonal block is singular");
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double ainv = 0.0, a = 0.0;
                for (int l = 0; l < n; ++l) {
                    ainv += dt[i * n + l] * kci[l * n + j];
                    a += kc[i * n + l] * dti[l * n + j];
                }
                host[0][(chi * n + i) * n + j] = ainv;
                host[1][(chi * n + i) * n + j] = a;
            }
    }
    for (int w = 0; w < 2; ++w) {
        std::vector<float> f(host[w].begin(), host[w].end());
        eofa_status s;
        // kept across eofa_set_system, which only changes their contents
        if (!c->dense[EOFA_F64][w] &&
            ((s = dalloc(c, &c->dense[EOFA_F64][w], sizeof(double) * 2 * n * n)) ||
             (s = dalloc(c, &c->dense[EOFA_F32][w], sizeof(float) * 2 * n * n))))
            return s;
        CK(cudaMemcpy(c->dense[EOFA_F64][w], host[w].data(), sizeof(double) * 2 * n * n, cudaMemcpyHostToDevice),
           "cudaMemcpy");
        CK(cudaMemcpy(c->dense[EOFA_F32][w], f.data(), sizeof(float) * 2 * n * n, cudaMemcpyHostToDevice),
           "cudaMemcpy");
    }
    const VecRef none{};
    eofa_status s0;
    if ((s0 = ensure_inner(c, EOFA_F32))) return s0;
    for (int P : {EOFA_F64, EOFA_F32}) {
        eofa_status s;
        // operands: the context's FP64 work vectors (before the solution is
        // imported), or the FP32 inner vectors
        const Inner& in = c->inner[EOFA_F32];
        const VecRef oa = P == EOFA_F64 ? c->x[1] : in.p, ev = P == EOFA_F64 ? c->t[0] : in.t,
                     ob = P == EOFA_F64 ? c->qo : in.q;
        const size_t bytes = (size_t)c->n5 * 24 * kWidth[P];
        for (VecRef v : {oa, ev, ob}) CK(cudaMemsetAsync(v.d, 0, bytes, st), "memset");
        if ((s = hop(c, P, KIND_D_EO, 0, oa, none, ev, red(c, FIN_NONE), nullptr, st)) ||
            (s = hop(c, P, KIND_D_OE, 1, ev, oa, ob, red(c, FIN_NONE), nullptr, st)) ||
            (s = hop(c, P, KIND_D_EO_DAG, 0, oa, none, ev, red(c, FIN_NONE), nullptr, st)) ||
            (s = hop(c, P, KIND_D_OE_DAG, 1, ev, oa, ob, red(c, FIN_NONE), nullptr, st)))
            return s;
    }
    CK(cudaStreamSynchronize(st), "sync");
    c->dense_ready = true;
    return EOFA_OK;
}

eofa_status solve_begin(eofa_ctx* c, const double* rhs, const double* sol, const eofa_solve_opts& o,
                        SolveState& ss, cudaStream_t st) {
    ss.t0 = Clock::now();
    c->exported = false;
    ss.P = o.inner;
    if (ss.P < 0 || ss.P > 3) return fail(c, EOFA_ERR_ARG, "opts.inner must be an eofa_prec");
    if (!(o.tol > 0.0)) return fail(c, EOFA_ERR_ARG, "opts.tol must be positive");
    if (o.precond != 0 && o.precond != 1) return fail(c, EOFA_ERR_ARG, "opts.precond must be 0 or 1");
    if (o.precond == 1) {
        if (!c->net_ready) return fail(c, EOFA_ERR_UNSUPPORTED, "no preconditioner: call eofa_set_preconditioner");
        if (ss.P != EOFA_F32) return fail(c, EOFA_ERR_UNSUPPORTED, "the learned preconditioner runs with inner FP32");
    }
    if (o.method != 0 && o.method != 1) return fail(c, EOFA_ERR_ARG, "opts.method must be 0 or 1");
    if (o.method == 1 && (ss.P > EOFA_F32 || o.precond != 0))
        return fail(c, EOFA_ERR_UNSUPPORTED, "the dense scheme runs with FP64 or FP32 inner and no preconditioner");
    c->method = o.method;
    ss.maxit = o.max_iter > 0 ? o.max_iter : 100000;
    ss.maxouter = o.max_outer > 0 ? o.max_outer : 100;
    ss.H = o.rhs_form == 0 ? 1 : 0;
    ss.xp = ss.P == EOFA_F64 ? EOFA_F64 : EOFA_F32;
    eofa_status s;
    if ((s = ensure_inner(c, ss.P))) return s;
    if ((s = autotune(c, ss.P, st)) || (s = autotune(c, EOFA_F64, st))) return s;
    if (c->method == 1 && (s = ensure_dense(c, st))) return s;
    c->timing = o.kernel_timing != 0;
    c->launches = 0;
    c->gcr_steps = c->gcr_fallbacks = 0;
    c->net_ms = 0.0;
    c->hop_ms = 0.0;
    c->hop_launches = 0;
    c->hop_bytes = 0.0;
    c->ev_used = 0;
    const VecRef none{};
    const Geom& g = c->g;
    const int Ls = g.Ls;
    CKL(layout_import(c->b[0], rhs, g, 0, ss.H, st), "import");
    CKL(layout_import(c->b[1], rhs, g, 1, ss.H, st), "import");
    CKL(blas_copy(0, c->t[0], 0, c->b[0], c->n5, Ls, 1.0, -1, red(c, FIN_STORE, 1), st), "norm");
    CKL(blas_copy(0, c->t[1], 0, c->b[1], c->n5, Ls, 1.0, -1, red(c, FIN_STORE, 2), st), "norm");
    if (o.use_guess) {
        CKL(layout_import(c->x[1], sol, g, 1, 0, st), "import");
        if (ss.H) {
            if ((s = hop(c, 0, KIND_LOC_DTINV, 1, none, c->x[1], c->t[1], red(c, FIN_NONE), nullptr, st)))
                return s;
            CKL(blas_copy(0, c->x[1], 0, c->t[1], c->n5, Ls, 1.0, -1, red(c, FIN_NONE), st), "copy");
        }
    } else {
        CKL(blas_zero(0, c->x[1], c->n5, Ls, st), "zero");
        ss.x_zero = true;
    }
    if ((s = hop(c, 0, KIND_LOC_DTMINV, 0, none, c->b[0], c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
    if ((s = hop(c, 0, KIND_SRC, 1, c->t[0], c->b[1], c->bto, red(c, FIN_NONE), nullptr, st))) return s;
    return enqueue_read(c, st);
}

// After the read-back of solve_begin: |b|^2, and the zero right-hand side.
eofa_status solve_check_rhs(eofa_ctx* c, double* sol, SolveState& ss, cudaStream_t st) {
    ss.bb = c->h_scal->store[1] + c->h_scal->store[2];
    if (!std::isfinite(ss.bb)) return fail(c, EOFA_ERR_NONFINITE, "right-hand side is not finite");
    if (ss.bb == 0.0) {
        CK(cudaMemsetAsync(sol, 0, (size_t)c->n5 * 2 * 24 * sizeof(double), st), "memset");
        ss.finished = true;
        ss.result = EOFA_OK;
        ss.rel = 0.0;
    }
    return EOFA_OK;
}

// r = b~o - S x_o in FP64 with |r|^2 into store[0]; read-back enqueued.
eofa_status outer_residual(eofa_ctx* c, const SolveState& ss, cudaStream_t st) {
    if (ss.x_zero) {  // r = b~o - S 0
        CKL(blas_copy(0, c->ro, 0, c->bto, c->n5, c->g.Ls, 1.0, -1, red(c, FIN_STORE, 0), st), "copy");
        return enqueue_read(c, st);
    }
    const VecRef none{};
    eofa_status s;
    if ((s = hop(c, 0, KIND_EO_MINV, 0, c->x[1], none, c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
    if ((s = hop(c, 0, KIND_OE_SCHUR, 1, c->t[0], c->x[1], c->qo, red(c, FIN_NONE), nullptr, st))) return s;
    CKL(blas_sub(c->ro, c->bto, c->qo, c->n5, c->g.Ls, red(c, FIN_STORE, 0), st), "sub");
    return enqueue_read(c, st);
}

// After the read-back of outer_residual: stop (converged, cap, timeout or
// non-finite) or go on.  Returns true when the outer loop must continue.
bool outer_decide(eofa_ctx* c, const eofa_solve_opts& o, SolveState& ss) {
    const double rr = c->h_scal->store[0];
    if (!std::isfinite(rr)) {
        ss.result = fail(c, EOFA_ERR_NONFINITE, "non-finite outer residual");
        return false;
    }
    ss.rel = std::sqrt(rr / ss.bb);
    if (ss.rel <= o.tol) { ss.result = EOFA_OK; return false; }
    if (ss.outer >= ss.maxouter || ss.total >= ss.maxit) {
        ss.result = fail(c, EOFA_ERR_NOT_CONVERGED, "iteration cap");
        return false;
    }
    if (o.timeout_ms > 0 && since(ss.t0) * 1e3 > (double)o.timeout_ms) {
        ss.result = fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms");
        return false;
    }
    return true;
}

double inner_tol_floor(const eofa_solve_opts& o, int P) {
    if (P == EOFA_F64) return 0.0;
    return o.inner_tol > 0.0 ? o.inner_tol : default_inner_tol(P);
}

// Phase 3: x_e = M^-1 (b_e + 1/2 D_h D~ x_o), the FP64 true residual of the
// full system, psi = D~ psi' (H form), export and statistics.
// host_sol (page-locked, may be NULL): the exported solution is copied there
// on the context's side stream, overlapping the true residual.
eofa_status solve_end(eofa_ctx* c, double* sol, const eofa_solve_opts& o, SolveState& ss,
                      eofa_solve_stats* stats, cudaStream_t st, double* host_sol = nullptr) {
    eofa_solve_stats S;
    std::memset(&S, 0, sizeof(S));
    const VecRef none{};
    const Geom& g = c->g;
    const int Ls = g.Ls;
    const size_t bytes = (size_t)c->n5 * 2 * 24 * sizeof(double);
    eofa_status s;
    if (host_sol && !c->side) {
        CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "cudaStreamCreate");
        for (auto& e : c->xev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (ss.bb == 0.0) {
        if (host_sol) CK(cudaMemcpyAsync(host_sol, sol, bytes, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(st), "sync");
        c->exported = true;
    } else {
        if ((s = hop(c, 0, KIND_RECON, 0, c->x[1], c->b[0], c->x[0], red(c, FIN_NONE), nullptr, st))) return s;
        // the solution first: psi = D~ psi' (H form) or psi' (K form)
        if (ss.H) {
            if ((s = hop(c, 0, KIND_LOC_DT, 0, none, c->x[0], c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
            if ((s = hop(c, 0, KIND_LOC_DT, 1, none, c->x[1], c->t[1], red(c, FIN_NONE), nullptr, st))) return s;
            CKL(layout_export(sol, c->t[0], g, 0, 0, st), "export");
            CKL(layout_export(sol, c->t[1], g, 1, 0, st), "export");
        } else {
            CKL(layout_export(sol, c->x[0], g, 0, 0, st), "export");
            CKL(layout_export(sol, c->x[1], g, 1, 0, st), "export");
        }
        c->exported = true;
        if (host_sol) {
            CK(cudaEventRecord(c->xev[0], st), "cudaEventRecord");
            CK(cudaStreamWaitEvent(c->side, c->xev[0], 0), "cudaStreamWaitEvent");
            CK(cudaMemcpyAsync(host_sol, sol, bytes, cudaMemcpyDeviceToHost, c->side), "cudaMemcpyAsync");
            CK(cudaEventRecord(c->xev[1], c->side), "cudaEventRecord");
        }
        // then the FP64 true residual of the full system
        if ((s = hop(c, 0, KIND_FULL, 0, c->x[1], c->x[0], c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
        if ((s = hop(c, 0, KIND_FULL, 1, c->x[0], c->x[1], c->t[1], red(c, FIN_NONE), nullptr, st))) return s;
        CKL(blas_sub(c->t[0], c->b[0], c->t[0], c->n5, Ls, red(c, FIN_STORE, 3), st), "sub");
        CKL(blas_sub(c->t[1], c->b[1], c->t[1], c->n5, Ls, red(c, FIN_STORE, 4), st), "sub");
        if (host_sol) CK(cudaStreamWaitEvent(st, c->xev[1], 0), "cudaStreamWaitEvent");
        if ((s = read_scal(c, st))) return s;
        S.true_res = std::sqrt((c->h_scal->store[3] + c->h_scal->store[4]) / ss.bb);
    }
    S.recur_res = ss.rel;
    S.outer_iters = ss.outer;
    S.inner_iters = ss.total;
    S.hop_ms = c->hop_ms;
    S.hop_launches = c->hop_launches;
    S.hop_bytes = c->hop_bytes;
    S.kernel_launches = c->launches;
    S.precond_iters = c->gcr_steps;
    S.precond_fallbacks = c->gcr_fallbacks;
    S.precond_ms = c->net_ms;
    eofa_status result = ss.result;
    if (result == EOFA_OK && ss.bb != 0.0 && !(S.true_res <= o.tol * 1.0000001))
        result = fail(c, EOFA_ERR_NOT_CONVERGED, "true residual above tol after the outer loop");
    S.status = result;
    S.seconds = since(ss.t0);
    if (stats) *stats = S;
    return result;
}

// host_sol: see solve_end; guess (may be NULL): where the initial guess is
// read instead of sol.
eofa_status solve_impl(eofa_ctx* c, const double* rhs, double* sol, const eofa_solve_opts& o,
                       eofa_solve_stats* stats, cudaStream_t st, double* host_sol = nullptr,
                       const double* guess = nullptr) {
    SolveState ss;
    eofa_status s;
    if ((s = solve_begin(c, rhs, guess ? guess : sol, o, ss, st))) return s;
    CK(cudaStreamSynchronize(st), "sync");
    if ((s = solve_check_rhs(c, sol, ss, st))) return s;
    const int Ls = c->g.Ls;
    while (!ss.finished) {
        if ((s = outer_residual(c, ss, st))) return s;
        CK(cudaStreamSynchronize(st), "sync");
        if (!outer_decide(c, o, ss)) break;
        const double itol = std::max(o.tol / ss.rel, inner_tol_floor(o, ss.P));
        // inner source r / |r| in precision P
        CKL(blas_copy(ss.P, c->inner[ss.P].r, 0, c->ro, c->n5, Ls, 1.0, 0, red(c, FIN_NONE), st), "copy");
        int its = 0;
        double irr = 0.0;
        eofa_status is = o.precond == 1
                             ? run_fgcr(c, itol, ss.maxit - ss.total, &its, st, ss.t0, o.timeout_ms)
                             : run_cgnr(c, ss.P, itol, ss.maxit - ss.total, &its, &irr, st, ss.t0, o.timeout_ms);
        ss.total += its;
        ++ss.outer;
        if (is == EOFA_ERR_NONFINITE || is == EOFA_ERR_TIMEOUT || is == EOFA_ERR_CUDA) {
            ss.result = is;
            break;
        }
        VecRef e = c->inner[ss.P].x;
        if (c->method == 1) {
            // the dense scheme's correction is in psi; the outer iterate is
            // psi' = D~^-1 psi
            if ((s = hop(c, ss.xp, KIND_LOC_DTINV, 1, VecRef{}, e, c->inner[ss.P].z, red(c, FIN_NONE), nullptr,
                         st)))
                return s;
            e = c->inner[ss.P].z;
        }
        CKL(blas_acc(c->x[1], ss.xp, e, c->n5, Ls, c->scal, 0, st), "acc");
        ss.x_zero = false;
    }
    return solve_end(c, sol, o, ss, stats, st, host_sol);
}

// ---------------------------------------------------------------------------
// batched solves: the whole FP64 defect correction of every system is one
// CUDA graph launch.  The graph holds, per system (parallel branches), the
// first FP64 residual and the first inner start, then a WHILE node whose
// body runs kChunk CG iterations of every system and, per system, the gate,
// the outer step (x += |r| e, FP64 residual r = b~o - S x_o) and the
// decision, which ends the system's outer loop or restarts its inner CGNR;
// a condition kernel over all systems closes the body.  Each phase's kernels
// return at once unless the system's device flags select them, so systems of
// different lattices, Ls and iteration counts advance independently.  The
// graph bakes in only context-owned buffers and is kept for later calls on
// the same contexts.
// ---------------------------------------------------------------------------
constexpr int kBatchMax = 32;

std::atomic<unsigned long long> g_ctx_uid{0};

struct BatchGraph {
    std::vector<unsigned long long> uids;
    int P = 0;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch_graphs;  // least recently used first
constexpr size_t kBatchGraphsKept = 4;

// Drop the kept batch graphs that involve a context (its operator changed
// or it is being destroyed).
void drop_batch_graphs(unsigned long long uid) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    for (size_t i = 0; i < g_batch_graphs.size();) {
        const auto& u = g_batch_graphs[i].uids;
        if (std::find(u.begin(), u.end(), uid) != u.end()) {
            cudaGraphExecDestroy(g_batch_graphs[i].exec);
            g_batch_graphs.erase(g_batch_graphs.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

// kernels of one system in one chunk of the batch graph (outer gate, step,
// decision and restart included), and of the first residual and start
constexpr int kBatchBodyKernels = 6 * kChunk + 11;
constexpr int kBatchStartKernels = 10;

// The outer step and the inner restart of system c in precision P: each
// kernel is gated by its device flag.
eofa_status batch_restart(eofa_ctx* c, int P, cudaStream_t st) {
    Inner& in = c->inner[P];
    const int* rs = &c->scal->o_skip_restart;
    CKL(blas_copy(P, in.r, 0, c->ro, c->n5, c->g.Ls, 1.0, 0, red(c, FIN_NONE), st, rs), "copy");
    return cg_start(c, P, rs, st);
}

eofa_status build_batch_graph(eofa_ctx* const* cs, int n, int P, cudaGraphExec_t* exec_out) {
    eofa_ctx* c = cs[0];  // errors are reported on the first context
    std::vector<cudaStream_t> str(n + 1, nullptr);
    std::vector<cudaEvent_t> evs(n + 1, nullptr);
    cudaGraph_t pro = nullptr, g = nullptr;
    eofa_status s = EOFA_OK;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        for (auto x : str) if (x) cudaStreamDestroy(x);
        for (auto x : evs) if (x) cudaEventDestroy(x);
        if (pro) cudaGraphDestroy(pro);
        if (g) cudaGraphDestroy(g);
    };
    for (int i = 0; i <= n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&str[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch streams"); }
    // fork/join capture helper: run f(i, stream) on a branch per system
    auto capture_branches = [&](auto&& f) -> eofa_status {
        cudaError_t ee = cudaEventRecord(evs[n], str[n]);
        for (int i = 0; i < n && ee == cudaSuccess; ++i) ee = cudaStreamWaitEvent(str[i], evs[n], 0);
        if (ee != cudaSuccess) return cuda_fail(c, ee, "fork");
        for (int i = 0; i < n; ++i) {
            eofa_status r = f(i, str[i]);
            if (r != EOFA_OK) return r;
        }
        for (int i = 0; i < n && ee == cudaSuccess; ++i) {
            ee = cudaEventRecord(evs[i], str[i]);
            if (ee == cudaSuccess) ee = cudaStreamWaitEvent(str[n], evs[i], 0);
        }
        return ee == cudaSuccess ? EOFA_OK : cuda_fail(c, ee, "join");
    };
    const VecRef none{};
    // first residual: r = b~o (no initial guess) or b~o - S x_o, then the
    // decision and the first inner start
    e = cudaStreamBeginCapture(str[n], cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "capture"); }
    s = capture_branches([&](int i, cudaStream_t st) -> eofa_status {
        eofa_ctx* ci = cs[i];
        DevScal* sc = ci->scal;
        eofa_status r;
        eofa_ctx* c = ci;  // CK/CKL report on this system
        CKL(blas_copy(0, ci->ro, 0, ci->bto, ci->n5, ci->g.Ls, 1.0, -1, red(ci, FIN_STORE, 0), st,
                      &sc->o_skip_copy), "copy");
        if ((r = hop(ci, 0, KIND_EO_MINV, 0, ci->x[1], none, ci->t[0], red(ci, FIN_NONE), &sc->o_skip_res, st)))
            return r;
        if ((r = hop(ci, 0, KIND_OE_SCHUR, 1, ci->t[0], ci->x[1], ci->qo, red(ci, FIN_NONE), &sc->o_skip_res, st)))
            return r;
        CKL(blas_sub(ci->ro, ci->bto, ci->qo, ci->n5, ci->g.Ls, red(ci, FIN_STORE, 0), st, &sc->o_skip_res), "sub");
        CKL(outer_decide_dev(sc, 1, st), "outer_decide");
        return batch_restart(ci, P, st);
    });
    cudaError_t e2 = cudaStreamEndCapture(str[n], &pro);
    if (s == EOFA_OK && e2 != cudaSuccess) s = cuda_fail(c, e2, "end capture");
    if (s != EOFA_OK) { cleanup(); return s; }
    // top graph: first residual and start (child graph) -> WHILE
    cudaGraphNode_t child, wn;
    e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, g, nullptr, 0, pro);
    cudaGraphConditionalHandle h;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    alignas(cudaGraphNodeParams) unsigned char npbuf[sizeof(cudaGraphNodeParams)];
    std::memset(npbuf, 0, sizeof(npbuf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(npbuf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wn, g, &child, nullptr, 1, &np);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "batch graph"); }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(str[n], body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(c, e, "capture body"); }
    const int xp = P == EOFA_F64 ? EOFA_F64 : EOFA_F32;
    s = capture_branches([&](int i, cudaStream_t st) -> eofa_status {
        eofa_ctx* ci = cs[i];
        DevScal* sc = ci->scal;
        eofa_ctx* c = ci;
        eofa_status r = EOFA_OK;
        for (int k = 0; k < kChunk && r == EOFA_OK; ++k) r = cg_iteration(ci, P, st, false);
        if (r != EOFA_OK) return r;
        CKL(outer_gate(sc, st), "outer_gate");
        const int* os = &sc->o_skip_step;
        CKL(blas_acc(ci->x[1], xp, ci->inner[P].x, ci->n5, ci->g.Ls, sc, 0, st, os), "acc");
        if ((r = hop(ci, 0, KIND_EO_MINV, 0, ci->x[1], none, ci->t[0], red(ci, FIN_NONE), os, st))) return r;
        if ((r = hop(ci, 0, KIND_OE_SCHUR, 1, ci->t[0], ci->x[1], ci->qo, red(ci, FIN_NONE), os, st))) return r;
        CKL(blas_sub(ci->ro, ci->bto, ci->qo, ci->n5, ci->g.Ls, red(ci, FIN_STORE, 0), st, os), "sub");
        CKL(outer_decide_dev(sc, 0, st), "outer_decide");
        return batch_restart(ci, P, st);
    });
    if (s == EOFA_OK) {
        ScalList L;
        std::memset(&L, 0, sizeof(L));
        L.n = n;
        for (int i = 0; i < n; ++i) L.s[i] = cs[i]->scal;
        e = outer_cond(h, L, str[n]);
        if (e != cudaSuccess) s = cuda_fail(c, e, "outer_cond");
    }
    cudaGraph_t cap = nullptr;
    e2 = cudaStreamEndCapture(str[n], &cap);
    if (s == EOFA_OK && e2 != cudaSuccess) s = cuda_fail(c, e2, "end capture body");
    if (s == EOFA_OK) {
        e = cudaGraphInstantiate(exec_out, g, 0);
        if (e != cudaSuccess) s = cuda_fail(c, e, "instantiate batch graph");
    }
    cleanup();
    return s;
}

// The kept graph of these contexts in precision P, built on first use.
eofa_status batch_graph(eofa_ctx* const* cs, int n, int P, cudaGraphExec_t* exec) {
    std::vector<unsigned long long> uids(n);
    for (int i = 0; i < n; ++i) uids[i] = cs[i]->uid;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (size_t i = 0; i < g_batch_graphs.size(); ++i)
            if (g_batch_graphs[i].P == P && g_batch_graphs[i].uids == uids) {
                BatchGraph b = g_batch_graphs[i];
                g_batch_graphs.erase(g_batch_graphs.begin() + (long)i);
                g_batch_graphs.push_back(b);
                *exec = b.exec;
                return EOFA_OK;
            }
    }
    cudaGraphExec_t x = nullptr;
    eofa_status s = build_batch_graph(cs, n, P, &x);
    if (s != EOFA_OK) return s;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    if (g_batch_graphs.size() >= kBatchGraphsKept) {
        cudaGraphExecDestroy(g_batch_graphs.front().exec);
        g_batch_graphs.erase(g_batch_graphs.begin());
    }
    BatchGraph b;
    b.uids = uids;
    b.P = P;
    b.exec = x;
    g_batch_graphs.push_back(b);
    *exec = x;
    return EOFA_OK;
}

// *failed: the system whose context holds the message of a failing status
// (0 for failures of the batch as a whole, reported on cs[0]).
eofa_status solve_batched_impl(eofa_ctx* const* cs, int n, const void* const* rhs, void* const* sol,
                               const eofa_solve_opts& o, eofa_solve_stats* stats, cudaStream_t st,
                               int* failed) {
    std::vector<SolveState> ss(n);
    eofa_status s;
    *failed = 0;
    for (int i = 0; i < n; ++i) {
        cs[i]->err.clear();
        if ((s = solve_begin(cs[i], (const double*)rhs[i], (const double*)sol[i], o, ss[i], st))) {
            *failed = i;
            return s;
        }
    }
    {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(cs[0], e, "batched solve start");
    }
    for (int i = 0; i < n; ++i)
        if ((s = solve_check_rhs(cs[i], (double*)sol[i], ss[i], st))) {
            *failed = i;
            return s;
        }
    const int P = ss[0].P;
    std::vector<long> launches0(n);
    for (int i = 0; i < n; ++i) launches0[i] = cs[i]->launches;
    cudaGraphExec_t exec = nullptr;
    s = batch_graph(cs, n, P, &exec);
    for (int i = 0; i < n; ++i) cs[i]->launches = launches0[i];  // the capture launched nothing
    if (s != EOFA_OK) return s;
    // every system's options, deadline and first-residual form, then the
    // one launch of the whole defect correction
    const int body_cap = ss[0].maxit / kChunk + ss[0].maxouter + 4;
    for (int i = 0; i < n; ++i) {
        eofa_ctx* c = cs[i];
        unsigned long long tns = 0;
        if (o.timeout_ms > 0) {
            const double left_ms = (double)o.timeout_ms - since(ss[i].t0) * 1e3;
            tns = left_ms > 1e-6 ? (unsigned long long)(left_ms * 1e6) : 1ull;
        }
        CKL(outer_begin(c->scal, o.tol, inner_tol_floor(o, P), ss[i].maxit, ss[i].maxouter, tns,
                        ss[i].finished ? 1 : 0, ss[i].x_zero ? 1 : 0, body_cap, st), "outer_begin");
    }
    if (const cudaError_t e = cudaGraphLaunch(exec, st); e != cudaSuccess)
        return cuda_fail(cs[0], e, "batched graph launch");
    for (int i = 0; i < n; ++i)
        if ((s = enqueue_read(cs[i], st))) return s;
    if (const cudaError_t e = cudaStreamSynchronize(st); e != cudaSuccess)
        return cuda_fail(cs[0], e, "batched solve");
    const int chunks = cs[0]->h_scal->o_body;
    for (int i = 0; i < n; ++i) {
        eofa_ctx* c = cs[i];
        const DevScal& h = *c->h_scal;
        c->launches += kBatchStartKernels + (long)kBatchBodyKernels * chunks + (i == 0 ? chunks : 0);
        if (ss[i].finished) continue;  // zero right-hand side
        ss[i].outer = h.outer;
        ss[i].total = h.total;
        ss[i].rel = h.rel;
        ss[i].finished = true;
        switch (h.o_status) {
            case EOFA_OK: ss[i].result = EOFA_OK; break;
            case EOFA_ERR_NONFINITE:
                ss[i].result = fail(c, EOFA_ERR_NONFINITE, "NaN or Inf in the defect correction");
                break;
            case EOFA_ERR_TIMEOUT: ss[i].result = fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms"); break;
            default: ss[i].result = fail(c, EOFA_ERR_NOT_CONVERGED, "iteration cap"); break;
        }
    }
    eofa_status first = EOFA_OK;
    for (int i = 0; i < n; ++i) {
        s = solve_end(cs[i], (double*)sol[i], o, ss[i], stats ? stats + i : nullptr, st);
        if (s != EOFA_OK && first == EOFA_OK) {
            first = s;
            *failed = i;
        }
    }
    return first;
}

eofa_status apply_impl(eofa_ctx* c, const void* in, void* out, int which, cudaStream_t st) {
    // which: 0 = K, 1 = K^dag, 2 = H + beta Delta P = g5 R5 K D~^-1
    const Geom& g = c->g;
    const VecRef none{};
    eofa_status s;
    CKL(layout_import(c->x[0], (const double*)in, g, 0, 0, st), "import");
    CKL(layout_import(c->x[1], (const double*)in, g, 1, 0, st), "import");
    if (which == 2) {
        if ((s = hop(c, 0, KIND_LOC_DTINV, 0, none, c->x[0], c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
        if ((s = hop(c, 0, KIND_LOC_DTINV, 1, none, c->x[1], c->t[1], red(c, FIN_NONE), nullptr, st))) return s;
        if ((s = hop(c, 0, KIND_FULL, 0, c->t[1], c->t[0], c->x[0], red(c, FIN_NONE), nullptr, st))) return s;
        if ((s = hop(c, 0, KIND_FULL, 1, c->t[0], c->t[1], c->x[1], red(c, FIN_NONE), nullptr, st))) return s;
        CKL(layout_export((double*)out, c->x[0], g, 0, 1, st), "export");
        CKL(layout_export((double*)out, c->x[1], g, 1, 1, st), "export");
        return EOFA_OK;
    }
    const int kind = which == 0 ? KIND_FULL : KIND_FULL_DAG;
    if ((s = hop(c, 0, kind, 0, c->x[1], c->x[0], c->t[0], red(c, FIN_NONE), nullptr, st))) return s;
    if ((s = hop(c, 0, kind, 1, c->x[0], c->x[1], c->t[1], red(c, FIN_NONE), nullptr, st))) return s;
    CKL(layout_export((double*)out, c->t[0], g, 0, 0, st), "export");
    CKL(layout_export((double*)out, c->t[1], g, 1, 0, st), "export");
    return EOFA_OK;
}

// ---------------------------------------------------------------------------
// EOFA action M_EOFA and heatbath (Eqs. eofa_action, eofa_heatbath)
// ---------------------------------------------------------------------------
// App. A, Moebius kernel, with c + d = b5, c - d = c5:
// Omega_+(s) = (-1)^(s+1) c5^(Ls-s-1) / b5^(Ls-s),  Omega_-(s) = (-1)^s c5^s / b5^(s+1)
OmegaW omega_of(const eofa_params& p, int pm) {
    OmegaW o{};
    const int Ls = p.Ls;
    for (int s = 0; s < Ls; ++s) {
        if (pm > 0)
            o.w[s] = ((s + 1) & 1 ? -1.0 : 1.0) * std::pow(p.c, Ls - s - 1) / std::pow(p.b, Ls - s);
        else
            o.w[s] = (s & 1 ? -1.0 : 1.0) * std::pow(p.c, s) / std::pow(p.b, s + 1);
    }
    return o;
}

// App. A: k = 2c (m2 - m1) (c+d)^(2Ls) / (N(m1) N(m2)), N(m) = b5^Ls + m c5^Ls, 2c = b5 + c5
double k_of(const eofa_params& p, double m1, double m2) {
    const double bl = std::pow(p.b, p.Ls), cl = std::pow(p.c, p.Ls);
    return (p.b + p.c) * (m2 - m1) * bl * bl / ((bl + m1 * cl) * (bl + m2 * cl));
}

void drop_graphs(eofa_ctx* c) {
    for (int m = 0; m < 2; ++m)
        for (int i = 0; i < 4; ++i) {
            if (c->cg_exec[m][i]) cudaGraphExecDestroy(c->cg_exec[m][i]);
            if (c->cg_first[m][i]) cudaGraphExecDestroy(c->cg_first[m][i]);
            c->cg_exec[m][i] = c->cg_first[m][i] = nullptr;
        }
    drop_batch_graphs(c->uid);
}

// Make the context solve H(mh) + beta Delta_pm(ma, mb) P_pm on its lattice
// and gauge field: new fifth-dimension coefficients.  The captured CG graphs
// hold the old ones as kernel arguments and the dense comparison matrices
// are built from them, so both are rebuilt on next use.
eofa_status set_system(eofa_ctx* c, const eofa_params& np) {
    if (np.pm != 1 && np.pm != -1) return fail(c, EOFA_ERR_ARG, "pm must be +1 or -1");
    if (!std::isfinite(np.m1) || !std::isfinite(np.m2) || !std::isfinite(np.m3) || !std::isfinite(np.beta))
        return fail(c, EOFA_ERR_ARG, "masses and beta must be finite");
    const eofa_params& o = c->p;
    if (np.m1 == o.m1 && np.m2 == o.m2 && np.m3 == o.m3 && np.beta == o.beta && np.pm == o.pm) return EOFA_OK;
    SCoef<double> k64;
    const char* why = "";
    eofa_status s = coef_from_params(np, k64, &why);
    if (s != EOFA_OK) return fail(c, s, why);
    c->p = np;
    c->c64 = k64;
    cast_coef(c->c64, c->c32);
    drop_graphs(c);
    c->dense_ready = false;
    return EOFA_OK;
}

eofa_status set_system(eofa_ctx* c, double mh, double ma, double mb, double beta, int pm) {
    eofa_params np = c->p;
    np.m1 = mh;
    np.m2 = ma;
    np.m3 = mb;
    np.beta = beta;
    np.pm = pm;
    return set_system(c, np);
}

// i-th canonical complex128 5D work field of the action calls
double* act_buf(eofa_ctx* c, size_t i) {
    while (c->act5.size() <= i) {
        void* p = nullptr;
        if (dalloc(c, &p, (size_t)c->n5 * 2 * 24 * sizeof(double)) != EOFA_OK) return nullptr;
        c->act5.push_back((double*)p);
    }
    return c->act5[i];
}

bool hard_error(eofa_status s) { return s != EOFA_OK && s != EOFA_ERR_NOT_CONVERGED; }

eofa_status solve_one(eofa_ctx* c, const double* rhs, double* sol, const eofa_solve_opts& o, eofa_solve_stats* stats,
                      cudaStream_t st) {
    eofa_status s = solve_impl(c, rhs, sol, o, stats, st);
    if (stats) stats->status = s;
    return s;
}

// the multi-dot partial sums and results of the context (allocated on first use)
eofa_status ensure_mdot(eofa_ctx* c) {
    if (c->mdot) return EOFA_OK;
    void* p = nullptr;
    eofa_status s = dalloc(c, &p, sizeof(double2) * (kMultiBlocks + 1) * kMultiMax);
    if (s != EOFA_OK) return s;
    c->mdot = (double*)p;
    return EOFA_OK;
}

// Chronological initial guess (Sec. V.B): with the previous solutions psi_k
// of the same term, x0 = sum_k c_k psi_k where
// sum_k c_k psi_l^dag A psi_k = psi_l^dag rhs, A the current system (H form);
// the small system by Gauss-Jordan elimination with partial pivoting.
// Returns false (no guess) when that system is numerically singular.
eofa_status forecast(eofa_ctx* c, double* const* prev, int n, const double* rhs, double* guess, bool* used,
                     cudaStream_t st) {
    *used = false;
    if (n < 1) return EOFA_OK;
    const long nc = c->n5 * 2 * 12;  // complex elements of a 5D field
    double* w = act_buf(c, 2);
    if (!w) return EOFA_ERR_OOM;
    eofa_status s0 = ensure_mdot(c);
    if (s0 != EOFA_OK) return s0;
    double* res = c->mdot + 2 * kMultiBlocks * kMultiMax;
    VecSet set{};
    set.n = n;
    for (int l = 0; l < n; ++l) set.v[l] = (const double2*)prev[l];
    std::vector<double> G(2 * n * n), b(2 * n), tmp(2 * kMultiMax);
    eofa_status s;
    for (int k = 0; k <= n; ++k) {
        const double* rhsk = rhs;
        if (k < n) {
            if ((s = apply_impl(c, prev[k], w, 2, st))) return s;
            rhsk = w;
        }
        CK(multidot(set, rhsk, nc, c->mdot, res, st), "multidot");
        c->launches += 2;
        CK(cudaMemcpyAsync(tmp.data(), res, sizeof(double2) * n, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(st), "sync");
        for (int l = 0; l < n; ++l) {
            double* dst = k < n ? &G[2 * (l * n + k)] : &b[2 * l];
            dst[0] = tmp[2 * l];
            dst[1] = tmp[2 * l + 1];
        }
    }
    // Gauss-Jordan on [G | b], complex entries as (re, im) pairs
    auto at = [&](int i, int j) -> double* { return &G[2 * (i * n + j)]; };
    double scale = 0.0;
    for (int i = 0; i < n * n; ++i) scale = std::max(scale, std::hypot(G[2 * i], G[2 * i + 1]));
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = 0.0;
        for (int i = col; i < n; ++i) {
            const double a = std::hypot(at(i, col)[0], at(i, col)[1]);
            if (a > best) best = a, piv = i;
        }
        if (!(best > 1e-13 * scale)) return EOFA_OK;
        if (piv != col) {
            for (int j = 0; j < n; ++j) std::swap(at(piv, j)[0], at(col, j)[0]), std::swap(at(piv, j)[1], at(col, j)[1]);
            std::swap(b[2 * piv], b[2 * col]);
            std::swap(b[2 * piv + 1], b[2 * col + 1]);
        }
        const double pr = at(col, col)[0], pi = at(col, col)[1], d = pr * pr + pi * pi;
        const double ir = pr / d, ii = -pi / d;  // 1 / pivot
        for (int j = 0; j < n; ++j) {
            double* e = at(col, j);
            const double er = e[0] * ir - e[1] * ii, ei = e[0] * ii + e[1] * ir;
            e[0] = er, e[1] = ei;
        }
        {
            const double br = b[2 * col] * ir - b[2 * col + 1] * ii, bi = b[2 * col] * ii + b[2 * col + 1] * ir;
            b[2 * col] = br, b[2 * col + 1] = bi;
        }
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            const double fr = at(i, col)[0], fi = at(i, col)[1];
            for (int j = 0; j < n; ++j) {
                const double* r = at(col, j);
                at(i, j)[0] -= fr * r[0] - fi * r[1];
                at(i, j)[1] -= fr * r[1] + fi * r[0];
            }
            b[2 * i] -= fr * b[2 * col] - fi * b[2 * col + 1];
            b[2 * i + 1] -= fr * b[2 * col + 1] + fi * b[2 * col];
        }
    }
    for (int l = 0; l < n; ++l) set.c[l] = make_double2(b[2 * l], b[2 * l + 1]);
    CKL(combine(guess, set, nc, st), "combine");
    *used = true;
    return EOFA_OK;
}

// M_EOFA(m1, m2) phi, Eq. (eofa_action): two H-form solves on the
// Omega_pm P_pm phi sources; the context's own system is restored by the
// caller.
eofa_status meofa_impl(eofa_ctx* c, double m1, double m2, const double* phi, double* out, const eofa_solve_opts& o0,
                       eofa_solve_stats* stats, cudaStream_t st) {
    const long V = 2L * c->g.Vh;
    const int Ls = c->g.Ls;
    eofa_solve_opts o = o0;
    o.rhs_form = 0;
    o.use_guess = 0;
    double* src = act_buf(c, 0);
    double* x = act_buf(c, 1);
    if (!src || !x) return EOFA_ERR_OOM;
    const double k = k_of(c->p, m1, m2);
    const OmegaW om_m = omega_of(c->p, -1), om_p = omega_of(c->p, +1);
    eofa_status s, first = EOFA_OK;
    // - k P_- Omega_-^dag H(m1)^-1 Omega_- P_- phi
    if ((s = set_system(c, m1, m1, m2, 0.0, -1))) return s;
    CKL(omega_in(src, phi, om_m, -1, V, Ls, st), "omega_in");
    s = solve_one(c, src, x, o, stats ? stats + 0 : nullptr, st);
    if (hard_error(s)) return s;
    if (s != EOFA_OK) first = s;
    CKL(omega_out(out, phi, 1.0, x, om_m, -1, -k, V, Ls, st), "omega_out");
    // + k P_+ Omega_+^dag [H(m2) - Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ phi
    if ((s = set_system(c, m2, m1, m2, -1.0, +1))) return s;
    CKL(omega_in(src, phi, om_p, +1, V, Ls, st), "omega_in");
    s = solve_one(c, src, x, o, stats ? stats + 1 : nullptr, st);
    if (hard_error(s)) return s;
    if (s != EOFA_OK && first == EOFA_OK) first = s;
    CKL(omega_out(out, out, 1.0, x, om_p, +1, k, V, Ls, st), "omega_out");
    CK(cudaStreamSynchronize(st), "sync");
    return first;
}

// EOFA pseudofermion force, Eq. (eofa_force): chi_1 = H(m1)^-1 Omega_- P_- phi,
// chi_2 = [H(m2) - Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ phi, then one kernel
// over the links.  D_EOFA(m) = D_DWF(m) D~(m)^-1 and D_DWF = D_W D~ + (1 - L)
// make the gauge derivative of D_EOFA that of D_W on every s-slice, for
// Moebius as for Shamir.
eofa_status force_impl(eofa_ctx* c, double m1, double m2, const double* phi, double* F, const eofa_solve_opts& o0,
                       eofa_solve_stats* stats, cudaStream_t st) {
    const long V = 2L * c->g.Vh;
    const int Ls = c->g.Ls;
    eofa_solve_opts o = o0;
    o.rhs_form = 0;
    o.use_guess = 0;
    double* src = act_buf(c, 0);
    double* chi1 = act_buf(c, 1);
    double* chi2 = act_buf(c, 3);
    if (!src || !chi1 || !chi2) return EOFA_ERR_OOM;
    const double k = k_of(c->p, m1, m2);
    eofa_status s, first = EOFA_OK;
    if ((s = set_system(c, m1, m1, m2, 0.0, -1))) return s;
    CKL(omega_in(src, phi, omega_of(c->p, -1), -1, V, Ls, st), "omega_in");
    s = solve_one(c, src, chi1, o, stats ? stats + 0 : nullptr, st);
    if (hard_error(s)) return s;
    if (s != EOFA_OK) first = s;
    if ((s = set_system(c, m2, m1, m2, -1.0, +1))) return s;
    CKL(omega_in(src, phi, omega_of(c->p, +1), +1, V, Ls, st), "omega_in");
    s = solve_one(c, src, chi2, o, stats ? stats + 1 : nullptr, st);
    if (hard_error(s)) return s;
    if (s != EOFA_OK && first == EOFA_OK) first = s;
    const void* l64[2] = {c->links[EOFA_F64][0], c->links[EOFA_F64][1]};
    if (c->g.gpmask) {
        // the stacked lattice's force (2 V links) in a work field, folded
        // onto the physical links
        double* Fs = act_buf(c, 2);
        if (!Fs) return EOFA_ERR_OOM;
        CKL(eofa_force_links(chi1, chi2, l64, Fs, c->g, k, st), "force");
        CKL(force_fold(Fs, F, V / 2 * 4 * 9, st), "force fold");
    } else {
        CKL(eofa_force_links(chi1, chi2, l64, F, c->g, k, st), "force");
    }
    CK(cudaStreamSynchronize(st), "sync");
    return first;
}

// phi = M_EOFA^(-1/2) eta by Eq. (eofa_heatbath): 2 np H-form solves, pole
// by pole, the minus term then the plus term; with nf > 0 each solve starts
// from the chronological guess built on the last nf solutions of its own term.
eofa_status heatbath_impl(eofa_ctx* c, double m1, double m2, int np, const double* alpha, const double* beta,
                          const double* pole_tol, int nf, const double* eta, double* phi, const eofa_solve_opts& o0,
                          eofa_solve_stats* stats, cudaStream_t st) {
    const long V = 2L * c->g.Vh;
    const int Ls = c->g.Ls;
    const double k = k_of(c->p, m1, m2);
    const OmegaW om_m = omega_of(c->p, -1), om_p = omega_of(c->p, +1);
    double a_tot = alpha[0];
    for (int l = 0; l < np; ++l) a_tot += alpha[l + 1] / (1.0 + beta[l]);
    // phi = (alpha_0 + sum_l alpha_l gamma_l) eta, then the 2 np solve terms
    CKL(omega_out(phi, eta, a_tot, nullptr, om_m, -1, 0.0, V, Ls, st), "omega_out");
    if (np == 0) {
        CK(cudaStreamSynchronize(st), "sync");
        return EOFA_OK;
    }
    double* src[2] = {act_buf(c, 0), act_buf(c, 1)};
    double* x1 = act_buf(c, 3);
    std::vector<double*> ring[2];
    for (int t = 0; t < 2; ++t)
        for (int j = 0; j < nf; ++j) ring[t].push_back(act_buf(c, 4 + t * nf + j));
    if (!src[0] || !src[1] || !x1) return EOFA_ERR_OOM;
    for (auto& r : ring)
        for (double* p : r)
            if (!p) return EOFA_ERR_OOM;
    CKL(omega_in(src[0], eta, om_m, -1, V, Ls, st), "omega_in");
    CKL(omega_in(src[1], eta, om_p, +1, V, Ls, st), "omega_in");
    eofa_status s, first = EOFA_OK;
    for (int l = 0; l < np; ++l) {
        const double g = 1.0 / (1.0 + beta[l]);
        const double cl = alpha[l + 1] * g * k * g;
        for (int t = 0; t < 2; ++t) {
            // t = 0: [H(m1) - gamma_l Delta_-(m1, m2) P_-]^-1, coefficient + alpha_l gamma_l^2 k
            // t = 1: [H(m2) - beta_l gamma_l Delta_+(m1, m2) P_+]^-1, coefficient - alpha_l gamma_l^2 k
            if (t == 0) s = set_system(c, m1, m1, m2, -g, -1);
            else s = set_system(c, m2, m1, m2, -beta[l] * g, +1);
            if (s) return s;
            eofa_solve_opts o = o0;
            o.rhs_form = 0;
            o.use_guess = 0;
            if (pole_tol && pole_tol[2 * l + t] > 0.0) o.tol = pole_tol[2 * l + t];
            double* x = nf ? ring[t][l % nf] : x1;
            if (nf) {
                // the previous solutions, oldest first; the slot written now
                // may still hold the oldest one (combine reads it before the
                // solve overwrites it)
                const int have = std::min(l, nf);
                std::vector<double*> prev;
                for (int j = l - have; j < l; ++j) prev.push_back(ring[t][j % nf]);
                bool used = false;
                if ((s = forecast(c, prev.data(), have, src[t], x, &used, st))) return s;
                o.use_guess = used ? 1 : 0;
            }
            eofa_solve_stats* sp = stats ? stats + 2 * l + t : nullptr;
            s = solve_one(c, src[t], x, o, sp, st);
            if (hard_error(s)) return s;
            if (s != EOFA_OK && first == EOFA_OK) first = s;
            CKL(omega_out(phi, phi, 1.0, x, t == 0 ? om_m : om_p, t == 0 ? -1 : +1, t == 0 ? cl : -cl, V, Ls, st),
                "omega_out");
        }
    }
    CK(cudaStreamSynchronize(st), "sync");
    return first;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

// gpmask = 0: the single-flavour lattice of p; otherwise G-parity in the
// directions of gpmask with the two flavours stacked along t
static eofa_status create_impl(const eofa_params* p, const void* gauge, int gpmask, void* stream, eofa_ctx** out) {
    if (!out) return EOFA_ERR_ARG;
    *out = nullptr;
    if (!p || !gauge) return EOFA_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (p->dims[i] < 2 || (p->dims[i] & 1)) return EOFA_ERR_ARG;
    if (p->pm != 1 && p->pm != -1) return EOFA_ERR_ARG;
    if (p->t_bc != 1 && p->t_bc != -1) return EOFA_ERR_ARG;
    if (p->Ls != 4 && p->Ls != 8 && p->Ls != 12 && p->Ls != 16) return EOFA_ERR_UNSUPPORTED;
    eofa_ctx* c = new (std::nothrow) eofa_ctx();
    if (!c) return EOFA_ERR_OOM;
    c->uid = ++g_ctx_uid;
    c->p = *p;
    Geom& g = c->g;
    g.X = p->dims[0]; g.Y = p->dims[1]; g.Z = p->dims[2];
    g.Tp = p->dims[3];
    g.T = gpmask ? 2 * g.Tp : g.Tp;
    g.gpmask = gpmask;
    g.Xh = g.X / 2;
    const long V = (long)g.X * g.Y * g.Z * g.T;
    if (V / 2 > (1L << 30)) { delete c; return EOFA_ERR_UNSUPPORTED; }
    g.Vh = (int)(V / 2);
    g.Ls = p->Ls;
    g.apmask = p->t_bc == -1 ? 8 : 0;
    c->n5 = (long)g.Vh * g.Ls;
    eofa_status s = build_coef(c);
    cudaStream_t st = (cudaStream_t)stream;
    auto bail = [&](eofa_status e) { eofa_destroy(c); return e; };
    if (s != EOFA_OK) return bail(s);
    for (int pr = 0; pr < 4; ++pr)
        for (int par = 0; par < 2; ++par)
            if ((s = dalloc(c, &c->links[pr][par], (size_t)g.Vh * 4 * 12 * kWidth[pr]))) return bail(s);
    for (int par = 0; par < 2; ++par) {
        if ((s = vec_alloc(c, 0, &c->b[par])) || (s = vec_alloc(c, 0, &c->x[par])) ||
            (s = vec_alloc(c, 0, &c->t[par])))
            return bail(s);
    }
    if ((s = vec_alloc(c, 0, &c->ro)) || (s = vec_alloc(c, 0, &c->bto)) || (s = vec_alloc(c, 0, &c->qo)))
        return bail(s);
    const int maxgrid = std::max(blas_max_grid(c->n5), g.Vh / 8 + 2);
    void* tmp = nullptr;
    if ((s = dalloc(c, &tmp, sizeof(double) * maxgrid))) return bail(s);
    c->partials = (double*)tmp;
    if ((s = dalloc(c, &tmp, 256))) return bail(s);
    c->counter = (unsigned*)tmp;
    if ((s = dalloc(c, &tmp, sizeof(DevScal)))) return bail(s);
    c->scal = (DevScal*)tmp;
    if ((s = dalloc(c, &tmp, 256))) return bail(s);
    c->d_flag = (int*)tmp;
    if (cudaMallocHost((void**)&c->h_scal, sizeof(DevScal)) != cudaSuccess) return bail(EOFA_ERR_OOM);
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->counter, 0, 256, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_flag, 0, 256, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->scal, 0, sizeof(DevScal), st)) != cudaSuccess)
        return bail(cuda_fail(c, e, "memset"));
    void* stacked = nullptr;  // G-parity: [U; U*], freed once imported
    if (gpmask) {
        const long n = (V / 2) * 4 * 9;  // complex entries of the physical U
        if ((e = cudaMalloc(&stacked, (size_t)n * 2 * 2 * sizeof(double))) != cudaSuccess)
            return bail(cuda_fail(c, e, "cudaMalloc"));
        if ((e = gparity_gauge((const double*)gauge, (double*)stacked, n, st)) != cudaSuccess) {
            cudaFree(stacked);
            return bail(cuda_fail(c, e, "G-parity gauge"));
        }
    }
    e = gauge_import(stacked ? (const double*)stacked : (const double*)gauge, g, c->links, c->d_flag, st);
    if (stacked) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFree(stacked);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "gauge import"));
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(c, e, "gauge check"));
    if (bad) return bail(EOFA_ERR_ARG);
    *out = c;
    return EOFA_OK;
}

eofa_status eofa_create(const eofa_params* p, const void* gauge, void* stream, eofa_ctx** out) {
    return create_impl(p, gauge, 0, stream, out);
}

eofa_status eofa_create_gparity(const eofa_params* p, const void* gauge, int gparity_dirs, void* stream,
                                eofa_ctx** out) {
    if (out) *out = nullptr;
    if (gparity_dirs < 1 || gparity_dirs > 15) return EOFA_ERR_ARG;
    return create_impl(p, gauge, gparity_dirs, stream, out);
}

eofa_status eofa_apply(eofa_ctx* ctx, const void* in, void* out, void* stream) {
    if (!ctx || !in || !out || in == out) return EOFA_ERR_ARG;
    return apply_impl(ctx, in, out, 0, (cudaStream_t)stream);
}

eofa_status eofa_apply_dag(eofa_ctx* ctx, const void* in, void* out, void* stream) {
    if (!ctx || !in || !out || in == out) return EOFA_ERR_ARG;
    return apply_impl(ctx, in, out, 1, (cudaStream_t)stream);
}

eofa_status eofa_apply_h(eofa_ctx* ctx, const void* in, void* out, void* stream) {
    if (!ctx || !in || !out || in == out) return EOFA_ERR_ARG;
    return apply_impl(ctx, in, out, 2, (cudaStream_t)stream);
}

eofa_status eofa_solve(eofa_ctx* ctx, const void* rhs, void* sol, const eofa_solve_opts* opts,
                       eofa_solve_stats* stats, void* stream) {
    if (!ctx || !rhs || !sol || !opts || rhs == sol) return EOFA_ERR_ARG;
    ctx->err.clear();
    eofa_status s = solve_impl(ctx, (const double*)rhs, (double*)sol, *opts, stats, (cudaStream_t)stream);
    if (stats) stats->status = s;
    return s;
}

eofa_status eofa_solve_host(eofa_ctx* ctx, const double* rhs, double* sol, const eofa_solve_opts* opts,
                            eofa_solve_stats* stats, void* stream) {
    if (!ctx || !rhs || !sol || !opts || rhs == sol) return EOFA_ERR_ARG;
    eofa_ctx* c = ctx;
    c->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    // a page-locked right-hand side (and initial guess) is read in place by
    // the import kernels (through NVLink-C2C on a Grace-Blackwell node); the
    // solution is exported to a device field and copied to a page-locked sol
    // by the copy engine while the true residual is computed
    cudaPointerAttributes ra{}, sa{};
    const bool rhs_pinned = cudaPointerGetAttributes(&ra, rhs) == cudaSuccess && ra.type == cudaMemoryTypeHost &&
                            ra.devicePointer;
    const bool sol_pinned = cudaPointerGetAttributes(&sa, sol) == cudaSuccess && sa.type == cudaMemoryTypeHost &&
                            sa.devicePointer;
    cudaGetLastError();  // the queries of pageable pointers may leave an error behind
    double* dsol = act_buf(c, 1);
    double* drhs = rhs_pinned ? (double*)ra.devicePointer : act_buf(c, 0);
    if (!dsol || !drhs) return fail(c, EOFA_ERR_OOM, "work fields of the host solve");
    const size_t bytes = (size_t)c->n5 * 2 * 24 * sizeof(double);
    if (!rhs_pinned) CK(cudaMemcpyAsync(drhs, rhs, bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    const double* guess = nullptr;
    if (opts->use_guess) {
        if (sol_pinned) guess = (const double*)sa.devicePointer;
        else CK(cudaMemcpyAsync(dsol, sol, bytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    }
    eofa_status s = solve_impl(c, drhs, dsol, *opts, stats, st, sol_pinned ? sol : nullptr, guess);
    if (stats) stats->status = s;
    if (!sol_pinned && c->exported)
        CK(cudaMemcpyAsync(sol, dsol, bytes, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return s;
}

eofa_status eofa_dot(eofa_ctx* ctx, const void* a, const void* b, long n, double* re, double* im, void* stream) {
    if (!ctx || !a || !b || n < 0 || !re || !im) return EOFA_ERR_ARG;
    eofa_ctx* c = ctx;
    c->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    eofa_status s = ensure_mdot(c);
    if (s != EOFA_OK) return s;
    double* res = c->mdot + 2 * kMultiBlocks * kMultiMax;
    VecSet set{};
    set.n = 1;
    set.v[0] = (const double2*)a;
    CK(multidot(set, (const double*)b, n, c->mdot, res, st), "multidot");
    double h[2];
    CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *re = h[0];
    *im = h[1];
    return EOFA_OK;
}

eofa_status eofa_force_norms(eofa_ctx* ctx, const void* force, double* f_rms, double* f_max, void* stream) {
    if (!ctx || !force || !f_rms || !f_max) return EOFA_ERR_ARG;
    eofa_ctx* c = ctx;
    c->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    eofa_status s = ensure_mdot(c);
    if (s != EOFA_OK) return s;
    // links of the physical lattice (G-parity: the force is folded onto them)
    const long nlinks = 4L * c->p.dims[0] * c->p.dims[1] * c->p.dims[2] * c->p.dims[3];
    double* res = c->mdot + 2 * kMultiBlocks * kMultiMax;
    CK(force_norm_sums((const double*)force, nlinks, c->mdot, res, st), "force_norm_sums");
    double h[2];
    CK(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *f_rms = std::sqrt(h[0]) / (double)nlinks;
    *f_max = std::sqrt(h[1]);
    return EOFA_OK;
}

eofa_status eofa_set_system(eofa_ctx* ctx, double m1, double m2, double m3, double beta, int pm) {
    if (!ctx) return EOFA_ERR_ARG;
    ctx->err.clear();
    return set_system(ctx, m1, m2, m3, beta, pm);
}

eofa_status eofa_apply_meofa(eofa_ctx* ctx, double m1, double m2, const void* phi, void* out,
                             const eofa_solve_opts* opts, eofa_solve_stats* stats, void* stream) {
    if (!ctx || !phi || !out || !opts || phi == out) return EOFA_ERR_ARG;
    ctx->err.clear();
    if (!std::isfinite(m1) || !std::isfinite(m2)) return fail(ctx, EOFA_ERR_ARG, "m1, m2 must be finite");
    if (stats) std::memset(stats, 0, 2 * sizeof(eofa_solve_stats));
    const eofa_params keep = ctx->p;
    eofa_status s = meofa_impl(ctx, m1, m2, (const double*)phi, (double*)out, *opts, stats, (cudaStream_t)stream);
    const std::string why = ctx->err;
    eofa_status r = set_system(ctx, keep);
    if (s == EOFA_OK && r != EOFA_OK) return r;
    ctx->err = why;
    return s;
}

eofa_status eofa_force(eofa_ctx* ctx, double m1, double m2, const void* phi, void* force,
                       const eofa_solve_opts* opts, eofa_solve_stats* stats, void* stream) {
    if (!ctx || !phi || !force || !opts) return EOFA_ERR_ARG;
    ctx->err.clear();
    if (!std::isfinite(m1) || !std::isfinite(m2)) return fail(ctx, EOFA_ERR_ARG, "m1, m2 must be finite");
    if (stats) std::memset(stats, 0, 2 * sizeof(eofa_solve_stats));
    const eofa_params keep = ctx->p;
    eofa_status s = force_impl(ctx, m1, m2, (const double*)phi, (double*)force, *opts, stats, (cudaStream_t)stream);
    const std::string why = ctx->err;
    eofa_status r = set_system(ctx, keep);
    if (s == EOFA_OK && r != EOFA_OK) return r;
    ctx->err = why;
    return s;
}

eofa_status eofa_heatbath(eofa_ctx* ctx, double m1, double m2, int np, const double* alpha, const double* beta,
                          const double* pole_tol, int forecast_n, const void* eta, void* phi,
                          const eofa_solve_opts* opts, eofa_solve_stats* stats, void* stream) {
    if (!ctx || !eta || !phi || !opts || eta == phi || np < 0 || !alpha || (np > 0 && !beta)) return EOFA_ERR_ARG;
    ctx->err.clear();
    if (forecast_n < 0 || forecast_n > kMultiMax)
        return fail(ctx, EOFA_ERR_ARG, "forecast_n must be in 0.." + std::to_string(kMultiMax));
    if (!std::isfinite(m1) || !std::isfinite(m2)) return fail(ctx, EOFA_ERR_ARG, "m1, m2 must be finite");
    for (int l = 0; l <= np; ++l)
        if (!std::isfinite(alpha[l])) return fail(ctx, EOFA_ERR_ARG, "alpha must be finite");
    for (int l = 0; l < np; ++l)
        if (!std::isfinite(beta[l]) || !(beta[l] > -1.0))
            return fail(ctx, EOFA_ERR_ARG, "every beta_l must be finite and > -1 (gamma_l = 1/(1+beta_l))");
    if (stats && np > 0) std::memset(stats, 0, 2 * (size_t)np * sizeof(eofa_solve_stats));
    const eofa_params keep = ctx->p;
    eofa_status s = heatbath_impl(ctx, m1, m2, np, alpha, beta, pole_tol, forecast_n, (const double*)eta,
                                  (double*)phi, *opts, stats, (cudaStream_t)stream);
    const std::string why = ctx->err;
    eofa_status r = set_system(ctx, keep);
    if (s == EOFA_OK && r != EOFA_OK) return r;
    ctx->err = why;
    return s;
}

eofa_status eofa_apply_batched(eofa_ctx* const* ctx, int n, const void* const* in, void* const* out, int dag,
                               void* stream) {
    if (n < 0 || (n > 0 && (!ctx || !in || !out))) return EOFA_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        eofa_status s = dag ? eofa_apply_dag(ctx[i], in[i], out[i], stream) : eofa_apply(ctx[i], in[i], out[i], stream);
        if (s != EOFA_OK) return s;
    }
    return EOFA_OK;
}

eofa_status eofa_solve_batched(eofa_ctx* const* ctx, int n, const void* const* rhs, void* const* sol,
                               const eofa_solve_opts* opts, eofa_solve_stats* stats, void* stream) {
    if (n < 0 || (n > 0 && (!ctx || !rhs || !sol || !opts))) return EOFA_ERR_ARG;
    if (n == 0) return EOFA_OK;  // nothing to solve (opts may be NULL)
    for (int i = 0; i < n; ++i) {
        if (!ctx[i] || !rhs[i] || !sol[i] || rhs[i] == sol[i]) return EOFA_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (ctx[j] == ctx[i]) return EOFA_ERR_ARG;  // one context per system
    }
    // kernel timing instruments the host-driven loop, the learned
    // preconditioner runs flexible GCR, and the dense comparison scheme has
    // no batched loop: these solve one by one
    // errors are reported on the first context, prefixed with the system
    auto report = [&](int k) {
        if (k > 0) ctx[0]->err = "system " + std::to_string(k) + ": " + ctx[k]->err;
    };
    if (opts->kernel_timing || opts->precond || opts->method || opts->inner < 0 || opts->inner > 3) {
        eofa_status first = EOFA_OK;
        for (int i = 0; i < n; ++i) {
            eofa_status s = eofa_solve(ctx[i], rhs[i], sol[i], opts, stats ? stats + i : nullptr, stream);
            if (s != EOFA_OK && first == EOFA_OK) {
                first = s;
                report(i);
            }
        }
        return first;
    }
    eofa_status first = EOFA_OK;
    for (int lo = 0; lo < n; lo += kBatchMax) {
        const int m = std::min(kBatchMax, n - lo);
        int failed = 0;
        eofa_status s = solve_batched_impl(ctx + lo, m, rhs + lo, sol + lo, *opts, stats ? stats + lo : nullptr,
                                           (cudaStream_t)stream, &failed);
        if (s != EOFA_OK && first == EOFA_OK) {
            first = s;
            report(lo + failed);
        }
    }
    return first;
}

void eofa_destroy(eofa_ctx* ctx) {
    if (!ctx) return;
    drop_batch_graphs(ctx->uid);
    for (void* p : ctx->allocs) cudaFree(p);
    for (cudaEvent_t e : ctx->evs) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->nev)
        if (e) cudaEventDestroy(e);
    for (auto& row : ctx->gev)
        for (cudaEvent_t e : row)
            if (e) cudaEventDestroy(e);
    for (int i = 0; i < 4; ++i) {
        for (int m = 0; m < 2; ++m) {
            if (ctx->cg_exec[m][i]) cudaGraphExecDestroy(ctx->cg_exec[m][i]);
            if (ctx->cg_first[m][i]) cudaGraphExecDestroy(ctx->cg_first[m][i]);
        }
    }
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (cudaEvent_t e : ctx->xev)
        if (e) cudaEventDestroy(e);
    if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
    delete ctx;
}

const char* eofa_status_string(eofa_status s) {
    switch (s) {
        case EOFA_OK: return "ok";
        case EOFA_ERR_ARG: return "invalid argument";
        case EOFA_ERR_UNSUPPORTED: return "unsupported parameters";
        case EOFA_ERR_SINGULAR: return "singular operator";
        case EOFA_ERR_NOT_CONVERGED: return "not converged";
        case EOFA_ERR_NONFINITE: return "non-finite value";
        case EOFA_ERR_TIMEOUT: return "timeout";
        case EOFA_ERR_CUDA: return "CUDA error";
        case EOFA_ERR_OOM: return "out of device memory";
        default: return "unknown status";
    }
}

const char* eofa_last_error(const eofa_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int eofa_tile_sites(const eofa_ctx* ctx, int prec, int kind) {
    if (!ctx || prec < 0 || prec > 3 || kind < 0 || kind > 3) return 0;
    return tile_sites(ctx->g.Ls, ctx->tuned[prec] ? ctx->tile[prec][kind] : 0);
}

int eofa_tile_variant(const eofa_ctx* ctx, int prec, int kind) {
    if (!ctx || prec < 0 || prec > 3 || kind < 0 || kind > 3) return -1;
    return ctx->tuned[prec] ? ctx->tile[prec][kind] : 0;
}

double eofa_tile_time(const eofa_ctx* ctx, int prec, int kind, int variant) {
    if (!ctx || prec < 0 || prec > 3 || kind < 0 || kind > 3 || variant < 0 || variant > 3) return -1.0;
    return ctx->tuned[prec] ? (double)ctx->tune_ms[prec][kind][variant] : 0.0;
}

double eofa_hop_bytes(const eofa_ctx* ctx, int prec, int with_local) {
    if (!ctx || prec < 0 || prec > 3) return 0.0;
    return hop_bytes_of(ctx, prec, with_local);
}

}  // extern "C"

// ===========================================================================
// eofa_apply_noalloc: K applied with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own pool and forbids allocations behind its back, or a
// latency-critical loop in which cudaMalloc's implicit device
// synchronisation is not acceptable.  This entry point needs no context:
// everything it works on besides the caller's inputs and output lives in
// one file-scope static device array, g_noalloc_scratch, which every GPU
// that loads the library holds until the process exits.
// ===========================================================================
namespace {

constexpr long kNoAllocMaxVol4 = 4096;     // 4D sites (e.g. 8^4)
constexpr long kNoAllocMaxSites5 = 32768;  // 5D sites V * Ls (e.g. 8^4 x 8)
constexpr size_t kNaHalf = kNoAllocMaxVol4 / 2;
constexpr size_t kNaLinks[4] = {kNaHalf * 4 * 12 * 8, kNaHalf * 4 * 12 * 4, kNaHalf * 4 * 12 * 2,
                                kNaHalf * 4 * 12 * 2};  // one parity, per precision
constexpr size_t kNaField = (size_t)(kNoAllocMaxSites5 / 2) * 24 * 8;  // one parity, FP64
constexpr size_t kNaLinkTotal = 2 * (kNaLinks[0] + kNaLinks[1] + kNaLinks[2] + kNaLinks[3]);
constexpr size_t kNaScratchBytes = kNaLinkTotal + 4 * kNaField + 256;

constexpr int kNaMaxDevices = 64;
unsigned char* g_noalloc_ptr[kNaMaxDevices] = {};  // device address of the scratch, per device
std::mutex g_noalloc_mu;

}  // namespace

// About 15 MiB: two-row links of both parities in four precisions, the
// input and output field in the even-odd layout, and the SU(3) check flag.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

namespace {

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// obtained once per device with cudaGetSymbolAddress, with that device
// current, and cached.
eofa_status noalloc_scratch(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return EOFA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return EOFA_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return EOFA_OK;
}

}  // namespace

extern "C" eofa_status eofa_apply_noalloc(const eofa_params* p, const void* gauge, const void* in, void* out,
                                          void* stream) {
    if (!p || !gauge || !in || !out || in == out) return EOFA_ERR_ARG;
    for (int i = 0; i < 4; ++i)
        if (p->dims[i] < 2 || (p->dims[i] & 1)) return EOFA_ERR_ARG;
    if (p->pm != 1 && p->pm != -1) return EOFA_ERR_ARG;
    if (p->t_bc != 1 && p->t_bc != -1) return EOFA_ERR_ARG;
    if (p->Ls != 4 && p->Ls != 8 && p->Ls != 12 && p->Ls != 16) return EOFA_ERR_UNSUPPORTED;
    const long V = (long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
    if (V > kNoAllocMaxVol4 || V * p->Ls > kNoAllocMaxSites5) return EOFA_ERR_UNSUPPORTED;
    SCoef<double> k;
    const char* why = "";
    eofa_status s = coef_from_params(*p, k, &why);
    if (s != EOFA_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the call reads the SU(3) flag back and waits for it, which a stream
    // capture cannot hold: refuse instead of invalidating the caller's capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return EOFA_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return EOFA_ERR_UNSUPPORTED;
    unsigned char* base = nullptr;
    if ((s = noalloc_scratch(&base)) != EOFA_OK) return s;

    Geom g;
    g.X = p->dims[0]; g.Y = p->dims[1]; g.Z = p->dims[2]; g.T = p->dims[3];
    g.Xh = g.X / 2;
    g.Vh = (int)(V / 2);
    g.Ls = p->Ls;
    g.apmask = p->t_bc == -1 ? 8 : 0;
    g.gpmask = 0;
    g.Tp = g.T;
    void* links[4][2];
    size_t off = 0;
    for (int pr = 0; pr < 4; ++pr)
        for (int par = 0; par < 2; ++par) {
            links[pr][par] = base + off;
            off += kNaLinks[pr];
        }
    VecRef fin[2], fout[2];
    for (int par = 0; par < 2; ++par) {
        fin[par] = VecRef{base + off, nullptr};
        off += kNaField;
        fout[par] = VecRef{base + off, nullptr};
        off += kNaField;
    }
    int* bad = reinterpret_cast<int*>(base + off);

    // the flag must start at zero: the array keeps the previous call's contents
    if (cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess) return EOFA_ERR_CUDA;
    if (gauge_import((const double*)gauge, g, links, bad, st) != cudaSuccess) return EOFA_ERR_CUDA;
    int hbad = 0;
    if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EOFA_ERR_CUDA;
    if (hbad) return EOFA_ERR_ARG;
    for (int par = 0; par < 2; ++par)
        if (layout_import(fin[par], (const double*)in, g, par, 0, st) != cudaSuccess) return EOFA_ERR_CUDA;
    for (int par = 0; par < 2; ++par) {
        HopArgs a;
        std::memset(&a, 0, sizeof(a));
        a.g = g;
        a.out_par = par;
        a.in = fin[1 - par].d;
        a.y = fin[par].d;
        a.out = fout[par].d;
        a.lk_out = links[EOFA_F64][par];
        a.lk_in = links[EOFA_F64][1 - par];
        a.rd.fin = FIN_NONE;
        if (launch_hop_f64(KIND_FULL, a, &k, st) != cudaSuccess) return EOFA_ERR_CUDA;
    }
    for (int par = 0; par < 2; ++par)
        if (layout_export((double*)out, fout[par], g, par, 0, st) != cudaSuccess) return EOFA_ERR_CUDA;
    return EOFA_OK;
}

// ===========================================================================
// learned preconditioner: stateless entry points for the network itself
// ===========================================================================

namespace {

struct DevBuf {
    std::vector<void*> p;
    ~DevBuf() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    cudaError_t get(T** out, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T));
        if (e != cudaSuccess) return e;
        p.push_back(q);
        *out = static_cast<T*>(q);
        return cudaSuccess;
    }
};

cudaError_t net_alloc(DevBuf& B, NetDev& n) {
    cudaError_t e = B.get(&n.Wm, (size_t)kNetWeights);
    for (int l = 0; l < kNetLayers && e == cudaSuccess; ++l) {
        e = B.get(&n.Wf[l], (size_t)81 * 32 * 32);
        if (e == cudaSuccess) e = B.get(&n.Wb[l], (size_t)81 * 32 * 32);
    }
    return e;
}

bool conv_geom(const int dims[4], int nslices, ConvGeom* g) {
    if (!dims || nslices <= 0) return false;
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 1) return false;
    const long V = (long)dims[0] * dims[1] * dims[2] * dims[3];
    if (V * nslices > (1L << 31)) return false;
    g->X = dims[0]; g->Y = dims[1]; g->Z = dims[2]; g->T = dims[3];
    g->V = (int)V;
    g->S = nslices;
    return true;
}

}  // namespace

extern "C" eofa_status eofa_net_forward(const float* weights, const int dims[4], int nslices, const void* in,
                                        void* out, void* stream) {
    ConvGeom g;
    if (!weights || !in || !out || !conv_geom(dims, nslices, &g)) return EOFA_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long rows = (long)g.V * g.S;
    DevBuf B;
    NetDev n;
    bf16 *a0, *a1, *a2;
    float* o32;
    cudaError_t e = net_alloc(B, n);
    if (e == cudaSuccess) e = B.get(&a0, rows * kCP);
    if (e == cudaSuccess) e = B.get(&a1, rows * kCP);
    if (e == cudaSuccess) e = B.get(&a2, rows * kCP);
    if (e == cudaSuccess) e = B.get(&o32, rows * kCP);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n.Wm, weights, sizeof(float) * kNetWeights, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = net_convert(n, st);
    if (e == cudaSuccess) e = pack_act((const float*)in, a0, rows, st);
    if (e == cudaSuccess) e = net_forward(n, g, a0, a1, a2, o32, st);
    if (e == cudaSuccess) e = unpack_out(o32, (float*)out, rows, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int fault = 0;
    if (e == cudaSuccess) e = net_fault(&fault);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EOFA_ERR_OOM : EOFA_ERR_CUDA;
    return fault ? EOFA_ERR_TIMEOUT : EOFA_OK;
}

extern "C" eofa_status eofa_net_backward(const float* weights, const int dims[4], int nslices, const void* in,
                                         const void* dout, float* dweights, void* din, void* stream) {
    ConvGeom g;
    if (!weights || !in || !dout || !dweights || !conv_geom(dims, nslices, &g)) return EOFA_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long rows = (long)g.V * g.S;
    DevBuf B;
    NetDev n;
    bf16 *a0, *a1, *a2, *dob, *d1, *d2;
    float *o32, *dout32, *dW, *din32 = nullptr;
    cudaError_t e = net_alloc(B, n);
    bf16** bufs[] = {&a0, &a1, &a2, &dob, &d1, &d2};
    for (auto b : bufs)
        if (e == cudaSuccess) e = B.get(b, rows * kCP);
    if (e == cudaSuccess) e = B.get(&o32, rows * kCP);
    if (e == cudaSuccess) e = B.get(&dout32, rows * kCP);
    if (e == cudaSuccess) e = B.get(&dW, (size_t)kNetWeights);
    if (e == cudaSuccess && din) e = B.get(&din32, rows * kCP);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n.Wm, weights, sizeof(float) * kNetWeights, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dW, 0, sizeof(float) * kNetWeights, st);
    if (e == cudaSuccess) e = net_convert(n, st);
    if (e == cudaSuccess) e = pack_act((const float*)in, a0, rows, st);
    if (e == cudaSuccess) e = net_forward(n, g, a0, a1, a2, o32, st);
    if (e == cudaSuccess) e = pad_f32((const float*)dout, dout32, rows, st);
    if (e == cudaSuccess) e = net_backward(n, g, a0, a1, a2, dout32, dW, din32, dob, d1, d2, st);
    if (e == cudaSuccess && din) e = unpack_out(din32, (float*)din, rows, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dweights, dW, sizeof(float) * kNetWeights, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int fault = 0;
    if (e == cudaSuccess) e = net_fault(&fault);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? EOFA_ERR_OOM : EOFA_ERR_CUDA;
    return fault ? EOFA_ERR_TIMEOUT : EOFA_OK;
}

// ===========================================================================
// learned preconditioner inside the solver
// ===========================================================================
namespace {

constexpr int kGcrM = 4;  // flexible GCR restart length

Reduce red2(eofa_ctx* c, int fin, int slot) {
    Reduce r;
    r.partials = c->partials2;
    r.counter = c->counter2;
    r.scal = c->scal;
    r.fin = fin;
    r.slot = slot;
    return r;
}

eofa_status ensure_learned(eofa_ctx* c) {
    if (c->act[0]) return EOFA_OK;
    const long rows = 2L * c->g.Vh * c->g.Ls;
    eofa_status s;
    void* p = nullptr;
    for (int i = 0; i < 3; ++i) {
        if ((s = dalloc(c, &p, sizeof(bf16) * rows * kCP))) return s;
        c->act[i] = (bf16*)p;
    }
    if ((s = dalloc(c, &p, sizeof(float) * rows * kCP))) return s;
    c->out32 = (float*)p;
    if ((s = vec_alloc(c, EOFA_F32, &c->gx)) || (s = vec_alloc(c, EOFA_F32, &c->gr))) return s;
    for (int k = 0; k < kGcrM; ++k)
        if ((s = vec_alloc(c, EOFA_F32, &c->gz[k])) || (s = vec_alloc(c, EOFA_F32, &c->gw[k]))) return s;
    const int maxgrid = std::max(blas_max_grid(c->n5), c->g.Vh / 8 + 2);
    if ((s = dalloc(c, &p, sizeof(double) * maxgrid))) return s;
    c->partials2 = (double*)p;
    if ((s = dalloc(c, &p, 256))) return s;
    c->counter2 = (unsigned*)p;
    CK(cudaMemset(c->counter2, 0, 256), "memset");
    if ((s = dalloc(c, &p, sizeof(float) * kNetWeights))) return s;
    c->net.Wm = (float*)p;
    for (int l = 0; l < kNetLayers; ++l) {
        if ((s = dalloc(c, &p, sizeof(bf16) * 81 * 32 * 32))) return s;
        c->net.Wf[l] = (bf16*)p;
        if ((s = dalloc(c, &p, sizeof(bf16) * 81 * 32 * 32))) return s;
        c->net.Wb[l] = (bf16*)p;
    }
    return EOFA_OK;
}

ConvGeom conv_geom_of(const eofa_ctx* c, int slices) {
    ConvGeom cg;
    cg.X = c->g.X; cg.Y = c->g.Y; cg.Z = c->g.Z; cg.T = c->g.T;
    cg.V = 2 * c->g.Vh;
    cg.S = slices;
    return cg;
}

// after a synchronisation: a tensor-core convolution that gave up on a
// bounded wait left its output unwritten
eofa_status check_net(eofa_ctx* c) {
    int f = 0;
    CK(net_fault(&f), "net_fault");
    if (f) return fail(c, EOFA_ERR_TIMEOUT, "tensor-core convolution: a bounded wait expired");
    return EOFA_OK;
}

// z = net(r) for every s-slice of an odd-parity FP32 field
eofa_status net_apply(eofa_ctx* c, VecRef in, VecRef out, cudaStream_t st) {
    CKL(embed_odd(in, c->act[0], c->g, -1, 1.0, c->scal, -1, st), "embed");
    CK(net_forward(c->net, conv_geom_of(c, c->g.Ls), c->act[0], c->act[1], c->act[2], c->out32, st), "net");
    c->launches += 3;
    CKL(extract_odd(c->out32, out, c->g, st), "extract");
    return EOFA_OK;
}

// <a, b> read back to the host (slots 4 and 5 are free during inner solves)
eofa_status dot_host(eofa_ctx* c, VecRef a, VecRef b, double* re, double* im, cudaStream_t st) {
    CKL(cdot(a, b, c->n5, c->g.Ls, red(c, FIN_STORE, 4), red2(c, FIN_STORE, 5), st), "cdot");
    eofa_status s;
    if ((s = read_scal(c, st))) return s;
    *re = c->h_scal->store[4];
    *im = c->h_scal->store[5];
    return EOFA_OK;
}

// Flexible GCR(kGcrM) on the Schur complement S in FP32 with the learned
// preconditioner: z_k = net(r), w_k = S z_k orthonormalised against the
// cycle's earlier w_j (modified Gram-Schmidt, the same combination applied
// to z_k), x += <w_k, r> z_k, r -= <w_k, r> w_k.  A restart cycle that does
// not halve |r| hands the rest of the solve to CGNR (the plain method
// stays the fallback).  Unit source in inner[F32].r, result in inner[F32].x.
eofa_status run_fgcr(eofa_ctx* c, double tol, int maxit, int* iters, cudaStream_t st, Clock::time_point t0,
                     long timeout_ms) {
    Inner& in = c->inner[EOFA_F32];
    const long n5 = c->n5;
    const int Ls = c->g.Ls;
    const VecRef none{};
    eofa_status s;
    if ((s = ensure_learned(c))) return s;
    for (cudaEvent_t& e : c->nev)
        if (!e) CK(cudaEventCreate(&e), "cudaEventCreate");
    CKL(blas_copy(EOFA_F32, c->gr, EOFA_F32, in.r, n5, Ls, 1.0, -1, red(c, FIN_NONE), st), "copy");
    CKL(blas_zero(EOFA_F32, c->gx, n5, Ls, st), "zero");
    double rr, im;
    if ((s = dot_host(c, c->gr, c->gr, &rr, &im, st))) return s;
    *iters = 0;
    auto finish = [&](eofa_status r) -> eofa_status {
        CKL(blas_copy(EOFA_F32, in.x, EOFA_F32, c->gx, n5, Ls, 1.0, -1, red(c, FIN_NONE), st), "copy");
        return r;
    };
    for (;;) {
        const double cycle_rr = rr;
        for (int k = 0; k < kGcrM; ++k) {
            CK(cudaEventRecord(c->nev[0], st), "cudaEventRecord");
            if ((s = net_apply(c, c->gr, c->gz[k], st))) return s;
            CK(cudaEventRecord(c->nev[1], st), "cudaEventRecord");
            if ((s = hop(c, EOFA_F32, KIND_EO_MINV, 0, c->gz[k], none, in.t, red(c, FIN_NONE), nullptr, st)))
                return s;
            if ((s = hop(c, EOFA_F32, KIND_OE_SCHUR, 1, in.t, c->gz[k], c->gw[k], red(c, FIN_NONE), nullptr, st)))
                return s;
            double br, bi;
            for (int j = 0; j < k; ++j) {
                if ((s = dot_host(c, c->gw[j], c->gw[k], &br, &bi, st))) return s;
                CKL(caxpby(c->gw[k], c->gw[j], n5, Ls, (float)-br, (float)-bi, 1.f, st), "caxpby");
                CKL(caxpby(c->gz[k], c->gz[j], n5, Ls, (float)-br, (float)-bi, 1.f, st), "caxpby");
            }
            double nn;
            if ((s = dot_host(c, c->gw[k], c->gw[k], &nn, &bi, st)) || (s = check_net(c))) return s;
            float nms = 0.f;
            CK(cudaEventElapsedTime(&nms, c->nev[0], c->nev[1]), "cudaEventElapsedTime");
            c->net_ms += nms;
            if (!(nn > 0.0) || !std::isfinite(nn)) break;  // no new direction: fall back below
            const float sc = (float)(1.0 / std::sqrt(nn));
            CKL(caxpby(c->gw[k], c->gw[k], n5, Ls, 0.f, 0.f, sc, st), "scale");
            CKL(caxpby(c->gz[k], c->gz[k], n5, Ls, 0.f, 0.f, sc, st), "scale");
            double ar, ai;
            if ((s = dot_host(c, c->gw[k], c->gr, &ar, &ai, st))) return s;
            CKL(caxpby(c->gx, c->gz[k], n5, Ls, (float)ar, (float)ai, 1.f, st), "caxpby");
            CKL(caxpby(c->gr, c->gw[k], n5, Ls, (float)-ar, (float)-ai, 1.f, st), "caxpby");
            if ((s = dot_host(c, c->gr, c->gr, &rr, &im, st))) return s;
            ++*iters;
            ++c->gcr_steps;
            if (!std::isfinite(rr)) return fail(c, EOFA_ERR_NONFINITE, "non-finite residual in flexible GCR");
            if (rr <= tol * tol) return finish(EOFA_OK);
            if (*iters >= maxit) return finish(EOFA_ERR_NOT_CONVERGED);
            if (timeout_ms > 0 && since(t0) * 1e3 > (double)timeout_ms)
                return fail(c, EOFA_ERR_TIMEOUT, "solve exceeded timeout_ms");
        }
        if (rr > 0.25 * cycle_rr) {
            // the cycle did not halve |r|: CGNR solves S e = r / |r|, x += |r| e
            ++c->gcr_fallbacks;
            const double rn = std::sqrt(rr);
            CKL(blas_copy(EOFA_F32, in.r, EOFA_F32, c->gr, n5, Ls, 1.0 / rn, -1, red(c, FIN_NONE), st), "copy");
            int cits = 0;
            double crr = 0.0;
            eofa_status cs = run_cgnr(c, EOFA_F32, tol / rn, maxit - *iters, &cits, &crr, st, t0, timeout_ms);
            *iters += cits;
            CKL(caxpby(in.x, c->gx, n5, Ls, 1.f, 0.f, (float)rn, st), "caxpby");
            return cs;
        }
    }
}

}  // namespace

extern "C" eofa_status eofa_set_preconditioner(eofa_ctx* ctx, const float* weights) {
    if (!ctx || !weights) return EOFA_ERR_ARG;
    eofa_ctx* c = ctx;
    eofa_status s;
    if ((s = ensure_learned(c))) return s;
    CK(cudaMemcpy(c->net.Wm, weights, sizeof(float) * kNetWeights, cudaMemcpyHostToDevice), "upload weights");
    CK(net_convert(c->net, nullptr), "convert weights");
    CK(cudaDeviceSynchronize(), "sync");
    c->net_ready = true;
    return EOFA_OK;
}

extern "C" eofa_status eofa_train_preconditioner(eofa_ctx* ctx, const void* const* sources, int n_sources,
                                                 const float* init_weights, const eofa_train_opts* opts,
                                                 float* weights_out, eofa_train_stats* stats, void* stream) {
    if (!ctx || !sources || n_sources <= 0 || !init_weights || !opts || !weights_out) return EOFA_ERR_ARG;
    if (opts->pairs <= 0 || opts->snapshot_every <= 0 || opts->epochs <= 0 || opts->batch <= 0 || !(opts->lr > 0.0) ||
        !(opts->solve_tol > 0.0) || opts->holdout < 0)
        return EOFA_ERR_ARG;
    for (int i = 0; i < n_sources; ++i)
        if (!sources[i]) return EOFA_ERR_ARG;
    eofa_ctx* c = ctx;
    c->err.clear();
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = Clock::now();
    eofa_status s;
    if ((s = ensure_inner(c, EOFA_F32)) || (s = ensure_learned(c))) return s;
    CK(cudaMemcpyAsync(c->net.Wm, init_weights, sizeof(float) * kNetWeights, cudaMemcpyHostToDevice, st), "upload");
    CK(net_convert(c->net, st), "convert");
    const Geom& g = c->g;
    const long V = 2L * g.Vh, n5 = c->n5;
    const int Ls = g.Ls, B = opts->batch;
    const int P = opts->pairs + opts->holdout;  // training pairs, then the held-out ones
    // the loss reduction shares the context's reduction buffers, sized for
    // one half-lattice 5D field: a batch holds at most Ls/2 full-lattice slices
    if (2L * B > Ls) return fail(c, EOFA_ERR_ARG, "train batch must be at most Ls/2");
    constexpr int kMaxSnap = 64;
    DevBuf D;
    bf16 *pr, *pe, *a0, *a1, *a2, *et, *dob, *d1, *d2;
    float *o32, *dout, *dW, *am, *av, *wdev;
    cudaError_t e = D.get(&pr, (size_t)P * V * kCP);
    if (e == cudaSuccess) e = D.get(&pe, (size_t)P * V * kCP);
    bf16** bb[] = {&a0, &a1, &a2, &et, &dob, &d1, &d2};
    for (auto b : bb)
        if (e == cudaSuccess) e = D.get(b, (size_t)B * V * kCP);
    if (e == cudaSuccess) e = D.get(&o32, (size_t)B * V * kCP);
    if (e == cudaSuccess) e = D.get(&dout, (size_t)B * V * kCP);
    if (e == cudaSuccess) e = D.get(&dW, (size_t)kNetWeights);
    if (e == cudaSuccess) e = D.get(&am, (size_t)kNetWeights);
    if (e == cudaSuccess) e = D.get(&av, (size_t)kNetWeights);
    if (e == cudaSuccess) e = D.get(&wdev, (size_t)B);
    std::vector<VecRef> snap(kMaxSnap);
    VecRef et5{}, rt5{};
    for (int i = 0; i < kMaxSnap && e == cudaSuccess; ++i) e = D.get((float**)&snap[i].d, (size_t)n5 * 24);
    if (e == cudaSuccess) e = D.get((float**)&et5.d, (size_t)n5 * 24);
    if (e == cudaSuccess) e = D.get((float**)&rt5.d, (size_t)n5 * 24);
    if (e == cudaSuccess) e = cudaMemsetAsync(am, 0, sizeof(float) * kNetWeights, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(av, 0, sizeof(float) * kNetWeights, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "training buffers");

    // ---- pairs from the solver's own iterates ----
    Inner& in = c->inner[EOFA_F32];
    const VecRef none{};
    std::vector<float> pw(P, 1.f);
    int have = 0, solves = 0;
    for (int j = 0; j < n_sources && have < P; ++j) {
        SolveState ss;
        eofa_solve_opts o;
        std::memset(&o, 0, sizeof(o));
        o.tol = 1e-10;
        o.inner = EOFA_F32;
        if ((s = solve_begin(c, (const double*)sources[j], (const double*)sources[j], o, ss, st))) return s;
        CK(cudaStreamSynchronize(st), "sync");
        if (c->h_scal->store[1] + c->h_scal->store[2] == 0.0) continue;
        if ((s = outer_residual(c, ss, st))) return s;
        CKL(blas_copy(EOFA_F32, in.r, 0, c->ro, n5, Ls, 1.0, 0, red(c, FIN_NONE), st), "copy");
        const double tol = opts->solve_tol;
        CKL(scal_init(c->scal, tol * tol, 100000, 0ull, st), "scal_init");
        if ((s = cg_start(c, EOFA_F32, nullptr, st))) return s;
        int ns = 1;  // snapshot 0 is the zero start vector
        CK(cudaMemsetAsync(snap[0].d, 0, sizeof(float) * n5 * 24, st), "memset");
        for (;;) {
            for (int i = 0; i < opts->snapshot_every; ++i)
                if ((s = cg_iteration(c, EOFA_F32, st, false))) return s;
            if ((s = read_scal(c, st))) return s;
            if (c->h_scal->nonfinite) return fail(c, EOFA_ERR_NONFINITE, "training solve");
            if (c->h_scal->done || c->h_scal->iters >= 100000) break;
            if (ns < kMaxSnap)
                CKL(blas_copy(EOFA_F32, snap[ns++], EOFA_F32, in.x, n5, Ls, 1.0, -1, red(c, FIN_NONE), st), "snap");
        }
        ++solves;
        for (int i = 0; i < ns && have < P; ++i) {
            // e = x* - x_k, r = S e
            CKL(blas_copy(EOFA_F32, et5, EOFA_F32, in.x, n5, Ls, 1.0, -1, red(c, FIN_NONE), st), "copy");
            CKL(caxpby(et5, snap[i], n5, Ls, -1.f, 0.f, 1.f, st), "caxpby");
            if ((s = hop(c, EOFA_F32, KIND_EO_MINV, 0, et5, none, in.t, red(c, FIN_NONE), nullptr, st))) return s;
            if ((s = hop(c, EOFA_F32, KIND_OE_SCHUR, 1, in.t, et5, rt5, red(c, FIN_NONE), nullptr, st))) return s;
            const int sl = have % Ls;
            CKL(slice_norm(rt5, g.Vh, Ls, sl, red(c, FIN_STORE, 4), st), "norm");
            CKL(slice_norm(et5, g.Vh, Ls, sl, red(c, FIN_STORE, 5), st), "norm");
            if ((s = read_scal(c, st))) return s;
            const double nr = c->h_scal->store[4], ne = c->h_scal->store[5];
            if (!(nr > 0.0) || !(ne > 0.0)) continue;
            const double sc = 1.0 / std::sqrt(nr);
            CKL(embed_odd(rt5, pr + (size_t)have * V * kCP, g, sl, sc, c->scal, -1, st), "embed");
            CKL(embed_odd(et5, pe + (size_t)have * V * kCP, g, sl, sc, c->scal, -1, st), "embed");
            pw[have] = (float)(nr / ne);
            ++have;
        }
    }
    if (have == 0) return fail(c, EOFA_ERR_ARG, "no training pairs (zero sources?)");
    const int ntrain = std::min(have, opts->pairs);
    const int nhold = have - ntrain;
    const ConvGeom cgB = conv_geom_of(c, B);
    std::vector<float> hw(B);
    // mean relative squared error of the current weights on pairs first .. first + count - 1
    auto eval_loss = [&](int first, int count, double* out) -> eofa_status {
        double sum = 0.0;
        for (int b0 = 0; b0 < count; b0 += B) {
            for (int b = 0; b < B; ++b) {
                const bool use = b0 + b < count;
                const int p = first + (use ? b0 + b : 0);
                CK(cudaMemcpyAsync(a0 + (size_t)b * V * kCP, pr + (size_t)p * V * kCP, sizeof(bf16) * V * kCP,
                                   cudaMemcpyDeviceToDevice, st), "batch");
                CK(cudaMemcpyAsync(et + (size_t)b * V * kCP, pe + (size_t)p * V * kCP, sizeof(bf16) * V * kCP,
                                   cudaMemcpyDeviceToDevice, st), "batch");
                hw[b] = use ? pw[p] : 0.f;
            }
            CK(cudaMemcpyAsync(wdev, hw.data(), sizeof(float) * B, cudaMemcpyHostToDevice, st), "weights");
            CK(net_forward(c->net, cgB, a0, a1, a2, o32, st), "forward");
            CK(loss_grad(o32, et, wdev, dout, g, B, red(c, FIN_STORE, 4), st), "loss");
            if ((s = read_scal(c, st))) return s;
            sum += c->h_scal->store[4] * B;
        }
        *out = count > 0 ? sum / count : 0.0;
        return EOFA_OK;
    };
    double hold_init = 0.0, hold_final = 0.0;
    if (nhold > 0 && (s = eval_loss(ntrain, nhold, &hold_init))) return s;

    // ---- Adam on the relative squared error ----
    std::vector<int> perm(ntrain);
    for (int i = 0; i < ntrain; ++i) perm[i] = i;
    unsigned long long lcg = 0x9e3779b97f4a7c15ull;  // fixed-seed shuffle of the pair order
    for (int i = ntrain - 1; i > 0; --i) {
        lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
        const int k = (int)((lcg >> 33) % (unsigned long long)(i + 1));
        std::swap(perm[i], perm[k]);
    }
    const int steps = std::max(1, (int)((long)opts->epochs * ntrain / B));
    double loss_first = 0.0, loss_last = 0.0;
    for (int step = 0; step < steps; ++step) {
        for (int b = 0; b < B; ++b) {
            const int p = perm[((long)step * B + b) % ntrain];
            CK(cudaMemcpyAsync(a0 + (size_t)b * V * kCP, pr + (size_t)p * V * kCP, sizeof(bf16) * V * kCP,
                               cudaMemcpyDeviceToDevice, st), "batch");
            CK(cudaMemcpyAsync(et + (size_t)b * V * kCP, pe + (size_t)p * V * kCP, sizeof(bf16) * V * kCP,
                               cudaMemcpyDeviceToDevice, st), "batch");
            hw[b] = pw[p];
        }
        CK(cudaMemcpyAsync(wdev, hw.data(), sizeof(float) * B, cudaMemcpyHostToDevice, st), "weights");
        CK(net_forward(c->net, cgB, a0, a1, a2, o32, st), "forward");
        Geom gB = g;  // loss over B slices of the full lattice
        CK(loss_grad(o32, et, wdev, dout, gB, B, red(c, FIN_STORE, 4), st), "loss");
        CK(cudaMemsetAsync(dW, 0, sizeof(float) * kNetWeights, st), "memset");
        CK(net_backward(c->net, cgB, a0, a1, a2, dout, dW, nullptr, dob, d1, d2, st), "backward");
        CK(adam_step(c->net.Wm, dW, am, av, kNetWeights, (float)opts->lr, 0.9f, 0.999f, 1e-8f, step + 1, st), "adam");
        CK(net_convert(c->net, st), "convert");
        if (step == 0 || step == steps - 1) {
            if ((s = read_scal(c, st))) return s;
            (step == 0 ? loss_first : loss_last) = c->h_scal->store[4];
            if (step == 0) loss_last = loss_first;
        }
    }
    if (nhold > 0 && (s = eval_loss(ntrain, nhold, &hold_final))) return s;
    CK(cudaMemcpyAsync(weights_out, c->net.Wm, sizeof(float) * kNetWeights, cudaMemcpyDeviceToHost, st), "download");
    CK(cudaStreamSynchronize(st), "sync");
    if ((s = check_net(c))) return s;
    c->net_ready = true;
    if (stats) {
        stats->holdout_pairs = nhold;
        stats->holdout_loss_init = hold_init;
        stats->holdout_loss_final = hold_final;
        stats->pairs = ntrain;
        stats->steps = steps;
        stats->solves = solves;
        stats->loss_first = loss_first;
        stats->loss_last = loss_last;
        stats->seconds = since(t0);
    }
    return EOFA_OK;
}
