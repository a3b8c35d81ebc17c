/*
 * eofa.h -- C ABI of the GB300 EOFA Dirac-equation solver (libeofa.so).
 *
 * The library solves the exact one flavor algorithm (EOFA) Dirac equation of
 * Jung, Kelly, Mawhinney, Murphy, arXiv:1706.05843,
 *
 *     ( H(m1) + beta Delta_pm(m2, m3) P_pm ) psi = phi,            Eq. (generic_eofa_system)
 *     H(m) = gamma_5 R_5 D_EOFA(m),                                 Sec. II
 *
 * for Moebius domain wall fermions.  Internally it rotates by gamma_5 R_5
 * (Eq. non_hermit_sys), right-preconditions with D~(m1)^-1 (Cayley form,
 * Eq. precond_mobius_eofa_system), so that the operator actually inverted is
 *
 *     K = D_DWF(m1) + pm * beta * u_pm (x) v_pm P_pm,               App. B
 *     D_DWF(m) = (b D_W + 1) + (c D_W - 1) L(m),                    Eq. (Ddwf)
 *
 * and solves the 4D even-odd Schur complement K_oo - K_oe K_ee^-1 K_eo
 * (App. B) by conjugate gradient on the normal equations, with the site-
 * diagonal inverse applied through the Sherman-Morrison formula
 * (Eq. sherman_morrison_mobius_inv).  psi = D~(m1) psi' recovers the
 * H-form solution.
 *
 * Notation: b, c are the Moebius coefficients b5, c5 of Eq. (Ddwf); the
 * paper writes them as b5 = c + d, c5 = c - d with d = 1/2.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice dims[4] = {X, Y, Z, T}; every extent even (checkerboarding),
 *    Ls even and in {4, 8, 12, 16} (EOFA_ERR_UNSUPPORTED otherwise).
 *  - Gauge field: device memory, complex128 (interleaved re, im doubles),
 *    C order U[t][z][y][x][mu][row][col], mu = 0..3 = x, y, z, t.  Links
 *    must be special unitary to 1e-10: the library keeps two rows and
 *    rebuilds the third as conj(row0 x row1).
 *  - 5D fermion fields: device memory, complex128,
 *    psi[t][z][y][x][s][spin][colour], 24 * Ls * X*Y*Z*T doubles.
 *  - Gamma matrices in the chiral basis: gamma_k = [[0,-i sigma_k],[i sigma_k,0]],
 *    gamma_4 = [[0,1],[1,0]], gamma_5 = diag(1,1,-1,-1); P_pm = (1 pm gamma_5)/2.
 *  - Hops across the t boundary carry t_bc (-1: antiperiodic); space is
 *    periodic, except in the G-parity directions of eofa_create_gparity.
 *  - Ownership: all field pointers belong to the caller and are not kept
 *    after a call returns.  eofa_create copies the gauge field into the
 *    context (compressed, even-odd blocked); the context owns its device
 *    workspace until eofa_destroy.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    eofa_apply* enqueue their work and return without synchronising;
 *    eofa_solve* return after the solve has finished (the caller's stream
 *    is ordered before and after it).  One context must not be used by
 *    two calls at the same time.
 *  - Errors: every call returns an eofa_status and never aborts or exits.
 *    eofa_last_error(ctx) gives a message for the last failing call.
 *    Non-convergence still writes the best solution and its statistics.
 */
#ifndef EOFA_H
#define EOFA_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EOFA_OK = 0,
    EOFA_ERR_ARG = 1,           /* bad argument (NULL, odd extent, |pm| != 1, non-SU(3) links) */
    EOFA_ERR_UNSUPPORTED = 2,   /* Ls outside the compiled set, |gamma/alpha| >= 1, ... */
    EOFA_ERR_SINGULAR = 3,      /* N(m) = 0 or Sherman-Morrison denominator ~ 0 */
    EOFA_ERR_NOT_CONVERGED = 4, /* max_iter / max_outer reached */
    EOFA_ERR_NONFINITE = 5,     /* NaN or Inf met in a reduction */
    EOFA_ERR_TIMEOUT = 6,       /* timeout_ms exceeded */
    EOFA_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    EOFA_ERR_OOM = 8            /* device allocation failed */
} eofa_status;

/* Storage precision of the inner Krylov solver (arithmetic is FP64 for
 * EOFA_F64 and FP32 for the others). */
typedef enum {
    EOFA_F64 = 0,
    EOFA_F32 = 1,
    EOFA_F16 = 2,   /* half spinors with one FP32 scale per 5D site */
    EOFA_BF16 = 3
} eofa_prec;

/* Physics parameters (Eq. Ddwf, Eq. generic_eofa_system). */
typedef struct {
    int dims[4];      /* X, Y, Z, T (each even) */
    int Ls;           /* fifth-dimension extent (even) */
    double M5;        /* domain wall height */
    double b, c;      /* Moebius b5, c5 */
    double m1;        /* mass of H(m1), of D_DWF(m1) and of D~(m1) */
    double m2, m3;    /* masses of the shift Delta_pm(m2, m3) */
    double beta;      /* coefficient of the shift (0: plain D_DWF / H solve) */
    int pm;           /* +1 or -1: chirality of the shift term */
    int t_bc;         /* +1 periodic or -1 antiperiodic time */
} eofa_params;

/* Solver options.  Zero-initialise and set what you need; tol is required. */
typedef struct {
    double tol;          /* target true relative residual ||b - A x|| / ||b|| */
    int max_iter;        /* cap on total inner CG iterations (0: 100000) */
    int inner;           /* eofa_prec of the inner solver (EOFA_F64 = plain FP64 CG) */
    double inner_tol;    /* inner relative tolerance of defect correction (0: per precision) */
    int max_outer;       /* cap on outer defect-correction steps (0: 100) */
    int precond;         /* 0: none.  1: learned preconditioner (needs eofa_set_preconditioner) */
    int use_guess;       /* 1: sol holds an initial guess on entry */
    int rhs_form;        /* 0: H form, rhs = phi, sol = psi.  1: K form, rhs = b, sol = psi' (K psi' = b) */
    int kernel_timing;   /* 1: time every hop kernel with CUDA events (no graph capture) */
    int method;          /* inner operator.  0: the Cayley form (right preconditioning by
                            D~(m1)^-1, O(Ls) site-diagonal inverse, App. B).  1: even-odd
                            on Eq. (non_hermit_sys) directly, with the dense Ls x Ls inverse
                            of its site-diagonal block (the "dense" scheme the paper compares
                            against, Sec. V.B); same outer loop, for comparison */
    long timeout_ms;     /* 0: none; otherwise wall-clock limit checked between chunks */
} eofa_solve_opts;

/* Statistics of one solve. */
typedef struct {
    int status;          /* eofa_status of the solve */
    int outer_iters;     /* defect-correction steps (1 for a plain FP64 solve) */
    int inner_iters;     /* CG iterations summed over all inner solves */
    int hop_launches;    /* hop kernels timed: every inner-solver hop with kernel_timing = 1;
                            otherwise a sample, the four hops of one CG iteration per inner
                            solve, timed by events inside the solver's CUDA graph */
    double true_res;     /* FP64 ||rhs - A sol|| / ||rhs|| on the full lattice */
    double recur_res;    /* last recursively updated residual (relative) */
    double seconds;      /* wall-clock time of the call */
    double hop_ms;       /* summed time of the timed hop kernels */
    double hop_bytes;    /* algorithmic bytes moved by the timed hop kernels */
    long kernel_launches;/* kernels this library launched during the call */
    int precond_iters;   /* flexible-GCR steps with the learned preconditioner (precond = 1) */
    int precond_fallbacks; /* inner solves handed to CGNR because a GCR cycle did not halve |r| */
    double precond_ms;   /* device time of the network applications (precond = 1; CUDA events) */
} eofa_solve_stats;

typedef struct eofa_ctx eofa_ctx;

/* Create a context: validates params, builds the fifth-dimension
 * coefficients (u_pm, v_pm, the cyclic-bidiagonal inverse and the
 * Sherman-Morrison factors of App. B) and copies the gauge field.
 * gauge: device pointer, layout above.  *out is NULL on failure. */
eofa_status eofa_create(const eofa_params *p, const void *gauge, void *stream,
                        eofa_ctx **out);

/* Create a context with G-parity boundary conditions (Sec. I): the light
 * doublet maps as (u, d) -> (d-bar, -u-bar) across the boundary of every
 * direction mu with bit mu of gparity_dirs set (1..15; bit 0 = x ... bit 3 =
 * t).  The operator acts on two flavours, psi_1 = u and psi_2 = C d-bar^T:
 * flavour 2 sees the conjugate links U*, and a hop across a G-parity
 * boundary changes flavour with psi_1(x + L mu^) = psi_2(x) and
 * psi_2(x + L mu^) = -psi_1(x); t_bc multiplies hops across the t boundary
 * as before.  p->dims and gauge are the physical lattice and links.
 * Every field of this context holds both flavours stacked along t:
 * 5D [f][t][z][y][x][s][spin][colour] and 4D [f][t][z][y][x][spin][colour],
 * twice the single-flavour size; internally the context is the
 * single-flavour solver on X x Y x Z x 2T, so every call (solve, action,
 * heatbath, force) works unchanged.  eofa_force returns the force on the
 * physical links (flavour 1's link plus the conjugate of flavour 2's). */
eofa_status eofa_create_gparity(const eofa_params *p, const void *gauge, int gparity_dirs,
                                void *stream, eofa_ctx **out);

/* out = K in, K = D_DWF(m1) + pm beta u_pm (x) v_pm P_pm (App. B).
 * in, out: device complex128 5D fields; in != out. */
eofa_status eofa_apply(eofa_ctx *ctx, const void *in, void *out, void *stream);

/* out = K^dag in. */
eofa_status eofa_apply_dag(eofa_ctx *ctx, const void *in, void *out, void *stream);

/* out = (H(m1) + beta Delta_pm(m2,m3) P_pm) in = g5 R5 K D~(m1)^-1 in
 * (Eq. generic_eofa_system). */
eofa_status eofa_apply_h(eofa_ctx *ctx, const void *in, void *out, void *stream);

/* Solve the EOFA system.  rhs, sol: device complex128 5D fields.
 * rhs_form 0 (H form): (H(m1) + beta Delta_pm P_pm) sol = rhs.
 * rhs_form 1 (K form): K sol = rhs.
 * Plain FP64 CGNR when opts->inner == EOFA_F64, otherwise restarted
 * defect correction (FP64 outer residual and update, inner CGNR in the
 * requested storage precision), Sec. V.A.  stats may be NULL. */
eofa_status eofa_solve(eofa_ctx *ctx, const void *rhs, void *sol,
                       const eofa_solve_opts *opts, eofa_solve_stats *stats,
                       void *stream);

/* eofa_solve with the right-hand side and the solution in HOST memory
 * (complex128, same layout), on `stream`; returns when the solution is in
 * `sol`.  A page-locked rhs (cudaHostAlloc, cudaHostRegister, torch
 * pin_memory) is read in place by the solver's import kernels through its
 * device mapping (over NVLink-C2C on a Grace-Blackwell node); a pageable one
 * is copied to a device work field first.  The solution is exported to a
 * device work field; into a page-locked sol it is copied by the copy engine
 * on a second stream of the context while the FP64 true residual is
 * computed, into a pageable sol after the solve.  The two 5D work fields are
 * allocated by the context on first use and kept (the same ones the action
 * calls use).  With opts->use_guess, sol holds the initial guess on entry
 * (read in place when page-locked).  sol is written whenever the solver has
 * produced a solution (EOFA_OK, EOFA_ERR_NOT_CONVERGED, EOFA_ERR_TIMEOUT,
 * and EOFA_ERR_NONFINITE met in the iterations); argument errors, a
 * non-finite right-hand side and CUDA errors leave it untouched.
 * End-to-end entry of the solve as Sec. V.A describes it (the paper has no
 * separate host form). */
eofa_status eofa_solve_host(eofa_ctx *ctx, const double *rhs, double *sol,
                            const eofa_solve_opts *opts, eofa_solve_stats *stats,
                            void *stream);

/* ---------------------------------------------------------------------------
 * EOFA action and heatbath (Sec. III.A Eq. eofa_action, Sec. III.B
 * Eq. eofa_heatbath, App. A).  These reuse the context's lattice and gauge
 * field with other masses, shifts and chiralities: eofa_set_system switches
 * the context's own system; the two action calls switch it per solve and
 * restore the caller's system before they return (also on failure).
 *
 * 4D fields (phi, out, eta): device complex128 [t][z][y][x][spin][colour],
 * 24 * X*Y*Z*T doubles.  Omega_pm and k are the App. A closed forms for the
 * context's Moebius b, c and Ls.  Every solve is an H-form eofa_solve with
 * the caller's opts (tol, inner precision, method, max_iter, timeout; rhs_form
 * and use_guess are set by the call).  A solve that does not converge
 * leaves its best iterate in the result and its status in stats; the call
 * then returns EOFA_ERR_NOT_CONVERGED after finishing every solve.  Any
 * other failing status stops the call.  The calls allocate canonical 5D work
 * fields (up to four plus two per forecast vector, 24 * Ls * X*Y*Z*T doubles
 * each) in the context on first use and keep them until eofa_destroy.
 * ------------------------------------------------------------------------- */

/* Make the context solve (H(m1) + beta Delta_pm(m2, m3) P_pm) psi = phi:
 * the fifth-dimension coefficients are rebuilt on the host; the captured
 * solver graphs are rebuilt at the next solve.  EOFA_ERR_ARG for |pm| != 1
 * or non-finite values; EOFA_ERR_SINGULAR as for eofa_create (the context
 * then keeps its previous system). */
eofa_status eofa_set_system(eofa_ctx *ctx, double m1, double m2, double m3, double beta, int pm);

/* out = M_EOFA(m1, m2) phi, Eq. (eofa_action):
 *   phi - k P_- Omega_-^dag H(m1)^-1 Omega_- P_- phi
 *       + k P_+ Omega_+^dag [H(m2) - Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ phi,
 * k = k(m1, m2).  Two H-form solves; stats: NULL or 2 entries (the minus,
 * then the plus term).  phi != out.  Returns after the work has finished. */
eofa_status eofa_apply_meofa(eofa_ctx *ctx, double m1, double m2, const void *phi, void *out,
                             const eofa_solve_opts *opts, eofa_solve_stats *stats, void *stream);

/* phi = M_EOFA(m1, m2)^(-1/2) eta through the rational approximation
 * x^(-1/2) ~ alpha[0] + sum_{l<np} alpha[l+1] / (x + beta[l]) in the form of
 * Eq. (eofa_heatbath): with gamma_l = 1 / (1 + beta_l),
 *   phi = alpha_0 eta + sum_l alpha_l gamma_l { eta
 *         + k gamma_l P_- Omega_-^dag [H(m1) - gamma_l Delta_-(m1, m2) P_-]^-1 Omega_- P_- eta
 *         - k gamma_l P_+ Omega_+^dag [H(m2) - beta_l gamma_l Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ eta }.
 * 2 np H-form solves, per pole the minus then the plus term.
 * alpha: np + 1 host doubles; beta: np host doubles, each > -1.
 * pole_tol: NULL, or 2 np host tolerances replacing opts->tol per solve
 *   (entry 2l the minus, 2l+1 the plus solve of pole l; <= 0 keeps
 *   opts->tol): the per-pole stopping conditions of Sec. V.B.
 * forecast_n: 0, or up to 8: each solve starts from the chronological
 *   guess of Sec. V.B, sum_k c_k psi_k over the last forecast_n solutions
 *   psi_k of the same term, with sum_k c_k psi_l^dag A psi_k = psi_l^dag b for
 *   the current system A and source b (Gauss-Jordan on the host; no guess
 *   when that small system is singular).
 * stats: NULL or 2 np entries in solve order.  eta != phi.  Returns after
 * the work has finished. */
eofa_status eofa_heatbath(eofa_ctx *ctx, double m1, double m2, int np, const double *alpha,
                          const double *beta, const double *pole_tol, int forecast_n,
                          const void *eta, void *phi, const eofa_solve_opts *opts,
                          eofa_solve_stats *stats, void *stream);

/* EOFA pseudofermion force of S = phi^dag M_EOFA(m1, m2) phi, Sec. III.C
 * Eq. (eofa_force): with chi_1 = H(m1)^-1 Omega_- P_- phi and
 * chi_2 = [H(m2) - Delta_+(m1, m2) P_+]^-1 Omega_+ P_+ phi (two H-form
 * solves),
 *   d^a S = k (g5 R5 chi_1)^dag (d^a D_W) chi_1 - k (g5 R5 chi_2)^dag (d^a D_W) chi_2,
 * d^a the derivative along U_mu(x) -> exp(s T^a) U_mu(x) at s = 0,
 * T^a = i lambda_a / 2 (Tr T^a T^b = -delta^ab / 2).  force: device
 * complex128 [t][z][y][x][mu][3][3] (the gauge layout) receives
 * F_mu(x) = sum_a T^a d^a S, anti-Hermitian and traceless.  The links are
 * the context's own.  stats: NULL or 2 entries (chi_1, chi_2).  Returns
 * after the work has finished. */
eofa_status eofa_force(eofa_ctx *ctx, double m1, double m2, const void *phi, void *force,
                       const eofa_solve_opts *opts, eofa_solve_stats *stats, void *stream);

/* Force norms of Sec. VI (Eqs. L2_force, Linf_force) of a force in the layout
 * eofa_force writes (device complex128 [t][z][y][x][mu][3][3] on the
 * context's physical lattice): with ||F_mu(x)||^2 = sum_a (F^a_mu(x))^2 =
 * 2 sum_ij |F_ij|^2 (Tr T^a T^b = -delta^ab / 2),
 * f_rms = [sum_{x,mu} ||F_mu(x)||^2]^(1/2) / (4V) as printed and
 * f_max = max_{x,mu} ||F_mu(x)||.  One pass over the force on the device;
 * synchronises stream. */
eofa_status eofa_force_norms(eofa_ctx *ctx, const void *force, double *f_rms, double *f_max,
                             void *stream);

/* <a, b> = sum_i conj(a_i) b_i over n complex128 elements of device arrays
 * (FP64, summed in a fixed order: the same result every call), for the
 * set-up and diagnostics around the solves (Rayleigh quotients, norms, the
 * heatbath error of Eq. heatbath_rel_err).  Uses the context's reduction
 * buffers; synchronises stream. */
eofa_status eofa_dot(eofa_ctx *ctx, const void *a, const void *b, long n, double *re, double *im,
                     void *stream);

/* out[i] = K in[i] (dag = 0) or K^dag in[i] (dag = 1) for n contexts,
 * which may have different lattices. */
eofa_status eofa_apply_batched(eofa_ctx *const *ctx, int n, const void *const *in,
                               void *const *out, int dag, void *stream);

/* n independent solves (one per context and rhs), possibly of different
 * lattice sizes; stats is an array of n entries (or NULL).  Returns the
 * first non-OK status.  The mixed-precision defect correction of Sec. IV
 * (Eq. generic_eofa_system solved on the even-odd Schur complement, FP64
 * outer residual and update, inner CGNR in opts->inner) of all n systems is
 * one CUDA graph launch: each system's outer decision (converged, caps,
 * deadline, non-finite) and inner restart are taken on the device, so the
 * systems advance independently and the host waits once.  The graph is
 * kept for later calls on the same contexts in the same order (dropped by
 * eofa_set_system or eofa_destroy of any of them).  Each system's outer
 * steps and inner iterations equal those of its eofa_solve.  With
 * opts->kernel_timing, opts->precond or opts->method set the systems are
 * solved one by one.  Contexts must be distinct.  More than 32 systems run
 * as several graphs of at most 32.  The message of a failing status is
 * reported on ctx[0] (eofa_last_error), prefixed "system i: " when it
 * belongs to another system. */
eofa_status eofa_solve_batched(eofa_ctx *const *ctx, int n, const void *const *rhs,
                               void *const *sol, const eofa_solve_opts *opts,
                               eofa_solve_stats *stats, void *stream);

/* Release the context and all its device memory. */
void eofa_destroy(eofa_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Learned preconditioner.  The paper preconditions only with even-odd and
 * Cayley form; this is an additional preconditioner for the inner solver.
 *
 * Network: three 3^4 convolutions over the full 4D lattice, periodic in
 * every direction, applied to each s-slice on its own (the slices are the
 * batch); real channels 24 -> 32 -> 32 -> 24 (the spinor's 12 complex
 * spin-colour components in the order [spin][colour][re, im]); no biases;
 * LeakyReLU with slope 0.1 after the first two layers.  On the device the
 * weights and activations are BF16 and the products accumulate in FP32 on
 * the tensor cores (forward and input-gradient products with tcgen05.mma
 * into tensor memory, weight gradients with mma.sync).  The tcgen05
 * convolution bounds its waits on the tensor cores; should one expire, the
 * call returns EOFA_ERR_TIMEOUT (forward, backward, training, and a solve
 * with the preconditioner) instead of a result.
 *
 * Weights: EOFA_NET_WEIGHTS host floats, the three layers one after another,
 * each as W[tap][co][ci] with (ci, co) = (24, 32), (32, 32), (32, 24) and
 * tap = ((dt*3 + dz)*3 + dy)*3 + dx for the neighbour offset
 * (dx-1, dy-1, dz-1, dt-1):  y[x][co] = sum_tap sum_ci W[tap][co][ci] in[x+off][ci].
 * ------------------------------------------------------------------------- */
#define EOFA_NET_WEIGHTS 207360

/* out = net(in) for nslices 4D fields of dims {X, Y, Z, T}.  in, out: device
 * FP32 arrays [slice][t][z][y][x][24].  Allocates and frees its own device
 * work space; synchronises stream. */
eofa_status eofa_net_forward(const float *weights, const int dims[4], int nslices,
                             const void *in, void *out, void *stream);

/* Gradients of a loss L through the network at input `in`: given
 * dout = dL/d(out) (device FP32, layout of out) writes dL/dW to the host
 * array dweights (EOFA_NET_WEIGHTS floats) and, if din is not NULL,
 * dL/d(in) to device memory.  Synchronises stream. */
eofa_status eofa_net_backward(const float *weights, const int dims[4], int nslices,
                              const void *in, const void *dout, float *dweights, void *din,
                              void *stream);

typedef struct {
    int pairs;            /* (residual, error) slice pairs to train on (e.g. 2000) */
    int snapshot_every;   /* CG iterations between snapshots of the iterate */
    int epochs;           /* passes over the pairs */
    int batch;            /* slices per Adam step, at most Ls/2 */
    double lr;            /* Adam step size */
    double solve_tol;     /* relative tolerance of the FP32 solves that make the pairs */
    int holdout;          /* further pairs, harvested after the training pairs and never
                             trained on, to measure what training gains (0: none) */
} eofa_train_opts;

typedef struct {
    int pairs, steps, solves;
    double loss_first;    /* mean relative squared error of the first step */
    double loss_last;     /* same, last step */
    double seconds;
    int holdout_pairs;        /* held-out pairs found (<= opts->holdout) */
    double holdout_loss_init; /* mean relative squared error on them, initial weights */
    double holdout_loss_final;/* same, trained weights */
} eofa_train_stats;

/* Train the network on the context's lattice.  For each source (device
 * complex128 5D fields, H form) the inner FP32 CGNR on the Schur complement
 * runs to solve_tol with snapshots x_k of its iterate; with the converged
 * x*, each snapshot gives the pair (r_k = S (x* - x_k), e_k = x* - x_k)
 * restricted to one s-slice.  Adam on the relative squared error
 * |net(r) - e|^2 / |e|^2 over the odd sites, starting from init_weights
 * (host; the random initial values are the caller's).  The trained weights
 * go to weights_out (host).  Sources must be enough to give `pairs` pairs;
 * with opts->holdout > 0 the sources' further pairs (up to holdout) are kept
 * out of training and the loss on them is reported for the initial and the
 * trained weights. */
eofa_status eofa_train_preconditioner(eofa_ctx *ctx, const void *const *sources, int n_sources,
                                      const float *init_weights, const eofa_train_opts *opts,
                                      float *weights_out, eofa_train_stats *stats, void *stream);

/* Load network weights (host FP32) into the context; eofa_solve with
 * opts->precond = 1 then runs the inner solve as flexible GCR(4) on the
 * Schur complement with z = net(r) as the preconditioner (FP32), falling back
 * to CGNR when a restart cycle fails to halve the residual.  The FP64 outer
 * defect correction and the true-residual check are unchanged. */
eofa_status eofa_set_preconditioner(eofa_ctx *ctx, const float *weights);

/* out = K in, the same result as eofa_apply, for callers that cannot call
 * cudaMalloc: for example a host framework that owns all device memory
 * through its own pool and forbids allocations behind its back, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation
 * is not acceptable.  The paper has no counterpart of this call; it exists
 * only for such callers.
 *
 * It needs no context and allocates nothing.  p, gauge, in and out are as
 * for eofa_create and eofa_apply (device pointers, layouts above).  The
 * work space -- two-row links, the even-odd copies of in and out, a check
 * flag -- is one static device array of about 15 MiB inside the library,
 * which every GPU that loads the library holds until the process exits.
 * Maximum size: X*Y*Z*T <= 4096 and X*Y*Z*T*Ls <= 32768 (e.g. 8^4 x 8);
 * larger lattices return EOFA_ERR_UNSUPPORTED before any device work.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any
 * stream capture.  The call checks that the links are SU(3) (EOFA_ERR_ARG
 * otherwise), which reads a flag back, so it returns after its work on
 * `stream` has finished; for the same reason it cannot be recorded into a
 * CUDA graph, and on a stream that is being captured it returns
 * EOFA_ERR_UNSUPPORTED without touching the capture.  Every call shares
 * the one array and it keeps the
 * last call's contents: calls that overlap on the GPU (other streams, other
 * host threads) race and must not be issued. */
eofa_status eofa_apply_noalloc(const eofa_params *p, const void *gauge, const void *in,
                               void *out, void *stream);

/* Measured throughput of the device's fused multiply-add pipe, a
 * measurement utility with no counterpart in the paper: prec EOFA_F64 or
 * EOFA_F32; a kernel of independent FMA chains (one CTA set per SM of the
 * current device) is timed with CUDA events on `stream` after a warm-up,
 * and *tflops receives 2 x FMAs / seconds / 1e12 (the best of `reps`
 * launches, reps >= 1).  Synchronises the stream.  EOFA_ERR_ARG for a bad
 * prec, reps or NULL tflops. */
eofa_status eofa_measure_fma(int prec, int reps, double *tflops, void *stream);

/* Static description of a status code. */
const char *eofa_status_string(eofa_status s);

/* Message of the last failing call on ctx (empty string if none). */
const char *eofa_last_error(const eofa_ctx *ctx);

/* Algorithmic bytes of one hop-kernel launch in storage precision prec:
 * per output 5D site 2*24 reals of spinor plus 8 two-row links shared
 * over Ls, plus 24 reals of the local vector when the kernel reads one. */
double eofa_hop_bytes(const eofa_ctx *ctx, int prec, int with_local);

/* 4D sites per CTA that the library's autotuner chose for hop kernel `kind`
 * of the inner solver (0: S step 1, 1: S step 2, 2: S^dag step 1, 3: S^dag
 * step 2) in precision prec; the default tile if that precision has not been
 * used by a solve yet.  Block and tile shapes are timed on the context's own
 * buffers at its first solve in a precision and cached per lattice shape. */
int eofa_tile_sites(const eofa_ctx *ctx, int prec, int kind);

/* The tile variant chosen for the same kernel: bit 0 set for the
 * alternative CTA shape, bit 1 set when the kernel is compiled with a
 * register cap (about 72 per thread: more resident warps; FP32 arithmetic
 * only).
 * 0 before the first solve in that precision, -1 for invalid arguments.
 * The environment variable EOFA_TILE_VARIANT=0..3, read when a context
 * first tunes a precision, replaces the timing by that fixed variant. */
int eofa_tile_variant(const eofa_ctx *ctx, int prec, int kind);

/* The autotuner's measurement behind that choice: milliseconds per launch of
 * tile variant `variant` (0..3) of hop kernel `kind` in precision prec, the
 * fastest of three rounds of three launches on the context's own buffers
 * (the dslash sweep over tile shapes; FP64 has variants 0 and 1 only).  0
 * when that variant was not timed (not compiled for the precision, the
 * variant fixed by EOFA_TILE_VARIANT, or no solve in that precision yet);
 * -1 for invalid arguments.  Contexts of a lattice shape already tuned in the
 * process report the first context's times. */
double eofa_tile_time(const eofa_ctx *ctx, int prec, int kind, int variant);

#ifdef __cplusplus
}
#endif

#endif /* EOFA_H */
