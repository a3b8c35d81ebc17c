/*
 * eofa_oracle.c -- plain, slow, FP64 CPU oracle for the EOFA Dirac-equation
 * solve of Jung, Kelly, Mawhinney, Murphy, "Domain wall fermion QCD with the
 * exact one flavor algorithm" (arXiv:1706.05843).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
 * run this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header, table or
 * helper with the CUDA library; both sides take their inputs from the seeded
 * generators in paper_1706_05843_gb300/inputs.py.
 *
 * Every operator here is the plain definition from the paper, written with
 * explicit 4x4 gamma matrices, explicit 3x3 links and explicit Ls x Ls
 * fifth-dimension matrices, with no even-odd blocking, fusion or reordering:
 *
 *   D_W, L, D_DWF      Eq. (Ddwf), Sec. II
 *   D_EOFA, D~         Eq. (eofa_dop), Eq. (eofa_dop_def), Sec. II
 *   M+-, Delta+-, k,   App. A (Moebius kernel, Eqs. mobius_Mp, mobius_Mm,
 *   Omega+-, D~^-1     mobius_Dp, mobius_Dm and the D~, D~^-1 closed forms)
 *   H = g5 R5 D_EOFA   Sec. II, above Eq. (eofa_action)
 *   EOFA system        Eq. (generic_eofa_system) / Eq. (hermit_indef_sys),
 *                      and its g5R5-rotated form Eq. (non_hermit_sys), App. B
 *   Cayley form K      Eq. (precond_mobius_eofa_system), Eq. (delta_rank_one),
 *                      u+-, v+- and Eqs. (Mooee_shift_p), (Mooee_shift_m)
 *   CGNR               conjugate gradient on the normal equations, App. B
 *
 * Parameters: the interface takes the Moebius coefficients b5 = b and c5 = c
 * of D_DWF = (b5 D_W + 1) + (c5 D_W - 1) L.  The paper writes them as
 * b5 = c + d and c5 = c - d with d = 1/2 (Sec. II); the oracle converts once,
 * cp = (b5 + c5)/2 and d = (b5 - c5)/2, and then uses the paper's (c, d)
 * formulas verbatim.  (The closed forms hold for any d, not only d = 1/2.)
 *
 * Readings of the paper taken here:
 *  - In (c5 D_W - 1) L the operator L acts first (the order in which
 *    D_DWF = D_EOFA D~ holds).
 *  - Chiral gamma basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *    gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
 *  - mu = 0, 1, 2, 3 is x, y, z, t; hops across the t boundary carry the
 *    factor t_bc (-1: antiperiodic), space is periodic.
 *  - u+- carry the D~ mass m1; v+- carry k(m2, m3) of the shift.
 *  - The +- in Eq. (precond_mobius_eofa_system) is the chirality of the
 *    shift (pm), i.e. K = D_DWF(m1) + pm * beta * u (x) v P_pm.
 *  - Solver residual: ||b - A x|| / ||b|| on the full, unpreconditioned
 *    system.
 *
 * Layouts (complex128, C order):
 *   gauge  U[t][z][y][x][mu][row][col]
 *   5D     psi[t][z][y][x][s][spin][colour]
 *   4D     chi[t][z][y][x][spin][colour]
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cd;

typedef struct {
    int dims[4];      /* X, Y, Z, T */
    int Ls;
    double M5;
    double b, c;      /* Moebius b5, c5 */
    double m1, m2, m3;
    double beta;      /* coefficient of the shift term */
    int pm;           /* +1 or -1: chirality of the shift term */
    int t_bc;         /* +1 periodic, -1 antiperiodic in time */
} oracle_params;

/* ------------------------------------------------------------------ */
/* basic helpers                                                       */
/* ------------------------------------------------------------------ */

static long vol4(const oracle_params *p)
{
    return (long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
}

static long len5(const oracle_params *p) { return vol4(p) * p->Ls * 12; }

static double paper_c(const oracle_params *p) { return 0.5 * (p->b + p->c); }
static double paper_d(const oracle_params *p) { return 0.5 * (p->b - p->c); }

/* integer power with sign-safe handling of negative exponents */
static double ipow(double x, int n)
{
    double r = 1.0;
    if (n < 0) { x = 1.0 / x; n = -n; }
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

static double sgn(int n) { return (n % 2 == 0) ? 1.0 : -1.0; }

static long site_index(const oracle_params *p, int x, int y, int z, int t)
{
    return (((long)t * p->dims[2] + z) * p->dims[1] + y) * p->dims[0] + x;
}

static void site_coords(const oracle_params *p, long i, int c[4])
{
    c[0] = (int)(i % p->dims[0]); i /= p->dims[0];
    c[1] = (int)(i % p->dims[1]); i /= p->dims[1];
    c[2] = (int)(i % p->dims[2]); i /= p->dims[2];
    c[3] = (int)i;
}

/* N(m) = (c+d)^Ls + m (c-d)^Ls, the normalisation of App. A. */
static double norm_N(const oracle_params *p, double m)
{
    double cp = paper_c(p), d = paper_d(p);
    return ipow(cp + d, p->Ls) + m * ipow(cp - d, p->Ls);
}

/* ------------------------------------------------------------------ */
/* gamma matrices (chiral basis)                                       */
/* ------------------------------------------------------------------ */

static cd GAM[5][4][4];   /* gamma_1..gamma_4 stored at 0..3, gamma_5 at 4 */
static int gam_ready = 0;

static void build_gammas(void)
{
    if (gam_ready) return;
    const cd sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAM, 0, sizeof(GAM));
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                GAM[k][a][2 + b] = -I * sig[k][a][b];
                GAM[k][2 + a][b] = I * sig[k][a][b];
            }
    for (int a = 0; a < 2; ++a) {
        GAM[3][a][2 + a] = 1;
        GAM[3][2 + a][a] = 1;
    }
    /* gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 */
    cd t1[4][4], t2[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cd s = 0;
            for (int k = 0; k < 4; ++k) s += GAM[0][i][k] * GAM[1][k][j];
            t1[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cd s = 0;
            for (int k = 0; k < 4; ++k) s += t1[i][k] * GAM[2][k][j];
            t2[i][j] = s;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cd s = 0;
            for (int k = 0; k < 4; ++k) s += t2[i][k] * GAM[3][k][j];
            GAM[4][i][j] = s;
        }
    gam_ready = 1;
}

/* Copy gamma matrix (mu = 0..3 -> gamma_1..gamma_4, mu = 4 -> gamma_5). */
void oracle_gamma(int mu, cd *out16)
{
    build_gammas();
    memcpy(out16, GAM[mu], sizeof(GAM[mu]));
}

/* chiral projector P_chi = (1 + chi gamma_5)/2 applied to one spinor */
static void proj_chi(int chi, const cd *in12, cd *out12)
{
    for (int a = 0; a < 4; ++a)
        for (int col = 0; col < 3; ++col) {
            cd s = 0;
            for (int b = 0; b < 4; ++b) {
                cd pab = 0.5 * ((a == b ? 1.0 : 0.0) + chi * GAM[4][a][b]);
                s += pab * in12[b * 3 + col];
            }
            out12[a * 3 + col] = s;
        }
}

static void gamma5_apply(const cd *in12, cd *out12)
{
    for (int a = 0; a < 4; ++a)
        for (int col = 0; col < 3; ++col) {
            cd s = 0;
            for (int b = 0; b < 4; ++b) s += GAM[4][a][b] * in12[b * 3 + col];
            out12[a * 3 + col] = s;
        }
}

/* ------------------------------------------------------------------ */
/* D_W: 4D Wilson operator, Eq. (Ddwf) second line                     */
/* ------------------------------------------------------------------ */

/*
 * D_W psi(x) = (4 - M5) psi(x)
 *   - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ].
 * Its adjoint is obtained element by element: the forward term
 * (1 - gamma) U(x) delta_{x+mu,x'} becomes (1 - gamma) U(x-mu)^dag
 * delta_{x-mu,x'} and the backward term becomes (1 + gamma) U(x)
 * delta_{x+mu,x'}, i.e. the two projectors trade places.
 *
 * Applied here to every s-slice of a 5D field (nslice = Ls; a 4D field is
 * nslice = 1).
 */
static void dw_apply(const oracle_params *p, const cd *U, const cd *in,
                     cd *out, int nslice, int dag)
{
    build_gammas();
    const long V = vol4(p);
    const double diag = 4.0 - p->M5;
    const double sf = dag ? +1.0 : -1.0; /* forward projector 1 + sf*gamma */
#pragma omp parallel for schedule(static)
    for (long xi = 0; xi < V; ++xi) {
        int co[4];
        site_coords(p, xi, co);
        for (int s = 0; s < nslice; ++s) {
            cd acc[12];
            const cd *src = in + (xi * nslice + s) * 12;
            for (int k = 0; k < 12; ++k) acc[k] = diag * src[k];
            for (int mu = 0; mu < 4; ++mu) {
                for (int dir = 0; dir < 2; ++dir) {
                    int cn[4] = {co[0], co[1], co[2], co[3]};
                    double phase = 1.0;
                    if (dir == 0) {
                        cn[mu] = (co[mu] + 1) % p->dims[mu];
                        if (mu == 3 && co[3] == p->dims[3] - 1) phase = p->t_bc;
                    } else {
                        cn[mu] = (co[mu] - 1 + p->dims[mu]) % p->dims[mu];
                        if (mu == 3 && co[3] == 0) phase = p->t_bc;
                    }
                    long ni = site_index(p, cn[0], cn[1], cn[2], cn[3]);
                    const cd *nb = in + (ni * nslice + s) * 12;
                    /* link: forward U_mu(x); backward U_mu(x-mu)^dag */
                    cd W[3][3];
                    if (dir == 0) {
                        const cd *u = U + (xi * 4 + mu) * 9;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) W[a][b] = u[a * 3 + b];
                    } else {
                        const cd *u = U + (ni * 4 + mu) * 9;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) W[a][b] = conj(u[b * 3 + a]);
                    }
                    /* colour multiply */
                    cd t[12];
                    for (int sp = 0; sp < 4; ++sp)
                        for (int a = 0; a < 3; ++a) {
                            cd sum = 0;
                            for (int b = 0; b < 3; ++b) sum += W[a][b] * nb[sp * 3 + b];
                            t[sp * 3 + a] = sum;
                        }
                    /* spin projector (1 + sg gamma_mu) */
                    double sg = (dir == 0) ? sf : -sf;
                    for (int sp = 0; sp < 4; ++sp)
                        for (int a = 0; a < 3; ++a) {
                            cd sum = t[sp * 3 + a];
                            for (int sq = 0; sq < 4; ++sq)
                                sum += sg * GAM[mu][sp][sq] * t[sq * 3 + a];
                            acc[sp * 3 + a] -= 0.5 * phase * sum;
                        }
                }
            }
            cd *dst = out + (xi * nslice + s) * 12;
            for (int k = 0; k < 12; ++k) dst[k] = acc[k];
        }
    }
}

void oracle_dw4(const oracle_params *p, const cd *U, const cd *in, cd *out, int dag)
{
    dw_apply(p, U, in, out, 1, dag);
}

void oracle_dw5(const oracle_params *p, const cd *U, const cd *in, cd *out, int dag)
{
    dw_apply(p, U, in, out, p->Ls, dag);
}

/* ------------------------------------------------------------------ */
/* fifth-dimension matrices                                            */
/* ------------------------------------------------------------------ */

/* (L_+)_{ss'} = -m delta_{Ls-1,s'} for s = 0, delta_{s-1,s'} otherwise;
 * (L_-)_{ss'} = (L_+)_{s's}.  Eq. (Ddwf). */
static double Lplus(int s, int sp, int Ls, double m)
{
    if (s == 0) return (sp == Ls - 1) ? -m : 0.0;
    return (sp == s - 1) ? 1.0 : 0.0;
}

void oracle_L_matrices(const oracle_params *p, double m, double *Lp, double *Lm)
{
    int Ls = p->Ls;
    for (int s = 0; s < Ls; ++s)
        for (int t = 0; t < Ls; ++t) {
            Lp[s * Ls + t] = Lplus(s, t, Ls, m);
            Lm[s * Ls + t] = Lplus(t, s, Ls, m);
        }
}

/*
 * out(x, s) = sum_s' [ A+_{ss'} P+ + A-_{ss'} P- ] in(x, s')  (trans = 0)
 * or with A+- transposed (trans = 1).  A+- real Ls x Ls, row major.
 * Either may be NULL (treated as zero).
 */
static void s_apply(const oracle_params *p, const double *Ap, const double *Am,
                    const cd *in, cd *out, int trans)
{
    build_gammas();
    const long V = vol4(p);
    const int Ls = p->Ls;
#pragma omp parallel for schedule(static)
    for (long xi = 0; xi < V; ++xi) {
        for (int s = 0; s < Ls; ++s) {
            cd acc[12];
            for (int k = 0; k < 12; ++k) acc[k] = 0;
            for (int t = 0; t < Ls; ++t) {
                const cd *src = in + (xi * Ls + t) * 12;
                cd pp[12], pm[12];
                proj_chi(+1, src, pp);
                proj_chi(-1, src, pm);
                double ap = 0.0, am = 0.0;
                if (Ap) ap = trans ? Ap[t * Ls + s] : Ap[s * Ls + t];
                if (Am) am = trans ? Am[t * Ls + s] : Am[s * Ls + t];
                for (int k = 0; k < 12; ++k) acc[k] += ap * pp[k] + am * pm[k];
            }
            cd *dst = out + (xi * Ls + s) * 12;
            for (int k = 0; k < 12; ++k) dst[k] = acc[k];
        }
    }
}

/* L = L+ P+ + L- P- (or its adjoint), mass m.  Eq. (Ddwf). */
void oracle_L(const oracle_params *p, double m, const cd *in, cd *out, int dag)
{
    int Ls = p->Ls;
    double *Lp = malloc(sizeof(double) * Ls * Ls);
    double *Lm = malloc(sizeof(double) * Ls * Ls);
    oracle_L_matrices(p, m, Lp, Lm);
    s_apply(p, Lp, Lm, in, out, dag);
    free(Lp);
    free(Lm);
}

/* ------------------------------------------------------------------ */
/* D_DWF, Eq. (Ddwf)                                                   */
/* ------------------------------------------------------------------ */

/*
 * D_DWF(m) psi = ((c+d) D_W + 1) psi + ((c-d) D_W - 1) (L psi)
 * D_DWF(m)^dag psi = ((c+d) D_W^dag + 1) psi + L^dag ((c-d) D_W^dag - 1) psi
 */
void oracle_ddwf(const oracle_params *p, const cd *U, double m, const cd *in,
                 cd *out, int dag)
{
    const long n = len5(p);
    const double cp = paper_c(p), d = paper_d(p);
    cd *t1 = malloc(sizeof(cd) * n);
    cd *t2 = malloc(sizeof(cd) * n);
    if (!dag) {
        oracle_dw5(p, U, in, t1, 0);          /* D_W psi */
        oracle_L(p, m, in, t2, 0);            /* L psi */
        cd *t3 = malloc(sizeof(cd) * n);
        oracle_dw5(p, U, t2, t3, 0);          /* D_W L psi */
        for (long i = 0; i < n; ++i)
            out[i] = (cp + d) * t1[i] + in[i] + (cp - d) * t3[i] - t2[i];
        free(t3);
    } else {
        oracle_dw5(p, U, in, t1, 1);          /* D_W^dag psi */
        for (long i = 0; i < n; ++i) t2[i] = (cp - d) * t1[i] - in[i];
        cd *t3 = malloc(sizeof(cd) * n);
        oracle_L(p, m, t2, t3, 1);            /* L^dag (...) */
        for (long i = 0; i < n; ++i) out[i] = (cp + d) * t1[i] + in[i] + t3[i];
        free(t3);
    }
    free(t1);
    free(t2);
}

/* D~(m) = d (1 - L) + c (1 + L), Eq. (eofa_dop_def); dag: L -> L^dag. */
void oracle_dtilde(const oracle_params *p, double m, const cd *in, cd *out, int dag)
{
    const long n = len5(p);
    const double cp = paper_c(p), d = paper_d(p);
    cd *t = malloc(sizeof(cd) * n);
    oracle_L(p, m, in, t, dag);
    for (long i = 0; i < n; ++i) out[i] = d * (in[i] - t[i]) + cp * (in[i] + t[i]);
    free(t);
}

/* ------------------------------------------------------------------ */
/* App. A closed forms (Moebius kernel)                                */
/* ------------------------------------------------------------------ */

/* k(mA, mB) = 2c (mB - mA) (c+d)^{2Ls} / (N(mA) N(mB)). */
double oracle_k(const oracle_params *p, double mA, double mB)
{
    double cp = paper_c(p), d = paper_d(p);
    return 2.0 * cp * (mB - mA) * ipow(cp + d, 2 * p->Ls) /
           (norm_N(p, mA) * norm_N(p, mB));
}

/* Omega_+-: the single column s' = 0 of the App. A expressions. */
void oracle_omega(const oracle_params *p, int pm, double *om)
{
    double cp = paper_c(p), d = paper_d(p);
    int Ls = p->Ls;
    for (int s = 0; s < Ls; ++s) {
        if (pm > 0)
            om[s] = sgn(s + 1) * ipow(cp - d, Ls - s - 1) / ipow(cp + d, Ls - s);
        else
            om[s] = sgn(s) * ipow(cp - d, s) / ipow(cp + d, s + 1);
    }
}

/* Delta_+-(mA, mB), Eqs. (mobius_Dp), (mobius_Dm). */
void oracle_delta(const oracle_params *p, double mA, double mB, int pm, double *D)
{
    double cp = paper_c(p), d = paper_d(p);
    int Ls = p->Ls;
    double den = norm_N(p, mA) * norm_N(p, mB);
    for (int s = 0; s < Ls; ++s)
        for (int t = 0; t < Ls; ++t) {
            double v;
            if (pm > 0)
                v = sgn(s + t) * 2.0 * cp * (mB - mA) * ipow(cp + d, s + t) *
                    ipow(cp - d, 2 * (Ls - 1) - s - t) / den;
            else
                v = sgn(s + t) * 2.0 * cp * (mB - mA) *
                    ipow(cp + d, 2 * (Ls - 1) - s - t) * ipow(cp - d, s + t) / den;
            D[s * Ls + t] = v;
        }
}

/* M_+-(m), Eqs. (mobius_Mp), (mobius_Mm).  Terms whose Heaviside factor
 * vanishes are skipped rather than multiplied by zero, so that c = d
 * (Shamir) never meets 0^(negative). */
void oracle_mpm(const oracle_params *p, double m, double *Mp, double *Mm)
{
    double cp = paper_c(p), d = paper_d(p);
    int Ls = p->Ls;
    double N = norm_N(p, m);
    double dg = (ipow(cp + d, Ls - 1) - m * ipow(cp - d, Ls - 1)) / N;
    for (int s = 0; s < Ls; ++s)
        for (int t = 0; t < Ls; ++t) {
            double vp = 0.0, vm = 0.0;
            if (s - t - 1 >= 0) {
                vp += sgn(s - t) * 2.0 * cp * ipow(cp + d, Ls - s + t - 1) *
                      ipow(cp - d, s - t - 1) / N;
                vm += sgn(t - s + 1) * 2.0 * cp * m * ipow(cp + d, s - t - 1) *
                      ipow(cp - d, Ls - s + t - 1) / N;
            }
            if (s == t) { vp += dg; vm += dg; }
            if (t - s - 1 >= 0) {
                vp += sgn(s - t + 1) * 2.0 * cp * m * ipow(cp + d, t - s - 1) *
                      ipow(cp - d, Ls + s - t - 1) / N;
                vm += sgn(s - t) * 2.0 * cp * ipow(cp + d, Ls + s - t - 1) *
                      ipow(cp - d, t - s - 1) / N;
            }
            Mp[s * Ls + t] = vp;
            Mm[s * Ls + t] = vm;
        }
}

/* D~(m)^{-1}, the App. A closed form, chirality blocks (row major). */
void oracle_dtilde_inv_matrices(const oracle_params *p, double m, double *Ip, double *Im)
{
    double cp = paper_c(p), d = paper_d(p);
    int Ls = p->Ls;
    double N = norm_N(p, m);
    for (int s = 0; s < Ls; ++s)
        for (int t = 0; t < Ls; ++t) {
            double vp = m * sgn(s - t + 1) * ipow(cp + d, t - s - 1) *
                        ipow(cp - d, Ls + s - t) / N;
            if (s - t >= 0)
                vp += sgn(s - t) * ipow(cp - d, s - t) / ipow(cp + d, s - t + 1);
            double vm = m * sgn(t - s + 1) * ipow(cp + d, s - t - 1) *
                        ipow(cp - d, Ls + t - s) / N;
            if (t - s >= 0)
                vm += sgn(t - s) * ipow(cp - d, t - s) / ipow(cp + d, t - s + 1);
            Ip[s * Ls + t] = vp;
            Im[s * Ls + t] = vm;
        }
}

void oracle_dtilde_inv(const oracle_params *p, double m, const cd *in, cd *out)
{
    int Ls = p->Ls;
    double *Ip = malloc(sizeof(double) * Ls * Ls);
    double *Im = malloc(sizeof(double) * Ls * Ls);
    oracle_dtilde_inv_matrices(p, m, Ip, Im);
    s_apply(p, Ip, Im, in, out, 0);
    free(Ip);
    free(Im);
}

/* ------------------------------------------------------------------ */
/* D_EOFA, H and the EOFA system                                       */
/* ------------------------------------------------------------------ */

/* D_EOFA(m) = D_W delta_ss' + M+(m) P+ + M-(m) P-, Eq. (eofa_dop_def);
 * dag: D_W^dag + M+^T P+ + M-^T P-. */
void oracle_deofa(const oracle_params *p, const cd *U, double m, const cd *in,
                  cd *out, int dag)
{
    const long n = len5(p);
    int Ls = p->Ls;
    double *Mp = malloc(sizeof(double) * Ls * Ls);
    double *Mm = malloc(sizeof(double) * Ls * Ls);
    oracle_mpm(p, m, Mp, Mm);
    cd *t = malloc(sizeof(cd) * n);
    oracle_dw5(p, U, in, out, dag);
    s_apply(p, Mp, Mm, in, t, dag);
    for (long i = 0; i < n; ++i) out[i] += t[i];
    free(t);
    free(Mp);
    free(Mm);
}

/* gamma_5 R_5, with (R_5)_{ss'} = delta_{s, Ls-1-s'} (Sec. II). */
void oracle_g5r5(const oracle_params *p, const cd *in, cd *out)
{
    build_gammas();
    const long V = vol4(p);
    int Ls = p->Ls;
#pragma omp parallel for schedule(static)
    for (long xi = 0; xi < V; ++xi)
        for (int s = 0; s < Ls; ++s)
            gamma5_apply(in + (xi * Ls + (Ls - 1 - s)) * 12, out + (xi * Ls + s) * 12);
}

/* H(m) = gamma_5 R_5 D_EOFA(m) (Hermitian). */
void oracle_h(const oracle_params *p, const cd *U, double m, const cd *in, cd *out)
{
    cd *t = malloc(sizeof(cd) * len5(p));
    oracle_deofa(p, U, m, in, t, 0);
    oracle_g5r5(p, t, out);
    free(t);
}

/* beta Delta_pm(m2, m3) P_pm applied to in (added into out when acc). */
static void shift_term(const oracle_params *p, const cd *in, cd *out)
{
    int Ls = p->Ls;
    double *D = malloc(sizeof(double) * Ls * Ls);
    oracle_delta(p, p->m2, p->m3, p->pm, D);
    for (int i = 0; i < Ls * Ls; ++i) D[i] *= p->beta;
    if (p->pm > 0) s_apply(p, D, NULL, in, out, 0);
    else s_apply(p, NULL, D, in, out, 0);
    free(D);
}

/* (H(m1) + beta Delta_pm(m2,m3) P_pm) psi, Eq. (generic_eofa_system). */
void oracle_apply_hsys(const oracle_params *p, const cd *U, const cd *in, cd *out)
{
    const long n = len5(p);
    cd *t = malloc(sizeof(cd) * n);
    oracle_h(p, U, p->m1, in, out);
    shift_term(p, in, t);
    for (long i = 0; i < n; ++i) out[i] += t[i];
    free(t);
}

/* A = D_EOFA(m1) + beta g5 R5 Delta_pm(m2,m3) P_pm, Eq. (non_hermit_sys);
 * dag: D_EOFA^dag + beta P_pm Delta_pm^T R5 g5. */
void oracle_apply_asys(const oracle_params *p, const cd *U, const cd *in, cd *out, int dag)
{
    const long n = len5(p);
    cd *t = malloc(sizeof(cd) * n);
    cd *t2 = malloc(sizeof(cd) * n);
    oracle_deofa(p, U, p->m1, in, out, dag);
    int Ls = p->Ls;
    double *D = malloc(sizeof(double) * Ls * Ls);
    oracle_delta(p, p->m2, p->m3, p->pm, D);
    for (int i = 0; i < Ls * Ls; ++i) D[i] *= p->beta;
    if (!dag) {
        if (p->pm > 0) s_apply(p, D, NULL, in, t, 0);
        else s_apply(p, NULL, D, in, t, 0);
        oracle_g5r5(p, t, t2);
    } else {
        oracle_g5r5(p, in, t);     /* (g5 R5)^dag = R5 g5 = g5 R5 */
        if (p->pm > 0) s_apply(p, D, NULL, t, t2, 1);
        else s_apply(p, NULL, D, t, t2, 1);
    }
    for (long i = 0; i < n; ++i) out[i] += t2[i];
    free(D);
    free(t);
    free(t2);
}

/* ------------------------------------------------------------------ */
/* Cayley-form operator K, Eq. (precond_mobius_eofa_system)            */
/* ------------------------------------------------------------------ */

/* u_pm (with the D~ mass m1) and k(m2, m3) of v_pm = k e_{Ls-1 | 0}. */
void oracle_uv(const oracle_params *p, double *u, double *kout)
{
    double cp = paper_c(p), d = paper_d(p);
    int Ls = p->Ls;
    double N1 = norm_N(p, p->m1);
    for (int s = 0; s < Ls; ++s) {
        if (p->pm > 0)
            u[s] = sgn(s) * ipow(cp - d, s) / ipow(cp + d, Ls + s + 1) * N1;
        else
            u[s] = sgn(s + 1) * ipow(cp - d, Ls - 1 - s) / ipow(cp + d, 2 * Ls - s) * N1;
    }
    *kout = oracle_k(p, p->m2, p->m3);
}

/*
 * K = D_DWF(m1) + pm beta Delta~_pm, Delta~_pm = u_pm (x) v_pm acting on
 * the P_pm component:
 *   (Delta~_+ psi)_s = k u+_s P+ psi_{Ls-1},    (Delta~_- psi)_s = k u-_s P- psi_0
 *   (Delta~_+^dag psi)_s = k delta_{s,Ls-1} P+ sum_s' u+_s' psi_s'   (and -)
 * Eqs. (Mooee_shift_p), (Mooee_shift_m).
 */
void oracle_apply_k(const oracle_params *p, const cd *U, const cd *in, cd *out, int dag)
{
    build_gammas();
    int Ls = p->Ls;
    oracle_ddwf(p, U, p->m1, in, out, dag);
    double *u = malloc(sizeof(double) * Ls);
    double k;
    oracle_uv(p, u, &k);
    const double coef = p->pm * p->beta * k;
    const int jstar = (p->pm > 0) ? Ls - 1 : 0;
    const long V = vol4(p);
#pragma omp parallel for schedule(static)
    for (long xi = 0; xi < V; ++xi) {
        cd pj[12];
        if (!dag) {
            proj_chi(p->pm, in + (xi * Ls + jstar) * 12, pj);
            for (int s = 0; s < Ls; ++s)
                for (int q = 0; q < 12; ++q) out[(xi * Ls + s) * 12 + q] += coef * u[s] * pj[q];
        } else {
            cd sum[12];
            for (int q = 0; q < 12; ++q) sum[q] = 0;
            for (int s = 0; s < Ls; ++s)
                for (int q = 0; q < 12; ++q) sum[q] += u[s] * in[(xi * Ls + s) * 12 + q];
            proj_chi(p->pm, sum, pj);
            for (int q = 0; q < 12; ++q) out[(xi * Ls + jstar) * 12 + q] += coef * pj[q];
        }
    }
    free(u);
}

/*
 * (K psi)(x, s) for every s at the listed 4D sites only (lexicographic
 * indices), written to out[i][s][spin][colour].  Same definitions as
 * oracle_apply_k, evaluated site by site for lattices too large for the
 * full-lattice oracle:  D_DWF psi = D_W chi + (psi - L psi) with
 * chi = (c+d) psi + (c-d) L psi, which is Eq. (Ddwf) regrouped, and chi is
 * site-local so D_W chi at x needs chi at x and its eight neighbours.
 */
static void chi_at(const oracle_params *p, const cd *psi, long xi, const double *Lp,
                   const double *Lm, cd *chi)
{
    const int Ls = p->Ls;
    const double cp = paper_c(p), d = paper_d(p);
    for (int s = 0; s < Ls; ++s) {
        cd acc[12];
        for (int k = 0; k < 12; ++k) acc[k] = (cp + d) * psi[(xi * Ls + s) * 12 + k];
        for (int t = 0; t < Ls; ++t) {
            cd pp[12], pmv[12];
            proj_chi(+1, psi + (xi * Ls + t) * 12, pp);
            proj_chi(-1, psi + (xi * Ls + t) * 12, pmv);
            for (int k = 0; k < 12; ++k)
                acc[k] += (cp - d) * (Lp[s * Ls + t] * pp[k] + Lm[s * Ls + t] * pmv[k]);
        }
        for (int k = 0; k < 12; ++k) chi[s * 12 + k] = acc[k];
    }
}

void oracle_apply_k_sites(const oracle_params *p, const cd *U, const cd *in,
                          const long *sites, long nsites, cd *out)
{
    build_gammas();
    const int Ls = p->Ls;
    double *Lp = malloc(sizeof(double) * Ls * Ls);
    double *Lm = malloc(sizeof(double) * Ls * Ls);
    oracle_L_matrices(p, p->m1, Lp, Lm);
    double *u = malloc(sizeof(double) * Ls);
    double k;
    oracle_uv(p, u, &k);
    const double coef = p->pm * p->beta * k;
    const int jstar = (p->pm > 0) ? Ls - 1 : 0;
    const double diag = 4.0 - p->M5;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nsites; ++i) {
        const long xi = sites[i];
        int co[4];
        site_coords(p, xi, co);
        cd *chi = malloc(sizeof(cd) * Ls * 12);
        cd *chn = malloc(sizeof(cd) * Ls * 12);
        chi_at(p, in, xi, Lp, Lm, chi);
        for (int s = 0; s < Ls; ++s) {
            cd acc[12];
            for (int q = 0; q < 12; ++q) acc[q] = diag * chi[s * 12 + q];
            /* psi - L psi */
            for (int t = 0; t < Ls; ++t) {
                cd pp[12], pmv[12];
                proj_chi(+1, in + (xi * Ls + t) * 12, pp);
                proj_chi(-1, in + (xi * Ls + t) * 12, pmv);
                for (int q = 0; q < 12; ++q)
                    acc[q] += (s == t ? in[(xi * Ls + t) * 12 + q] : 0)
                              - (Lp[s * Ls + t] * pp[q] + Lm[s * Ls + t] * pmv[q]);
            }
            for (int c = 0; c < 12; ++c) out[(i * Ls + s) * 12 + c] = acc[c];
        }
        for (int mu = 0; mu < 4; ++mu)
            for (int dir = 0; dir < 2; ++dir) {
                int cn[4] = {co[0], co[1], co[2], co[3]};
                double phase = 1.0;
                if (dir == 0) {
                    cn[mu] = (co[mu] + 1) % p->dims[mu];
                    if (mu == 3 && co[3] == p->dims[3] - 1) phase = p->t_bc;
                } else {
                    cn[mu] = (co[mu] - 1 + p->dims[mu]) % p->dims[mu];
                    if (mu == 3 && co[3] == 0) phase = p->t_bc;
                }
                long ni = site_index(p, cn[0], cn[1], cn[2], cn[3]);
                chi_at(p, in, ni, Lp, Lm, chn);
                cd W[3][3];
                if (dir == 0) {
                    const cd *uu = U + (xi * 4 + mu) * 9;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) W[a][b] = uu[a * 3 + b];
                } else {
                    const cd *uu = U + (ni * 4 + mu) * 9;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) W[a][b] = conj(uu[b * 3 + a]);
                }
                double sg = (dir == 0) ? -1.0 : 1.0;
                for (int s = 0; s < Ls; ++s) {
                    cd t[12];
                    for (int sp = 0; sp < 4; ++sp)
                        for (int a = 0; a < 3; ++a) {
                            cd sum = 0;
                            for (int b = 0; b < 3; ++b) sum += W[a][b] * chn[s * 12 + sp * 3 + b];
                            t[sp * 3 + a] = sum;
                        }
                    for (int sp = 0; sp < 4; ++sp)
                        for (int a = 0; a < 3; ++a) {
                            cd sum = t[sp * 3 + a];
                            for (int sq = 0; sq < 4; ++sq) sum += sg * GAM[mu][sp][sq] * t[sq * 3 + a];
                            out[(i * Ls + s) * 12 + sp * 3 + a] -= 0.5 * phase * sum;
                        }
                }
            }
        /* + pm beta k u_s P_pm psi_{j*} */
        cd pj[12];
        proj_chi(p->pm, in + (xi * Ls + jstar) * 12, pj);
        for (int s = 0; s < Ls; ++s)
            for (int q = 0; q < 12; ++q) out[(i * Ls + s) * 12 + q] += coef * u[s] * pj[q];
        free(chi);
        free(chn);
    }
    free(Lp); free(Lm); free(u);
}

/* ------------------------------------------------------------------ */
/* vector helpers with a fixed summation order                         */
/* ------------------------------------------------------------------ */

#define RED_BLOCK 4096

static double norm2(const cd *v, long n)
{
    long nb = (n + RED_BLOCK - 1) / RED_BLOCK;
    double *part = malloc(sizeof(double) * (nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
    for (long b = 0; b < nb; ++b) {
        double s = 0;
        long hi = (b + 1) * RED_BLOCK < n ? (b + 1) * RED_BLOCK : n;
        for (long i = b * RED_BLOCK; i < hi; ++i)
            s += creal(v[i]) * creal(v[i]) + cimag(v[i]) * cimag(v[i]);
        part[b] = s;
    }
    double s = 0;
    for (long b = 0; b < nb; ++b) s += part[b];
    free(part);
    return s;
}

double oracle_norm2(const cd *v, long n) { return norm2(v, n); }

/* ------------------------------------------------------------------ */
/* CG on the normal equations                                          */
/* ------------------------------------------------------------------ */

typedef void (*op_fn)(const oracle_params *, const cd *, const cd *, cd *, int);

typedef struct {
    int iters;
    int converged;
    double true_res;
    double recur_res;
} oracle_stats;

/*
 * Solve A x = b by CG on A^dag A x = A^dag b, x0 = 0 unless use_guess.
 * Stops when the recursively updated residual ||r|| <= tol ||b||, then
 * recomputes the true residual ||b - A x|| / ||b||.  maxit bounds the work
 * (a bounded sample for timing passes a small maxit).
 */
static int cgnr(const oracle_params *p, const cd *U, op_fn A, const cd *b, cd *x,
                double tol, int maxit, int use_guess, oracle_stats *st)
{
    const long n = len5(p);
    cd *r = malloc(sizeof(cd) * n), *z = malloc(sizeof(cd) * n);
    cd *pv = malloc(sizeof(cd) * n), *q = malloc(sizeof(cd) * n);
    double bb = norm2(b, n);
    if (use_guess) {
        A(p, U, x, q, 0);
        for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    } else {
        memset(x, 0, sizeof(cd) * n);
        memcpy(r, b, sizeof(cd) * n);
    }
    A(p, U, r, z, 1);
    memcpy(pv, z, sizeof(cd) * n);
    double zz = norm2(z, n);
    double rr = norm2(r, n);
    int it = 0, conv = (rr <= tol * tol * bb);
    while (!conv && it < maxit) {
        A(p, U, pv, q, 0);
        double qq = norm2(q, n);
        double alpha = zz / qq;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * pv[i];
            r[i] -= alpha * q[i];
        }
        rr = norm2(r, n);
        ++it;
        if (rr <= tol * tol * bb) { conv = 1; break; }
        A(p, U, r, z, 1);
        double zz_new = norm2(z, n);
        double beta = zz_new / zz;
        zz = zz_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) pv[i] = z[i] + beta * pv[i];
    }
    A(p, U, x, q, 0);
    for (long i = 0; i < n; ++i) q[i] = b[i] - q[i];
    if (st) {
        st->iters = it;
        st->converged = conv;
        st->true_res = sqrt(norm2(q, n) / bb);
        st->recur_res = sqrt(rr / bb);
    }
    free(r); free(z); free(pv); free(q);
    return conv ? 0 : 1;
}

/*
 * H-form solve: psi with (H(m1) + beta Delta_pm(m2,m3) P_pm) psi = phi,
 * by CGNR on the g5R5-rotated system A psi = g5 R5 phi, Eq. (non_hermit_sys)
 * (the g5R5 factor cancels in the normal equations).  No even-odd or Cayley
 * preconditioning: those are exact reformulations checked on the GPU side.
 */
int oracle_solve_h(const oracle_params *p, const cd *U, const cd *phi, cd *psi,
                   double tol, int maxit, int use_guess, oracle_stats *st)
{
    const long n = len5(p);
    cd *b = malloc(sizeof(cd) * n);
    oracle_g5r5(p, phi, b);
    int rc = cgnr(p, U, oracle_apply_asys, b, psi, tol, maxit, use_guess, st);
    free(b);
    return rc;
}

/* K-form solve: psi' with K psi' = b, CGNR on K directly. */
int oracle_solve_k(const oracle_params *p, const cd *U, const cd *b, cd *psi,
                   double tol, int maxit, int use_guess, oracle_stats *st)
{
    return cgnr(p, U, oracle_apply_k, b, psi, tol, maxit, use_guess, st);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
