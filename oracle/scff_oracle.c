/*
 * scff_oracle.c -- plain FP64 CPU oracle for the molecular transition form
 * factor.  TEST INFRASTRUCTURE ONLY: it is built and called by the tests, by
 * the smoke check and by the benchmark's CPU-baseline leg, never by the
 * product path.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (the definition, Sec. "Analytic Method", the AO-basis form
 * of Eq. fSreal with Eq. PhiTDM):
 *
 *   f_s(q) = scale * sum_{mu,nu} T^s[mu][nu] * Int phi_mu(r) phi_nu(r) e^{+i q.r} d^3r
 *
 * over real contracted Cartesian Gaussians
 *
 *   phi_mu(r) = R_mu * sum_k c_k N_k (x-Ax)^a (y-Ay)^b (z-Az)^c exp(-alpha_k |r-A|^2)
 *
 * where N_k normalises each primitive (Appendix A, Eq. defprimitive and the
 * normalisation that follows it, written with sigma^2 = 1/(2 alpha)) and R_mu
 * optionally rescales the contraction to <phi|phi> = 1.
 *
 * Route (deliberately not the paper's Hermite/monomial route): every ordered
 * pair of functions and every pair of primitives is integrated separately,
 * with no i<->j folding.  Per axis the polynomial (x-A)^a (x-B)^b is expanded
 * about the Gaussian-product centre P by the binomial theorem (the content of
 * Eq. bCoefficients), and the 1-D moments
 *
 *   J_t(q) = Int y^t exp(-p y^2 + i q y) dy
 *
 * come from J_0 = sqrt(pi/p) exp(-q^2/4p), J_1 = (iq/2p) J_0 and
 * J_{t+1} = (iq J_t + t J_{t-1}) / (2p)  (integration by parts).
 * The integral is K_AB e^{i q.P} prod_axes sum_t e_t J_t with
 * K_AB = exp(-alpha beta |A-B|^2 / p), the Gaussian product theorem in its
 * exponent form (Eqs. sigmaTidbits, positionTidbits with sigma^2 = 1/(2 alpha)).
 * Accumulation over function pairs runs in long double.
 *
 * Basis conventions: shell codes 0 = s, 1 = p, 2 = Cartesian d, 3 = Cartesian
 * f, -1 = sp; the Cartesian components of a shell of angular momentum l are
 * ordered by descending x power, then descending y power (x,y,z;
 * xx,xy,xz,yy,yz,zz; xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz); an sp shell
 * gives s,px,py,pz and stores its s coefficients before its p coefficients.
 *
 * Pure (spherical-harmonic) d and f shells (flag bits ORACLE_PURE_D and
 * ORACLE_PURE_F) follow Appendix A, Eq. defprimitive: each primitive is a sum
 * of Cartesian terms k_i x^a y^b z^c with one normalisation constant N for the
 * whole sum, N^-2 = sum_ij k_i k_j prod_axes Int x^(a_i+a_j) exp(-x^2/sigma^2) dx
 * (the printed double sum; terms with an odd exponent sum vanish).  The 2l+1
 * functions are the real solid harmonics, ordered m = -l..l:
 *   d: xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2
 *   f: 3x^2y-y^3, xyz, 4yz^2-x^2y-y^3, 2z^3-3x^2z-3y^2z, 4xz^2-x^3-xy^2,
 *      x^2z-y^2z, x^3-3xy^2
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2

#define ORACLE_RENORM 1
#define ORACLE_PURE_D 2
#define ORACLE_PURE_F 4

#define MAX_TERMS 3

typedef struct {
    int atom;
    int nterm;              /* Cartesian terms of the angular factor */
    int pw[MAX_TERMS][3];   /* their exponents */
    double k[MAX_TERMS];    /* their coefficients k_i */
    int nprim;
    const double *alpha;    /* nprim exponents */
    double *w;              /* nprim normalised weights c_k N_k R */
} ofn_t;

typedef struct {
    int nterm;
    int pw[MAX_TERMS][3];
    double k[MAX_TERMS];
} pure_t;

/* Real solid harmonics, m = -l..l (unnormalised polynomials). */
static const pure_t PURE_D[5] = {
    {1, {{1, 1, 0}}, {1.0}},
    {1, {{0, 1, 1}}, {1.0}},
    {3, {{0, 0, 2}, {2, 0, 0}, {0, 2, 0}}, {2.0, -1.0, -1.0}},
    {1, {{1, 0, 1}}, {1.0}},
    {2, {{2, 0, 0}, {0, 2, 0}}, {1.0, -1.0}},
};
static const pure_t PURE_F[7] = {
    {2, {{2, 1, 0}, {0, 3, 0}}, {3.0, -1.0}},
    {1, {{1, 1, 1}}, {1.0}},
    {3, {{0, 1, 2}, {2, 1, 0}, {0, 3, 0}}, {4.0, -1.0, -1.0}},
    {3, {{0, 0, 3}, {2, 0, 1}, {0, 2, 1}}, {2.0, -3.0, -3.0}},
    {3, {{1, 0, 2}, {3, 0, 0}, {1, 2, 0}}, {4.0, -1.0, -1.0}},
    {2, {{2, 0, 1}, {0, 2, 1}}, {1.0, -1.0}},
    {2, {{3, 0, 0}, {1, 2, 0}}, {1.0, -3.0}},
};

static int is_pure(int l, int flags) {
    return (l == 2 && (flags & ORACLE_PURE_D)) || (l == 3 && (flags & ORACLE_PURE_F));
}

static int nfn_of(int l, int flags) {
    if (is_pure(l, flags)) return 2 * l + 1;
    switch (l) {
    case 0: return 1;
    case 1: return 3;
    case 2: return 6;
    case 3: return 10;
    case -1: return 4;
    default: return -1;
    }
}

/* Cartesian exponents of component i of shell code l. */
static void powers_of(int l, int i, int pw[3]) {
    static const int P1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    static const int P2[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1},
                                 {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
    static const int P3[10][3] = {{3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1},
                                  {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};
    pw[0] = pw[1] = pw[2] = 0;
    if (l == 1) memcpy(pw, P1[i], sizeof(int) * 3);
    else if (l == 2) memcpy(pw, P2[i], sizeof(int) * 3);
    else if (l == 3) memcpy(pw, P3[i], sizeof(int) * 3);
    else if (l == -1 && i > 0) memcpy(pw, P1[i - 1], sizeof(int) * 3);
}

/* Primitive normalisation, Appendix A with a single Cartesian term (k = 1):
 * N = [ prod_axes sigma^{1+2a} Gamma(a + 1/2) ]^{-1/2},  sigma = (2 alpha)^{-1/2}. */
double scff_oracle_prim_norm(double alpha, int a, int b, int c) {
    const double sigma = 1.0 / sqrt(2.0 * alpha);
    const int e[3] = {a, b, c};
    double prod = 1.0;
    for (int i = 0; i < 3; ++i)
        prod *= pow(sigma, 1.0 + 2.0 * e[i]) * tgamma(e[i] + 0.5);
    return 1.0 / sqrt(prod);
}

/* Appendix A normalisation of a primitive whose angular factor is the sum of
 * Cartesian terms k_i x^a_i y^b_i z^c_i:
 * N = [ sum_ij k_i k_j prod_axes sigma^{1+n} Gamma((n+1)/2) ]^{-1/2} with n the
 * axis exponent sum of terms i and j; odd n contributes zero. */
static double multi_term_norm(double alpha, int nterm, const int pw[][3], const double *k) {
    const double sigma = 1.0 / sqrt(2.0 * alpha);
    double sum = 0.0;
    for (int i = 0; i < nterm; ++i)
        for (int j = 0; j < nterm; ++j) {
            double prod = k[i] * k[j];
            for (int ax = 0; ax < 3; ++ax) {
                const int n = pw[i][ax] + pw[j][ax];
                if (n & 1) {
                    prod = 0.0;
                    break;
                }
                prod *= pow(sigma, 1.0 + n) * tgamma(0.5 * (n + 1));
            }
            sum += prod;
        }
    return 1.0 / sqrt(sum);
}

/* Int x^{2a} exp(-p x^2) dx = Gamma(a + 1/2) / p^{a + 1/2}. */
static double even_moment(int a, double p) {
    return tgamma(a + 0.5) / pow(p, a + 0.5);
}

/* Int x^n exp(-p x^2) dx for any n >= 0 (zero for odd n). */
static double moment(int n, double p) {
    return (n & 1) ? 0.0 : even_moment(n / 2, p);
}

int scff_oracle_nbf(int n_shells, const int32_t *shell_l, int flags) {
    int nbf = 0;
    for (int s = 0; s < n_shells; ++s) {
        int n = nfn_of(shell_l[s], flags);
        if (n < 0) return ORACLE_EINVAL;
        nbf += n;
    }
    return nbf;
}

/* Builds the function table; caller frees fns[i].w and fns. */
static int build_functions(int n_atoms, int n_shells, const int32_t *shell_atom,
                           const int32_t *shell_l, const int32_t *shell_nprim,
                           const double *exps, const double *coefs, int flags,
                           ofn_t **out, int *nbf_out) {
    const int renorm = flags & ORACLE_RENORM;
    int nbf = scff_oracle_nbf(n_shells, shell_l, flags);
    if (nbf <= 0) return ORACLE_EINVAL;
    ofn_t *fns = (ofn_t *)calloc((size_t)nbf, sizeof(ofn_t));
    if (!fns) return ORACLE_ENOMEM;
    size_t eoff = 0, coff = 0;
    int f = 0;
    for (int s = 0; s < n_shells; ++s) {
        const int l = shell_l[s], np = shell_nprim[s];
        if (np <= 0 || shell_atom[s] < 0 || shell_atom[s] >= n_atoms) {
            for (int i = 0; i < f; ++i) free(fns[i].w);
            free(fns);
            return ORACLE_EINVAL;
        }
        const int nf = nfn_of(l, flags);
        const int pure = is_pure(l, flags);
        for (int i = 0; i < nf; ++i, ++f) {
            ofn_t *fn = &fns[f];
            fn->atom = shell_atom[s];
            if (pure) {
                const pure_t *h = (l == 2) ? &PURE_D[i] : &PURE_F[i];
                fn->nterm = h->nterm;
                memcpy(fn->pw, h->pw, sizeof(fn->pw));
                memcpy(fn->k, h->k, sizeof(fn->k));
            } else {
                fn->nterm = 1;
                powers_of(l, i, fn->pw[0]);
                fn->k[0] = 1.0;
            }
            fn->nprim = np;
            fn->alpha = exps + eoff;
            fn->w = (double *)malloc(sizeof(double) * (size_t)np);
            const double *c = coefs + coff + ((l == -1 && i > 0) ? (size_t)np : 0);
            for (int k = 0; k < np; ++k)
                fn->w[k] = c[k] * (pure ? multi_term_norm(fn->alpha[k], fn->nterm, fn->pw, fn->k)
                                        : scff_oracle_prim_norm(fn->alpha[k], fn->pw[0][0], fn->pw[0][1],
                                                                fn->pw[0][2]));
            if (renorm) {
                /* <phi|phi> = sum_kk' w_k w_k' sum_ij k_i k_j prod_axes Int x^(a_i+a_j) e^{-(a_k+a_k') x^2} */
                double nrm = 0.0;
                for (int k = 0; k < np; ++k)
                    for (int kk = 0; kk < np; ++kk) {
                        const double p = fn->alpha[k] + fn->alpha[kk];
                        double ang = 0.0;
                        for (int ti = 0; ti < fn->nterm; ++ti)
                            for (int tj = 0; tj < fn->nterm; ++tj)
                                ang += fn->k[ti] * fn->k[tj] * moment(fn->pw[ti][0] + fn->pw[tj][0], p) *
                                       moment(fn->pw[ti][1] + fn->pw[tj][1], p) *
                                       moment(fn->pw[ti][2] + fn->pw[tj][2], p);
                        nrm += fn->w[k] * fn->w[kk] * ang;
                    }
                const double r = 1.0 / sqrt(nrm);
                for (int k = 0; k < np; ++k) fn->w[k] *= r;
            }
        }
        eoff += (size_t)np;
        coff += (size_t)np * (l == -1 ? 2 : 1);
    }
    *out = fns;
    *nbf_out = nbf;
    return ORACLE_OK;
}

static void free_functions(ofn_t *fns, int nbf) {
    for (int i = 0; i < nbf; ++i) free(fns[i].w);
    free(fns);
}

/* Coefficients e_t of (y + u)^a (y + v)^b = sum_t e_t y^t (binomial theorem). */
static int binomial_product(int a, double u, int b, double v, double e[7]) {
    double ea[4] = {0, 0, 0, 0}, eb[4] = {0, 0, 0, 0};
    /* (y+u)^a = sum_i C(a,i) u^{a-i} y^i */
    static const double C[4][4] = {{1, 0, 0, 0}, {1, 1, 0, 0}, {1, 2, 1, 0}, {1, 3, 3, 1}};
    for (int i = 0; i <= a; ++i) ea[i] = C[a][i] * pow(u, a - i);
    for (int j = 0; j <= b; ++j) eb[j] = C[b][j] * pow(v, b - j);
    for (int t = 0; t < 7; ++t) e[t] = 0.0;
    for (int i = 0; i <= a; ++i)
        for (int j = 0; j <= b; ++j) e[i + j] += ea[i] * eb[j];
    return a + b;
}

/* sum_t e_t J_t(q) with J from the integration-by-parts recurrence. */
static double complex axis_factor(const double e[7], int tmax, double p, double q) {
    double complex J[7];
    J[0] = sqrt(M_PI / p) * exp(-q * q / (4.0 * p));
    if (tmax >= 1) J[1] = (I * q / (2.0 * p)) * J[0];
    for (int t = 1; t < tmax; ++t) J[t + 1] = (I * q * J[t] + (double)t * J[t - 1]) / (2.0 * p);
    double complex s = 0.0;
    for (int t = 0; t <= tmax; ++t) s += e[t] * J[t];
    return s;
}

/* Int phi_mu phi_nu e^{i q.r} d^3r for one q (all primitive pairs). */
static double complex pair_integral(const ofn_t *m, const ofn_t *n, const double *A,
                                    const double *B, const double q[3]) {
    double complex total = 0.0;
    double AB2 = 0.0;
    for (int i = 0; i < 3; ++i) AB2 += (A[i] - B[i]) * (A[i] - B[i]);
    for (int k = 0; k < m->nprim; ++k) {
        const double al = m->alpha[k];
        for (int kk = 0; kk < n->nprim; ++kk) {
            const double be = n->alpha[kk];
            const double p = al + be;
            const double K = exp(-al * be * AB2 / p);
            double P[3];
            double phase = 0.0;
            for (int i = 0; i < 3; ++i) {
                P[i] = (al * A[i] + be * B[i]) / p;
                phase += q[i] * P[i];
            }
            double complex ang = 0.0;
            for (int ti = 0; ti < m->nterm; ++ti)
                for (int tj = 0; tj < n->nterm; ++tj) {
                    double complex prod = m->k[ti] * n->k[tj];
                    for (int i = 0; i < 3; ++i) {
                        double e[7];
                        const int tmax = binomial_product(m->pw[ti][i], P[i] - A[i], n->pw[tj][i], P[i] - B[i], e);
                        prod *= axis_factor(e, tmax, p, q[i]);
                    }
                    ang += prod;
                }
            total += m->w[k] * n->w[kk] * K * ang * cexp(I * phase);
        }
    }
    return total;
}

/*
 * f_out[s][iq][0..1] = Re, Im of f_s(q_iq).  T is [n_states][nbf][nbf]
 * row-major; q is [n_q][3]; flags = ORACLE_RENORM | ORACLE_PURE_D | ORACLE_PURE_F.
 * With term_out non-NULL, term_out[s][iq] = |scale| sum_{mu,nu} |T^s_{mu nu}
 * integral_{mu nu}(q)|, the sum of the magnitudes of the function-pair terms
 * whose sum is f_s(q) (the scale against which the rounding of the terms
 * acts).  Returns 0 or a negative error code.
 */
static int form_factor_impl(int n_atoms, const double *xyz, int n_shells,
                            const int32_t *shell_atom, const int32_t *shell_l,
                            const int32_t *shell_nprim, const double *exps,
                            const double *coefs, int flags, int n_states,
                            const double *T, int64_t n_q, const double *q,
                            double scale, double *f_out, double *term_out, int n_threads) {
    if (n_atoms <= 0 || n_shells <= 0 || n_states <= 0 || n_q < 0 || !xyz || !T || !f_out)
        return ORACLE_EINVAL;
    ofn_t *fns = NULL;
    int nbf = 0;
    int rc = build_functions(n_atoms, n_shells, shell_atom, shell_l, shell_nprim, exps,
                             coefs, flags, &fns, &nbf);
    if (rc) return rc;
    const size_t nn = (size_t)nbf * nbf;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int fail = 0;
#pragma omp parallel
    {
        long double *acc = (long double *)malloc(sizeof(long double) * 3 * (size_t)n_states);
        if (!acc) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t iq = 0; iq < n_q; ++iq) {
            if (!acc) continue;
            for (int s = 0; s < 3 * n_states; ++s) acc[s] = 0.0L;
            const double *qv = q + 3 * iq;
            for (int mu = 0; mu < nbf; ++mu) {
                const double *A = xyz + 3 * fns[mu].atom;
                for (int nu = 0; nu < nbf; ++nu) {
                    const double *B = xyz + 3 * fns[nu].atom;
                    const double complex v = pair_integral(&fns[mu], &fns[nu], A, B, qv);
                    const double vr = creal(v), vi = cimag(v);
                    const double va = term_out ? cabs(v) : 0.0;
                    for (int s = 0; s < n_states; ++s) {
                        const long double t = T[(size_t)s * nn + (size_t)mu * nbf + nu];
                        acc[2 * s] += t * vr;
                        acc[2 * s + 1] += t * vi;
                        if (term_out) acc[2 * n_states + s] += fabsl(t) * va;
                    }
                }
            }
            for (int s = 0; s < n_states; ++s) {
                f_out[((size_t)s * n_q + iq) * 2] = (double)(scale * acc[2 * s]);
                f_out[((size_t)s * n_q + iq) * 2 + 1] = (double)(scale * acc[2 * s + 1]);
                if (term_out) term_out[(size_t)s * n_q + iq] = (double)(fabs(scale) * acc[2 * n_states + s]);
            }
        }
        free(acc);
    }
    free_functions(fns, nbf);
    return fail ? ORACLE_ENOMEM : ORACLE_OK;
}

int scff_oracle_form_factor(int n_atoms, const double *xyz, int n_shells,
                            const int32_t *shell_atom, const int32_t *shell_l,
                            const int32_t *shell_nprim, const double *exps,
                            const double *coefs, int flags, int n_states,
                            const double *T, int64_t n_q, const double *q,
                            double scale, double *f_out, int n_threads) {
    return form_factor_impl(n_atoms, xyz, n_shells, shell_atom, shell_l, shell_nprim, exps, coefs,
                            flags, n_states, T, n_q, q, scale, f_out, NULL, n_threads);
}

/* f_out as scff_oracle_form_factor, plus term_out[s][iq] (see form_factor_impl). */
int scff_oracle_form_factor_terms(int n_atoms, const double *xyz, int n_shells,
                                  const int32_t *shell_atom, const int32_t *shell_l,
                                  const int32_t *shell_nprim, const double *exps,
                                  const double *coefs, int flags, int n_states,
                                  const double *T, int64_t n_q, const double *q,
                                  double scale, double *f_out, double *term_out, int n_threads) {
    if (!term_out) return ORACLE_EINVAL;
    return form_factor_impl(n_atoms, xyz, n_shells, shell_atom, shell_l, shell_nprim, exps, coefs,
                            flags, n_states, T, n_q, q, scale, f_out, term_out, n_threads);
}

/*
 * Function table for tests (Cartesian shells only: flags may hold
 * ORACLE_RENORM alone): per function its atom, Cartesian exponents and
 * normalised primitive weights (w_out holds sum_k nprim entries in function
 * order; nprim_out[f] gives the count).  Returns nbf or a negative code.
 */
int scff_oracle_functions(int n_atoms, int n_shells, const int32_t *shell_atom,
                          const int32_t *shell_l, const int32_t *shell_nprim,
                          const double *exps, const double *coefs, int flags,
                          int32_t *atom_out, int32_t *pw_out, int32_t *nprim_out,
                          double *alpha_out, double *w_out) {
    if (flags & ~ORACLE_RENORM) return ORACLE_EINVAL;
    ofn_t *fns = NULL;
    int nbf = 0;
    int rc = build_functions(n_atoms, n_shells, shell_atom, shell_l, shell_nprim, exps,
                             coefs, flags, &fns, &nbf);
    if (rc) return rc;
    size_t o = 0;
    for (int f = 0; f < nbf; ++f) {
        atom_out[f] = fns[f].atom;
        for (int i = 0; i < 3; ++i) pw_out[3 * f + i] = fns[f].pw[0][i];
        nprim_out[f] = fns[f].nprim;
        for (int k = 0; k < fns[f].nprim; ++k, ++o) {
            alpha_out[o] = fns[f].alpha[k];
            w_out[o] = fns[f].w[k];
        }
    }
    free_functions(fns, nbf);
    return nbf;
}

int scff_oracle_version(void) { return 1; }

/*
 * Transition densities Phi_s(r) = scale * sum_{mu,nu} T^s[mu][nu] phi_mu(r) phi_nu(r)
 * at n_r points r[n_r][3] (the real-space integrand of Eq. fSreal, which the
 * FFT method tabulates).  out[s][ir].  Same basis conventions and flags as
 * scff_oracle_form_factor.  Returns 0 or a negative error code.
 */
int scff_oracle_density(int n_atoms, const double *xyz, int n_shells, const int32_t *shell_atom,
                        const int32_t *shell_l, const int32_t *shell_nprim, const double *exps,
                        const double *coefs, int flags, int n_states, const double *T, int64_t n_r,
                        const double *r, double scale, double *out, int n_threads) {
    if (n_atoms <= 0 || n_shells <= 0 || n_states <= 0 || n_r < 0 || !xyz || !T || !out) return ORACLE_EINVAL;
    ofn_t *fns = NULL;
    int nbf = 0;
    int rc = build_functions(n_atoms, n_shells, shell_atom, shell_l, shell_nprim, exps, coefs, flags, &fns, &nbf);
    if (rc) return rc;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int fail = 0;
#pragma omp parallel
    {
        double *phi = (double *)malloc(sizeof(double) * (size_t)nbf);
        if (!phi) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t ir = 0; ir < n_r; ++ir) {
            if (!phi) continue;
            const double *rv = r + 3 * ir;
            for (int mu = 0; mu < nbf; ++mu) {
                const ofn_t *fn = &fns[mu];
                const double *A = xyz + 3 * fn->atom;
                const double d[3] = {rv[0] - A[0], rv[1] - A[1], rv[2] - A[2]};
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double ang = 0.0;
                for (int t = 0; t < fn->nterm; ++t)
                    ang += fn->k[t] * pow(d[0], fn->pw[t][0]) * pow(d[1], fn->pw[t][1]) * pow(d[2], fn->pw[t][2]);
                double rad = 0.0;
                for (int k = 0; k < fn->nprim; ++k) rad += fn->w[k] * exp(-fn->alpha[k] * r2);
                phi[mu] = ang * rad;
            }
            for (int s = 0; s < n_states; ++s) {
                long double acc = 0.0L;
                const double *Ts = T + (size_t)s * nbf * nbf;
                for (int mu = 0; mu < nbf; ++mu)
                    for (int nu = 0; nu < nbf; ++nu) acc += (long double)Ts[(size_t)mu * nbf + nu] * phi[mu] * phi[nu];
                out[(size_t)s * n_r + ir] = (double)(scale * acc);
            }
        }
        free(phi);
    }
    free_functions(fns, nbf);
    return fail ? ORACLE_ENOMEM : ORACLE_OK;
}
