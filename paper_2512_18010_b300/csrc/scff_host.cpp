// Host runtime of the form-factor library: context, handles, validation,
// basis ingest (normalisation, primitive-shell records, pair list), q-grids
// and dispatch of the device kernels.  Implements include/scff.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/scff.h"
#include "scff_internal.h"
#include "tc_internal.h"

using namespace scff;

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

static scff_status fail(scff_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation)                                              \
                return fail(SCFF_ERR_OOM, "%s: %s", #call, cudaGetErrorString(e_));           \
            return fail(SCFF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));              \
        }                                                                                     \
    } while (0)

extern "C" const char *scff_last_error(void) { return g_last_error.c_str(); }

namespace scff {
// Lets other translation units of the library report an error message.
scff_status set_last_error(scff_status code, const char *msg) {
    g_last_error = msg;
    return code;
}
}  // namespace scff

// ------------------------------------------------------------------ objects

#include "scff_objects.h"

static scff_status grow(scff_ctx *c, DevBuf &b, size_t bytes) {
    if (bytes <= b.cap) return SCFF_OK;
    // Kernels of earlier calls may still read the old buffer.
    CUDA_TRY(cudaDeviceSynchronize());
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = bytes + bytes / 8 + 256;
    CUDA_TRY(cudaMalloc(&b.p, want));
    b.cap = want;
    (void)c;
    return SCFF_OK;
}

#define TRY(x)                          \
    do {                                \
        scff_status s_ = (x);           \
        if (s_ != SCFF_OK) return s_;   \
    } while (0)

// ------------------------------------------------------------------ context

extern "C" scff_status scff_create(scff_ctx **out, int device, uint64_t hbm_budget_bytes) {
    if (!out) return fail(SCFF_ERR_INVALID_ARG, "scff_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SCFF_ERR_INVALID_ARG, "scff_create: device %d of %d", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    CUDA_TRY(pairprep_init());
    scff_ctx *c = new scff_ctx();
    c->device = device;
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
        delete c;
        return fail(SCFF_ERR_CUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
    }
    c->budget = hbm_budget_bytes ? hbm_budget_bytes : (uint64_t)(0.9 * (double)fr);
    if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
        if (c->d_err) cudaFree(c->d_err);
        delete c;
        return fail(SCFF_ERR_OOM, "scff_create: status word allocation failed");
    }
    cudaMemset(c->d_err, 0, sizeof(int));
    for (auto &ev : c->ev) cudaEventCreate(&ev);
    *out = c;
    return SCFF_OK;
}

extern "C" scff_status scff_set_tc_drain(scff_ctx *c, int drain_every) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_tc_drain: NULL context");
    if (drain_every < -1) return fail(SCFF_ERR_INVALID_ARG, "scff_set_tc_drain: %d", drain_every);
    c->drain_every = drain_every;
    return SCFF_OK;
}

// The W generator variant a call in this precision asks for (tc_variant_resolve
// decides what the grid and kind allow): the context's mode, or the kind's default.
int zstage_mode(const scff_ctx *c, int precision) {
    if (c->tc_zstage >= 0) return c->tc_zstage;
    const int k = tc_kind_of_precision(precision);
    return k >= 0 ? tc_variant_preferred(k) : 0;
}

extern "C" scff_status scff_last_path(scff_ctx *c, int32_t *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_last_path: NULL argument");
    for (int i = 0; i < 3; ++i) out[i] = c->last_path[i];
    return SCFF_OK;
}

extern "C" scff_status scff_set_tc_variant(scff_ctx *c, int mode) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_tc_variant: NULL context");
    if (mode < -1 || mode > 4) return fail(SCFF_ERR_INVALID_ARG, "scff_set_tc_variant: %d", mode);
    c->tc_zstage = mode;
    return SCFF_OK;
}

extern "C" scff_status scff_set_tc_zstage(scff_ctx *c, int mode) { return scff_set_tc_variant(c, mode); }

extern "C" scff_status scff_set_timing(scff_ctx *c, int enable) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_timing: NULL context");
    c->timing = enable ? 1 : 0;
    c->timed_valid = 0;
    return SCFF_OK;
}

extern "C" scff_status scff_last_timing(scff_ctx *c, double *ms_out) {
    if (!c || !ms_out) return fail(SCFF_ERR_INVALID_ARG, "scff_last_timing: NULL argument");
    if (!c->timed_valid) return fail(SCFF_ERR_NOT_FOUND, "scff_last_timing: no timed call since timing was enabled");
    cudaSetDevice(c->device);
    CUDA_TRY(cudaEventSynchronize(c->ev[2]));
    float a = 0.f, b = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
    ms_out[0] = b;        // q-evaluation kernel(s)
    ms_out[1] = a;        // pair-prep, geometry and tables
    ms_out[2] = a + b;    // whole device pipeline of the call
    return SCFF_OK;
}

static void free_basis(scff_basis_s *b) {
    PairSetDev &d = b->dev;
    cudaFree(d.rec_xyz);
    cudaFree(d.rec_alpha);
    cudaFree(d.rec_type);
    cudaFree(d.rec_fn0);
    cudaFree(d.rec_w);
    cudaFree(d.pair_rec);
    cudaFree(b->cmap_idx);
    cudaFree(b->cmap_c);
    delete b;
}
static void free_trans(scff_trans_s *t) {
    cudaFree(t->d_T);
    delete t;
}

static void drop_screened(scff_ctx *c, scff_trans_s *t) {
    for (size_t i = 0; i < c->screened.size();) {
        if (!t || c->screened[i]->trans == t) {
            cudaFree(c->screened[i]->dev.pair_rec);
            delete c->screened[i];
            c->screened.erase(c->screened.begin() + i);
        } else {
            ++i;
        }
    }
}
static void free_grid(scff_qgrid_s *g) {
    cudaFree(g->d_qx);
    cudaFree(g->d_qy);
    cudaFree(g->d_qz);
    cudaFree(g->d_q);
    delete g;
}

static void free_plan_any(struct scff_plan_s *p);

extern "C" void scff_destroy(scff_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    drop_screened(c, nullptr);
    for (auto *t : c->transs) free_trans(t);
    for (auto *b : c->bases) free_basis(b);
    for (auto *g : c->grids) free_grid(g);
    for (auto *p : c->plans) free_plan_any(p);
    scff_sph_cache_free(c->sph);
    DevBuf *bufs[] = {&c->coef, &c->geom, &c->gx, &c->gy, &c->gz, &c->fstage, &c->f2stage, &c->tc_ws, &c->sph_ws, &c->fft_ws};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    cudaFree(c->d_err);
    cudaFreeHost(c->h_err);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : c->band_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_st) cudaStreamDestroy(c->copy_st);
    if (c->progress_h) cudaFreeHost(c->progress_h);
    delete c;
}

extern "C" int64_t scff_kernel_launches(scff_ctx *c) { return c ? c->launches : -1; }

// ------------------------------------------------------------------ basis ingest

namespace {

struct HostRec {
    int atom;
    double alpha;
    int type;
    int fn0;
    double w[kRecW];
};

// (2n-1)!! with (-1)!! = 1
double dfact_odd(int n) {
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

// Cartesian exponents of the functions of each record type.
void type_powers(int type, int j, int pw[3]) {
    for (int ax = 0; ax < 3; ++ax)
        pw[ax] = type == REC_SP ? (j == 0 ? 0 : cart_pow(1, j - 1, ax)) : cart_pow(rec_lmax(type), j, ax);
}

// Unit-norm factor of x^a y^b z^c exp(-alpha r^2):
// N^2 = (2 alpha/pi)^{3/2} (4 alpha)^{a+b+c} / ((2a-1)!! (2b-1)!! (2c-1)!!).
double prim_norm(double alpha, const int pw[3]) {
    const int L = pw[0] + pw[1] + pw[2];
    const double n2 = pow(2.0 * alpha / M_PI, 1.5) * pow(4.0 * alpha, L) /
                      (dfact_odd(pw[0]) * dfact_odd(pw[1]) * dfact_odd(pw[2]));
    return sqrt(n2);
}

// <x^a y^b z^c e^{-a1 r^2} | x^a y^b z^c e^{-a2 r^2}> on one centre:
// prod_axes (2a-1)!! / (2p)^a * sqrt(pi/p), p = a1 + a2.
double same_centre_overlap(double p, const int pw[3]) {
    double v = pow(M_PI / p, 1.5);
    for (int i = 0; i < 3; ++i) v *= dfact_odd(pw[i]) / pow(2.0 * p, pw[i]);
    return v;
}

// <x^a y^b z^c e^{-p r^2/2} | x^a' y^b' z^c' e^{-p r^2/2}> on one centre:
// per axis Int x^n e^{-p x^2} dx = (n-1)!! / (2p)^{n/2} sqrt(pi/p) for even n, 0 for odd n.
double mono_overlap(double p, const int pa[3], const int pb[3]) {
    double v = pow(M_PI / p, 1.5);
    for (int i = 0; i < 3; ++i) {
        const int n = pa[i] + pb[i];
        if (n & 1) return 0.0;
        v *= dfact_odd(n / 2) / pow(2.0 * p, n / 2);
    }
    return v;
}

// Real solid harmonics of the pure d and f shells, m = -l..l, as Cartesian
// polynomials: up to three terms (k, exponents) each.
struct PureTerm {
    double k;
    int pw[3];
};
struct PureFn {
    int n;
    PureTerm t[kMaxPureTerms];
};
const PureFn kPureD[5] = {
    {1, {{1, {1, 1, 0}}}},
    {1, {{1, {0, 1, 1}}}},
    {3, {{2, {0, 0, 2}}, {-1, {2, 0, 0}}, {-1, {0, 2, 0}}}},
    {1, {{1, {1, 0, 1}}}},
    {2, {{1, {2, 0, 0}}, {-1, {0, 2, 0}}}},
};
const PureFn kPureF[7] = {
    {2, {{3, {2, 1, 0}}, {-1, {0, 3, 0}}}},
    {1, {{1, {1, 1, 1}}}},
    {3, {{4, {0, 1, 2}}, {-1, {2, 1, 0}}, {-1, {0, 3, 0}}}},
    {3, {{2, {0, 0, 3}}, {-3, {2, 0, 1}}, {-3, {0, 2, 1}}}},
    {3, {{4, {1, 0, 2}}, {-1, {3, 0, 0}}, {-1, {1, 2, 0}}}},
    {2, {{1, {2, 0, 1}}, {-1, {0, 2, 1}}}},
    {2, {{1, {3, 0, 0}}, {-3, {1, 2, 0}}}},
};

// Coefficients of pure function m of shell l on the unit-norm Cartesian
// components: phi_m = sum_i k_i (N_m / n_i) chi_i, where N_m normalises the
// whole polynomial primitive (Appendix A) and n_i the single term.  Both
// scale as alpha^{(2l+3)/4}, so the ratio is exponent-independent and equal
// contraction renormalisation factors cancel; it is evaluated at alpha = 1/2.
void pure_coefficients(int l, int m, int cart_out[kMaxPureTerms], double coef_out[kMaxPureTerms], int *n_out) {
    const PureFn &h = (l == 2) ? kPureD[m] : kPureF[m];
    const double alpha = 0.5, p = 2.0 * alpha;
    double norm2 = 0.0;
    for (int i = 0; i < h.n; ++i)
        for (int j = 0; j < h.n; ++j) norm2 += h.t[i].k * h.t[j].k * mono_overlap(p, h.t[i].pw, h.t[j].pw);
    const double Nm = 1.0 / sqrt(norm2);
    const int ncart = (l + 1) * (l + 2) / 2;
    for (int i = 0; i < h.n; ++i) {
        int ci = -1;
        for (int j = 0; j < ncart; ++j) {
            int pw[3];
            for (int ax = 0; ax < 3; ++ax) pw[ax] = cart_pow(l, j, ax);
            if (pw[0] == h.t[i].pw[0] && pw[1] == h.t[i].pw[1] && pw[2] == h.t[i].pw[2]) ci = j;
        }
        cart_out[i] = ci;
        coef_out[i] = h.t[i].k * Nm / prim_norm(alpha, h.t[i].pw);
    }
    *n_out = h.n;
}

template <typename T>
scff_status upload(T **dst, const std::vector<T> &src) {
    *dst = nullptr;
    if (src.empty()) return SCFF_OK;
    CUDA_TRY(cudaMalloc((void **)dst, sizeof(T) * src.size()));
    CUDA_TRY(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return SCFF_OK;
}

}  // namespace

extern "C" scff_status scff_basis(scff_ctx *c, int n_atoms, const double *xyz, int n_shells,
                                  const int32_t *shell_atom, const int32_t *shell_l, const int32_t *shell_nprim,
                                  const double *exps, const double *coefs, uint32_t flags, scff_basis_h *out,
                                  int32_t *nbf_out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: NULL context or output");
    *out = nullptr;
    if (n_atoms <= 0 || n_shells <= 0 || !xyz || !shell_atom || !shell_l || !shell_nprim || !exps || !coefs)
        return fail(SCFF_ERR_INVALID_ARG, "scff_basis: empty basis or NULL array");
    for (int i = 0; i < 3 * n_atoms; ++i)
        if (!isfinite(xyz[i])) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: non-finite coordinate %d", i);
    if (flags & ~(SCFF_RENORM_CONTRACTED | SCFF_PURE_D | SCFF_PURE_F))
        return fail(SCFF_ERR_INVALID_ARG, "scff_basis: unknown flag bits 0x%x", flags);
    std::vector<HostRec> recs;
    size_t eoff = 0, coff = 0;
    int nbf = 0, nuser = 0;
    bool any_pure = false;
    std::vector<int32_t> cm_idx;  // [ncart][kMaxPureTerms]
    std::vector<double> cm_c;
    const bool renorm = (flags & SCFF_RENORM_CONTRACTED) != 0;
    for (int s = 0; s < n_shells; ++s) {
        const int l = shell_l[s], np = shell_nprim[s], at = shell_atom[s];
        if (l > 3) return fail(SCFF_ERR_UNSUPPORTED_L, "scff_basis: shell %d has l=%d (Cartesian f is the maximum)", s, l);
        if (l < -1) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d has invalid code %d", s, l);
        if (np < 1 || np > 64) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d has %d primitives", s, np);
        if (at < 0 || at >= n_atoms) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d on atom %d", s, at);
        const int type = (l == 0) ? REC_S : (l == 1) ? REC_P : (l == 2) ? REC_D : (l == 3) ? REC_F : REC_SP;
        const int nf = rec_nfn(type);
        for (int k = 0; k < np; ++k)
            if (!(exps[eoff + k] > 0.0) || !isfinite(exps[eoff + k]))
                return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d exponent %d is not positive", s, k);
        const int ncoef = np * (type == REC_SP ? 2 : 1);
        for (int k = 0; k < ncoef; ++k)
            if (!isfinite(coefs[coff + k])) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d coefficient %d", s, k);
        // weights w[j][k] = c_k N_k(j) R_j
        std::vector<double> w((size_t)nf * np);
        for (int j = 0; j < nf; ++j) {
            int pw[3];
            type_powers(type, j, pw);
            const double *c = coefs + coff + ((type == REC_SP && j > 0) ? np : 0);
            for (int k = 0; k < np; ++k) w[(size_t)j * np + k] = c[k] * prim_norm(exps[eoff + k], pw);
            if (renorm) {
                double ov = 0.0;
                for (int k = 0; k < np; ++k)
                    for (int kk = 0; kk < np; ++kk)
                        ov += w[(size_t)j * np + k] * w[(size_t)j * np + kk] *
                              same_centre_overlap(exps[eoff + k] + exps[eoff + kk], pw);
                if (!(ov > 0.0)) return fail(SCFF_ERR_INVALID_ARG, "scff_basis: shell %d function %d has zero norm", s, j);
                const double r = 1.0 / sqrt(ov);
                for (int k = 0; k < np; ++k) w[(size_t)j * np + k] *= r;
            }
        }
        for (int k = 0; k < np; ++k) {
            HostRec r;
            r.atom = at;
            r.alpha = exps[eoff + k];
            r.type = type;
            r.fn0 = nbf;
            for (int j = 0; j < kRecW; ++j) r.w[j] = j < nf ? w[(size_t)j * np + k] : 0.0;
            recs.push_back(r);
        }
        // caller functions -> Cartesian components
        const bool pure = (l == 2 && (flags & SCFF_PURE_D)) || (l == 3 && (flags & SCFF_PURE_F));
        cm_idx.resize((size_t)(nbf + nf) * kMaxPureTerms, -1);
        cm_c.resize((size_t)(nbf + nf) * kMaxPureTerms, 0.0);
        if (pure) {
            any_pure = true;
            std::vector<int> used(nf, 0);
            for (int m = 0; m < 2 * l + 1; ++m) {
                int cart[kMaxPureTerms], n = 0;
                double co[kMaxPureTerms];
                pure_coefficients(l, m, cart, co, &n);
                for (int i = 0; i < n; ++i) {
                    const int a = nbf + cart[i];
                    if (cart[i] < 0 || used[cart[i]] >= kMaxPureTerms)
                        return fail(SCFF_ERR_INVALID_ARG, "scff_basis: internal pure-shell table error");
                    cm_idx[(size_t)a * kMaxPureTerms + used[cart[i]]] = nuser + m;
                    cm_c[(size_t)a * kMaxPureTerms + used[cart[i]]] = co[i];
                    ++used[cart[i]];
                }
            }
            nuser += 2 * l + 1;
        } else {
            for (int j = 0; j < nf; ++j) {
                cm_idx[(size_t)(nbf + j) * kMaxPureTerms] = nuser + j;
                cm_c[(size_t)(nbf + j) * kMaxPureTerms] = 1.0;
            }
            nuser += nf;
        }
        nbf += nf;
        eoff += np;
        coff += ncoef;
    }
    // pair list sorted by class L
    const int nrec = (int)recs.size();
    std::vector<int2> buckets[kNumClasses];
    for (int a = 0; a < nrec; ++a)
        for (int b = a; b < nrec; ++b) {
            const int L = rec_lmax(recs[a].type) + rec_lmax(recs[b].type);
            buckets[L].push_back(make_int2(a, b));
        }
    scff_basis_s *B = new scff_basis_s();
    B->ctx = c;
    B->nbf = nuser;
    PairSetDev &d = B->dev;
    d.n_rec = nrec;
    d.nbf = nbf;
    std::vector<int2> pairs;
    d.pair_off[0] = 0;
    d.row_off[0] = d.krow_off[0] = d.axrow_off[0] = 0;
    int64_t axrows = 0;
    for (int L = 0; L < kNumClasses; ++L) {
        pairs.insert(pairs.end(), buckets[L].begin(), buckets[L].end());
        const int64_t np = (int64_t)buckets[L].size();
        d.pair_off[L + 1] = d.pair_off[L] + (int)np;
        d.row_off[L + 1] = d.row_off[L] + np * mono_count(L);
        d.krow_off[L + 1] = d.krow_off[L] + np * vw_count(L);
        axrows += np * (L + 1);
        d.axrow_off[L + 1] = axrows;
    }
    d.n_pair = (int)pairs.size();
    d.n_rows = d.row_off[kNumClasses];
    d.n_krows = d.krow_off[kNumClasses];
    d.n_axrows = axrows;
    std::vector<double> rx(3 * (size_t)nrec), ra(nrec), rw(kRecW * (size_t)nrec);
    std::vector<int32_t> rt(nrec), rf(nrec);
    for (int i = 0; i < nrec; ++i) {
        for (int k = 0; k < 3; ++k) rx[3 * i + k] = xyz[3 * recs[i].atom + k];
        ra[i] = recs[i].alpha;
        rt[i] = recs[i].type;
        rf[i] = recs[i].fn0;
        for (int j = 0; j < kRecW; ++j) rw[kRecW * i + j] = recs[i].w[j];
    }
    scff_status st = SCFF_OK;
    cudaSetDevice(c->device);
    if ((st = upload(&d.rec_xyz, rx)) || (st = upload(&d.rec_alpha, ra)) || (st = upload(&d.rec_type, rt)) ||
        (st = upload(&d.rec_fn0, rf)) || (st = upload(&d.rec_w, rw)) || (st = upload(&d.pair_rec, pairs)) ||
        (any_pure && ((st = upload(&B->cmap_idx, cm_idx)) || (st = upload(&B->cmap_c, cm_c))))) {
        free_basis(B);
        return st;
    }
    c->bases.push_back(B);
    *out = B;
    if (nbf_out) *nbf_out = nuser;
    return SCFF_OK;
}

extern "C" scff_status scff_transitions(scff_ctx *c, scff_basis_h b, int n_states, const double *T, int on_dev,
                                        scff_trans_h *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_transitions: NULL context or output");
    *out = nullptr;
    if (!b || std::find(c->bases.begin(), c->bases.end(), b) == c->bases.end())
        return fail(SCFF_ERR_NOT_FOUND, "scff_transitions: unknown basis handle");
    if (n_states <= 0 || !T) return fail(SCFF_ERR_INVALID_ARG, "scff_transitions: n_states=%d, T=%p", n_states, (const void *)T);
    const size_t bytes = sizeof(double) * (size_t)n_states * b->nbf * b->nbf;
    const int ncart = b->dev.nbf;
    const size_t cbytes = sizeof(double) * (size_t)n_states * ncart * ncart;
    cudaSetDevice(c->device);
    scff_trans_s *t = new scff_trans_s();
    t->ctx = c;
    t->basis = b;
    t->S = n_states;
    t->d_T = nullptr;
    if (cudaMalloc(&t->d_T, cbytes) != cudaSuccess) {
        delete t;
        return fail(SCFF_ERR_OOM, "scff_transitions: cannot allocate %zu bytes", cbytes);
    }
    cudaError_t e = cudaSuccess;
    if (!b->cmap_idx) {
        e = cudaMemcpy(t->d_T, T, bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
        // a device-to-device copy may return early: the caller may free T after this call
        if (e == cudaSuccess && on_dev) e = cudaStreamSynchronize(0);
    } else {
        // pure shells: expand T to the Cartesian components on the device
        const double *Tu = T;
        double *stage = nullptr;
        if (!on_dev) {
            if (cudaMalloc(&stage, bytes) != cudaSuccess) {
                free_trans(t);
                return fail(SCFF_ERR_OOM, "scff_transitions: cannot allocate %zu staging bytes", bytes);
            }
            e = cudaMemcpy(stage, T, bytes, cudaMemcpyHostToDevice);
            Tu = stage;
        }
        if (e == cudaSuccess)
            e = launch_pure_to_cart(n_states, ncart, b->nbf, b->cmap_idx, b->cmap_c, Tu, t->d_T, 0);
        if (e == cudaSuccess) {
            ++c->launches;
            e = cudaStreamSynchronize(0);
        }
        if (stage) cudaFree(stage);
    }
    if (e != cudaSuccess) {
        free_trans(t);
        return fail(SCFF_ERR_CUDA, "scff_transitions: copy failed: %s", cudaGetErrorString(e));
    }
    c->transs.push_back(t);
    *out = t;
    return SCFF_OK;
}

int scff_axes_antisym(const double *qx, int nx, const double *qy, int ny, const double *qz, int nz) {
    const double *ax[3] = {qx, qy, qz};
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < n[a]; ++i)
            if (!(ax[a][n[a] - 1 - i] == -ax[a][i])) return 0;
    return 1;
}

// Whether a job on grid g computes half its points (Hermitian symmetry).
static int grid_half(const scff_ctx *c, const scff_qgrid_s *g) {
    return (c->hermitian && g->product && g->antisym && g->n > 1) ? 1 : 0;
}

extern "C" scff_status scff_set_hermitian(scff_ctx *c, int enable) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_hermitian: NULL context");
    c->hermitian = enable ? 1 : 0;
    return SCFF_OK;
}

extern "C" scff_status scff_set_download_bands(scff_ctx *c, int n_bands) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_download_bands: NULL context");
    if (n_bands < 0 || n_bands > kMaxBands)
        return fail(SCFF_ERR_INVALID_ARG, "scff_set_download_bands: %d bands (0..%d)", n_bands, kMaxBands);
    c->bands = n_bands;
    return SCFF_OK;
}

extern "C" scff_status scff_qgrid_product(scff_ctx *c, const double *qx, int nx, const double *qy, int ny,
                                          const double *qz, int nz, scff_qgrid_h *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_product: NULL context or output");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || !qx || !qy || !qz)
        return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_product: axis sizes %d %d %d", nx, ny, nz);
    const double *ax[3] = {qx, qy, qz};
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < n[a]; ++i)
            if (!isfinite(ax[a][i])) return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_product: non-finite q");
    cudaSetDevice(c->device);
    scff_qgrid_s *g = new scff_qgrid_s();
    g->ctx = c;
    g->product = 1;
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->n = (int64_t)nx * ny * nz;
    g->d_qx = g->d_qy = g->d_qz = g->d_q = nullptr;
    g->hx.assign(qx, qx + nx);
    g->hy.assign(qy, qy + ny);
    g->hz.assign(qz, qz + nz);
    g->antisym = scff_axes_antisym(qx, nx, qy, ny, qz, nz);
    {
        double m[3] = {0, 0, 0};
        for (int i = 0; i < nx; ++i) m[0] = std::max(m[0], fabs(qx[i]));
        for (int i = 0; i < ny; ++i) m[1] = std::max(m[1], fabs(qy[i]));
        for (int i = 0; i < nz; ++i) m[2] = std::max(m[2], fabs(qz[i]));
        g->qmax = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    }
    scff_status st;
    if ((st = upload(&g->d_qx, g->hx)) || (st = upload(&g->d_qy, g->hy)) || (st = upload(&g->d_qz, g->hz))) {
        free_grid(g);
        return st;
    }
    c->grids.push_back(g);
    *out = g;
    return SCFF_OK;
}

extern "C" scff_status scff_qgrid_list(scff_ctx *c, const double *q, int64_t n, scff_qgrid_h *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_list: NULL context or output");
    *out = nullptr;
    if (n < 0 || (n > 0 && !q)) return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_list: n=%lld", (long long)n);
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(q[i])) return fail(SCFF_ERR_INVALID_ARG, "scff_qgrid_list: non-finite q");
    cudaSetDevice(c->device);
    scff_qgrid_s *g = new scff_qgrid_s();
    g->ctx = c;
    g->product = 0;
    g->nx = g->ny = g->nz = 0;
    g->n = n;
    g->d_qx = g->d_qy = g->d_qz = g->d_q = nullptr;
    for (int64_t i = 0; i < n; ++i)
        g->qmax = std::max(g->qmax, sqrt(q[3 * i] * q[3 * i] + q[3 * i + 1] * q[3 * i + 1] + q[3 * i + 2] * q[3 * i + 2]));
    if (n > 0) {
        std::vector<double> v(q, q + 3 * n);
        g->hq = v;
        scff_status st = upload(&g->d_q, v);
        if (st) {
            free_grid(g);
            return st;
        }
    }
    c->grids.push_back(g);
    *out = g;
    return SCFF_OK;
}

extern "C" int64_t scff_qgrid_size(scff_ctx *c, scff_qgrid_h g) {
    if (!c || !g || std::find(c->grids.begin(), c->grids.end(), g) == c->grids.end()) return -1;
    return g->n;
}

template <typename V>
static void release_from(std::vector<V *> &v, V *h, void (*fr)(V *)) {
    auto it = std::find(v.begin(), v.end(), h);
    if (it == v.end()) return;
    v.erase(it);
    fr(h);
}

extern "C" void scff_release_basis(scff_ctx *c, scff_basis_h h) {
    if (!c || !h) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    // transitions built on this basis go with it
    for (size_t i = 0; i < c->transs.size();) {
        if (c->transs[i]->basis == h) {
            drop_screened(c, c->transs[i]);
            free_trans(c->transs[i]);
            c->transs.erase(c->transs.begin() + i);
        } else {
            ++i;
        }
    }
    release_from(c->bases, h, free_basis);
}
extern "C" void scff_release_transitions(scff_ctx *c, scff_trans_h h) {
    if (!c || !h) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (std::find(c->transs.begin(), c->transs.end(), h) != c->transs.end()) drop_screened(c, h);
    release_from(c->transs, h, free_trans);
}
extern "C" void scff_release_qgrid(scff_ctx *c, scff_qgrid_h h) {
    if (!c || !h) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    release_from(c->grids, h, free_grid);
}

// ------------------------------------------------------------------ form factor

// Footprint of one configuration (coefficients, geometry, tables, workspace).
static size_t ff_footprint(const PairSetDev &ps, const scff_qgrid_s *g, int S, int precision, const FFChoice &ch) {
    const bool fp64 = precision == SCFF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const int S_pad = (S + ch.SB - 1) / ch.SB * ch.SB;
    size_t foot = (size_t)S_pad * ps.n_rows * rsz + (size_t)ps.n_pair * 4 * sizeof(double) + 64;
    if (ch.use_tc) {
        const int kind = tc_kind_of_precision(precision);
        foot += tc_workspace_bytes(ps, S, g->nx, g->ny, g->nz, kind);
    } else if (g->product) {
        foot += (size_t)ps.n_pair * (g->nx + g->ny + g->nz) * 2 * rsz;
    }
    return foot;
}

// Host destination of a call with host outputs: the tensor-core path may copy
// the result there itself, band by band, overlapped with its launches (done).
struct HostOut {
    void *f, *f2;
    bool done;
};

// Pair-prep and q-evaluation of one configuration into device outputs (and,
// with ho, possibly already downloaded to ho's host buffers).
static scff_status ff_run(scff_ctx *c, const PairSetDev &ps, scff_trans_s *t, scff_qgrid_s *g, int precision,
                          double scale, void *fdev, void *f2dev, const FFChoice &ch, cudaStream_t st,
                          HostOut *ho = nullptr) {
    const int S = t->S;
    const int64_t nq = g->n;
    const bool fp64 = precision == SCFF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const int SB = ch.SB;
    const int S_pad = (S + SB - 1) / SB * SB;
    const size_t coef_bytes = (size_t)S_pad * ps.n_rows * rsz;
    const size_t geom_bytes = (size_t)ps.n_pair * 4 * sizeof(double) + 64;
    TRY(grow(c, c->coef, coef_bytes + 256));
    TRY(grow(c, c->geom, geom_bytes));
    CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[0], st));
    CUDA_TRY(launch_pair_geom(ps, (double *)c->geom.p, st));
    ++c->launches;
    CUDA_TRY(launch_pairprep(ps, t->d_T, S, SB, S_pad, fp64 ? (double *)c->coef.p : nullptr,
                             fp64 ? nullptr : (float *)c->coef.p, &c->launches, st));
    if (ch.use_tc) {
        const int kind = tc_kind_of_precision(precision);
        const size_t tc_bytes = tc_workspace_bytes(ps, S, g->nx, g->ny, g->nz, kind);
        TcArgs ta;
        memset(&ta, 0, sizeof(ta));
        ta.ps = &ps;
        ta.coef32 = (const float *)c->coef.p;
        ta.SB = SB;
        ta.pair_geom = (const double *)c->geom.p;
        ta.qx = g->d_qx;
        ta.qy = g->d_qy;
        ta.qz = g->d_qz;
        ta.nx = g->nx;
        ta.ny = g->ny;
        ta.nz = g->nz;
        ta.S = S;
        ta.scale = scale;
        ta.f = (float *)fdev;
        ta.f2 = (float *)f2dev;
        ta.err = c->d_err;
        TRY(grow(c, c->tc_ws, tc_bytes + 1024));
        ta.ws = c->tc_ws.p;
        ta.ws_bytes = c->tc_ws.cap;
        ta.ev_mark = c->timing ? c->ev[1] : nullptr;
        ta.kind = kind;
        tc_axes_abs_max(g->hx.data(), g->nx, g->hy.data(), g->ny, g->hz.data(), g->nz, ta.qabs);
        ta.drain_every = ch.drain;
        ta.zstage = ch.zs;
        ta.half = grid_half(c, g);
        int used = 1;
        if (ho && c->bands != 1) {
            if (!c->copy_st) CUDA_TRY(cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
            for (auto &e : c->band_ev)
                if (!e) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            if (!c->progress_h) {
                const size_t pb = sizeof(int) * 8 * (size_t)tc_num_sms();
                CUDA_TRY(cudaHostAlloc((void **)&c->progress_h, pb, cudaHostAllocMapped));
                memset(c->progress_h, 0, pb);
                CUDA_TRY(cudaHostGetDevicePointer((void **)&c->progress_d, c->progress_h, 0));
            }
            ta.n_bands = c->bands;
            ta.f_host = (float *)ho->f;
            ta.f2_host = (float *)ho->f2;
            ta.copy_st = c->copy_st;
            ta.progress_dev = c->progress_d;
            ta.progress_host = c->progress_h;
            ta.ev_done = c->band_ev[0];
            ta.ev_copied = c->band_ev[1];
            ta.bands_used = &used;
        }
        int variant_used = 0;
        ta.variant_used = &variant_used;
        CUDA_TRY(launch_tc_form_factor(ta, &c->launches, st));
        if (ho) ho->done = used > 1;
        c->last_path[0] = 2;
        c->last_path[1] = precision;
        c->last_path[2] = variant_used;
    } else {
        DirectArgs a;
        memset(&a, 0, sizeof(a));
        a.ps = &ps;
        a.coef = c->coef.p;
        a.nq = grid_half(c, g) ? (nq + 1) / 2 : nq;
        a.nq_out = nq;
        a.S = S;
        a.SB = SB;
        a.scale = scale;
        a.f = fdev;
        a.f2 = f2dev;
        a.err_flag = c->d_err;
        if (g->product) {
            const size_t el = 2 * rsz;
            TRY(grow(c, c->gx, (size_t)ps.n_pair * g->nx * el + 256));
            TRY(grow(c, c->gy, (size_t)ps.n_pair * g->ny * el + 256));
            TRY(grow(c, c->gz, (size_t)ps.n_pair * g->nz * el + 256));
            CUDA_TRY(launch_axis_tables(ps, (double *)c->geom.p, g->d_qx, g->nx, 0, c->gx.p, fp64, st));
            CUDA_TRY(launch_axis_tables(ps, (double *)c->geom.p, g->d_qy, g->ny, 1, c->gy.p, fp64, st));
            CUDA_TRY(launch_axis_tables(ps, (double *)c->geom.p, g->d_qz, g->nz, 2, c->gz.p, fp64, st));
            c->launches += 3;
            a.gx = c->gx.p;
            a.gy = c->gy.p;
            a.gz = c->gz.p;
            a.qax = g->d_qx;
            a.qay = g->d_qy;
            a.qaz = g->d_qz;
            a.nx = g->nx;
            a.ny = g->ny;
            a.nz = g->nz;
        } else {
            a.qlist = g->d_q;
            a.pair_geom = (const double *)c->geom.p;
        }
        if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[1], st));
        CUDA_TRY(launch_direct(a, fp64 ? 1 : 0, g->product ? 0 : 1, &c->launches, st));
        c->last_path[0] = fp64 ? 0 : 1;
        c->last_path[1] = fp64 ? SCFF_FP64 : SCFF_FP32;
        c->last_path[2] = 0;
    }
    if (c->timing) {
        CUDA_TRY(cudaEventRecord(c->ev[2], st));
        c->timed_valid = 1;
    }
    return SCFF_OK;
}

// Shape key of the autotuner: log2 buckets of pair monomial rows, states and
// grid points, and the requested precision.
static uint64_t tune_key(const PairSetDev &ps, int S, int64_t nq, int precision) {
    auto lg = [](double x) { return (uint64_t)std::max(0.0, std::floor(std::log2(std::max(1.0, x)) * 2.0)); };
    return (lg((double)ps.n_rows) << 32) | (lg((double)S) << 24) | (lg((double)nq) << 8) | (uint64_t)precision;
}

// Times every candidate configuration once on this job (outputs go to the
// device staging buffers) and keeps the fastest.  All candidates meet the
// accuracy of the requested precision: the tensor-core path with TMEM drains
// of 8 k-chunks (the TMEM accumulation error grows linearly with the drain
// length, and 16 gives only about 1% speed for twice the error, so it is not
// a candidate), and the FP32 direct path (1e-6) for the 1e-5-grade modes.
static scff_status autotune(scff_ctx *c, const PairSetDev &ps, scff_trans_s *t, scff_qgrid_s *g, int precision,
                            cudaStream_t st, FFChoice *best) {
    const size_t rsz = sizeof(float);
    const int S = t->S;
    const int64_t nq = g->n;
    std::vector<FFChoice> cand;
    // tensor cores with both W generator variants (bitwise the same results) unless the
    // context fixes one, then the FP32 direct path's state blocks
    const int kind = tc_kind_of_precision(precision);
    for (int zs : {4, 3, 2, 1, 0})
        if ((c->tc_zstage < 0 || c->tc_zstage == zs) && kind >= 0 && tc_variant_resolve(kind, zs, g->nz % 128 == 0) == zs)
            cand.push_back({1, 8, 8, zs});
    for (int sb : {8, 12, 16}) cand.push_back({0, 0, sb, 0});
    TRY(grow(c, c->fstage, (size_t)S * nq * 2 * rsz + 256));
    TRY(grow(c, c->f2stage, (size_t)S * nq * rsz + 256));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    *best = cand[0];
    const int saved_timing = c->timing;
    c->timing = 0;
    for (const FFChoice &ch : cand) {
        if (ff_footprint(ps, g, S, precision, ch) > c->budget) continue;
        scff_status s = ff_run(c, ps, t, g, precision, 1.0, c->fstage.p, c->f2stage.p, ch, st);  // warm-up
        if (s != SCFF_OK) continue;
        cudaEventRecord(e0, st);
        s = ff_run(c, ps, t, g, precision, 1.0, c->fstage.p, c->f2stage.p, ch, st);
        cudaEventRecord(e1, st);
        if (s != SCFF_OK || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            *best = ch;
        }
    }
    c->timing = saved_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_ms[tune_key(ps, S, nq, precision)] = best_ms;
    return SCFF_OK;
}

// ---- error-bounded pair screening

static ScreenedSet *find_screened(scff_ctx *c, scff_trans_s *t, scff_qgrid_s *g) {
    for (ScreenedSet *e : c->screened)
        if (e->trans == t && e->eps == c->screen_eps && fabs(e->qmax - g->qmax) <= 1e-12 * (1.0 + g->qmax)) return e;
    return nullptr;
}

// Up to 64 q points of the grid itself: the 8 nearest the origin and a
// seeded sample, so max over them of |f_s| never exceeds its grid maximum.
static std::vector<double> probe_points(const scff_qgrid_s *g) {
    std::vector<double> q;
    if (g->product) {
        auto nearest2 = [](const std::vector<double> &ax) {
            std::vector<int> idx(ax.size());
            for (size_t i = 0; i < ax.size(); ++i) idx[i] = (int)i;
            std::sort(idx.begin(), idx.end(), [&](int a, int b) { return fabs(ax[a]) < fabs(ax[b]); });
            idx.resize(std::min<size_t>(2, idx.size()));
            return idx;
        };
        for (int ix : nearest2(g->hx))
            for (int iy : nearest2(g->hy))
                for (int iz : nearest2(g->hz)) q.insert(q.end(), {g->hx[ix], g->hy[iy], g->hz[iz]});
        uint64_t x = 0x9E3779B97F4A7C15ull;
        while (q.size() < 3 * 64 && q.size() < (size_t)(3 * g->n)) {
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            q.insert(q.end(), {g->hx[x % g->nx], g->hy[(x >> 20) % g->ny], g->hz[(x >> 40) % g->nz]});
        }
    } else {
        const int64_t n = std::min<int64_t>(g->n, 64);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t j = g->n <= 64 ? i : (i * (g->n / 64));
            q.insert(q.end(), {g->hq[3 * j], g->hq[3 * j + 1], g->hq[3 * j + 2]});
        }
    }
    return q;
}

// Drops every pair whose bounded contribution, summed over the dropped pairs,
// stays below eps * F_s for every state s, where F_s is the largest |f_s| at
// the probe points (a lower bound of max |f_s| on the grid): the screened
// result then differs from the exact one by at most eps * max_q |f_s(q)|.
static scff_status get_screened(scff_ctx *c, scff_basis_s *b, scff_trans_s *t, scff_qgrid_s *g, cudaStream_t st,
                                ScreenedSet **out) {
    if (ScreenedSet *e = find_screened(c, t, g)) {
        *out = e;
        return SCFF_OK;
    }
    const PairSetDev &ps = b->dev;
    const int S = t->S;
    // the bounds and the probe values come from the FP64 coefficients and the
    // FP64 path, so that only FP64 rounding is left in the error argument
    const int SB = direct_state_block(S, true);
    const int S_pad = (S + SB - 1) / SB * SB;
    TRY(grow(c, c->coef, (size_t)S_pad * ps.n_rows * sizeof(double) + 256));
    TRY(grow(c, c->geom, (size_t)ps.n_pair * 4 * sizeof(double) + 64));
    CUDA_TRY(launch_pair_geom(ps, (double *)c->geom.p, st));
    CUDA_TRY(launch_pairprep(ps, t->d_T, S, SB, S_pad, (double *)c->coef.p, nullptr, &c->launches, st));
    std::vector<double> qp = probe_points(g);
    const int np = (int)(qp.size() / 3);
    double *d_bound = nullptr, *d_fp = nullptr;
    double *d_q = nullptr;
    const size_t nb = (size_t)ps.n_pair * S;
    if (cudaMalloc(&d_bound, sizeof(double) * std::max<size_t>(nb, 1)) != cudaSuccess ||
        cudaMalloc(&d_fp, sizeof(double) * 2 * (size_t)S * std::max(np, 1)) != cudaSuccess ||
        cudaMalloc(&d_q, sizeof(double) * std::max<size_t>(qp.size(), 3)) != cudaSuccess) {
        cudaFree(d_bound);
        cudaFree(d_fp);
        cudaFree(d_q);
        return fail(SCFF_ERR_OOM, "scff_form_factor: screening buffers");
    }
    std::vector<double> hb(nb), hf(2 * (size_t)S * np);
    scff_status rc = SCFF_OK;
    do {
        if (launch_pair_bounds(ps, (const double *)c->coef.p, SB, S, g->qmax, d_bound, st) != cudaSuccess ||
            cudaMemcpyAsync(d_q, qp.data(), sizeof(double) * qp.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = fail(SCFF_ERR_CUDA, "scff_form_factor: screening launch failed");
            break;
        }
        DirectArgs a;
        memset(&a, 0, sizeof(a));
        a.ps = &ps;
        a.coef = c->coef.p;
        a.qlist = d_q;
        a.pair_geom = (const double *)c->geom.p;
        a.nq = np;
        a.S = S;
        a.SB = SB;
        a.scale = 1.0;
        a.f = d_fp;
        a.err_flag = c->d_err;
        if (launch_direct(a, 1, 1, &c->launches, st) != cudaSuccess ||
            cudaMemcpyAsync(hb.data(), d_bound, sizeof(double) * nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hf.data(), d_fp, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(SCFF_ERR_CUDA, "scff_form_factor: screening probe failed");
            break;
        }
    } while (0);
    cudaFree(d_bound);
    cudaFree(d_fp);
    cudaFree(d_q);
    if (rc != SCFF_OK) return rc;
    std::vector<double> F(S, 0.0);
    for (int s = 0; s < S; ++s)
        for (int i = 0; i < np; ++i) {
            const double re = hf[2 * ((size_t)s * np + i)], im = hf[2 * ((size_t)s * np + i) + 1];
            F[s] = std::max(F[s], sqrt(re * re + im * im) * (1.0 - 1e-9));  // margin for the FP64 probe
        }
    // greedy: smallest relative bound first, stop at the first pair that does not fit
    std::vector<double> score(ps.n_pair);
    for (int p = 0; p < ps.n_pair; ++p) {
        double m = 0.0;
        for (int s = 0; s < S; ++s) {
            const double bb = hb[(size_t)p * S + s];
            m = std::max(m, F[s] > 0 ? bb / F[s] : (bb > 0 ? 1e300 : 0.0));
        }
        score[p] = m;
    }
    std::vector<int> order(ps.n_pair);
    for (int p = 0; p < ps.n_pair; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return score[x] < score[y]; });
    std::vector<char> keep(ps.n_pair, 1);
    std::vector<double> cum(S, 0.0);
    for (int p : order) {
        bool fits = true;
        for (int s = 0; s < S && fits; ++s) fits = cum[s] + hb[(size_t)p * S + s] <= c->screen_eps * F[s];
        if (!fits) break;
        for (int s = 0; s < S; ++s) cum[s] += hb[(size_t)p * S + s];
        keep[p] = 0;
    }
    // compacted pair list, still ordered by class
    std::vector<int2> all(ps.n_pair), kept;
    CUDA_TRY(cudaMemcpy(all.data(), ps.pair_rec, sizeof(int2) * ps.n_pair, cudaMemcpyDeviceToHost));
    ScreenedSet *e = new ScreenedSet();
    e->trans = t;
    e->eps = c->screen_eps;
    e->qmax = g->qmax;
    e->dev = ps;
    e->total = ps.n_pair;
    e->dev.pair_off[0] = 0;
    e->dev.row_off[0] = e->dev.krow_off[0] = e->dev.axrow_off[0] = 0;
    for (int L = 0; L < kNumClasses; ++L) {
        int cnt = 0;
        for (int p = ps.pair_off[L]; p < ps.pair_off[L + 1]; ++p)
            if (keep[p]) {
                kept.push_back(all[p]);
                ++cnt;
            }
        e->dev.pair_off[L + 1] = e->dev.pair_off[L] + cnt;
        e->dev.row_off[L + 1] = e->dev.row_off[L] + (int64_t)cnt * mono_count(L);
        e->dev.krow_off[L + 1] = e->dev.krow_off[L] + (int64_t)cnt * vw_count(L);
        e->dev.axrow_off[L + 1] = e->dev.axrow_off[L] + (int64_t)cnt * (L + 1);
    }
    e->dev.n_pair = (int)kept.size();
    e->dev.n_rows = e->dev.row_off[kNumClasses];
    e->dev.n_krows = e->dev.krow_off[kNumClasses];
    e->dev.n_axrows = e->dev.axrow_off[kNumClasses];
    e->kept = (int)kept.size();
    e->dev.pair_rec = nullptr;
    if (!kept.empty()) {
        scff_status us = upload(&e->dev.pair_rec, kept);
        if (us != SCFF_OK) {
            delete e;
            return us;
        }
    }
    c->screened.push_back(e);
    *out = e;
    return SCFF_OK;
}

extern "C" scff_status scff_set_screening(scff_ctx *c, double eps) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_screening: NULL context");
    if (!(eps >= 0.0 && eps < 1.0)) return fail(SCFF_ERR_INVALID_ARG, "scff_set_screening: eps %g", eps);
    c->screen_eps = eps;
    return SCFF_OK;
}

extern "C" scff_status scff_screening_info(scff_ctx *c, scff_trans_h t, scff_qgrid_h g, int64_t *out) {
    if (!c || !t || !g || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_screening_info: NULL argument");
    ScreenedSet *e = find_screened(c, t, g);
    if (!e) return fail(SCFF_ERR_NOT_FOUND, "scff_screening_info: no screened pair set for this job");
    out[0] = e->kept;
    out[1] = e->total;
    out[2] = e->dev.n_krows;
    out[3] = t->basis->dev.n_krows;
    return SCFF_OK;
}

extern "C" scff_status scff_set_autotune(scff_ctx *c, int enable) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_set_autotune: NULL context");
    c->autotune = enable ? 1 : 0;
    return SCFF_OK;
}

extern "C" scff_status scff_autotune_choice(scff_ctx *c, scff_basis_h b, scff_trans_h t, scff_qgrid_h g,
                                            int precision, int32_t *out) {
    if (!c || !b || !t || !g || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_autotune_choice: NULL argument");
    const ScreenedSet *se = c->screen_eps > 0 ? find_screened(c, t, g) : nullptr;
    auto it = c->tune.find(tune_key(se ? se->dev : b->dev, t->S, g->n, precision));
    if (it == c->tune.end()) return fail(SCFF_ERR_NOT_FOUND, "scff_autotune_choice: shape not tuned yet");
    out[0] = it->second.use_tc;
    out[1] = it->second.drain;
    out[2] = it->second.SB;
    out[3] = (int32_t)(1000.0f * c->tune_ms[it->first]);  // microseconds of the best candidate
    out[4] = it->second.zs;
    return SCFF_OK;
}

extern "C" scff_status scff_form_factor(scff_ctx *c, scff_basis_h b, scff_trans_h t, scff_qgrid_h g, int precision,
                                        double scale, void *f_out, void *f2_out, int out_on_device, void *stream) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_form_factor: NULL context");
    if (!b || std::find(c->bases.begin(), c->bases.end(), b) == c->bases.end())
        return fail(SCFF_ERR_NOT_FOUND, "scff_form_factor: unknown basis handle");
    if (!t || std::find(c->transs.begin(), c->transs.end(), t) == c->transs.end())
        return fail(SCFF_ERR_NOT_FOUND, "scff_form_factor: unknown transitions handle");
    if (!g || std::find(c->grids.begin(), c->grids.end(), g) == c->grids.end())
        return fail(SCFF_ERR_NOT_FOUND, "scff_form_factor: unknown q-grid handle");
    if (t->basis != b) return fail(SCFF_ERR_INVALID_ARG, "scff_form_factor: transitions belong to another basis");
    if (precision < SCFF_FP64 || precision > SCFF_FP16X2)
        return fail(SCFF_ERR_INVALID_ARG, "scff_form_factor: precision %d", precision);
    if (!f_out) return fail(SCFF_ERR_INVALID_ARG, "scff_form_factor: f_out is NULL");
    if (!isfinite(scale)) return fail(SCFF_ERR_INVALID_ARG, "scff_form_factor: scale is not finite");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int S = t->S;
    const int64_t nq = g->n;
    const bool fp64 = precision == SCFF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const bool tc_prec = tc_kind_of_precision(precision) >= 0;
    const bool tc_path = tc_prec && g->product;
    int dev_sms = 148;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c->device);
    const int direct_sb = fp64 ? direct_state_block_fp64(S, grid_half(c, g) ? (nq + 1) / 2 : nq, dev_sms)
                               : direct_state_block(S, false);
    FFChoice ch = {tc_path ? 1 : 0, c->drain_every >= 0 ? c->drain_every : 8, tc_path ? 8 : direct_sb,
                   zstage_mode(c, precision)};
    const PairSetDev *ps = &b->dev;
    if (c->screen_eps > 0 && nq > 0) {
        ScreenedSet *se = nullptr;
        TRY(get_screened(c, b, t, g, st, &se));
        ps = &se->dev;
    }
    if (c->autotune && tc_prec && g->product && nq > 0) {
        const uint64_t key = tune_key(*ps, S, nq, precision);
        auto it = c->tune.find(key);
        if (it == c->tune.end()) {
            FFChoice best;
            TRY(autotune(c, *ps, t, g, precision, st, &best));
            it = c->tune.emplace(key, best).first;
        }
        ch = it->second;
    }
    // footprint check (admission)
    const size_t out_bytes = (size_t)S * nq * rsz * 3;
    const size_t foot = ff_footprint(*ps, g, S, precision, ch) + (out_on_device ? 0 : out_bytes);
    if (foot > c->budget)
        return fail(SCFF_ERR_ADMISSION, "scff_form_factor: footprint %zu bytes exceeds the budget %llu", foot,
                    (unsigned long long)c->budget);
    void *fdev = f_out, *f2dev = f2_out;
    if (!out_on_device) {
        TRY(grow(c, c->fstage, (size_t)S * nq * 2 * rsz + 256));
        fdev = c->fstage.p;
        if (f2_out) {
            TRY(grow(c, c->f2stage, (size_t)S * nq * rsz + 256));
            f2dev = c->f2stage.p;
        }
    }
    if (ps->n_pair == 0) {  // every pair screened away: the result is zero to within eps
        if (nq > 0) {
            CUDA_TRY(cudaMemsetAsync(fdev, 0, (size_t)S * nq * 2 * rsz, st));
            if (f2dev) CUDA_TRY(cudaMemsetAsync(f2dev, 0, (size_t)S * nq * rsz, st));
        }
    }
    HostOut ho = {f_out, f2_out, false};
    if (ps->n_pair != 0) TRY(ff_run(c, *ps, t, g, precision, scale, fdev, f2dev, ch, st, out_on_device ? nullptr : &ho));
    if (!out_on_device) {
        if (nq > 0 && !ho.done) {
            CUDA_TRY(cudaMemcpyAsync(f_out, fdev, (size_t)S * nq * 2 * rsz, cudaMemcpyDeviceToHost, st));
            if (f2_out) CUDA_TRY(cudaMemcpyAsync(f2_out, f2dev, (size_t)S * nq * rsz, cudaMemcpyDeviceToHost, st));
        }
        CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (*c->h_err) return fail(SCFF_ERR_TIMEOUT, "scff_form_factor: a device-side wait timed out (code %d)", *c->h_err);
    }
    return SCFF_OK;
}

// Separable integral of every state's form factor against wx(qx) wy(qy) wz(qz).
extern "C" scff_status scff_separable_integral(scff_ctx *c, scff_basis_h b, scff_trans_h t, const double *qx,
                                               const double *wx, int nx, const double *qy, const double *wy, int ny,
                                               const double *qz, const double *wz, int nz, double scale,
                                               double *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_separable_integral: NULL argument");
    if (!b || std::find(c->bases.begin(), c->bases.end(), b) == c->bases.end())
        return fail(SCFF_ERR_NOT_FOUND, "scff_separable_integral: unknown basis handle");
    if (!t || std::find(c->transs.begin(), c->transs.end(), t) == c->transs.end() || t->basis != b)
        return fail(SCFF_ERR_NOT_FOUND, "scff_separable_integral: unknown or mismatched transitions handle");
    if (nx < 1 || ny < 1 || nz < 1 || !qx || !wx || !qy || !wy || !qz || !wz || !isfinite(scale))
        return fail(SCFF_ERR_INVALID_ARG, "scff_separable_integral: empty axis or NULL array");
    cudaSetDevice(c->device);
    const PairSetDev &ps = b->dev;
    const int S = t->S, SB = 4, S_pad = (S + 3) / 4 * 4;
    const int n[3] = {nx, ny, nz};
    const double *hq[3] = {qx, qy, qz}, *hw[3] = {wx, wy, wz};
    size_t bytes = (size_t)ps.n_pair * 32 + 256;
    const size_t coef_off = bytes;
    bytes += (size_t)S_pad * ps.n_rows * 8 + 256;
    const size_t ax_off = bytes;
    bytes += sizeof(double) * 2 * (size_t)(nx + ny + nz) + 256;
    const size_t sums_off = bytes;
    bytes += sizeof(double2) * 3 * (size_t)(ps.n_axrows + 1) + 256;
    const size_t part_off = bytes;
    bytes += sizeof(double2) * (size_t)S * (ps.n_pair + 1) + 256;
    const size_t out_off = bytes;
    bytes += sizeof(double) * 2 * S + 256;
    void *buf = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return fail(SCFF_ERR_OOM, "scff_separable_integral: %zu bytes", bytes);
    uint8_t *B = static_cast<uint8_t *>(buf);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    double *geom = reinterpret_cast<double *>(B);
    double *coef = reinterpret_cast<double *>(B + al(coef_off));
    double *dq[3], *dw[3];
    size_t o = al(ax_off);
    for (int a = 0; a < 3; ++a) {
        dq[a] = reinterpret_cast<double *>(B + o);
        o += sizeof(double) * n[a];
        dw[a] = reinterpret_cast<double *>(B + o);
        o += sizeof(double) * n[a];
    }
    double2 *sums = reinterpret_cast<double2 *>(B + al(sums_off));
    double2 *part = reinterpret_cast<double2 *>(B + al(part_off));
    double *dout = reinterpret_cast<double *>(B + al(out_off));
    scff_status rc = SCFF_OK;
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        e = cudaMemcpy(dq[a], hq[a], sizeof(double) * n[a], cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dw[a], hw[a], sizeof(double) * n[a], cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = launch_pair_geom(ps, geom, 0);
    if (e == cudaSuccess) e = launch_pairprep(ps, t->d_T, S, SB, S_pad, coef, nullptr, &c->launches, 0);
    const double *cq[3] = {dq[0], dq[1], dq[2]}, *cw[3] = {dw[0], dw[1], dw[2]};
    if (e == cudaSuccess)
        e = launch_separable(ps, geom, coef, SB, S, cq, cw, n, sums, part, scale, dout, &c->launches, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = fail(SCFF_ERR_CUDA, "scff_separable_integral: %s", cudaGetErrorString(e));
    cudaFree(buf);
    return rc;
}

// Reads the device status word after all work on `stream` has finished.
extern "C" scff_status scff_alu_peak(scff_ctx *c, int fp64, int iters, double *tflops, double *ms) {
    if (!c || !tflops || !ms) return fail(SCFF_ERR_INVALID_ARG, "scff_alu_peak: NULL argument");
    if (iters < 1 || iters > (1 << 24)) return fail(SCFF_ERR_INVALID_ARG, "scff_alu_peak: iters must be 1..2^24");
    if (fp64 < 0 || fp64 > 2) return fail(SCFF_ERR_INVALID_ARG, "scff_alu_peak: mode %d (0 FP32, 1 FP64, 2 f32x2)", fp64);
    cudaSetDevice(c->device);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(measure_alu_peak(fp64, iters, tflops, ms));
    return SCFF_OK;
}

extern "C" scff_status scff_wait_selftest(scff_ctx *c, int64_t tries) {
    if (!c || tries < 1 || tries > (int64_t)1 << 24)
        return fail(SCFF_ERR_INVALID_ARG, "scff_wait_selftest: tries must be 1..2^24");
    cudaSetDevice(c->device);
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    CUDA_TRY(launch_wait_selftest((long long)tries, c->d_err, 0));
    ++c->launches;
    int h = 0;
    CUDA_TRY(cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(c->d_err, 0, sizeof(int)));
    if (h) return fail(SCFF_ERR_TIMEOUT, "scff_wait_selftest: the device-side wait gave up as intended (code %d)", h);
    return SCFF_OK;
}

extern "C" scff_status scff_sync(scff_ctx *c, void *stream) {
    if (!c) return fail(SCFF_ERR_INVALID_ARG, "scff_sync: NULL context");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (*c->h_err) return fail(SCFF_ERR_TIMEOUT, "scff_sync: a device-side wait timed out (code %d)", *c->h_err);
    return SCFF_OK;
}

// ------------------------------------------------------------------ batches (plans)
//
// A plan holds a fixed list of form-factor jobs and every device buffer their
// evaluation needs.  Tensor-core jobs (product grids, split precisions) are
// grouped so that each group's tables and A images fit the workspace; a
// group is evaluated by one persistent launch over all of its tiles.  The
// other jobs run the direct path one after the other.  scff_plan_run only
// launches kernels (no allocation, no synchronisation), so it can be
// captured; scff_plan_run_graph captures it once and replays the graph.

struct PlanJob {
    scff_job job;
    int tc;            // tensor-core job
    int group;         // group index (tensor-core jobs)
    size_t region;     // offset of the job's tables and A image in the group area
    int S, S_pad, SB;
    int half;          // Hermitian half of an antisymmetric product grid
};

struct scff_plan_s {
    scff_ctx *ctx;
    int precision;
    int tc_kind;
    int SB;
    std::vector<PlanJob> jobs;
    std::vector<std::vector<int>> groups;
    std::vector<size_t> group_desc, group_items;  // offsets in dev
    std::vector<int> group_nitems;
    std::vector<char> group_zs;                   // W generator variant of each group's launch
    int pair = 0;                                 // jobs laid out for the CTA-pair launch
    int oct = 0;                                  // ... in the octant form (on antisymmetric grids)
    size_t off_queue = 0;                         // device int: the launches' work-queue counter
    void *dev = nullptr;
    size_t dev_bytes = 0;
    size_t off_geom = 0, off_coef = 0, off_tab = 0, off_group = 0;
    size_t tab_stride = 0;
    // Per-job prep of a tensor-core group runs on kLanes streams forked from
    // the launch stream (job k of the group on lane k mod kLanes), each lane
    // with its own pair-geometry and coefficient scratch at lane x lane_stride.
    static constexpr int kLanes = 4;
    size_t lane_stride = 0;
    cudaStream_t lane[kLanes] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kLanes] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    int64_t launches_per_run = 0;
};

static size_t up1k(size_t x) { return (x + 1023) / 1024 * 1024; }

extern "C" scff_status scff_plan_create(scff_ctx *c, int n_jobs, const scff_job *jobs, int precision,
                                        uint64_t workspace_bytes, scff_plan_h *out) {
    if (!c || !out) return fail(SCFF_ERR_INVALID_ARG, "scff_plan_create: NULL context or output");
    *out = nullptr;
    if (n_jobs <= 0 || !jobs) return fail(SCFF_ERR_INVALID_ARG, "scff_plan_create: no jobs");
    if (precision < SCFF_FP64 || precision > SCFF_FP16X2)
        return fail(SCFF_ERR_INVALID_ARG, "scff_plan_create: precision %d", precision);
    cudaSetDevice(c->device);
    const bool tc_prec = tc_kind_of_precision(precision) >= 0;
    const bool fp64 = precision == SCFF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    scff_plan_s *P = new scff_plan_s();
    P->ctx = c;
    P->precision = precision;
    P->tc_kind = tc_kind_of_precision(precision);
    // jobs laid out for the CTA-pair launch when that variant is asked for (it never changes a result)
    {
        const int v = P->tc_kind >= 0 ? tc_variant_resolve(P->tc_kind, zstage_mode(c, precision), false) : 0;
        P->pair = tc_prefetch_ok(P->tc_kind) && (v == 3 || v == 4) ? 1 : 0;
        P->oct = v == 4 ? 1 : 0;
    }
    P->SB = fp64 ? 4 : 8;
    uint64_t budget = workspace_bytes ? workspace_bytes : std::min<uint64_t>(c->budget, 64ull << 30);
    size_t geom_max = 256, coef_max = 256, tab_max = 256;
    for (int i = 0; i < n_jobs; ++i) {
        const scff_job &j = jobs[i];
        if (!j.basis || std::find(c->bases.begin(), c->bases.end(), j.basis) == c->bases.end() || !j.trans ||
            std::find(c->transs.begin(), c->transs.end(), j.trans) == c->transs.end() || !j.grid ||
            std::find(c->grids.begin(), c->grids.end(), j.grid) == c->grids.end()) {
            delete P;
            return fail(SCFF_ERR_NOT_FOUND, "scff_plan_create: job %d has an unknown handle", i);
        }
        if (j.trans->basis != j.basis || !j.f_out || !isfinite(j.scale)) {
            delete P;
            return fail(SCFF_ERR_INVALID_ARG, "scff_plan_create: job %d is inconsistent", i);
        }
        PlanJob pj;
        pj.job = j;
        pj.tc = tc_prec && j.grid->product;
        pj.half = grid_half(c, j.grid);
        pj.group = -1;
        pj.region = 0;
        pj.S = j.trans->S;
        pj.SB = pj.tc ? 8 : direct_state_block(pj.S, fp64);
        pj.S_pad = (pj.S + pj.SB - 1) / pj.SB * pj.SB;
        const PairSetDev &ps = j.basis->dev;
        geom_max = std::max(geom_max, (size_t)ps.n_pair * 4 * sizeof(double));
        coef_max = std::max(coef_max, (size_t)pj.S_pad * ps.n_rows * (pj.tc ? sizeof(float) : rsz));
        if (!pj.tc && j.grid->product)
            tab_max = std::max(tab_max, (size_t)ps.n_pair * std::max(j.grid->nx, std::max(j.grid->ny, j.grid->nz)) * 2 * rsz);
        P->jobs.push_back(pj);
    }
    // Greedy grouping of tensor-core jobs by footprint, largest first.
    std::vector<int> order;
    for (int i = 0; i < n_jobs; ++i)
        if (P->jobs[i].tc) order.push_back(i);
    auto bytes_of = [&](int i) {
        const PlanJob &pj = P->jobs[i];
        return up1k(tc_job_bytes(pj.job.basis->dev, pj.S, pj.job.grid->nx, pj.job.grid->ny, pj.job.grid->nz,
                                 P->tc_kind));
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes_of(a) > bytes_of(b); });
    const size_t fixed = up1k(geom_max) + up1k(coef_max) + 3 * up1k(tab_max);
    if (fixed >= budget) {
        delete P;
        return fail(SCFF_ERR_ADMISSION, "scff_plan_create: workspace budget %llu below the fixed scratch %zu",
                    (unsigned long long)budget, fixed);
    }
    const size_t area_budget = budget - fixed;
    size_t area_max = 0, cur = 0;
    for (int i : order) {
        const size_t b = bytes_of(i);
        if (b > area_budget) {
            delete P;
            return fail(SCFF_ERR_ADMISSION, "scff_plan_create: job %d needs %zu bytes, above the budget %zu", i, b,
                        area_budget);
        }
        if (P->groups.empty() || cur + b > area_budget) {
            P->groups.emplace_back();
            cur = 0;
        }
        P->jobs[i].group = (int)P->groups.size() - 1;
        P->jobs[i].region = cur;
        P->groups.back().push_back(i);
        cur += b;
        area_max = std::max(area_max, cur);
    }
    // descriptors and work lists of every group (kept for the plan's lifetime)
    size_t desc_bytes = 0;
    std::vector<std::vector<TcJobDev>> gdesc(P->groups.size());
    std::vector<std::vector<int4>> gitems(P->groups.size());
    P->off_geom = 0;
    P->off_coef = up1k(geom_max);
    P->lane_stride = up1k(geom_max) + up1k(coef_max);
    P->off_tab = (size_t)scff_plan_s::kLanes * P->lane_stride;
    P->tab_stride = up1k(tab_max);
    P->off_group = P->off_tab + 3 * P->tab_stride;
    const size_t off_desc = P->off_group + up1k(area_max);
    for (size_t g = 0; g < P->groups.size(); ++g) {
        P->group_desc.push_back(off_desc + desc_bytes);
        desc_bytes += up1k(sizeof(TcJobDev) * P->groups[g].size());
        P->group_items.push_back(0);
        P->group_nitems.push_back(0);
        P->group_zs.push_back(0);
    }
    // work lists need the descriptors (tile counts), which need addresses: allocate first
    size_t items_bytes = 0;
    std::vector<size_t> nitems_est(P->groups.size(), 0);
    for (size_t g = 0; g < P->groups.size(); ++g) {
        for (int i : P->groups[g]) {
            const PlanJob &pj = P->jobs[i];
            const int64_t M = (int64_t)pj.S * pj.job.grid->nx;
            const int64_t N = (int64_t)pj.job.grid->ny * pj.job.grid->nz;
            // column tiles: 128 columns, or 32 octant points in the octant form
            const int64_t Noct = (int64_t)((pj.job.grid->ny + 1) / 2) * ((pj.job.grid->nz + 1) / 2);
            const int64_t n_nt = std::max((N + 127) / 128, (Noct + 31) / 32);
            nitems_est[g] += (size_t)tc_max_items(((M + 127) / 128) * n_nt);
        }
        items_bytes += up1k(sizeof(int4) * nitems_est[g]);
    }
    P->off_queue = off_desc + desc_bytes + items_bytes;  // work-queue counter of the persistent launches
    P->dev_bytes = P->off_queue + 1024;
    if (cudaMalloc(&P->dev, P->dev_bytes) != cudaSuccess) {
        delete P;
        return fail(SCFF_ERR_OOM, "scff_plan_create: cannot allocate %zu bytes", P->dev_bytes);
    }
    uint8_t *base = static_cast<uint8_t *>(P->dev);
    size_t ioff = off_desc + desc_bytes;
    for (size_t g = 0; g < P->groups.size(); ++g) {
        for (int i : P->groups[g]) {
            const PlanJob &pj = P->jobs[i];
            TcArgs ta;
            memset(&ta, 0, sizeof(ta));
            ta.ps = &pj.job.basis->dev;
            ta.S = pj.S;
            ta.nx = pj.job.grid->nx;
            ta.ny = pj.job.grid->ny;
            ta.nz = pj.job.grid->nz;
            ta.scale = pj.job.scale;
            ta.f = (float *)pj.job.f_out;
            ta.f2 = (float *)pj.job.f2_out;
            ta.kind = P->tc_kind;
            ta.half = pj.half;
            ta.pair = P->pair;
            ta.oct = P->oct && pj.half;
            TcJobDev jd;
            memset(&jd, 0, sizeof(jd));
            tc_job_desc(ta, base + P->off_group + pj.region, &jd);
            gdesc[g].push_back(jd);
        }
        tc_build_items(gdesc[g].data(), (int)gdesc[g].size(), gitems[g]);
        if (gitems[g].size() > nitems_est[g]) {
            cudaFree(P->dev);
            delete P;
            return fail(SCFF_ERR_INVALID_ARG, "scff_plan_create: work list larger than its reserved space");
        }
        P->group_items[g] = ioff;
        P->group_nitems[g] = (int)gitems[g].size();
        P->group_zs[g] = (char)tc_variant_for(P->tc_kind, zstage_mode(c, precision), gdesc[g].data(), (int)gdesc[g].size());
        ioff += up1k(sizeof(int4) * nitems_est[g]);
        cudaError_t e1 = cudaMemcpy(base + P->group_desc[g], gdesc[g].data(), sizeof(TcJobDev) * gdesc[g].size(),
                                    cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(base + P->group_items[g], gitems[g].data(), sizeof(int4) * gitems[g].size(),
                                    cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaFree(P->dev);
            delete P;
            return fail(SCFF_ERR_CUDA, "scff_plan_create: descriptor upload failed");
        }
    }
    // Kernel attributes are set outside any later stream capture.
    for (size_t g = 0; g < P->groups.size(); ++g)
        tc_launch_persistent(P->tc_kind, P->group_zs[g], nullptr, nullptr, 0, 0, nullptr, 0, nullptr, 0);
    // prep lanes (streams and events of the fork and join)
    bool lanes_ok = cudaEventCreateWithFlags(&P->fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l < scff_plan_s::kLanes && lanes_ok; ++l)
        lanes_ok = cudaStreamCreateWithFlags(&P->lane[l], cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&P->join_ev[l], cudaEventDisableTiming) == cudaSuccess;
    if (!lanes_ok) {
        free_plan_any(P);
        return fail(SCFF_ERR_CUDA, "scff_plan_create: stream or event creation failed");
    }
    c->plans.push_back(P);
    *out = P;
    return SCFF_OK;
}

static scff_status plan_launch(scff_plan_s *P, cudaStream_t st, int64_t *launches) {
    scff_ctx *c = P->ctx;
    uint8_t *base = static_cast<uint8_t *>(P->dev);
    double *geom = reinterpret_cast<double *>(base + P->off_geom);
    void *coef = base + P->off_coef;
    const bool fp64 = P->precision == SCFF_FP64;
    CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    for (size_t g = 0; g < P->groups.size(); ++g) {
        // the group's jobs are prepared on the lanes, after everything before on st
        // (the previous group's launch still reads the shared group area)
        CUDA_TRY(cudaEventRecord(P->fork_ev, st));
        for (int l = 0; l < scff_plan_s::kLanes; ++l) CUDA_TRY(cudaStreamWaitEvent(P->lane[l], P->fork_ev, 0));
        int k = 0;
        for (int i : P->groups[g]) {
            const PlanJob &pj = P->jobs[i];
            const PairSetDev &ps = pj.job.basis->dev;
            const int l = k++ % scff_plan_s::kLanes;
            cudaStream_t ls = P->lane[l];
            double *lgeom = reinterpret_cast<double *>(base + (size_t)l * P->lane_stride + P->off_geom);
            void *lcoef = base + (size_t)l * P->lane_stride + P->off_coef;
            CUDA_TRY(launch_pair_geom(ps, lgeom, ls));
            ++*launches;
            CUDA_TRY(launch_pairprep(ps, pj.job.trans->d_T, pj.S, pj.SB, pj.S_pad, nullptr, (float *)lcoef, launches, ls));
            TcArgs ta;
            memset(&ta, 0, sizeof(ta));
            ta.ps = &ps;
            ta.coef32 = (const float *)lcoef;
            ta.SB = pj.SB;
            ta.pair_geom = lgeom;
            ta.qx = pj.job.grid->d_qx;
            ta.qy = pj.job.grid->d_qy;
            ta.qz = pj.job.grid->d_qz;
            ta.nx = pj.job.grid->nx;
            ta.ny = pj.job.grid->ny;
            ta.nz = pj.job.grid->nz;
            ta.S = pj.S;
            ta.scale = pj.job.scale;
            ta.f = (float *)pj.job.f_out;
            ta.f2 = (float *)pj.job.f2_out;
            ta.kind = P->tc_kind;
            ta.half = pj.half;
            ta.pair = P->pair;
            ta.oct = P->oct && pj.half;
            tc_axes_abs_max(pj.job.grid->hx.data(), ta.nx, pj.job.grid->hy.data(), ta.ny, pj.job.grid->hz.data(), ta.nz,
                            ta.qabs);
            CUDA_TRY(tc_prep_job(ta, base + P->off_group + pj.region, nullptr, launches, ls));
        }
        for (int l = 0; l < scff_plan_s::kLanes; ++l) {
            CUDA_TRY(cudaEventRecord(P->join_ev[l], P->lane[l]));
            CUDA_TRY(cudaStreamWaitEvent(st, P->join_ev[l], 0));
        }
        const int drain = c->drain_every >= 0 ? c->drain_every : 8;
        CUDA_TRY(tc_launch_persistent(P->tc_kind, P->group_zs[g],
                                      reinterpret_cast<const TcJobDev *>(base + P->group_desc[g]),
                                      reinterpret_cast<const int4 *>(base + P->group_items[g]), P->group_nitems[g],
                                      drain, c->d_err, tc_num_sms(), launches, st, nullptr,
                                      reinterpret_cast<int *>(base + P->off_queue)));
    }
    for (const PlanJob &pj : P->jobs) {
        if (pj.tc) continue;
        const PairSetDev &ps = pj.job.basis->dev;
        const scff_qgrid_s *gq = pj.job.grid;
        CUDA_TRY(launch_pair_geom(ps, geom, st));
        ++*launches;
        CUDA_TRY(launch_pairprep(ps, pj.job.trans->d_T, pj.S, pj.SB, pj.S_pad, fp64 ? (double *)coef : nullptr,
                                 fp64 ? nullptr : (float *)coef, launches, st));
        DirectArgs a;
        memset(&a, 0, sizeof(a));
        a.ps = &ps;
        a.coef = coef;
        a.nq = pj.half ? (gq->n + 1) / 2 : gq->n;
        a.nq_out = gq->n;
        a.S = pj.S;
        a.SB = pj.SB;
        a.scale = pj.job.scale;
        a.f = pj.job.f_out;
        a.f2 = pj.job.f2_out;
        a.err_flag = c->d_err;
        if (gq->product) {
            void *t0 = base + P->off_tab, *t1 = base + P->off_tab + P->tab_stride,
                 *t2 = base + P->off_tab + 2 * P->tab_stride;
            CUDA_TRY(launch_axis_tables(ps, geom, gq->d_qx, gq->nx, 0, t0, fp64, st));
            CUDA_TRY(launch_axis_tables(ps, geom, gq->d_qy, gq->ny, 1, t1, fp64, st));
            CUDA_TRY(launch_axis_tables(ps, geom, gq->d_qz, gq->nz, 2, t2, fp64, st));
            *launches += 3;
            a.gx = t0;
            a.gy = t1;
            a.gz = t2;
            a.qax = gq->d_qx;
            a.qay = gq->d_qy;
            a.qaz = gq->d_qz;
            a.nx = gq->nx;
            a.ny = gq->ny;
            a.nz = gq->nz;
        } else {
            a.qlist = gq->d_q;
            a.pair_geom = geom;
        }
        CUDA_TRY(launch_direct(a, fp64 ? 1 : 0, gq->product ? 0 : 1, launches, st));
    }
    return SCFF_OK;
}

static bool plan_known(scff_ctx *c, scff_plan_h p) {
    return c && p && std::find(c->plans.begin(), c->plans.end(), p) != c->plans.end();
}

extern "C" scff_status scff_plan_run(scff_ctx *c, scff_plan_h p, void *stream) {
    if (!plan_known(c, p)) return fail(SCFF_ERR_NOT_FOUND, "scff_plan_run: unknown plan");
    cudaSetDevice(c->device);
    int64_t n = 0;
    scff_status s = plan_launch(p, (cudaStream_t)stream, &n);
    c->launches += n;
    p->launches_per_run = n;
    return s;
}

extern "C" scff_status scff_plan_run_graph(scff_ctx *c, scff_plan_h p, void *stream) {
    if (!plan_known(c, p)) return fail(SCFF_ERR_NOT_FOUND, "scff_plan_run_graph: unknown plan");
    if (!stream) return fail(SCFF_ERR_INVALID_ARG, "scff_plan_run_graph: capture needs a non-default stream");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!p->exec) {
        CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int64_t n = 0;
        scff_status s = plan_launch(p, st, &n);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (s != SCFF_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(SCFF_ERR_CUDA, "scff_plan_run_graph: capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&p->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            p->exec = nullptr;
            return fail(SCFF_ERR_CUDA, "scff_plan_run_graph: instantiate failed: %s", cudaGetErrorString(e));
        }
        p->graph = g;
        p->launches_per_run = n;
    }
    CUDA_TRY(cudaGraphLaunch(p->exec, st));
    c->launches += p->launches_per_run;
    return SCFF_OK;
}

extern "C" scff_status scff_plan_info(scff_ctx *c, scff_plan_h p, int64_t *info) {
    if (!plan_known(c, p) || !info) return fail(SCFF_ERR_NOT_FOUND, "scff_plan_info: unknown plan");
    int64_t items = 0, tcj = 0;
    for (int n : p->group_nitems) items += n;
    for (const PlanJob &pj : p->jobs) tcj += pj.tc;
    info[0] = (int64_t)p->jobs.size();
    info[1] = tcj;
    info[2] = (int64_t)p->groups.size();
    info[3] = items;
    info[4] = (int64_t)p->dev_bytes;
    info[5] = p->launches_per_run;
    return SCFF_OK;
}

static void free_plan(scff_plan_s *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (int l = 0; l < scff_plan_s::kLanes; ++l) {
        if (p->lane[l]) cudaStreamDestroy(p->lane[l]);
        if (p->join_ev[l]) cudaEventDestroy(p->join_ev[l]);
    }
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    cudaFree(p->dev);
    delete p;
}
static void free_plan_any(struct scff_plan_s *p) { free_plan(p); }

extern "C" void scff_release_plan(scff_ctx *c, scff_plan_h p) {
    if (!plan_known(c, p)) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->plans.erase(std::find(c->plans.begin(), c->plans.end(), p));
    free_plan(p);
}
