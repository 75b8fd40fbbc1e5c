// Host side of the spherical method (scff_spherical): the molecule-independent
// coefficient tables (Theta of Appendix B, Gaunt coefficients of Eq. YYY) and
// the orchestration of the kernels in kernels_sph.cu and kernels_tc.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "scff_internal.h"
#include "scff_objects.h"
#include "sph_common.h"
#include "sph_internal.h"
#include "tc_internal.h"

using namespace scff;

namespace scff {
scff_status set_last_error(scff_status code, const char *msg);
}

namespace {

scff_status sfail(scff_status code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return scff::set_last_error(code, buf);
}

#define SCUDA(call)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return sfail(SCFF_ERR_CUDA, "scff_spherical: %s", cudaGetErrorString(e_)); \
    } while (0)

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on P_n).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

constexpr int kThetaMono = mono_count(kMaxPairL);  // 84 monomials of degree <= 6
constexpr int kThetaLam = (kMaxPairL + 1) * (kMaxPairL + 1);  // 49 (lambda, mu)

// Theta^{uvw}_{lambda mu} = Int x^u y^v z^w conj(Y_lambda^mu) dOmega over the
// unit sphere (Appendix B defines Theta by q_x^u q_y^v q_z^w = q^n sum Theta
// Y_lambda^mu; since the Y are orthonormal this projection is that
// coefficient).  The integrand is a polynomial of degree <= 12 on the sphere,
// so 8 Gauss-Legendre nodes in cos(theta) and 16 equally spaced phi integrate
// it exactly.  Entries outside the selection rules (lambda > n, lambda and n
// of different parity) are set to zero exactly.
std::vector<double> theta_table() {
    std::vector<double> gx, gw;
    gauss_legendre(8, gx, gw);
    const int nphi = 16;
    std::vector<double> out(2 * (size_t)kThetaMono * kThetaLam, 0.0);
    double p[(kMaxPairL + 1) * (kMaxPairL + 2) / 2];
    for (int mi = 0; mi < kThetaMono; ++mi) {
        const int u = mono_u(mi), v = mono_v(mi), w = mono_w(mi), n = u + v + w;
        for (int lam = 0; lam <= kMaxPairL; ++lam) {
            if (lam > n || ((n - lam) & 1)) continue;
            for (int mu = -lam; mu <= lam; ++mu) {
                double re = 0.0, im = 0.0;
                for (int a = 0; a < 8; ++a) {
                    const double ct = gx[a], st = sqrt(1.0 - ct * ct);
                    sph::plm_all(lam, ct, p);
                    const double pl = sph::plm_signed(p, lam, mu);
                    for (int b = 0; b < nphi; ++b) {
                        const double ph = 2.0 * M_PI * b / nphi;
                        const double mono = pow(st * cos(ph), u) * pow(st * sin(ph), v) * pow(ct, w);
                        const double wt = gw[a] * (2.0 * M_PI / nphi) * mono * pl;
                        re += wt * cos(mu * ph);
                        im -= wt * sin(mu * ph);
                    }
                }
                const size_t o = 2 * ((size_t)mi * kThetaLam + sph::lm_index(lam, mu));
                out[o] = re;
                out[o + 1] = im;
            }
        }
    }
    return out;
}

}  // namespace

// Molecule-independent tables of the spherical method, cached per context.
struct SphCache {
    bool plm_ready = false;    // device table of Legendre recurrence coefficients filled
    double2 *theta = nullptr;  // [84][49]
    int lmax = -1, lam = -1;   // Gaunt table key
    int *goff = nullptr;       // [NR + 1]
    int2 *gidx = nullptr;      // (lambda mu index, L M index) per entry
    double *gval = nullptr;
    int nent = 0;
};

void scff_sph_cache_free(SphCache *c) {
    if (!c) return;
    cudaFree(c->theta);
    cudaFree(c->goff);
    cudaFree(c->gidx);
    cudaFree(c->gval);
    delete c;
}

namespace {

// Gaunt coefficients G(lambda mu, L M -> l m) = Int Y_lambda^mu Y_L^M conj(Y_l^m)
// = 2 pi delta_{m, mu+M} Int p_lambda^mu p_L^M p_l^m dx for l <= lmax,
// lambda <= lam, |l - lambda| <= L <= l + lambda with lambda + L + l even.  The
// integrand is a polynomial of degree lambda + L + l <= 92, so 64
// Gauss-Legendre nodes integrate it exactly.  Entries are grouped by output
// (l, m) in CSR form; an entry holds (index of (lambda, mu) among the
// harmonics of lambda's parity | parity << 16, index of (L, M)).
scff_status build_gaunt(SphCache *cache, int lmax, int lam) {
    const int Lmax = lmax + lam;
    std::vector<double> gx, gw;
    gauss_legendre(64, gx, gw);
    const int ntri = (Lmax + 1) * (Lmax + 2) / 2;
    std::vector<double> P((size_t)64 * ntri);
    for (int a = 0; a < 64; ++a) sph::plm_all(Lmax, gx[a], &P[(size_t)a * ntri]);
    const int NR = (lmax + 1) * (lmax + 1);
    std::vector<int> off(NR + 1, 0);
    std::vector<int2> idx;
    std::vector<double> val;
    for (int l = 0; l <= lmax; ++l)
        for (int m = -l; m <= l; ++m) {
            for (int la = 0; la <= lam; ++la)
                for (int mu = -la; mu <= la; ++mu) {
                    const int M = m - mu;
                    for (int L = std::abs(l - la); L <= l + la; L += 2) {
                        if (std::abs(M) > L) continue;
                        double g = 0.0;
                        for (int a = 0; a < 64; ++a) {
                            const double *p = &P[(size_t)a * ntri];
                            g += gw[a] * sph::plm_signed(p, la, mu) * sph::plm_signed(p, L, M) *
                                 sph::plm_signed(p, l, m);
                        }
                        g *= 2.0 * M_PI;
                        if (fabs(g) < 1e-15) continue;
                        idx.push_back(make_int2(sph_parity_sub(la, mu) | ((la & 1) << 16), sph::lm_index(L, M)));
                        val.push_back(g);
                    }
                }
            off[sph::lm_index(l, m) + 1] = (int)idx.size();
        }
    cudaFree(cache->goff);
    cudaFree(cache->gidx);
    cudaFree(cache->gval);
    cache->goff = nullptr;
    cache->gidx = nullptr;
    cache->gval = nullptr;
    if (cudaMalloc(&cache->goff, sizeof(int) * off.size()) != cudaSuccess ||
        cudaMalloc(&cache->gidx, sizeof(int2) * std::max<size_t>(1, idx.size())) != cudaSuccess ||
        cudaMalloc(&cache->gval, sizeof(double) * std::max<size_t>(1, val.size())) != cudaSuccess)
        return sfail(SCFF_ERR_OOM, "scff_spherical: cannot allocate the Gaunt table");
    if (cudaMemcpy(cache->goff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!idx.empty() &&
         cudaMemcpy(cache->gidx, idx.data(), sizeof(int2) * idx.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!val.empty() &&
         cudaMemcpy(cache->gval, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        return sfail(SCFF_ERR_CUDA, "scff_spherical: cannot upload the Gaunt table");
    cache->lmax = lmax;
    cache->lam = lam;
    cache->nent = (int)idx.size();
    return SCFF_OK;
}

scff_status get_cache(scff_ctx *c, int lmax, int lam, SphCache **out) {
    if (!c->sph) c->sph = new SphCache();
    SphCache *k = c->sph;
    if (!k->plm_ready) {
        if (launch_sph_plm_init(0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
            return sfail(SCFF_ERR_CUDA, "scff_spherical: cannot fill the Legendre coefficient table");
        k->plm_ready = true;
    }
    if (!k->theta) {
        const std::vector<double> t = theta_table();
        if (cudaMalloc(&k->theta, sizeof(double) * t.size()) != cudaSuccess)
            return sfail(SCFF_ERR_OOM, "scff_spherical: cannot allocate the Theta table");
        if (cudaMemcpy(k->theta, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return sfail(SCFF_ERR_CUDA, "scff_spherical: cannot upload the Theta table");
    }
    if (k->lmax != lmax || k->lam != lam) {
        scff_status s = build_gaunt(k, lmax, lam);
        if (s != SCFF_OK) return s;
    }
    *out = k;
    return SCFF_OK;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" scff_status scff_spherical(scff_ctx *c, scff_basis_h b, scff_trans_h t, const scff_sph_grid *grid,
                                      int precision, double scale, void *R_out, void *f_out, void *f2_out,
                                      void *iso_out, int out_on_device, void *stream) {
    if (!c || !grid) return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: NULL context or grid");
    if (!b || std::find(c->bases.begin(), c->bases.end(), b) == c->bases.end())
        return sfail(SCFF_ERR_NOT_FOUND, "scff_spherical: unknown basis handle");
    if (!t || std::find(c->transs.begin(), c->transs.end(), t) == c->transs.end() || t->basis != b)
        return sfail(SCFF_ERR_NOT_FOUND, "scff_spherical: unknown transitions handle");
    const bool fp64 = precision == SCFF_FP64;
    const bool tc = precision == SCFF_BF16X3 || precision == SCFF_TF32X3 || precision == SCFF_BF16X2;
    if (!fp64 && !tc)
        return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: precision %d (FP64, BF16X3, TF32X3 or BF16X2)", precision);
    const int lmax = grid->lmax, nq = grid->n_q, nt = grid->n_theta, np = grid->n_phi;
    if (lmax < 0 || lmax > sph::kMaxLmax)
        return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: lmax %d outside 0..%d", lmax, sph::kMaxLmax);
    if (nq < 0 || (nq > 0 && !grid->q) || nt < 0 || np < 0 || (nt > 0) != (np > 0) || (nt > 0 && (!grid->theta || !grid->phi)))
        return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: bad radial or angular grid");
    for (int i = 0; i < nq; ++i)
        if (!(grid->q[i] >= 0.0) || !isfinite(grid->q[i]))
            return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: radial q[%d] = %g", i, grid->q[i]);
    for (int i = 0; i < nt; ++i)
        if (!isfinite(grid->theta[i])) return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: theta[%d]", i);
    for (int i = 0; i < np; ++i)
        if (!isfinite(grid->phi[i])) return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: phi[%d]", i);
    if ((f_out || f2_out) && nt == 0)
        return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: f requested without an angular grid");
    if (!isfinite(scale)) return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: scale is not finite");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const PairSetDev &ps = b->dev;
    const int S = t->S;
    if (nq == 0) return SCFF_OK;
    // highest pair degree present
    int lam = 0;
    for (int L = 0; L < kNumClasses; ++L)
        if (ps.pair_off[L + 1] > ps.pair_off[L]) lam = L;
    const int Lmax = lmax + lam, NL = Lmax + 1, NLM = NL * NL;
    const int NR = (lmax + 1) * (lmax + 1);
    const int64_t K = ps.n_axrows;
    const int kind = precision == SCFF_BF16X2 ? 0 : precision == SCFF_BF16X3 ? 1 : 2;
    // the even and odd parity jobs: rows (s, lambda mu of that parity), k = (pair, n of that parity)
    SphParity kp[2];
    int nsub[2];
    int64_t Kj[2], Kj_pad[2];
    for (int par = 0; par < 2; ++par) {
        kp[par].par = par;
        kp[par].off[0] = 0;
        for (int L = 0; L < kNumClasses; ++L)
            kp[par].off[L + 1] = kp[par].off[L] + (int64_t)(ps.pair_off[L + 1] - ps.pair_off[L]) * sph_parity_count(L, par);
        Kj[par] = kp[par].off[kNumClasses];
        Kj_pad[par] = tc ? tc_generic_kpad(kind, Kj[par]) : std::max<int64_t>(Kj[par], 1);
        nsub[par] = sph_parity_rows(lam, par);
    }
    if ((K + 1) * nq * (int64_t)NL >= INT32_MAX || (int64_t)(ps.n_pair + 1) * NLM >= INT32_MAX)
        return sfail(SCFF_ERR_INVALID_ARG, "scff_spherical: tables exceed 2^31 entries (split the radial grid)");
    SphCache *cache = nullptr;
    {
        scff_status s = get_cache(c, lmax, lam, &cache);
        if (s != SCFF_OK) return s;
    }
    // ---- workspace plan
    const size_t el = fp64 ? sizeof(double2) : sizeof(float2);
    const int SB = 4, S_pad = (S + SB - 1) / SB * SB;
    const int M2 = S * nq;
    const int64_t NZ = (int64_t)nq * NLM;
    const int64_t K2 = NR, K2_pad = tc ? tc_generic_kpad(kind, K2) : K2;
    size_t o = 0;
    const size_t o_coef = o;   o = up256(o + sizeof(double) * (size_t)S_pad * ps.n_rows);
    const size_t o_geom = o;   o = up256(o + sizeof(double) * 4 * (size_t)ps.n_pair);
    const size_t o_q = o;      o = up256(o + sizeof(double) * (size_t)(nq + nt + np));
    const size_t o_rho = o;    o = up256(o + el * (size_t)(K + 1) * nq * NL);
    const size_t o_y = o;      o = up256(o + el * (size_t)(ps.n_pair + 1) * NLM);
    size_t o_kofs[2], o_A[2], o_Z[2];
    for (int par = 0; par < 2; ++par) {
        o_kofs[par] = o;
        o = up256(o + sizeof(int2) * (size_t)Kj_pad[par]);
        o_A[par] = o;
        o = up256(o + sizeof(double2) * (size_t)S * nsub[par] * Kj_pad[par]);
        o_Z[par] = o;
        o = up256(o + el * (size_t)S * nsub[par] * NZ);
    }
    const size_t o_R = o;      o = up256(o + sizeof(double2) * (size_t)M2 * NR);
    const size_t o_T1 = o;     o = up256(o + el * (size_t)(NR + 1) * std::max(nt, 1));
    const size_t o_T2 = o;     o = up256(o + el * (size_t)(2 * lmax + 2) * std::max(np, 1));
    const size_t o_k2 = o;     o = up256(o + sizeof(int2) * (size_t)K2_pad);
    const size_t tcw = tc ? std::max(tc_generic_bytes(kind, S * nsub[0], Kj[0]) + tc_generic_bytes(kind, S * nsub[1], Kj[1]),
                                     tc_generic_bytes(kind, M2, K2)) +
                                sizeof(int4) * (size_t)((S * nsub[0] + 127) / 128 + (S * nsub[1] + 127) / 128 +
                                                        (M2 + 127) / 128) *
                                    (size_t)((std::max<int64_t>(NZ, (int64_t)nt * np) + 127) / 128) + 4096
                          : 0;
    const size_t o_tc = o;     o = up256(o + tcw);
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const size_t bytes_R = (size_t)M2 * NR * 2 * rsz, bytes_iso = (size_t)M2 * rsz;
    const size_t bytes_f = (size_t)M2 * nt * np * 2 * rsz, bytes_f2 = (size_t)M2 * nt * np * rsz;
    const size_t o_out = o;
    if (!out_on_device) o = up256(o + up256(bytes_R) + up256(bytes_iso) + up256(bytes_f) + up256(bytes_f2));
    // |f|^2 alone still needs f as the contraction's output
    const size_t o_ftmp = o;
    if (f2_out && !f_out) o = up256(o + bytes_f);
    const size_t total = o + 1024;
    if (total > c->budget)
        return sfail(SCFF_ERR_ADMISSION, "scff_spherical: footprint %zu bytes exceeds the budget %llu", total,
                     (unsigned long long)c->budget);
    if (c->sph_ws.cap < total) {
        cudaFree(c->sph_ws.p);
        c->sph_ws.p = nullptr;
        c->sph_ws.cap = 0;
        if (cudaMalloc(&c->sph_ws.p, total) != cudaSuccess)
            return sfail(SCFF_ERR_OOM, "scff_spherical: cannot allocate %zu bytes of workspace", total);
        c->sph_ws.cap = total;
    }
    uint8_t *w = static_cast<uint8_t *>(c->sph_ws.p);
    double *coef = reinterpret_cast<double *>(w + o_coef);
    double *geom = reinterpret_cast<double *>(w + o_geom);
    double *dq = reinterpret_cast<double *>(w + o_q), *dth = dq + nq, *dph = dth + nt;
    void *rho = w + o_rho, *ytab = w + o_y, *T1 = w + o_T1, *T2 = w + o_T2;
    int2 *kofs2 = reinterpret_cast<int2 *>(w + o_k2);
    double2 *R64 = reinterpret_cast<double2 *>(w + o_R);
    uint8_t *outs = w + o_out;
    void *dR = out_on_device ? R_out : (R_out ? (void *)outs : nullptr);
    void *diso = out_on_device ? iso_out : (iso_out ? (void *)(outs + up256(bytes_R)) : nullptr);
    void *df = out_on_device ? f_out : (f_out ? (void *)(outs + up256(bytes_R) + up256(bytes_iso)) : nullptr);
    void *df2 = out_on_device ? f2_out
                              : (f2_out ? (void *)(outs + up256(bytes_R) + up256(bytes_iso) + up256(bytes_f)) : nullptr);

    SCUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    SCUDA(cudaMemcpyAsync(dq, grid->q, sizeof(double) * nq, cudaMemcpyHostToDevice, st));
    if (nt > 0) {
        SCUDA(cudaMemcpyAsync(dth, grid->theta, sizeof(double) * nt, cudaMemcpyHostToDevice, st));
        SCUDA(cudaMemcpyAsync(dph, grid->phi, sizeof(double) * np, cudaMemcpyHostToDevice, st));
    }
    // ---- pair-prep (FP64 coefficients) and pair geometry
    SCUDA(launch_pair_geom(ps, geom, st));
    ++c->launches;
    SCUDA(launch_pairprep(ps, t->d_T, S, SB, S_pad, coef, nullptr, &c->launches, st));
    // ---- tables: rho (+ zero row), y (+ zero row), k offsets, W tensor
    SCUDA(cudaMemsetAsync(static_cast<uint8_t *>(rho) + el * (size_t)K * nq * NL, 0, el * (size_t)nq * NL, st));
    SCUDA(cudaMemsetAsync(static_cast<uint8_t *>(ytab) + el * (size_t)ps.n_pair * NLM, 0, el * (size_t)NLM, st));
    SCUDA(launch_sph_radial(ps, geom, dq, nq, NL, fp64 ? 1 : 0, rho, st));
    SCUDA(launch_sph_ypair(ps, geom, Lmax, fp64 ? 1 : 0, ytab, st));
    c->launches += 2;
    for (int par = 0; par < 2; ++par) {
        if (nsub[par] == 0) continue;
        SCUDA(launch_sph_kofs(ps, kp[par], Kj_pad[par], nq, NL, NLM, reinterpret_cast<int2 *>(w + o_kofs[par]), st));
        SCUDA(launch_sph_wdense(ps, coef, SB, S, kp[par], nsub[par], cache->theta, Kj_pad[par],
                                reinterpret_cast<double2 *>(w + o_A[par]), st));
        c->launches += 2;
    }
    // ---- Z = W (rho y): the dense contraction over (pair, n), one job per parity
    if (fp64) {
        for (int par = 0; par < 2; ++par) {
            if (nsub[par] == 0) continue;
            Gemm64Args g;
            memset(&g, 0, sizeof(g));
            g.A = reinterpret_cast<const double2 *>(w + o_A[par]);
            g.lda = Kj_pad[par];
            g.K = Kj[par];
            g.M = S * nsub[par];
            g.nx = nsub[par];
            g.Y = static_cast<const double2 *>(rho);
            g.Z = static_cast<const double2 *>(ytab);
            g.kofs = reinterpret_cast<const int2 *>(w + o_kofs[par]);
            g.nz = NLM;
            g.ylm = 1;
            g.ystride = NL;
            g.N = NZ;
            g.scale = 1.0;
            g.C = reinterpret_cast<double2 *>(w + o_Z[par]);
            SCUDA(launch_gen_gemm64(g, st));
            ++c->launches;
        }
    } else {
        TcGenericArgs g[2];
        int nj = 0;
        for (int par = 0; par < 2; ++par) {
            if (nsub[par] == 0) continue;
            TcGenericArgs &a = g[nj++];
            memset(&a, 0, sizeof(a));
            a.kind = kind;
            a.A = reinterpret_cast<const double2 *>(w + o_A[par]);
            a.lda = Kj_pad[par];
            a.K = Kj[par];
            a.M = S * nsub[par];
            a.nx = nsub[par];
            a.Y = static_cast<const float2 *>(rho);
            a.Z = static_cast<const float2 *>(ytab);
            a.kofs = reinterpret_cast<const int2 *>(w + o_kofs[par]);
            a.nz = NLM;
            a.ylm = 1;
            a.ystride = NL;
            a.N = NZ;
            a.scale = 1.0f;
            a.C = reinterpret_cast<float2 *>(w + o_Z[par]);
            a.drain_every = c->drain_every >= 0 ? c->drain_every : 8;
            a.err = c->d_err;
            a.ws = w + o_tc;
            a.ws_bytes = tcw;
        }
        SCUDA(tc_run_generic_multi(g, nj, &c->launches, st));
    }
    // ---- R = Gaunt-coupled Z (scaled), then the outputs that follow from it
    SCUDA(launch_sph_gaunt(w + o_Z[0], w + o_Z[1], nsub[0], nsub[1], fp64 ? 1 : 0, S, nq, NLM, NR, cache->goff,
                           cache->gidx, cache->gval, scale, R64, st));
    ++c->launches;
    if (dR) {
        if (fp64)
            SCUDA(cudaMemcpyAsync(dR, R64, sizeof(double2) * (size_t)M2 * NR, cudaMemcpyDeviceToDevice, st));
        else {
            SCUDA(launch_sph_r_to_f32(R64, (int64_t)M2 * NR, static_cast<float2 *>(dR), st));
            ++c->launches;
        }
    }
    if (diso) {
        SCUDA(launch_sph_iso(R64, M2, NR, fp64 ? 1 : 0, diso, st));
        ++c->launches;
    }
    if (df || df2) {
        SCUDA(cudaMemsetAsync(static_cast<uint8_t *>(T1) + el * (size_t)NR * nt, 0, el * (size_t)nt, st));
        SCUDA(cudaMemsetAsync(static_cast<uint8_t *>(T2) + el * (size_t)(2 * lmax + 1) * np, 0, el * (size_t)np, st));
        SCUDA(launch_sph_angular_tables(dth, nt, dph, np, lmax, fp64 ? 1 : 0, T1, T2, st));
        SCUDA(launch_sph_angular_kofs(NR, K2_pad, lmax, nt, np, kofs2, st));
        c->launches += 3;
        void *fdst = df ? df : (void *)(w + o_ftmp);
        if (fp64) {
            Gemm64Args g;
            memset(&g, 0, sizeof(g));
            g.A = R64;
            g.lda = NR;
            g.K = K2;
            g.M = M2;
            g.nx = nq;
            g.Y = static_cast<const double2 *>(T1);
            g.Z = static_cast<const double2 *>(T2);
            g.kofs = kofs2;
            g.nz = np;
            g.ylm = 0;
            g.ystride = 1;
            g.N = (int64_t)nt * np;
            g.scale = 1.0;
            g.C = static_cast<double2 *>(fdst);
            g.C2 = static_cast<double *>(df2);
            SCUDA(launch_gen_gemm64(g, st));
            ++c->launches;
        } else {
            TcGenericArgs g;
            memset(&g, 0, sizeof(g));
            g.kind = kind;
            g.A = R64;
            g.lda = NR;
            g.K = K2;
            g.M = M2;
            g.nx = nq;
            g.Y = static_cast<const float2 *>(T1);
            g.Z = static_cast<const float2 *>(T2);
            g.kofs = kofs2;
            g.nz = np;
            g.ylm = 0;
            g.ystride = 1;
            g.N = (int64_t)nt * np;
            g.scale = 1.0f;
            g.C = static_cast<float2 *>(fdst);
            g.C2 = static_cast<float *>(df2);
            g.drain_every = c->drain_every >= 0 ? c->drain_every : 8;
            g.err = c->d_err;
            g.ws = w + o_tc;
            g.ws_bytes = tcw;
            SCUDA(tc_run_generic(g, &c->launches, st));
        }
    }
    if (!out_on_device) {
        if (R_out) SCUDA(cudaMemcpyAsync(R_out, dR, bytes_R, cudaMemcpyDeviceToHost, st));
        if (iso_out) SCUDA(cudaMemcpyAsync(iso_out, diso, bytes_iso, cudaMemcpyDeviceToHost, st));
        if (f_out) SCUDA(cudaMemcpyAsync(f_out, df, bytes_f, cudaMemcpyDeviceToHost, st));
        if (f2_out) SCUDA(cudaMemcpyAsync(f2_out, df2, bytes_f2, cudaMemcpyDeviceToHost, st));
    }
    SCUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCUDA(cudaStreamSynchronize(st));
    if (*c->h_err) return sfail(SCFF_ERR_TIMEOUT, "scff_spherical: a device-side wait timed out (code %d)", *c->h_err);
    return SCFF_OK;
}
