// scff_form_factor_static: the FP64 form factor on an explicit q list without
// any device allocation.
//
// Who needs this: programs that cannot or must not call cudaMalloc while they
// run -- a host framework whose caching allocator already owns nearly all of
// the device memory (a fresh cudaMalloc would fail or fragment its pool), a
// latency-bound serving loop where cudaMalloc/cudaFree would synchronise the
// device mid-stream, or a plugin whose host application forbids it to manage
// device memory.  Such callers pass their own device buffers for T, q and the
// outputs; every intermediate array of the evaluation (primitive-shell
// records, pair list, pair geometry, folded coefficients and the status word)
// lives in one file-scope device array of fixed size, g_scratch, that is part
// of the library image and is held by every GPU that loads the library until
// the process exits.
//
// Host-side staging of the records and pairs uses static host storage, so the
// call makes no heap allocation either.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/scff.h"
#include "scff_internal.h"

namespace scff {

// set by the host runtime (scff_host.cpp); records the calling thread's error
scff_status set_last_error(scff_status code, const char *msg);

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxRecords = 256;                     // primitive-shell records
constexpr int kMaxPairs = kMaxRecords * (kMaxRecords + 1) / 2;
constexpr int kMaxDevices = 64;
constexpr int kSB = 4;                               // state block of the FP64 kernels

// The scratch array.  Host code must not take its address directly: in host
// code the name is a stand-in, not a device address; the device address comes
// from cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Byte layout of g_scratch (each piece 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffErr = 0;
constexpr size_t kOffXyz = 256;
constexpr size_t kOffAlpha = kOffXyz + align256(sizeof(double) * 3 * kMaxRecords);
constexpr size_t kOffType = kOffAlpha + align256(sizeof(double) * kMaxRecords);
constexpr size_t kOffFn0 = kOffType + align256(sizeof(int32_t) * kMaxRecords);
constexpr size_t kOffW = kOffFn0 + align256(sizeof(int32_t) * kMaxRecords);
constexpr size_t kOffPairs = kOffW + align256(sizeof(double) * kRecW * kMaxRecords);
constexpr size_t kOffGeom = kOffPairs + align256(sizeof(int2) * kMaxPairs);
constexpr size_t kOffCoef = kOffGeom + align256(sizeof(double) * 4 * kMaxPairs);
static_assert(kOffCoef < kScratchBytes, "scratch layout");
constexpr size_t kCoefBytes = kScratchBytes - kOffCoef;

// Host staging in static storage (one call at a time, under g_mu).
struct HostStage {
    double xyz[3 * kMaxRecords];
    double alpha[kMaxRecords];
    int32_t type[kMaxRecords];
    int32_t fn0[kMaxRecords];
    double w[kRecW * kMaxRecords];
    int2 pairs[kMaxPairs];
    int err;
};
static HostStage g_host;
static std::mutex g_mu;

scff_status err(scff_status code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

// Device address of g_scratch in the current device's current context.  It
// is looked up on every call (the lookup allocates nothing), so an address
// never outlives the context it belongs to: after cudaDeviceReset the next
// call resolves the array of the new context instead of using a stale one.
scff_status scratch_address(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(SCFF_ERR_CUDA, "scff_form_factor_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: device %d", dev);
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return err(SCFF_ERR_CUDA, "scff_form_factor_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    *out = static_cast<unsigned char *>(p);
    return SCFF_OK;
}

double dfact_odd(int n) {
    double r = 1.0;
    for (int k = 2 * n - 1; k > 1; k -= 2) r *= k;
    return r;
}

void powers(int type, int j, int pw[3]) {
    for (int ax = 0; ax < 3; ++ax)
        pw[ax] = type == REC_SP ? (j == 0 ? 0 : cart_pow(1, j - 1, ax)) : cart_pow(rec_lmax(type), j, ax);
}

// Unit-norm factor of x^a y^b z^c exp(-alpha r^2).
double prim_norm(double alpha, const int pw[3]) {
    const int L = pw[0] + pw[1] + pw[2];
    return sqrt(pow(2.0 * alpha / M_PI, 1.5) * pow(4.0 * alpha, L) /
                (dfact_odd(pw[0]) * dfact_odd(pw[1]) * dfact_odd(pw[2])));
}

double self_overlap(double p, const int pw[3]) {
    double v = pow(M_PI / p, 1.5);
    for (int i = 0; i < 3; ++i) v *= dfact_odd(pw[i]) / pow(2.0 * p, pw[i]);
    return v;
}

}  // namespace
}  // namespace scff

using namespace scff;

extern "C" scff_status scff_form_factor_static(int n_atoms, const double *xyz, int n_shells, const int32_t *shell_atom,
                                               const int32_t *shell_l, const int32_t *shell_nprim,
                                               const double *exponents, const double *coefficients, uint32_t flags,
                                               int n_states, const double *T_dev, int64_t n_q, const double *q_dev,
                                               double scale, double *f_dev, double *f2_dev, void *stream) {
    if (n_atoms <= 0 || n_shells <= 0 || !xyz || !shell_atom || !shell_l || !shell_nprim || !exponents ||
        !coefficients)
        return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: empty basis or NULL array");
    if (n_states <= 0 || !T_dev || n_q < 0 || (n_q > 0 && (!q_dev || !f_dev)) || !isfinite(scale))
        return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: bad states, T, q or output argument");
    std::lock_guard<std::mutex> lock(g_mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *scr = nullptr;
    scff_status rc = scratch_address(&scr);
    if (rc != SCFF_OK) return rc;

    // ---- basis ingest into static host storage: records, then pairs by class
    if (flags & ~SCFF_RENORM_CONTRACTED)
        return err(SCFF_ERR_INVALID_ARG,
                   "scff_form_factor_static: only SCFF_RENORM_CONTRACTED is accepted (pure shells need scff_basis)");
    const bool renorm = (flags & SCFF_RENORM_CONTRACTED) != 0;
    int nrec = 0, nbf = 0;
    size_t eo = 0, co = 0;
    for (int s = 0; s < n_shells; ++s) {
        const int l = shell_l[s], np = shell_nprim[s], at = shell_atom[s];
        if (l > 3) return err(SCFF_ERR_UNSUPPORTED_L, "scff_form_factor_static: shell %d has l=%d", s, l);
        if (l < -1 || np < 1 || np > 64 || at < 0 || at >= n_atoms)
            return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: shell %d is invalid", s);
        if (nrec + np > kMaxRecords)
            return err(SCFF_ERR_INVALID_ARG,
                       "scff_form_factor_static: more than %d primitive-shell records (the static scratch limit)",
                       kMaxRecords);
        const int type = (l == 0) ? REC_S : (l == 1) ? REC_P : (l == 2) ? REC_D : (l == 3) ? REC_F : REC_SP;
        const int nf = rec_nfn(type);
        for (int k = 0; k < np; ++k)
            if (!(exponents[eo + k] > 0.0) || !isfinite(exponents[eo + k]))
                return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: shell %d exponent %d", s, k);
        for (int k = 0; k < np; ++k) {
            HostStage &h = g_host;
            const int r = nrec + k;
            for (int i = 0; i < 3; ++i) h.xyz[3 * r + i] = xyz[3 * at + i];
            h.alpha[r] = exponents[eo + k];
            h.type[r] = type;
            h.fn0[r] = nbf;
        }
        for (int j = 0; j < kRecW; ++j) {
            int pw[3];
            if (j < nf) powers(type, j, pw);
            const double *c = coefficients + co + ((type == REC_SP && j > 0) ? np : 0);
            double ov = 0.0;
            for (int k = 0; k < np; ++k) {
                const double wk = j < nf ? c[k] * prim_norm(exponents[eo + k], pw) : 0.0;
                if (!isfinite(wk)) return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: shell %d coefficient", s);
                g_host.w[kRecW * (nrec + k) + j] = wk;
            }
            if (j < nf && renorm) {
                for (int k = 0; k < np; ++k)
                    for (int kk = 0; kk < np; ++kk)
                        ov += g_host.w[kRecW * (nrec + k) + j] * g_host.w[kRecW * (nrec + kk) + j] *
                              self_overlap(exponents[eo + k] + exponents[eo + kk], pw);
                if (!(ov > 0.0)) return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: shell %d has zero norm", s);
                const double r = 1.0 / sqrt(ov);
                for (int k = 0; k < np; ++k) g_host.w[kRecW * (nrec + k) + j] *= r;
            }
        }
        nrec += np;
        nbf += nf;
        eo += np;
        co += (size_t)np * (type == REC_SP ? 2 : 1);
    }
    for (int i = 0; i < 3 * n_atoms; ++i)
        if (!isfinite(xyz[i])) return err(SCFF_ERR_INVALID_ARG, "scff_form_factor_static: non-finite coordinate");

    PairSetDev ps;
    ps.n_rec = nrec;
    ps.nbf = nbf;
    int np_all = 0;
    ps.pair_off[0] = 0;
    ps.row_off[0] = ps.krow_off[0] = ps.axrow_off[0] = 0;
    for (int L = 0; L < kNumClasses; ++L) {
        int cnt = 0;
        for (int a = 0; a < nrec; ++a)
            for (int b = a; b < nrec; ++b)
                if (rec_lmax(g_host.type[a]) + rec_lmax(g_host.type[b]) == L) g_host.pairs[np_all + cnt++] = make_int2(a, b);
        np_all += cnt;
        ps.pair_off[L + 1] = np_all;
        ps.row_off[L + 1] = ps.row_off[L] + (int64_t)cnt * mono_count(L);
        ps.krow_off[L + 1] = ps.krow_off[L] + (int64_t)cnt * vw_count(L);
        ps.axrow_off[L + 1] = ps.axrow_off[L] + (int64_t)cnt * (L + 1);
    }
    ps.n_pair = np_all;
    ps.n_rows = ps.row_off[kNumClasses];
    ps.n_krows = ps.krow_off[kNumClasses];
    ps.n_axrows = ps.axrow_off[kNumClasses];
    const int S_pad = (n_states + kSB - 1) / kSB * kSB;
    const size_t coef_bytes = (size_t)S_pad * (size_t)ps.n_rows * sizeof(double);
    if (coef_bytes > kCoefBytes)
        return err(SCFF_ERR_INVALID_ARG,
                   "scff_form_factor_static: %d states x %lld coefficient rows need %zu bytes, above the %zu-byte "
                   "static scratch limit",
                   n_states, (long long)ps.n_rows, coef_bytes, kCoefBytes);

    ps.rec_xyz = reinterpret_cast<double *>(scr + kOffXyz);
    ps.rec_alpha = reinterpret_cast<double *>(scr + kOffAlpha);
    ps.rec_type = reinterpret_cast<int32_t *>(scr + kOffType);
    ps.rec_fn0 = reinterpret_cast<int32_t *>(scr + kOffFn0);
    ps.rec_w = reinterpret_cast<double *>(scr + kOffW);
    ps.pair_rec = reinterpret_cast<int2 *>(scr + kOffPairs);
    double *geom = reinterpret_cast<double *>(scr + kOffGeom);
    double *coef = reinterpret_cast<double *>(scr + kOffCoef);
    int *d_err = reinterpret_cast<int *>(scr + kOffErr);

#define STATIC_CUDA(call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return err(SCFF_ERR_CUDA, "scff_form_factor_static: %s: %s", #call,        \
                                          cudaGetErrorString(e_));                                         \
    } while (0)

    // ---- upload (pageable host source: each copy has consumed g_host when it returns)
    STATIC_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    STATIC_CUDA(cudaMemcpyAsync(ps.rec_xyz, g_host.xyz, sizeof(double) * 3 * nrec, cudaMemcpyHostToDevice, st));
    STATIC_CUDA(cudaMemcpyAsync(ps.rec_alpha, g_host.alpha, sizeof(double) * nrec, cudaMemcpyHostToDevice, st));
    STATIC_CUDA(cudaMemcpyAsync(ps.rec_type, g_host.type, sizeof(int32_t) * nrec, cudaMemcpyHostToDevice, st));
    STATIC_CUDA(cudaMemcpyAsync(ps.rec_fn0, g_host.fn0, sizeof(int32_t) * nrec, cudaMemcpyHostToDevice, st));
    STATIC_CUDA(cudaMemcpyAsync(ps.rec_w, g_host.w, sizeof(double) * kRecW * nrec, cudaMemcpyHostToDevice, st));
    STATIC_CUDA(cudaMemcpyAsync(ps.pair_rec, g_host.pairs, sizeof(int2) * ps.n_pair, cudaMemcpyHostToDevice, st));

    // ---- the same kernels as scff_form_factor (FP64, explicit q list)
    STATIC_CUDA(launch_pair_geom(ps, geom, st));
    STATIC_CUDA(launch_pairprep(ps, T_dev, n_states, kSB, S_pad, coef, nullptr, nullptr, st));
    DirectArgs a;
    memset(&a, 0, sizeof(a));
    a.ps = &ps;
    a.coef = coef;
    a.qlist = q_dev;
    a.pair_geom = geom;
    a.nq = n_q;
    a.S = n_states;
    a.SB = kSB;
    a.scale = scale;
    a.f = f_dev;
    a.f2 = f2_dev;
    a.err_flag = d_err;
    STATIC_CUDA(launch_direct(a, 1, 1, nullptr, st));

    // ---- status word back to the host (static storage), then wait
    STATIC_CUDA(cudaMemcpyAsync(&g_host.err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaStreamSynchronize(st));
#undef STATIC_CUDA
    if (g_host.err) return err(SCFF_ERR_TIMEOUT, "scff_form_factor_static: a device-side wait timed out");
    return SCFF_OK;
}
