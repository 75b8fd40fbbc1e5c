// Host side of the FFT method (scff_fft_form_factor): box and grid checks,
// workspace, and the launches of kernels_fft.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "fft_internal.h"
#include "scff_internal.h"
#include "scff_objects.h"

using namespace scff;

namespace scff {
scff_status set_last_error(scff_status code, const char *msg);
}

namespace {

scff_status ffail(scff_status code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return scff::set_last_error(code, buf);
}

#define FCUDA(call)                                                                                          \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return ffail(SCFF_ERR_CUDA, "scff_fft_form_factor: %s", cudaGetErrorString(e_)); \
    } while (0)

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

extern "C" scff_status scff_fft_form_factor(scff_ctx *c, scff_basis_h b, scff_trans_h t, const scff_fft_grid *grid,
                                            int precision, double scale, void *f_out, void *f2_out,
                                            double *parseval_out, int out_on_device, void *stream) {
    if (!c || !grid) return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: NULL context or grid");
    if (!b || std::find(c->bases.begin(), c->bases.end(), b) == c->bases.end())
        return ffail(SCFF_ERR_NOT_FOUND, "scff_fft_form_factor: unknown basis handle");
    if (!t || std::find(c->transs.begin(), c->transs.end(), t) == c->transs.end() || t->basis != b)
        return ffail(SCFF_ERR_NOT_FOUND, "scff_fft_form_factor: unknown transitions handle");
    if (precision != SCFF_FP64 && precision != SCFF_FP32)
        return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: precision %d (FP64 or FP32)", precision);
    for (int i = 0; i < 3; ++i) {
        const int n = grid->n[i];
        if (n < 4 || n > 1024 || (n & (n - 1)))
            return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: n[%d] = %d is not a power of two in 4..1024", i, n);
        if (!(grid->dq[i] > 0.0) || !isfinite(grid->dq[i]) || !isfinite(grid->centre[i]))
            return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: dq[%d] or centre[%d] invalid", i, i);
    }
    if (!(grid->threshold >= 0.0 && grid->threshold < 1.0))
        return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: threshold %g outside [0, 1)", grid->threshold);
    if (!isfinite(scale)) return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: scale is not finite");
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = precision == SCFF_FP64;
    const PairSetDev &ps = b->dev;
    const int S = t->S, nbf = ps.nbf, nbf_pad = (nbf + 31) / 32 * 32;
    const int nx = grid->n[0], ny = grid->n[1], nz = grid->n[2];
    const int64_t npts = (int64_t)nx * ny * nz;
    const int nfield = (S + 1) / 2;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    // states per register sweep (FP32 12, 8 or 4; FP64 8 or 4: as many as there are states)
    // and points per tile (the largest whose function values fit in shared memory)
    const int sbf = fp64 ? (S > 4 ? 8 : 4) : (S > 8 ? 12 : S > 4 ? 8 : 4);
    int tp = 0;
    for (int cand : {128, 64, 32}) {
        if (fp64 ? cand == 128 : cand == 64) continue;
        if (fft_density_smem(fp64 ? 1 : 0, nbf_pad, sbf, cand) <= 220 * 1024) {
            tp = cand;
            break;
        }
    }
    if (!tp)
        return ffail(SCFF_ERR_INVALID_ARG, "scff_fft_form_factor: %d functions exceed the tile's shared memory", nbf);
    // ---- workspace: packed fields, T in the arithmetic type, host staging, Parseval sums
    size_t o = 0;
    const size_t o_field = o;
    o = up256(o + 2 * rsz * (size_t)nfield * npts);
    const size_t o_T = o;
    o = up256(o + (fp64 ? 0 : sizeof(float) * (size_t)S * nbf * nbf));
    const size_t o_par = o;
    o = up256(o + sizeof(double) * 2 * (size_t)S);
    const int64_t kpad = fft_pair_kpad(nbf);
    const int nsweep = (S + sbf - 1) / sbf;
    const size_t o_tsym = o;
    o = up256(o + rsz * (size_t)nsweep * kpad * sbf);
    const size_t o_pairs = o;
    o = up256(o + sizeof(int2) * (size_t)kpad);
    const size_t bytes_f = 2 * rsz * (size_t)S * npts, bytes_f2 = rsz * (size_t)S * npts;
    const size_t o_phase = o;
    o = up256(o + sizeof(double2) * (size_t)(nx + ny + nz));
    const size_t o_recg = o;
    o = up256(o + (fp64 ? 0 : 2 * sizeof(float4) * (size_t)ps.n_rec));
    const size_t o_recw = o;
    o = up256(o + (fp64 ? 0 : sizeof(float) * kRecW * (size_t)ps.n_rec));
    const size_t o_out = o;
    if (!out_on_device) o = up256(o + up256(bytes_f) + up256(bytes_f2));
    const size_t total = o + 1024;
    if (total > c->budget)
        return ffail(SCFF_ERR_ADMISSION, "scff_fft_form_factor: footprint %zu bytes exceeds the budget %llu", total,
                     (unsigned long long)c->budget);
    if (c->fft_ws.cap < total) {
        cudaFree(c->fft_ws.p);
        c->fft_ws.p = nullptr;
        c->fft_ws.cap = 0;
        if (cudaMalloc(&c->fft_ws.p, total) != cudaSuccess)
            return ffail(SCFF_ERR_OOM, "scff_fft_form_factor: cannot allocate %zu bytes of workspace", total);
        c->fft_ws.cap = total;
    }
    uint8_t *w = static_cast<uint8_t *>(c->fft_ws.p);
    void *field = w + o_field;
    double *par = reinterpret_cast<double *>(w + o_par);
    void *df = out_on_device ? f_out : (f_out ? (void *)(w + o_out) : nullptr);
    void *df2 = out_on_device ? f2_out : (f2_out ? (void *)(w + o_out + up256(bytes_f)) : nullptr);
    FCUDA(cudaMemsetAsync(par, 0, sizeof(double) * 2 * S, st));
    const void *Tdev = t->d_T;
    if (!fp64) {
        FCUDA(launch_cast_f64_to_f32(t->d_T, (int64_t)S * nbf * nbf, reinterpret_cast<float *>(w + o_T), st));
        ++c->launches;
        Tdev = w + o_T;
    }
    // ---- box: side L = 2 pi / dq centred at centre, n points from the low corner
    double L[3], dx[3], xmin[3];
    for (int i = 0; i < 3; ++i) {
        L[i] = 2.0 * M_PI / grid->dq[i];
        dx[i] = L[i] / grid->n[i];
        xmin[i] = grid->centre[i] - 0.5 * L[i];
    }
    const double vpix = dx[0] * dx[1] * dx[2];
    FCUDA(launch_fft_tsym(Tdev, fp64 ? 1 : 0, nbf, S, sbf, w + o_tsym, reinterpret_cast<int2 *>(w + o_pairs), st));
    ++c->launches;
    FCUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int), st));
    // ---- 1. density tabulation and contraction
    FftDensityArgs da;
    memset(&da, 0, sizeof(da));
    da.ps = ps;
    da.nbf = nbf;
    da.nbf_pad = nbf_pad;
    da.S = S;
    da.T = Tdev;
    da.out = field;
    for (int i = 0; i < 3; ++i) {
        da.xmin[i] = xmin[i];
        da.dx[i] = dx[i];
    }
    da.nx = nx;
    da.ny = ny;
    da.nz = nz;
    da.npts = npts;
    da.cut = grid->threshold > 0.0 ? -log(grid->threshold) : 0.0;
    da.scale = scale;
    da.vpix = vpix;
    da.parseval = par;
    da.tsym = w + o_tsym;
    da.pairs = reinterpret_cast<const int2 *>(w + o_pairs);
    da.kpad = kpad;
    da.err = c->d_err;
    if (!fp64) {
        da.recg = reinterpret_cast<const float4 *>(w + o_recg);
        da.recw = reinterpret_cast<const float *>(w + o_recw);
        FCUDA(launch_fft_record_prep(da, reinterpret_cast<float4 *>(w + o_recg), reinterpret_cast<float *>(w + o_recw), st));
        ++c->launches;
    }
    FCUDA(launch_fft_density(da, fp64 ? 1 : 0, sbf, tp, st));
    ++c->launches;
    // ---- 2. three in-place passes, z, y, x
    const int64_t cap_elems = fp64 ? 4096 : 8192;  // complex elements of one CTA's line buffer
    for (int ax = 2; ax >= 0; --ax) {
        FftAxisArgs fa;
        memset(&fa, 0, sizeof(fa));
        fa.data = field;
        fa.n = grid->n[ax];
        fa.logn = ilog2(fa.n);
        const int64_t lines = (int64_t)nfield * npts / fa.n;
        if (ax == 2) {
            fa.es = 1;
            int64_t W = std::max<int64_t>(1, cap_elems / fa.n);
            while (W > 1 && lines % W) W >>= 1;
            fa.W = (int)W;
        } else {
            fa.es = ax == 1 ? nz : (int64_t)ny * nz;
            fa.inner = fa.es;
            fa.block_stride = (int64_t)grid->n[ax] * fa.es;
            int64_t W = std::min<int64_t>(std::max<int64_t>(1, cap_elems / fa.n), fa.inner);
            while (W > 1 && fa.inner % W) W >>= 1;
            fa.W = (int)W;
        }
        FCUDA(launch_fft_axis(fa, fp64 ? 1 : 0, lines / fa.W, st));
        ++c->launches;
    }
    // ---- 3. unpack, order, rephase
    FftUnpackArgs ua;
    memset(&ua, 0, sizeof(ua));
    ua.data = field;
    ua.S = S;
    for (int i = 0; i < 3; ++i) {
        ua.n[i] = grid->n[i];
        ua.dq[i] = grid->dq[i];
        ua.xmin[i] = xmin[i];
    }
    ua.vpix = vpix;
    ua.dq3_over_2pi3 = grid->dq[0] * grid->dq[1] * grid->dq[2] / (8.0 * M_PI * M_PI * M_PI);
    ua.f = df;
    ua.f2 = df2;
    ua.parseval = par;
    ua.phase = reinterpret_cast<double2 *>(w + o_phase);
    FCUDA(launch_fft_unpack(ua, fp64 ? 1 : 0, st));
    c->launches += 2;
    if (!out_on_device) {
        if (f_out) FCUDA(cudaMemcpyAsync(f_out, df, bytes_f, cudaMemcpyDeviceToHost, st));
        if (f2_out) FCUDA(cudaMemcpyAsync(f2_out, df2, bytes_f2, cudaMemcpyDeviceToHost, st));
    }
    if (parseval_out)
        FCUDA(cudaMemcpyAsync(parseval_out, par, sizeof(double) * 2 * S, cudaMemcpyDeviceToHost, st));
    FCUDA(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    FCUDA(cudaStreamSynchronize(st));
    if (*c->h_err)
        return ffail(SCFF_ERR_TIMEOUT, "scff_fft_form_factor: a device-side wait timed out (code %d)", *c->h_err);
    return SCFF_OK;
}
