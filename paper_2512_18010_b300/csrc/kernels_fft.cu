// FFT method (Sec. "The (Fast) Fourier Transform", Eqs. Falbega, continuFFT,
// fftABC, qabc; Sec. "Fast Fourier Transform Method"):
//
//   1. tabulate the basis functions on a box of points and contract them with
//      the transition matrices, Phi_s(r) = sum_{mu nu} T^s_{mu nu} phi_mu(r) phi_nu(r)
//      (fft_density_kernel: one tile of points per CTA, the functions of the
//      tile in shared memory, the contraction as a register-tiled product
//      against T staged through shared memory; primitives whose Gaussian
//      factor is below the threshold are dropped and all-zero tiles skip the
//      contraction, as in the paper's tabulation);
//   2. a 3-D discrete Fourier sum with the +i sign, one radix-2 pass per axis
//      in shared memory (fft_axis_kernel), two states packed per complex
//      field (Phi_a + i Phi_b, both real);
//   3. unpack the pair, order the frequencies from -n/2, and apply the pixel
//      volume and the phase of the box corner (fft_unpack_kernel):
//      f_s(q) = V_pix e^{i q.x_min} sum_a Phi_s(x_a) e^{2 pi i alpha.a / n}.
#include <math.h>

#include "device_common.cuh"
#include "fft_internal.h"
#include "scff_internal.h"

namespace scff {

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

__device__ __forceinline__ float fexp(float x) { return expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ void sincos_pi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincos_pi(double x, double *s, double *c) { sincospi(x, s, c); }

__device__ __forceinline__ void rec_powers(int type, int j, int pw[3]) {
    for (int ax = 0; ax < 3; ++ax)
        pw[ax] = type == REC_SP ? (j == 0 ? 0 : cart_pow(1, j - 1, ax)) : cart_pow(rec_lmax(type), j, ax);
}

constexpr int kFftThreads = 512;
constexpr int kFftWarps = kFftThreads / 32;
constexpr int kPairChunk = 256;  // (mu <= nu) pairs per staged chunk

// Tsym[sweep][k][q] for the pairs k = (mu <= nu) of the basis in row order
// (mu ascending, nu = mu..nbf-1): T_mu,mu on the diagonal and T_mu,nu + T_nu,mu
// above it, for states s = sweep * SBF + q (zero beyond S and beyond the last
// pair); pairs[k] = (mu, nu), (-1, -1) for the padding.
template <typename R>
__global__ void fft_tsym_kernel(const R *__restrict__ T, int nbf, int S, int sbf, int64_t kpad, int nsweep,
                                R *__restrict__ tsym, int2 *__restrict__ pairs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nsweep * kpad * sbf) return;
    const int q = (int)(idx % sbf);
    const int64_t k = (idx / sbf) % kpad;
    const int sweep = (int)(idx / ((int64_t)sbf * kpad));
    const int64_t kf = (int64_t)nbf * (nbf + 1) / 2;
    R v = R(0);
    int2 pr = make_int2(-1, -1);
    if (k < kf) {
        // invert k = mu nbf - mu (mu - 1) / 2 + (nu - mu)
        const double bq = 2.0 * nbf + 1.0;
        int mu = (int)floor((bq - sqrt(bq * bq - 8.0 * (double)k)) * 0.5);
        while (mu > 0 && (int64_t)mu * nbf - (int64_t)mu * (mu - 1) / 2 > k) --mu;
        while ((int64_t)(mu + 1) * nbf - (int64_t)(mu + 1) * mu / 2 <= k) ++mu;
        const int nu = mu + (int)(k - ((int64_t)mu * nbf - (int64_t)mu * (mu - 1) / 2));
        pr = make_int2(mu, nu);
        const int s = sweep * sbf + q;
        if (s < S) {
            const R *Ts = T + (size_t)s * nbf * nbf;
            v = Ts[(size_t)mu * nbf + nu];
            if (mu != nu) v += Ts[(size_t)nu * nbf + mu];
        }
    }
    tsym[idx] = v;
    if (sweep == 0 && q == 0) pairs[k] = pr;
}

// Phi_s(r) = sum_{mu <= nu} Tsym^s_{mu nu} phi_mu(r) phi_nu(r).  The pair
// products are state-independent, so each is formed once per point and used
// for the SBF states of a sweep held in registers.
//
// CTA: TP points (TP / 32 contiguous per lane) x 16 warps (the function values
// of the tile hold one CTA per SM, so its own warps hide the latencies).  The pairs stream
// through shared memory in chunks (1-D bulk async copies of the contiguous
// Tsym and pair rows, double-buffered on mbarriers with bounded waits); warp w
// takes pairs w, w + 16, ... of a chunk, so its lanes read the same Tsym row
// (broadcast) at different points.  A pair with a function that is
// identically zero on the tile (its Gaussians underflow, or the threshold
// dropped every primitive) is skipped by the whole warp: an exact pruning.
// smem: phi[nbf_pad][TP], active[nbf_pad] (bytes), 2 stages of
// (Tsym[kPairChunk][SBF], pairs[kPairChunk]), one state's partial densities [warps][TP].
template <typename R, int SBF, int TP>
__global__ void __launch_bounds__(kFftThreads) fft_density_kernel(FftDensityArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int PT = TP / 32;
    constexpr uint32_t T_BYTES = kPairChunk * SBF * sizeof(R), P_BYTES = kPairChunk * sizeof(int2);
    constexpr uint32_t STAGE = T_BYTES + P_BYTES;
    static_assert(T_BYTES % 16 == 0 && STAGE % 16 == 0, "bulk copies move multiples of 16 bytes");
    unsigned char *stage0 = smem_raw;  // [2][STAGE]
    R *part = reinterpret_cast<R *>(smem_raw + 2 * STAGE);
    R *phi = part + (size_t)kFftWarps * TP;
    unsigned char *active = reinterpret_cast<unsigned char *>(phi + (size_t)a.nbf_pad * TP);
    // the active pairs of the current chunk, compacted: (mu, nu, index in chunk)
    int4 *alist = reinterpret_cast<int4 *>(((uintptr_t)(active + a.nbf_pad) + 15) & ~uintptr_t(15));
    int *wcnt = reinterpret_cast<int *>(alist + kPairChunk);  // [kPairChunk / 32] counts per warp
    __shared__ __align__(8) uint64_t bars[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * TP;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbarrier_init();
    }
    for (int e = tid; e < a.nbf_pad * TP; e += kFftThreads) phi[e] = R(0);
    __syncthreads();
    // ---- 1. basis function values at the tile's points: kFftThreads / TP
    // groups of TP threads, group g taking the records whose first function
    // index is g modulo the group count, so all primitives of a function are
    // added by one thread in record order (the values do not depend on the
    // grouping)
    static_assert(kFftThreads % TP == 0, "whole groups of TP threads");
    constexpr int kTabGroups = kFftThreads / TP;
    if constexpr (sizeof(R) == 4) {
        // FP32: the displacement from a record's centre is ((i - ia) - fa) dx
        // per axis, an exact integer difference less a fraction, so it keeps
        // its relative accuracy however close the point is to the centre
        const int pt = tid % TP, grp = tid / TP;
        const int64_t p = p0 + pt;
        if (p < a.npts) {
            const float ci = (float)(p % a.nz), bi = (float)((p / a.nz) % a.ny),
                        ai = (float)(p / ((int64_t)a.ny * a.nz));
            const float dxf = (float)a.dx[0], dyf = (float)a.dx[1], dzf = (float)a.dx[2];
            const float cutf = (float)a.cut;
            for (int rec = 0; rec < a.ps.n_rec; ++rec) {
                const int fn0 = a.ps.rec_fn0[rec];
                if (fn0 % kTabGroups != grp) continue;
                const float4 gi = a.recg[2 * rec], gf = a.recg[2 * rec + 1];
                const float d[3] = {((ai - gi.x) - gf.x) * dxf, ((bi - gi.y) - gf.y) * dyf,
                                    ((ci - gi.z) - gf.z) * dzf};
                const float ex = gi.w * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (cutf > 0.f && ex > cutf) continue;
                const float g = expf(-ex);
                if (g == 0.f) continue;
                const int type = a.ps.rec_type[rec];
                const int nf = rec_nfn(type);
                for (int j = 0; j < nf; ++j) {
                    int pw[3];
                    rec_powers(type, j, pw);
                    float v = a.recw[kRecW * rec + j] * g;
                    for (int ax = 0; ax < 3; ++ax)
                        for (int k = 0; k < pw[ax]; ++k) v *= d[ax];
                    phi[(size_t)(fn0 + j) * TP + pt] += (R)v;
                }
            }
        }
    } else {
        const int pt = tid % TP, grp = tid / TP;
        const int64_t p = p0 + pt;
        if (p < a.npts) {
            const int c = (int)(p % a.nz), b = (int)((p / a.nz) % a.ny), aa = (int)(p / ((int64_t)a.ny * a.nz));
            const double rx = a.xmin[0] + aa * a.dx[0], ry = a.xmin[1] + b * a.dx[1], rz = a.xmin[2] + c * a.dx[2];
            for (int rec = 0; rec < a.ps.n_rec; ++rec) {
                if (a.ps.rec_fn0[rec] % kTabGroups != grp) continue;
                const double dxr = rx - a.ps.rec_xyz[3 * rec], dyr = ry - a.ps.rec_xyz[3 * rec + 1],
                             dzr = rz - a.ps.rec_xyz[3 * rec + 2];
                const double ex = a.ps.rec_alpha[rec] * (dxr * dxr + dyr * dyr + dzr * dzr);
                if (a.cut > 0.0 && ex > a.cut) continue;
                const R g = fexp((R)(-ex));
                if (g == R(0)) continue;
                const int type = a.ps.rec_type[rec], fn0 = a.ps.rec_fn0[rec];
                const int nf = rec_nfn(type);
                const R d[3] = {(R)dxr, (R)dyr, (R)dzr};
                for (int j = 0; j < nf; ++j) {
                    int pw[3];
                    rec_powers(type, j, pw);
                    R v = (R)a.ps.rec_w[kRecW * rec + j] * g;
                    for (int ax = 0; ax < 3; ++ax)
                        for (int k = 0; k < pw[ax]; ++k) v *= d[ax];
                    // row-major points within a lane's group: point pt lives at lane*PT+i
                    phi[(size_t)(fn0 + j) * TP + pt] += v;
                }
            }
        }
    }
    __syncthreads();
    for (int mu = tid; mu < a.nbf_pad; mu += kFftThreads) {
        bool nzf = false;
        if (mu < a.nbf)
            for (int i = 0; i < TP && !nzf; ++i) nzf = phi[(size_t)mu * TP + i] != R(0);
        active[mu] = nzf ? 1 : 0;
    }
    __syncthreads();
    // ---- 2. state sweeps; chunk g (global count over the sweeps) sits in stage g & 1
    const int nchunks = (int)(a.kpad / kPairChunk);
    const int nsweep = (a.S + SBF - 1) / SBF;
    int g = 0;
    bool ok = true;
    auto issue = [&](int sweep, int c, int gg) {
        unsigned char *st = stage0 + (gg & 1) * STAGE;
        mbar_arrive_expect_tx(&bars[gg & 1], STAGE);
        bulk_g2s(st, static_cast<const R *>(a.tsym) + ((size_t)sweep * a.kpad + (size_t)c * kPairChunk) * SBF,
                 T_BYTES, &bars[gg & 1]);
        bulk_g2s(st + T_BYTES, a.pairs + (size_t)c * kPairChunk, P_BYTES, &bars[gg & 1]);
    };
    for (int sweep = 0; sweep < nsweep && ok; ++sweep) {
        R tot[SBF][PT];
#pragma unroll
        for (int q = 0; q < SBF; ++q)
#pragma unroll
            for (int i = 0; i < PT; ++i) tot[q][i] = R(0);
        if (tid == 0) {
            fence_proxy_async_smem();
            issue(sweep, 0, g);
            if (nchunks > 1) issue(sweep, 1, g + 1);
        }
        for (int c = 0; c < nchunks; ++c, ++g) {
            const bool got = mbar_wait(&bars[g & 1], (g >> 1) & 1);
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            const unsigned char *st = stage0 + (g & 1) * STAGE;
            const R *Tc = reinterpret_cast<const R *>(st);
            const int2 *pc = reinterpret_cast<const int2 *>(st + T_BYTES);
            // compact the chunk's active pairs (both functions nonzero on the
            // tile), in chunk order, so the product loop has neither branches
            // nor dependent index loads
            static_assert(kPairChunk <= kFftThreads && kPairChunk % 32 == 0, "one thread per pair of a chunk");
            bool act = false;
            int2 prc = make_int2(-1, -1);
            if (tid < kPairChunk) {
                prc = pc[tid];
                act = prc.x >= 0 && active[prc.x] && active[prc.y];
            }
            const unsigned am = __ballot_sync(0xffffffffu, act);
            if (tid < kPairChunk && lane == 0) wcnt[warp] = __popc(am);
            __syncthreads();
            int n_act = 0, off = 0;
#pragma unroll
            for (int w = 0; w < kPairChunk / 32; ++w) {
                const int cw = wcnt[w];
                if (w < warp) off += cw;
                n_act += cw;
            }
            if (act) alist[off + __popc(am & ((1u << lane) - 1u))] = make_int4(prc.x, prc.y, tid, 0);
            __syncthreads();
            R acc[SBF][PT];
#pragma unroll
            for (int q = 0; q < SBF; ++q)
#pragma unroll
                for (int i = 0; i < PT; ++i) acc[q][i] = R(0);
#pragma unroll 2
            for (int t = warp; t < n_act; t += kFftWarps) {
                const int4 e = alist[t];
                const int kk = e.z;
                const R *pa = phi + (size_t)e.x * TP + lane * PT;
                const R *pb = phi + (size_t)e.y * TP + lane * PT;
                R prod[PT];
#pragma unroll
                for (int i = 0; i < PT; ++i) prod[i] = pa[i] * pb[i];
                const R *tr = Tc + (size_t)kk * SBF;
#pragma unroll
                for (int q = 0; q < SBF; ++q) {
                    const R t = tr[q];
#pragma unroll
                    for (int i = 0; i < PT; ++i) acc[q][i] = fma(t, prod[i], acc[q][i]);
                }
            }
#pragma unroll
            for (int q = 0; q < SBF; ++q)
#pragma unroll
                for (int i = 0; i < PT; ++i) tot[q][i] += acc[q][i];
            __syncthreads();
            if (tid == 0 && c + 2 < nchunks) {
                fence_proxy_async_smem();
                issue(sweep, c + 2, g + 2);
            }
        }
        if (!ok) break;
        // reduce the warps' partial sums state by state and write the fields
        // (point index lane * PT + i)
#pragma unroll
        for (int q = 0; q < SBF; ++q) {
#pragma unroll
            for (int i = 0; i < PT; ++i) part[(size_t)warp * TP + lane * PT + i] = tot[q][i];
            __syncthreads();
            const int s = sweep * SBF + q;
            if (tid < TP) {
                R v = R(0);
                for (int w = 0; w < kFftWarps; ++w) v += part[(size_t)w * TP + tid];
                v *= (R)a.scale;
                const int64_t p = p0 + tid;
                double sq = 0.0;
                if (s < a.S && p < a.npts) {
                    R *field = static_cast<R *>(a.out) + ((size_t)(s >> 1) * a.npts + p) * 2;
                    field[s & 1] = v;
                    if ((s & 1) == 0 && s + 1 == a.S) field[1] = R(0);
                    sq = (double)v * (double)v;
                }
                // Parseval over the tile's points (TP is a multiple of 32)
                for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
                if (lane == 0 && s < a.S && a.parseval) atomicAdd(&a.parseval[2 * s], sq * a.vpix);
            }
            __syncthreads();
        }
    }
    if (!ok && tid == 0) {
        flag_error(a.err, kDevErrTimeout);
        // let the copies still in flight land before the CTA's shared memory goes away
        mbar_wait(&bars[g & 1], (g >> 1) & 1);
        mbar_wait(&bars[(g + 1) & 1], ((g + 1) >> 1) & 1);
    }
}

// One radix-2 pass along one axis for W lines of length n (a power of two):
// out[alpha] = sum_a in[a] e^{+2 pi i alpha a / n}, in place.  Lines are
// loaded into shared memory in bit-reversed order, then log2(n) butterfly
// stages run with twiddles from a table of the n/2 roots of unity.
template <typename R>
__global__ void __launch_bounds__(256) fft_axis_kernel(FftAxisArgs a) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *buf = reinterpret_cast<V *>(smem_raw);
    V *tw = buf + (size_t)a.W * a.n;
    V *data = reinterpret_cast<V *>(a.data);
    const int n = a.n, W = a.W, logn = a.logn;
    // line group -> base address of line 0 of the group and the stride between lines
    const int64_t g = blockIdx.x;
    int64_t base;
    int64_t lstride;
    if (a.es == 1) {
        base = g * W * (int64_t)n;  // W consecutive contiguous lines
        lstride = n;
    } else {
        const int64_t groups_per_block = a.inner / W;  // inner: lines adjacent in memory (stride 1)
        const int64_t blk = g / groups_per_block, w0 = (g % groups_per_block) * W;
        base = blk * a.block_stride + w0;
        lstride = 1;
    }
    for (int k = threadIdx.x; k < n / 2; k += blockDim.x) {
        R sn, cs;
        sincos_pi((R)(2 * k) / (R)n, &sn, &cs);
        tw[k].x = cs;
        tw[k].y = sn;
    }
    for (int idx = threadIdx.x; idx < W * n; idx += blockDim.x) {
        int w, k;
        if (a.es == 1) {
            w = idx / n;
            k = idx % n;
        } else {
            k = idx / W;
            w = idx % W;
        }
        const unsigned rev = __brev((unsigned)k) >> (32 - logn);
        buf[(size_t)w * n + rev] = data[base + w * lstride + (int64_t)k * a.es];
    }
    __syncthreads();
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1, step = n / len;
        for (int t = threadIdx.x; t < W * (n / 2); t += blockDim.x) {
            const int w = t / (n / 2), j = t % (n / 2);
            const int blk = j / half, k = j % half;
            V *line = buf + (size_t)w * n + blk * len;
            const V u = line[k], x = line[k + half], c = tw[k * step];
            const V v = {x.x * c.x - x.y * c.y, x.x * c.y + x.y * c.x};
            line[k] = V{u.x + v.x, u.y + v.y};
            line[k + half] = V{u.x - v.x, u.y - v.y};
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < W * n; idx += blockDim.x) {
        int w, k;
        if (a.es == 1) {
            w = idx / n;
            k = idx % n;
        } else {
            k = idx / W;
            w = idx % W;
        }
        data[base + w * lstride + (int64_t)k * a.es] = buf[(size_t)w * n + k];
    }
}

// f[s][ix][iy][iz] at q = dq (i - n/2): unpack state s from its packed field,
// order from the most negative frequency, times scale-free V_pix e^{i q.x_min}
// (Phi already carries the scale).
template <typename R>
__global__ void fft_unpack_kernel(FftUnpackArgs a) {
    using V = typename C2<R>::T;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npts = (int64_t)a.n[0] * a.n[1] * a.n[2];
    const int64_t total = (int64_t)a.S * npts;
    double sq = 0.0;
    int s = 0;
    if (idx < total) {
        s = (int)(idx / npts);
        const int64_t p = idx % npts;
        const int iz = (int)(p % a.n[2]), iy = (int)((p / a.n[2]) % a.n[1]), ix = (int)(p / ((int64_t)a.n[1] * a.n[2]));
        const int al[3] = {ix - a.n[0] / 2, iy - a.n[1] / 2, iz - a.n[2] / 2};
        const int i3[3] = {(al[0] + a.n[0]) & (a.n[0] - 1), (al[1] + a.n[1]) & (a.n[1] - 1), (al[2] + a.n[2]) & (a.n[2] - 1)};
        const int j3[3] = {(-al[0] + a.n[0]) & (a.n[0] - 1), (-al[1] + a.n[1]) & (a.n[1] - 1), (-al[2] + a.n[2]) & (a.n[2] - 1)};
        const V *field = reinterpret_cast<const V *>(a.data) + (size_t)(s >> 1) * npts;
        const V G = field[((int64_t)i3[0] * a.n[1] + i3[1]) * a.n[2] + i3[2]];
        const V Gm = field[((int64_t)j3[0] * a.n[1] + j3[1]) * a.n[2] + j3[2]];
        double fr, fi;
        if ((s & 1) == 0) {  // (G + conj(Gm)) / 2
            fr = 0.5 * ((double)G.x + (double)Gm.x);
            fi = 0.5 * ((double)G.y - (double)Gm.y);
        } else {  // (G - conj(Gm)) / (2i)
            fr = 0.5 * ((double)G.y + (double)Gm.y);
            fi = -0.5 * ((double)G.x - (double)Gm.x);
        }
        // e^{i q.x_min} as the product of the three per-axis factors
        const double2 px = a.phase[ix], py = a.phase[a.n[0] + iy], pz = a.phase[a.n[0] + a.n[1] + iz];
        const double xyr = px.x * py.x - px.y * py.y, xyi = px.x * py.y + px.y * py.x;
        const double cs = xyr * pz.x - xyi * pz.y, sn = xyr * pz.y + xyi * pz.x;
        const double vr = a.vpix * (fr * cs - fi * sn), vi = a.vpix * (fr * sn + fi * cs);
        V out;
        out.x = (R)vr;
        out.y = (R)vi;
        if (a.f) reinterpret_cast<V *>(a.f)[idx] = out;
        if (a.f2) reinterpret_cast<R *>(a.f2)[idx] = out.x * out.x + out.y * out.y;
        sq = vr * vr + vi * vi;
    }
    // Parseval, momentum side: warp sums, then one atomic per block when the
    // block lies within one state (npts a multiple of the block size), else
    // one per warp (npts is a multiple of 32, so a warp never spans two
    // states).  Every thread of the block reaches the shuffles (no early return).
    __shared__ double wsum[8];
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (npts % blockDim.x == 0) {
        if (lane == 0) wsum[wid] = sq;
        __syncthreads();
        if (threadIdx.x == 0 && idx < total && a.parseval) {
            double b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w];
            atomicAdd(&a.parseval[2 * s + 1], b * a.dq3_over_2pi3);
        }
    } else if (lane == 0 && idx < total && a.parseval) {
        atomicAdd(&a.parseval[2 * s + 1], sq * a.dq3_over_2pi3);
    }
}

// Per-axis factors e^{i dq_k al x_min,k} of the box-corner phase, al = i - n_k/2.
__global__ void fft_phase_table_kernel(FftUnpackArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n[0] + a.n[1] + a.n[2]) return;
    const int ax = i < a.n[0] ? 0 : (i < a.n[0] + a.n[1] ? 1 : 2);
    const int j = i - (ax > 0 ? a.n[0] : 0) - (ax > 1 ? a.n[1] : 0);
    double sn, cs;
    sincos(a.dq[ax] * (j - a.n[ax] / 2) * a.xmin[ax], &sn, &cs);
    a.phase[i] = make_double2(cs, sn);
}

__global__ void cast_f64_to_f32_kernel(const double *__restrict__ in, int64_t n, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_cast_f64_to_f32(const double *in, int64_t n, float *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cast_f64_to_f32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

__global__ void fft_record_prep_kernel(FftDensityArgs a, float4 *__restrict__ recg, float *__restrict__ recw) {
    const int rec = blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= a.ps.n_rec) return;
    float ia[3], fa[3];
    for (int ax = 0; ax < 3; ++ax) {
        const double gc = (a.ps.rec_xyz[3 * rec + ax] - a.xmin[ax]) / a.dx[ax];
        const double fl = floor(gc);
        ia[ax] = (float)fl;
        fa[ax] = (float)(gc - fl);
    }
    recg[2 * rec] = make_float4(ia[0], ia[1], ia[2], (float)a.ps.rec_alpha[rec]);
    recg[2 * rec + 1] = make_float4(fa[0], fa[1], fa[2], 0.f);
    for (int j = 0; j < kRecW; ++j) recw[kRecW * rec + j] = (float)a.ps.rec_w[kRecW * rec + j];
}

cudaError_t launch_fft_record_prep(const FftDensityArgs &a, float4 *recg, float *recw, cudaStream_t st) {
    if (a.ps.n_rec == 0) return cudaSuccess;
    fft_record_prep_kernel<<<(a.ps.n_rec + 127) / 128, 128, 0, st>>>(a, recg, recw);
    return cudaGetLastError();
}

template <typename R, int SBF, int TP>
static cudaError_t density_t(const FftDensityArgs &a, cudaStream_t st) {
    const size_t smem = fft_density_smem(sizeof(R) == 8, a.nbf_pad, SBF, TP);
    cudaError_t e = cudaFuncSetAttribute(fft_density_kernel<R, SBF, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.npts + TP - 1) / TP;
    fft_density_kernel<R, SBF, TP><<<(unsigned)tiles, kFftThreads, smem, st>>>(a);
    return cudaGetLastError();
}

size_t fft_density_smem(int fp64, int nbf_pad, int sbf, int tp) {
    const size_t rs = fp64 ? sizeof(double) : sizeof(float);
    const size_t stage = (size_t)kPairChunk * sbf * rs + (size_t)kPairChunk * sizeof(int2);
    return 2 * stage + rs * ((size_t)kFftWarps * tp + (size_t)nbf_pad * tp) + (size_t)nbf_pad + 16 +
           sizeof(int4) * kPairChunk + sizeof(int) * (kPairChunk / 32) + 128;
}

int64_t fft_pair_kpad(int nbf) {
    const int64_t kf = (int64_t)nbf * (nbf + 1) / 2;
    return (kf + kPairChunk - 1) / kPairChunk * kPairChunk;
}

cudaError_t launch_fft_tsym(const void *T, int fp64, int nbf, int S, int sbf, void *tsym, int2 *pairs,
                            cudaStream_t st) {
    const int64_t kpad = fft_pair_kpad(nbf);
    const int nsweep = (S + sbf - 1) / sbf;
    const int64_t tot = (int64_t)nsweep * kpad * sbf;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        fft_tsym_kernel<double><<<blocks, 256, 0, st>>>((const double *)T, nbf, S, sbf, kpad, nsweep, (double *)tsym,
                                                        pairs);
    else
        fft_tsym_kernel<float><<<blocks, 256, 0, st>>>((const float *)T, nbf, S, sbf, kpad, nsweep, (float *)tsym,
                                                       pairs);
    return cudaGetLastError();
}

// Instantiated shapes: FP32 (12|8|4 states) x (128|32 points); FP64 (8|4) x (64|32).
cudaError_t launch_fft_density(const FftDensityArgs &a, int fp64, int sbf, int tp, cudaStream_t st) {
    if (a.npts == 0) return cudaSuccess;
    if (fp64) {
        if (tp == 64) return sbf == 8 ? density_t<double, 8, 64>(a, st) : density_t<double, 4, 64>(a, st);
        if (tp == 32) return sbf == 8 ? density_t<double, 8, 32>(a, st) : density_t<double, 4, 32>(a, st);
        return cudaErrorInvalidValue;
    }
    if (tp == 128) {
        if (sbf == 12) return density_t<float, 12, 128>(a, st);
        if (sbf == 8) return density_t<float, 8, 128>(a, st);
        return density_t<float, 4, 128>(a, st);
    }
    if (tp == 32) {
        if (sbf == 12) return density_t<float, 12, 32>(a, st);
        if (sbf == 8) return density_t<float, 8, 32>(a, st);
        return density_t<float, 4, 32>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fft_axis(const FftAxisArgs &a, int fp64, int64_t n_groups, cudaStream_t st) {
    const size_t el = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t smem = el * ((size_t)a.W * a.n + a.n / 2);
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(fft_axis_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fft_axis_kernel<double><<<(unsigned)n_groups, 256, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(fft_axis_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fft_axis_kernel<float><<<(unsigned)n_groups, 256, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_fft_unpack(const FftUnpackArgs &a, int fp64, cudaStream_t st) {
    const int64_t tot = (int64_t)a.S * a.n[0] * a.n[1] * a.n[2];
    if (tot == 0) return cudaSuccess;
    const int nax = a.n[0] + a.n[1] + a.n[2];
    fft_phase_table_kernel<<<(nax + 127) / 128, 128, 0, st>>>(a);
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        fft_unpack_kernel<double><<<blocks, 256, 0, st>>>(a);
    else
        fft_unpack_kernel<float><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace scff
