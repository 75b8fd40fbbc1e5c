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

constexpr int kFftThreads = 256;
constexpr int kMuBlock = 32;  // functions per contraction pass (8 warps x 4)

// smem: phi[nbf_pad][TP] and the staged transposed T block Tt[nbf_pad][kMuBlock],
// then the per-warp partial densities [8][TP].
template <typename R, int TP>
__global__ void __launch_bounds__(kFftThreads) fft_density_kernel(FftDensityArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *phi = reinterpret_cast<R *>(smem_raw);
    R *Tt = phi + (size_t)a.nbf_pad * TP;
    R *part = Tt + (size_t)a.nbf_pad * kMuBlock;
    __shared__ int any_nonzero;
    constexpr int PT = TP / 32;  // points per lane: lane + 32 i, i < PT
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * TP;
    if (tid == 0) any_nonzero = 0;
    for (int e = tid; e < a.nbf_pad * TP; e += kFftThreads) phi[e] = R(0);
    __syncthreads();
    // ---- 1. basis function values at the tile's points
    if (tid < TP) {
        const int64_t p = p0 + tid;
        if (p < a.npts) {
            const int c = (int)(p % a.nz), b = (int)((p / a.nz) % a.ny), aa = (int)(p / ((int64_t)a.ny * a.nz));
            const double rx = a.xmin[0] + aa * a.dx[0], ry = a.xmin[1] + b * a.dx[1], rz = a.xmin[2] + c * a.dx[2];
            bool nz = false;
            for (int rec = 0; rec < a.ps.n_rec; ++rec) {
                const double dxr = rx - a.ps.rec_xyz[3 * rec], dyr = ry - a.ps.rec_xyz[3 * rec + 1],
                             dzr = rz - a.ps.rec_xyz[3 * rec + 2];
                const double ex = a.ps.rec_alpha[rec] * (dxr * dxr + dyr * dyr + dzr * dzr);
                if (a.cut > 0.0 && ex > a.cut) continue;
                const R g = fexp((R)(-ex));
                const int type = a.ps.rec_type[rec], fn0 = a.ps.rec_fn0[rec];
                const int nf = rec_nfn(type);
                const R d[3] = {(R)dxr, (R)dyr, (R)dzr};
                for (int j = 0; j < nf; ++j) {
                    int pw[3];
                    rec_powers(type, j, pw);
                    R v = (R)a.ps.rec_w[kRecW * rec + j] * g;
                    for (int ax = 0; ax < 3; ++ax)
                        for (int k = 0; k < pw[ax]; ++k) v *= d[ax];
                    phi[(size_t)(fn0 + j) * TP + tid] += v;
                }
                nz = true;
            }
            if (nz) any_nonzero = 1;
        }
    }
    __syncthreads();
    const bool skip = any_nonzero == 0;
    // ---- 2. Phi_s = sum_mu phi_mu (sum_nu T_mu,nu phi_nu), state by state
    for (int s = 0; s < a.S; ++s) {
        R dens[PT];
#pragma unroll
        for (int i = 0; i < PT; ++i) dens[i] = R(0);
        if (!skip) {
            const R *Ts = static_cast<const R *>(a.T) + (size_t)s * a.nbf * a.nbf;
            for (int mu0 = 0; mu0 < a.nbf; mu0 += kMuBlock) {
                // Tt[nu][j] = T[mu0 + j][nu]
                for (int e = tid; e < kMuBlock * a.nbf_pad; e += kFftThreads) {
                    const int j = e / a.nbf_pad, nu = e % a.nbf_pad;
                    const int mu = mu0 + j;
                    Tt[(size_t)nu * kMuBlock + j] = (mu < a.nbf && nu < a.nbf) ? Ts[(size_t)mu * a.nbf + nu] : R(0);
                }
                __syncthreads();
                R acc[4][PT];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int i = 0; i < PT; ++i) acc[j][i] = R(0);
                const int jw = warp * 4;
                for (int nu = 0; nu < a.nbf; ++nu) {
                    R t[4], v[PT];
#pragma unroll
                    for (int j = 0; j < 4; ++j) t[j] = Tt[(size_t)nu * kMuBlock + jw + j];
#pragma unroll
                    for (int i = 0; i < PT; ++i) v[i] = phi[(size_t)nu * TP + lane + 32 * i];
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int i = 0; i < PT; ++i) acc[j][i] = fma(t[j], v[i], acc[j][i]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int mu = mu0 + jw + j;
                    if (mu < a.nbf) {
#pragma unroll
                        for (int i = 0; i < PT; ++i)
                            dens[i] = fma(phi[(size_t)mu * TP + lane + 32 * i], acc[j][i], dens[i]);
                    }
                }
                __syncthreads();
            }
        }
        // reduce the eight warps' partial sums
#pragma unroll
        for (int i = 0; i < PT; ++i) part[warp * TP + lane + 32 * i] = dens[i];
        __syncthreads();
        if (tid < TP) {
            R v = R(0);
            for (int w = 0; w < kFftThreads / 32; ++w) v += part[w * TP + tid];
            v *= (R)a.scale;
            const int64_t p = p0 + tid;
            double sq = 0.0;
            if (p < a.npts) {
                R *field = static_cast<R *>(a.out) + ((size_t)(s >> 1) * a.npts + p) * 2;
                field[s & 1] = v;
                if ((s & 1) == 0 && s + 1 == a.S) field[1] = R(0);
                sq = (double)v * (double)v;
            }
            // Parseval: sum over the tile's points, one atomic per warp
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
            if (lane == 0 && a.parseval) atomicAdd(&a.parseval[2 * s], sq * a.vpix);
        }
        __syncthreads();
    }
}

// One radix-2 pass along one axis for W lines of length n (a power of two):
// out[alpha] = sum_a in[a] e^{+2 pi i alpha a / n}, in place.  Lines are
// loaded into shared memory in bit-reversed order, then log2(n) butterfly
// stages run with twiddles from a table of the n/2 roots of unity.
template <typename R>
__global__ void __launch_bounds__(256) fft_axis_kernel(FftAxisArgs a) {
    using V = typename C2<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
        const double ph = a.dq[0] * al[0] * a.xmin[0] + a.dq[1] * al[1] * a.xmin[1] + a.dq[2] * al[2] * a.xmin[2];
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double vr = a.vpix * (fr * cs - fi * sn), vi = a.vpix * (fr * sn + fi * cs);
        V out;
        out.x = (R)vr;
        out.y = (R)vi;
        if (a.f) reinterpret_cast<V *>(a.f)[idx] = out;
        if (a.f2) reinterpret_cast<R *>(a.f2)[idx] = out.x * out.x + out.y * out.y;
        sq = vr * vr + vi * vi;
    }
    // Parseval, momentum side: one atomic per warp.  npts is a multiple of 32,
    // so a warp never spans two states; every thread of the block reaches the
    // shuffle (no early return).
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0 && idx < total && a.parseval) atomicAdd(&a.parseval[2 * s + 1], sq * a.dq3_over_2pi3);
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

template <typename R, int TP>
static cudaError_t density_t(const FftDensityArgs &a, cudaStream_t st) {
    const size_t smem = sizeof(R) * ((size_t)a.nbf_pad * TP + (size_t)a.nbf_pad * kMuBlock + 8 * TP);
    cudaError_t e = cudaFuncSetAttribute(fft_density_kernel<R, TP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (a.npts + TP - 1) / TP;
    fft_density_kernel<R, TP><<<(unsigned)tiles, kFftThreads, smem, st>>>(a);
    return cudaGetLastError();
}

size_t fft_density_smem(int fp64, int nbf_pad, int tp) {
    const size_t rs = fp64 ? sizeof(double) : sizeof(float);
    return rs * ((size_t)nbf_pad * tp + (size_t)nbf_pad * kMuBlock + 8 * (size_t)tp);
}

cudaError_t launch_fft_density(const FftDensityArgs &a, int fp64, int tp, cudaStream_t st) {
    if (a.npts == 0) return cudaSuccess;
    if (fp64) {
        if (tp == 128) return density_t<double, 128>(a, st);
        if (tp == 64) return density_t<double, 64>(a, st);
        return density_t<double, 32>(a, st);
    }
    if (tp == 128) return density_t<float, 128>(a, st);
    if (tp == 64) return density_t<float, 64>(a, st);
    return density_t<float, 32>(a, st);
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
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        fft_unpack_kernel<double><<<blocks, 256, 0, st>>>(a);
    else
        fft_unpack_kernel<float><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace scff
