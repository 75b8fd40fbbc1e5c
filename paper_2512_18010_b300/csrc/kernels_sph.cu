// Spherical method (Sec. "Analytic Method", Eqs. SphericalMethod, RTensor,
// WTensor and YYY; Appendix B for the monomial-to-spherical coefficients):
//
//   f_s(q) = sum_{l <= l_max, m} Y_l^m(q^) R^s_lm(|q|).
//
// Per pair p (centre P, exponent p, folded coefficients D^s_uvw of the
// Cartesian method) the monomials are projected on spherical harmonics,
// q_x^u q_y^v q_z^w = q^n sum Theta^{uvw}_{lambda mu} Y_lambda^mu(q^) (n = u+v+w),
// the phase is expanded in plane waves,
// e^{iq.P} = 4 pi sum_{LM} i^L j_L(q|P|) Y_L^M(q^) conj(Y_L^M(P^)),
// and the two harmonics of q^ are coupled by Gaunt coefficients
// G(lambda mu, L M -> l m) = Int Y_lambda^mu Y_L^M conj(Y_l^m) dOmega.
// Grouping the sums the B300 way, the pair sum becomes one dense complex
// contraction per job,
//   Z^s[(lambda mu), (q, L M)] = sum_{(p, n)} W^{s,n}_{p,lambda mu} rho_{p,n,L}(q) y_{p,LM},
//   W^{s,n}_{p,lambda mu} = sum_{u+v+w=n} D^s_uvw Theta^{uvw}_{lambda mu}   (the W tensor),
//   rho_{p,n,L}(q) = exp(-q^2/4p) q^n j_L(q|P|),   y_{p,LM} = 4 pi i^L conj(Y_L^M(P^)),
// Theta vanishes unless lambda and n have the same parity, so the contraction
// splits into an even job (n and lambda even) and an odd job, each over its
// own k = (pair, n) and rows (s, lambda mu): half the work of the full one.
// This is followed by a small Gaunt contraction
//   R^s_lm(q) = sum_{lambda mu, L} G(lambda mu, L (m-mu) -> l m) Z^s[(lambda mu), (q, L (m-mu))]
// and, for a tabulated angular grid, a second dense contraction
//   f_s(q, theta, phi) = sum_{lm} R^s_lm(q) p_l^m(cos theta) e^{i m phi}.
// The dense contractions run on the tensor cores (kernels_tc.cu,
// tc_run_generic) or, in FP64, in gen_gemm64_kernel below.  Tables are built
// in FP64 (spherical Bessel functions by Miller's downward recurrence).
#include <math.h>

#include "device_common.cuh"
#include "scff_internal.h"
#include "sph_common.h"
#include "sph_internal.h"

namespace scff {

using sph::kMaxBigL;

// Recurrence coefficients of the associated Legendre functions for l <= kMaxBigL
// (sph::plm_coefficients), filled once per device by sph_plm_init_kernel.
constexpr int kPlmTri = (kMaxBigL + 1) * (kMaxBigL + 2) / 2;
__device__ double g_plm_ab[2 * kPlmTri];

__global__ void sph_plm_init_kernel() {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kPlmTri) return;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= t) ++l;
    const int m = t - l * (l + 1) / 2;
    sph::plm_coefficients(l, m, g_plm_ab + 2 * t);
}

__device__ __forceinline__ int pair_class(const PairSetDev &ps, int pr) {
    int L = 0;
    while (L < kMaxPairL && pr >= ps.pair_off[L + 1]) ++L;
    return L;
}

__device__ __forceinline__ int axrow_class(const PairSetDev &ps, int64_t k) {
    int L = 0;
    while (L < kMaxPairL && k >= ps.axrow_off[L + 1]) ++L;
    return L;
}

// rho[(k, iq, L)] for the rows k = (pair, n) of one pair and one radial q.
template <typename V>
__global__ void sph_radial_kernel(PairSetDev ps, const double *__restrict__ geom, const double *__restrict__ q,
                                  int nq, int NL, V *__restrict__ table) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ps.n_pair * nq) return;
    const int pr = (int)(idx / nq), iq = (int)(idx % nq);
    const int Lc = pair_class(ps, pr);
    const int64_t k0 = ps.axrow_off[Lc] + (int64_t)(pr - ps.pair_off[Lc]) * (Lc + 1);
    const double Px = geom[4 * pr], Py = geom[4 * pr + 1], Pz = geom[4 * pr + 2], inv4p = geom[4 * pr + 3];
    const double r = sqrt(Px * Px + Py * Py + Pz * Pz);
    const double qq = q[iq];
    double j[kMaxBigL + 1];
    sph::sph_bessel_all(NL, qq * r, j);
    const double g = exp(-qq * qq * inv4p);
    double qn = 1.0;
    for (int n = 0; n <= Lc; ++n) {
        V *row = table + ((size_t)(k0 + n) * nq + iq) * NL;
        const double a = g * qn;
        for (int L = 0; L < NL; ++L) {
            V v;
            v.x = a * j[L];
            v.y = 0;
            row[L] = v;
        }
        qn *= qq;
    }
}

// y[p][LM] = 4 pi i^L conj(Y_L^M(P^)) for L <= Lmax (P at the origin: P^ = z^);
// one thread per (pair, |M|) writes the +M and -M entries of every L.
template <typename V>
__global__ void sph_ypair_kernel(PairSetDev ps, const double *__restrict__ geom, int Lmax, V *__restrict__ table) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ps.n_pair * (Lmax + 1)) return;
    const int pr = (int)(idx / (Lmax + 1)), M = (int)(idx % (Lmax + 1));
    const double Px = geom[4 * pr], Py = geom[4 * pr + 1], Pz = geom[4 * pr + 2];
    const double r = sqrt(Px * Px + Py * Py + Pz * Pz);
    const double x = r > 0.0 ? Pz / r : 1.0;
    const double phi = r > 0.0 ? atan2(Py, Px) : 0.0;
    double col[kMaxBigL + 1];
    sph::plm_column_tab(Lmax, M, x, g_plm_ab, col);
    double sn, cs;
    sincos(M * phi, &sn, &cs);
    const int NLM = (Lmax + 1) * (Lmax + 1);
    V *row = table + (size_t)pr * NLM;
    const double four_pi = 12.566370614359172;
    const double sgn = (M & 1) ? -1.0 : 1.0;  // p_L^{-M} = (-1)^M p_L^M
    for (int L = M; L <= Lmax; ++L) {
        // i^L
        const double ir = (L & 1) ? 0.0 : ((L & 2) ? -1.0 : 1.0);
        const double ii = (L & 1) ? ((L & 2) ? -1.0 : 1.0) : 0.0;
        const double a = four_pi * col[L - M];
        // conj(Y_L^M) = p e^{-i M phi}
        double yr = a * cs, yi = -a * sn;
        V v;
        v.x = ir * yr - ii * yi;
        v.y = ir * yi + ii * yr;
        row[sph::lm_index(L, M)] = v;
        if (M > 0) {
            // conj(Y_L^{-M}) = (-1)^M p e^{+i M phi}
            yr = sgn * a * cs;
            yi = sgn * a * sn;
            v.x = ir * yr - ii * yi;
            v.y = ir * yi + ii * yr;
            row[sph::lm_index(L, -M)] = v;
        }
    }
}

// Compact k of one parity job -> (class, pair, n, axis row).
__device__ __forceinline__ bool sph_k_decode(const PairSetDev &ps, const SphParity &kp, int64_t k, int *Lc_out,
                                             int *pr_out, int *n_out, int64_t *axrow_out) {
    if (k >= kp.off[kNumClasses]) return false;
    int Lc = 0;
    while (Lc < kMaxPairL && k >= kp.off[Lc + 1]) ++Lc;
    const int cnt = sph_parity_count(Lc, kp.par);
    const int64_t local = k - kp.off[Lc];
    const int pl = (int)(local / cnt);
    const int n = kp.par + 2 * (int)(local % cnt);
    *Lc_out = Lc;
    *pr_out = ps.pair_off[Lc] + pl;
    *n_out = n;
    *axrow_out = ps.axrow_off[Lc] + (int64_t)pl * (Lc + 1) + n;
    return true;
}

// kofs of one parity job: k = (pair, n) reads rho at axis row (pair, n) and y
// at row pair; padding k reads the zero rows.
__global__ void sph_kofs_kernel(PairSetDev ps, SphParity kp, int64_t K_pad, int nq, int NL, int NLM,
                                int2 *__restrict__ kofs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K_pad) return;
    int Lc, pr, n;
    int64_t ax;
    if (sph_k_decode(ps, kp, k, &Lc, &pr, &n, &ax))
        kofs[k] = make_int2((int)(ax * nq * NL), pr * NLM);
    else
        kofs[k] = make_int2((int)(ps.n_axrows * nq * NL), ps.n_pair * NLM);
}

// W tensor of one parity job as a dense complex matrix
// A[(s, sub)][k = (pair, n)], sub the index of (lambda, mu) among the
// harmonics of that parity:
// W = i^(n mod 2) sum_{u+v+w=n} c^s_uvw Theta^{uvw}_{lambda mu} (the folded
// pair-prep coefficients c carry the sign of i^n; the odd-n factor i is
// restored here).  theta is [monomial][49] over lambda <= 6.
__global__ void sph_wdense_kernel(PairSetDev ps, const double *__restrict__ coef64, int SB, int S, SphParity kp,
                                  int n_sub, const double2 *__restrict__ theta, int64_t K_pad,
                                  double2 *__restrict__ A) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)S * n_sub * K_pad) return;
    const int m = (int)(idx / K_pad);
    const int64_t k = idx % K_pad;
    const int s = m / n_sub, sub = m % n_sub;
    int lam = kp.par, base = 0;
    while (sub >= base + 2 * lam + 1) {
        base += 2 * lam + 1;
        lam += 2;
    }
    const int lm = sph::lm_index(lam, sub - base - lam);
    double2 acc = make_double2(0.0, 0.0);
    int Lc, pr, n;
    int64_t ax;
    if (sph_k_decode(ps, kp, k, &Lc, &pr, &n, &ax)) {
        const int pr_local = pr - ps.pair_off[Lc];
        if (lam <= n) {
            const int64_t rowbase = ps.row_off[Lc] + (int64_t)pr_local * mono_count(Lc);
            const double *cs = coef64 + ((size_t)(s / SB) * ps.n_rows) * SB + (s % SB);
            for (int u = n; u >= 0; --u)
                for (int v = n - u; v >= 0; --v) {
                    const int mi = mono_index(u, v, n - u - v);
                    const double c = cs[(size_t)(rowbase + mi) * SB];
                    const double2 t = theta[mi * 49 + lm];
                    acc.x = fma(c, t.x, acc.x);
                    acc.y = fma(c, t.y, acc.y);
                }
            if (n & 1) acc = make_double2(-acc.y, acc.x);
        }
    }
    A[idx] = acc;
}

// R^s_lm(q) = scale * sum_entries G Z^s[(lambda mu), (q, L M)], with Z held
// as the even and odd jobs' outputs [S][n_sub][nq x NLM]; an entry's x field
// is sub | (parity << 16).
template <typename VZ>
__global__ void sph_gaunt_kernel(const VZ *__restrict__ Ze, const VZ *__restrict__ Zo, int ne, int no, int S,
                                 int nq, int NLM, int NR, const int *__restrict__ goff,
                                 const int2 *__restrict__ gidx, const double *__restrict__ gval, double scale,
                                 double2 *__restrict__ R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)S * nq * NR) return;
    const int o = (int)(idx % NR);
    const int64_t sq = idx / NR;
    const int iq = (int)(sq % nq), s = (int)(sq / nq);
    const int64_t N = (int64_t)nq * NLM;
    double re = 0.0, im = 0.0;
    for (int e = goff[o]; e < goff[o + 1]; ++e) {
        const int2 ix = gidx[e];
        const int sub = ix.x & 0xFFFF;
        const bool odd = (ix.x >> 16) != 0;
        const VZ *Z = odd ? Zo : Ze;
        const int nsub = odd ? no : ne;
        const VZ z = Z[((size_t)s * nsub + sub) * N + (size_t)iq * NLM + ix.y];
        const double g = gval[e];
        re = fma(g, (double)z.x, re);
        im = fma(g, (double)z.y, im);
    }
    R[idx] = make_double2(scale * re, scale * im);
}

// iso[s][q] = (1/4pi) sum_lm |R_lm|^2; out is float or double.
template <typename T>
__global__ void sph_iso_kernel(const double2 *__restrict__ R, int64_t n_sq, int NR, T *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_sq) return;
    double a = 0.0;
    for (int o = 0; o < NR; ++o) {
        const double2 v = R[idx * NR + o];
        a = fma(v.x, v.x, fma(v.y, v.y, a));
    }
    out[idx] = (T)(a * 0.07957747154594767);  // 1 / (4 pi)
}

__global__ void sph_r_to_f32_kernel(const double2 *__restrict__ R, int64_t n, float2 *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] = make_float2((float)R[idx].x, (float)R[idx].y);
}

// Angular tables: T1[(l m)][itheta] = p_l^m(cos theta), T2[(m + lmax)][iphi] = e^{i m phi};
// one thread per (theta, |m|) fills the +m and -m rows.
template <typename V>
__global__ void sph_theta_table_kernel(const double *__restrict__ theta, int nt, int lmax, V *__restrict__ T1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nt * (lmax + 1)) return;
    const int it = idx / (lmax + 1), m = idx % (lmax + 1);
    double col[sph::kMaxLmax + 1];
    sph::plm_column_tab(lmax, m, cos(theta[it]), g_plm_ab, col);
    const double sgn = (m & 1) ? -1.0 : 1.0;
    for (int l = m; l <= lmax; ++l) {
        V v;
        v.x = col[l - m];
        v.y = 0;
        T1[(size_t)sph::lm_index(l, m) * nt + it] = v;
        if (m > 0) {
            v.x = sgn * col[l - m];
            T1[(size_t)sph::lm_index(l, -m) * nt + it] = v;
        }
    }
}

template <typename V>
__global__ void sph_phi_table_kernel(const double *__restrict__ phi, int np, int lmax, V *__restrict__ T2) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (2 * lmax + 1) * np) return;
    const int m = idx / np - lmax, ip = idx % np;
    double sn, cs;
    sincos(m * phi[ip], &sn, &cs);
    V v;
    v.x = cs;
    v.y = sn;
    T2[idx] = v;
}

__global__ void sph_angular_kofs_kernel(int NR, int64_t K_pad, int lmax, int nt, int np, int2 *__restrict__ kofs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K_pad) return;
    if (k < NR) {
        int l = (int)sqrtf((float)k);
        while (l * l > k) --l;
        while ((l + 1) * (l + 1) <= k) ++l;
        const int m = (int)k - l * l - l;
        kofs[k] = make_int2((int)k * nt, (m + lmax) * np);
    } else {
        kofs[k] = make_int2(NR * nt, (2 * lmax + 1) * np);
    }
}

// ------------------------------------------------------------------ FP64 two-table contraction

// C[(s, ix), n] = scale * sum_k A[m][k] Y[kofs[k].x + iy(n)] Z[kofs[k].y + iz(n)],
// the FP64 counterpart of the tensor-core contraction: 64 x 64 output tiles,
// 256 threads with 4 x 4 complex outputs each, k in steps of 16 through
// shared memory (A tile loaded, W tile generated from the two tables).
constexpr int G64_BM = 64, G64_BN = 64, G64_BK = 16;

__global__ void __launch_bounds__(256) gen_gemm64_kernel(Gemm64Args a) {
    __shared__ double2 As[G64_BK][G64_BM + 1];
    __shared__ double2 Ws[G64_BK][G64_BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * G64_BM, n0 = blockIdx.x * G64_BN;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
    // column decomposition of this thread's W loads: column n0 + (threadIdx.x % 64)
    const int wc = threadIdx.x % G64_BN, wk0 = threadIdx.x / G64_BN;  // 4 k-rows per pass
    const int64_t wn = (int64_t)n0 + wc;
    const bool wvalid = wn < a.N;
    int iy = 0, iz = 0;
    if (wvalid) {
        iz = (int)(wn % a.nz);
        iy = (int)(wn / a.nz);
        if (a.ylm) {
            int l = (int)sqrtf((float)iz);
            while (l * l > iz) --l;
            while ((l + 1) * (l + 1) <= iz) ++l;
            iy = iy * a.ystride + l;
        }
    }
    for (int64_t k0 = 0; k0 < a.K; k0 += G64_BK) {
        // A tile: 64 rows x 16 k
        for (int e = threadIdx.x; e < G64_BM * G64_BK; e += 256) {
            const int r = e / G64_BK, kk = e % G64_BK;
            const int m = m0 + r;
            const int64_t k = k0 + kk;
            As[kk][r] = (m < a.M && k < a.K) ? a.A[(size_t)m * a.lda + k] : make_double2(0.0, 0.0);
        }
        // W tile: 16 k x 64 columns
        for (int kk = wk0; kk < G64_BK; kk += 256 / G64_BN) {
            const int64_t k = k0 + kk;
            double2 w = make_double2(0.0, 0.0);
            if (wvalid && k < a.K) {
                const int2 ko = a.kofs[k];
                const double2 y = a.Y[(size_t)ko.x + iy], z = a.Z[(size_t)ko.y + iz];
                w = make_double2(y.x * z.x - y.y * z.y, y.x * z.y + y.y * z.x);
            }
            Ws[kk][wc] = w;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < G64_BK; ++kk) {
            double2 av[4], wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) wv[j] = Ws[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(av[i].x, wv[j].x, fma(-av[i].y, wv[j].y, acc[i][j].x));
                    acc[i][j].y = fma(av[i].x, wv[j].y, fma(av[i].y, wv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= a.M) continue;
        const int sidx = m / a.nx, ix = m % a.nx;
        double2 *crow = a.C + (size_t)sidx * a.nx * a.N + (size_t)ix * a.N;
        double *c2row = a.C2 ? a.C2 + (size_t)sidx * a.nx * a.N + (size_t)ix * a.N : nullptr;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t n = (int64_t)n0 + tx + 16 * j;
            if (n < a.N) {
                const double2 v = make_double2(a.scale * acc[i][j].x, a.scale * acc[i][j].y);
                crow[n] = v;
                if (c2row) c2row[n] = v.x * v.x + v.y * v.y;
            }
        }
    }
}

// ------------------------------------------------------------------ launchers

static unsigned blocks_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_sph_plm_init(cudaStream_t st) {
    sph_plm_init_kernel<<<blocks_of(kPlmTri, 256), 256, 0, st>>>();
    return cudaGetLastError();
}

cudaError_t launch_sph_radial(const PairSetDev &ps, const double *geom, const double *q, int nq, int NL, int fp64,
                              void *table, cudaStream_t st) {
    const int64_t tot = (int64_t)ps.n_pair * nq;
    if (tot == 0) return cudaSuccess;
    if (fp64)
        sph_radial_kernel<double2><<<blocks_of(tot, 128), 128, 0, st>>>(ps, geom, q, nq, NL, (double2 *)table);
    else
        sph_radial_kernel<float2><<<blocks_of(tot, 128), 128, 0, st>>>(ps, geom, q, nq, NL, (float2 *)table);
    return cudaGetLastError();
}

cudaError_t launch_sph_ypair(const PairSetDev &ps, const double *geom, int Lmax, int fp64, void *table,
                             cudaStream_t st) {
    const int64_t tot = (int64_t)ps.n_pair * (Lmax + 1);
    if (tot == 0) return cudaSuccess;
    if (fp64)
        sph_ypair_kernel<double2><<<blocks_of(tot, 128), 128, 0, st>>>(ps, geom, Lmax, (double2 *)table);
    else
        sph_ypair_kernel<float2><<<blocks_of(tot, 128), 128, 0, st>>>(ps, geom, Lmax, (float2 *)table);
    return cudaGetLastError();
}

cudaError_t launch_sph_kofs(const PairSetDev &ps, const SphParity &kp, int64_t K_pad, int nq, int NL, int NLM,
                            int2 *kofs, cudaStream_t st) {
    sph_kofs_kernel<<<blocks_of(K_pad, 256), 256, 0, st>>>(ps, kp, K_pad, nq, NL, NLM, kofs);
    return cudaGetLastError();
}

cudaError_t launch_sph_wdense(const PairSetDev &ps, const double *coef64, int SB, int S, const SphParity &kp,
                              int n_sub, const double2 *theta, int64_t K_pad, double2 *A, cudaStream_t st) {
    const int64_t tot = (int64_t)S * n_sub * K_pad;
    if (tot == 0) return cudaSuccess;
    sph_wdense_kernel<<<blocks_of(tot, 256), 256, 0, st>>>(ps, coef64, SB, S, kp, n_sub, theta, K_pad, A);
    return cudaGetLastError();
}

cudaError_t launch_sph_gaunt(const void *Ze, const void *Zo, int ne, int no, int fp64, int S, int nq, int NLM,
                             int NR, const int *goff, const int2 *gidx, const double *gval, double scale, double2 *R,
                             cudaStream_t st) {
    const int64_t tot = (int64_t)S * nq * NR;
    if (tot == 0) return cudaSuccess;
    if (fp64)
        sph_gaunt_kernel<double2><<<blocks_of(tot, 256), 256, 0, st>>>(
            (const double2 *)Ze, (const double2 *)Zo, ne, no, S, nq, NLM, NR, goff, gidx, gval, scale, R);
    else
        sph_gaunt_kernel<float2><<<blocks_of(tot, 256), 256, 0, st>>>(
            (const float2 *)Ze, (const float2 *)Zo, ne, no, S, nq, NLM, NR, goff, gidx, gval, scale, R);
    return cudaGetLastError();
}

cudaError_t launch_sph_iso(const double2 *R, int64_t n_sq, int NR, int fp64, void *out, cudaStream_t st) {
    if (n_sq == 0) return cudaSuccess;
    if (fp64)
        sph_iso_kernel<double><<<blocks_of(n_sq, 256), 256, 0, st>>>(R, n_sq, NR, (double *)out);
    else
        sph_iso_kernel<float><<<blocks_of(n_sq, 256), 256, 0, st>>>(R, n_sq, NR, (float *)out);
    return cudaGetLastError();
}

cudaError_t launch_sph_r_to_f32(const double2 *R, int64_t n, float2 *out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    sph_r_to_f32_kernel<<<blocks_of(n, 256), 256, 0, st>>>(R, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sph_angular_tables(const double *theta, int nt, const double *phi, int np, int lmax, int fp64,
                                      void *T1, void *T2, cudaStream_t st) {
    if (fp64) {
        sph_theta_table_kernel<double2><<<blocks_of((int64_t)nt * (lmax + 1), 128), 128, 0, st>>>(theta, nt, lmax,
                                                                                                  (double2 *)T1);
        sph_phi_table_kernel<double2><<<blocks_of((int64_t)(2 * lmax + 1) * np, 256), 256, 0, st>>>(
            phi, np, lmax, (double2 *)T2);
    } else {
        sph_theta_table_kernel<float2><<<blocks_of((int64_t)nt * (lmax + 1), 128), 128, 0, st>>>(theta, nt, lmax,
                                                                                                 (float2 *)T1);
        sph_phi_table_kernel<float2><<<blocks_of((int64_t)(2 * lmax + 1) * np, 256), 256, 0, st>>>(
            phi, np, lmax, (float2 *)T2);
    }
    return cudaGetLastError();
}

cudaError_t launch_sph_angular_kofs(int NR, int64_t K_pad, int lmax, int nt, int np, int2 *kofs, cudaStream_t st) {
    sph_angular_kofs_kernel<<<blocks_of(K_pad, 256), 256, 0, st>>>(NR, K_pad, lmax, nt, np, kofs);
    return cudaGetLastError();
}

cudaError_t launch_gen_gemm64(const Gemm64Args &a, cudaStream_t st) {
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    dim3 grid(blocks_of(a.N, G64_BN), blocks_of(a.M, G64_BM));
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gen_gemm64_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace scff
