// Pair-prep (Gaussian product theorem + monomial coefficients), per-axis
// Gaussian x phase tables, and the direct q-evaluation kernels (FP64/FP32).
//
// Method (Sec. "Analytic Method"): for a pair of primitive shells r1 = (A, alpha),
// r2 = (B, beta) the Gaussian product theorem (Eqs. sigmaTidbits,
// positionTidbits) gives p = alpha + beta, P = (alpha A + beta B)/p and the
// prefactor K = (pi/p)^{3/2} exp(-alpha beta |A-B|^2 / p), which is
// (2 pi)^{3/2} sigma_ij^3 exp(-r_ij^2 / (2 sigma-bar_ij^2)) of Eq. Mij with
// sigma^2 = 1/(2 alpha).  Per axis the polynomial (y + P - A)^a (y + P - B)^a'
// has binomial coefficients b_t (Eq. bCoefficients) and the Fourier integral
// turns into exp(-q^2/(4p)) sum_u i^u C^u q^u with
// C^u = sum_m b_{u+2m} sigma^{2(u+m)} (u+2m)! / (m! u! 2^m)  (Eq. Ccoefficients).
// Folding every function pair of the two shells with its contraction weights
// and T^s gives one real coefficient per (pair, monomial q_x^u q_y^v q_z^w,
// state) -- the D-tensor of Eq. DTensor contracted with T -- and
//     f_s(q) = sum_pairs exp(-q^2/4p) e^{i q.P} sum_uvw i^{u+v+w} D q^u q^v q^w.
// The factor i^n is stored as a sign in the coefficient; odd n contribute to
// the imaginary part of the polynomial.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "device_common.cuh"
#include "scff_internal.h"

namespace scff {

// ------------------------------------------------------------------ helpers

// Cartesian exponent of function j of a record type along axis ax
// (s; p: x,y,z; d: xx,xy,xz,yy,yz,zz; sp: s,x,y,z; f: xxx,xxy,...,zzz).
__host__ __device__ constexpr int fn_pow(int type, int j, int ax) {
    return type == REC_SP ? (j == 0 ? 0 : cart_pow(1, j - 1, ax)) : cart_pow(rec_lmax(type), j, ax);
}

// (u+2m)! / (m! u! 2^m), the Hermite-to-monomial factor of Eq. Ccoefficients.
__device__ __forceinline__ double herm_mono_factor(int u, int m) {
    double num = 1.0;
    for (int k = 2; k <= u + 2 * m; ++k) num *= k;
    double den = 1.0;
    for (int k = 2; k <= m; ++k) den *= k;
    for (int k = 2; k <= u; ++k) den *= k;
    for (int k = 0; k < m; ++k) den *= 2.0;
    return num / den;
}

// C^u for exponents (a, a2) along one axis, PA = P - A, PB = P - B, s2 = 1/(2p).
__device__ double c_coef(int a, int a2, int u, double PA, double PB, double s2) {
    const int deg = a + a2;
    if (u > deg) return 0.0;
    // binomial coefficients of (y+PA)^a and (y+PB)^a2 (a, a2 <= 3)
    double ea[4], eb[4];
    for (int i = 0; i <= 3; ++i) {
        ea[i] = 0.0;
        eb[i] = 0.0;
    }
    {
        double bc = 1.0;  // C(a, i) PA^(a-i)
        for (int i = 0; i <= a; ++i) {
            double pw = 1.0;
            for (int k = 0; k < a - i; ++k) pw *= PA;
            ea[i] = bc * pw;
            bc = bc * (a - i) / (i + 1);
        }
        bc = 1.0;
        for (int i = 0; i <= a2; ++i) {
            double pw = 1.0;
            for (int k = 0; k < a2 - i; ++k) pw *= PB;
            eb[i] = bc * pw;
            bc = bc * (a2 - i) / (i + 1);
        }
    }
    double c = 0.0;
    double s2pow = 1.0;
    for (int i = 0; i < u; ++i) s2pow *= s2;  // sigma^{2u}
    for (int m = 0; u + 2 * m <= deg; ++m) {
        const int t = u + 2 * m;
        double bt = 0.0;
        for (int i = 0; i <= a; ++i) {
            const int j = t - i;
            if (j >= 0 && j <= a2) bt += ea[i] * eb[j];
        }
        c += bt * s2pow * herm_mono_factor(u, m);
        s2pow *= s2;  // sigma^{2(u+m)} for the next m
    }
    return c;
}

// ------------------------------------------------------------------ pair geometry

__global__ void pair_geom_kernel(PairSetDev ps, double *__restrict__ geom) {
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= ps.n_pair) return;
    const int2 rr = ps.pair_rec[pr];
    const double a = ps.rec_alpha[rr.x], b = ps.rec_alpha[rr.y];
    const double p = a + b;
    for (int ax = 0; ax < 3; ++ax)
        geom[4 * pr + ax] = (a * ps.rec_xyz[3 * rr.x + ax] + b * ps.rec_xyz[3 * rr.y + ax]) / p;
    geom[4 * pr + 3] = 0.25 / p;
}

cudaError_t launch_pair_geom(const PairSetDev &ps, double *pair_geom, cudaStream_t st) {
    if (ps.n_pair == 0) return cudaSuccess;
    pair_geom_kernel<<<(ps.n_pair + 127) / 128, 128, 0, st>>>(ps, pair_geom);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K1 pair-prep

// One thread per (pair, monomial) row: the geometry, the prefactor K and the
// C tables are computed once (C in shared memory, indexed by the functions'
// exponents) and reused for every state.
constexpr int kPrepThreads = 128;
constexpr int kPrepStates = 8;  // states per register block

// T entries staged per block and state block: the symmetrised T^s_ij (+ T^s_ji)
// of every function pair of every pair the block's rows belong to.  A block
// holds 128 consecutive rows; a pair of degree L has (L+1)(L+2)(L+3)/6 rows and
// at most 1.6 times as many function pairs, so the block's pairs have at most
// 1.6 x 128 + 2 x 100 (the two pairs cut by the block's ends) function pairs.
constexpr int kPrepMaxFnPairs = 416;
// dynamic shared memory: the staged T, then the function-pair offsets (kPrepThreads + 1 ints)
constexpr int kPrepTsmBytes = kPrepMaxFnPairs * kPrepStates * (int)sizeof(double) + 1024;

__global__ void __launch_bounds__(kPrepThreads) pairprep_kernel(PairSetDev ps, const double *__restrict__ T,
                                                                int S, int S_pad, int SB,
                                                                double *__restrict__ coef64,
                                                                float *__restrict__ coef32) {
    __shared__ double Csm[3 * 4 * 4][kPrepThreads];  // C[ax][a][a2] of this thread's row
    extern __shared__ double Tsm[];                  // [function pair of the block][kPrepStates], then foff
    // first function pair of each of the block's pairs
    int *foff = reinterpret_cast<int *>(Tsm + kPrepMaxFnPairs * kPrepStates);
    const int64_t row0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t row = row0 + threadIdx.x;
    const bool valid = row < ps.n_rows;
    const int tid = threadIdx.x;
    auto pair_of = [&](int64_t r) {
        int L = 0;
        while (L < kMaxPairL && r >= ps.row_off[L + 1]) ++L;
        return ps.pair_off[L] + (int)((r - ps.row_off[L]) / mono_count(L));
    };
    // the block's pairs p_lo..p_lo + np - 1 and their function-pair offsets
    const int p_lo = pair_of(row0);
    const int64_t row_last = row0 + (int64_t)blockDim.x <= ps.n_rows ? row0 + blockDim.x - 1 : ps.n_rows - 1;
    const int np = pair_of(row_last) - p_lo + 1;
    if (tid < np) {
        const int2 rr = ps.pair_rec[p_lo + tid];
        foff[tid + 1] = rec_nfn(ps.rec_type[rr.x]) * rec_nfn(ps.rec_type[rr.y]);
    }
    __syncthreads();
    if (tid == 0) {
        foff[0] = 0;
        for (int t = 0; t < np; ++t) foff[t + 1] += foff[t];
    }
    __syncthreads();
    const int nfp = foff[np];
    const bool staged = nfp <= kPrepMaxFnPairs;  // else (never for s..f shells) read T from global memory

    int L = 0;
    while (L < kMaxPairL && valid && row >= ps.row_off[L + 1]) ++L;
    const int mL = mono_count(L);
    const int64_t local = valid ? row - ps.row_off[L] : 0;
    const int pr = valid ? ps.pair_off[L] + (int)(local / mL) : p_lo;
    const int m = (int)(local % mL);
    const int2 rr = ps.pair_rec[pr];
    const double al = ps.rec_alpha[rr.x], be = ps.rec_alpha[rr.y];
    const double p = al + be;
    const double s2 = 0.5 / p;
    double PA[3], PB[3], ab2 = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        const double A = ps.rec_xyz[3 * rr.x + ax], B = ps.rec_xyz[3 * rr.y + ax];
        const double P = (al * A + be * B) / p;
        PA[ax] = P - A;
        PB[ax] = P - B;
        ab2 += (A - B) * (A - B);
    }
    const double K = pow(M_PI / p, 1.5) * exp(-al * be * ab2 / p);
    const int e[3] = {mono_u(m), mono_v(m), mono_w(m)};
    const int t1 = ps.rec_type[rr.x], t2 = ps.rec_type[rr.y];
    const int l1 = rec_lmax(t1), l2 = rec_lmax(t2);
    for (int ax = 0; ax < 3; ++ax)
        for (int a = 0; a <= l1; ++a)
            for (int a2 = 0; a2 <= l2; ++a2) Csm[(ax * 4 + a) * 4 + a2][tid] = c_coef(a, a2, e[ax], PA[ax], PB[ax], s2);
    const int n1 = rec_nfn(t1), n2 = rec_nfn(t2);
    const int f1 = ps.rec_fn0[rr.x], f2 = ps.rec_fn0[rr.y];
    const int nbf = ps.nbf;
    const bool same = (rr.x == rr.y);
    const int n = e[0] + e[1] + e[2];
    const double sgn = K * ((n & 2) ? -1.0 : 1.0);  // i^n = +1, +i, -1, -i
    const double *Tmine = Tsm + (size_t)foff[pr - p_lo] * kPrepStates;
    // states in register blocks of kPrepStates: the function-pair factor
    // w_i w_j D (state-independent) is formed once per block, and each state
    // adds T^s_ij (+ T^s_ji) times it
    const size_t nn = (size_t)nbf * nbf;
    // blockIdx.y takes every gridDim.y-th block of states (more blocks in flight than rows alone give)
    for (int s0 = blockIdx.y * kPrepStates; s0 < S_pad; s0 += gridDim.y * kPrepStates) {
        const int ns = min(kPrepStates, S - s0);
        if (staged) {
            // the symmetrised T of the block's function pairs for these states, once per block
            __syncthreads();
            for (int q = tid; q < nfp * kPrepStates; q += blockDim.x) {
                const int u = q % kPrepStates, fp = q / kPrepStates;
                int t = 0, hi = np - 1;  // the pair t with foff[t] <= fp < foff[t + 1]
                while (t < hi) {
                    const int mid = (t + hi + 1) >> 1;
                    if (foff[mid] <= fp) t = mid;
                    else hi = mid - 1;
                }
                const int2 qr = ps.pair_rec[p_lo + t];
                const int m2 = rec_nfn(ps.rec_type[qr.y]);
                const int i = (fp - foff[t]) / m2, j = (fp - foff[t]) % m2;
                const int g1 = ps.rec_fn0[qr.x] + i, g2 = ps.rec_fn0[qr.y] + j;
                double tw = 0.0;
                if (u < ns) {
                    tw = T[(size_t)(s0 + u) * nn + (size_t)g1 * nbf + g2];
                    if (qr.x != qr.y) tw += T[(size_t)(s0 + u) * nn + (size_t)g2 * nbf + g1];
                }
                Tsm[q] = tw;
            }
            __syncthreads();
        }
        double acc[kPrepStates];
#pragma unroll
        for (int u = 0; u < kPrepStates; ++u) acc[u] = 0.0;
        if (ns > 0 && valid) {
            for (int i = 0; i < n1; ++i) {
                const double wi = ps.rec_w[kRecW * rr.x + i];
                const int ai = fn_pow(t1, i, 0), bi = fn_pow(t1, i, 1), ci = fn_pow(t1, i, 2);
                for (int j = 0; j < n2; ++j) {
                    const int aj = fn_pow(t2, j, 0), bj = fn_pow(t2, j, 1), cj = fn_pow(t2, j, 2);
                    const double D = Csm[(0 * 4 + ai) * 4 + aj][tid] * Csm[(1 * 4 + bi) * 4 + bj][tid] *
                                     Csm[(2 * 4 + ci) * 4 + cj][tid];
                    if (D == 0.0) continue;
                    const double w = wi * ps.rec_w[kRecW * rr.y + j] * D;
                    if (staged) {
                        const double *ts = Tmine + (size_t)(i * n2 + j) * kPrepStates;
#pragma unroll
                        for (int u = 0; u < kPrepStates; ++u)
                            if (u < ns) acc[u] = fma(ts[u], w, acc[u]);
                    } else {
                        const double *Tij = T + (size_t)s0 * nn + (size_t)(f1 + i) * nbf + (f2 + j);
                        const double *Tji = T + (size_t)s0 * nn + (size_t)(f2 + j) * nbf + (f1 + i);
#pragma unroll
                        for (int u = 0; u < kPrepStates; ++u) {
                            if (u < ns) {
                                double tw = Tij[u * nn];
                                if (!same) tw += Tji[u * nn];
                                acc[u] = fma(tw, w, acc[u]);
                            }
                        }
                    }
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int u = 0; u < kPrepStates; ++u) {
                const int s = s0 + u;
                if (s >= S_pad) break;
                const double val = sgn * acc[u];
                const size_t idx = ((size_t)(s / SB) * ps.n_rows + row) * SB + (s % SB);
                if (coef64) coef64[idx] = val;
                if (coef32) coef32[idx] = (float)val;
            }
        }
    }
}

cudaError_t pairprep_init() {
    // the staged T takes the block beyond 48 KB of shared memory: the attribute
    // is set once per device (when a context is created, or by the first launch
    // on a device that has none, e.g. through the allocation-free entry)
    constexpr int kDevs = 64;
    static bool done[kDevs] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kDevs && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(pairprep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPrepTsmBytes);
    if (e == cudaSuccess && dev >= 0 && dev < kDevs) done[dev] = true;
    return e;
}

cudaError_t launch_pairprep(const PairSetDev &ps, const double *T, int S, int SB, int S_pad,
                            double *coef64, float *coef32, int64_t *launches, cudaStream_t st) {
    if (ps.n_rows == 0) return cudaSuccess;
    const cudaError_t ei = pairprep_init();
    if (ei != cudaSuccess) return ei;
    const unsigned grid = (unsigned)((ps.n_rows + kPrepThreads - 1) / kPrepThreads);
    const unsigned sblocks = (unsigned)std::max(1, (S_pad + kPrepStates - 1) / kPrepStates);
    pairprep_kernel<<<dim3(grid, sblocks), kPrepThreads, kPrepTsmBytes, st>>>(ps, T, S, S_pad, SB, coef64, coef32);
    if (launches) ++*launches;
    return cudaGetLastError();
}

// ------------------------------------------------------------------ axis tables

template <typename V>
__global__ void axis_table_kernel(int n_pair, const double *__restrict__ geom,
                                  const double *__restrict__ qaxis, int n, int axis, V *__restrict__ table) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_pair * n) return;
    const int pr = (int)(idx / n), i = (int)(idx % n);
    const double q = qaxis[i];
    const double P = geom[4 * pr + axis], inv4p = geom[4 * pr + 3];
    double sn, cs;
    sincos(q * P, &sn, &cs);  // FP64 range reduction of the phase
    const double amp = exp(-q * q * inv4p);
    V v;
    v.x = amp * cs;
    v.y = amp * sn;
    table[idx] = v;
}

cudaError_t launch_axis_tables(const PairSetDev &ps, const double *pair_geom, const double *qaxis,
                               int n, int axis, void *table, int fp64, cudaStream_t st) {
    const int64_t tot = (int64_t)ps.n_pair * n;
    if (tot == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        axis_table_kernel<double2><<<blocks, 256, 0, st>>>(ps.n_pair, pair_geom, qaxis, n, axis,
                                                           (double2 *)table);
    else
        axis_table_kernel<float2><<<blocks, 256, 0, st>>>(ps.n_pair, pair_geom, qaxis, n, axis,
                                                          (float2 *)table);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pure shells -> Cartesian T

__global__ void pure_to_cart_kernel(int S, int ncart, int nuser, const int32_t *__restrict__ idx,
                                    const double *__restrict__ c, const double *__restrict__ Tu,
                                    double *__restrict__ Tc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nn = (int64_t)ncart * ncart;
    if (t >= (int64_t)S * nn) return;
    const int s = (int)(t / nn);
    const int a = (int)((t % nn) / ncart), b = (int)(t % ncart);
    const double *T = Tu + (size_t)s * nuser * nuser;
    double v = 0.0;
    for (int e = 0; e < kMaxPureTerms; ++e) {
        const int i = idx[a * kMaxPureTerms + e];
        if (i < 0) break;
        double row = 0.0;
        for (int f = 0; f < kMaxPureTerms; ++f) {
            const int j = idx[b * kMaxPureTerms + f];
            if (j < 0) break;
            row = fma(c[b * kMaxPureTerms + f], T[(size_t)i * nuser + j], row);
        }
        v = fma(c[a * kMaxPureTerms + e], row, v);
    }
    Tc[t] = v;
}

cudaError_t launch_pure_to_cart(int S, int ncart, int nuser, const int32_t *idx, const double *c,
                                const double *Tu, double *Tc, cudaStream_t st) {
    const int64_t tot = (int64_t)S * ncart * ncart;
    if (tot == 0) return cudaSuccess;
    pure_to_cart_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(S, ncart, nuser, idx, c, Tu, Tc);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K2 direct q-evaluation

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };

constexpr int kDirectThreads = 128;
constexpr int kChunkBytes = 8192;
constexpr int kMaxChunkPairs = kChunkBytes / 32;  // most pairs of a staged chunk (FP64, SB = 4, L = 0)

struct DirectParams {
    PairSetDev ps;
    const void *coef;
    const void *gx, *gy, *gz;
    const double *qax, *qay, *qaz;
    int nx, ny, nz;
    const double *qlist;
    const double *pair_geom;
    int64_t nq;      // points computed
    int64_t nq_out;  // points of the output grid (state stride); > nq: mirror into the rest
    int S;
    double scale;
    void *f, *f2;
    int *err;
    int part;  // kPartContinue: start from the raw sums in f; kPartFinal: write scaled f and |f|^2
    // product grid with nz a multiple of the block size: every block's points
    // share (ix, iy), so the x and y table factors of a pair are the same for
    // the whole block and are formed once per block into shared memory
    int xy_uniform;
};

// Pair classes of degree >= kHighClass (pairs with an f shell) run in a second
// launch of their own, so that the registers their long unrolled monomial
// sums need do not lower the occupancy of the common s/p/d classes.  The
// first launch leaves unscaled sums in f and the second continues from them.
constexpr int kHighClass = 5;
constexpr int kPartContinue = 1;
constexpr int kPartFinal = 2;

// Gaussian x phase factor of one pair at this thread's q point.
template <typename R, bool LIST>
__device__ __forceinline__ typename Cplx<R>::T pair_factor(const DirectParams &p, int pr, int ix, int iy,
                                                           int iz, double qx, double qy, double qz, double q2) {
    using V = typename Cplx<R>::T;
    V g;
    if constexpr (!LIST) {
        const V a = static_cast<const V *>(p.gx)[(int64_t)pr * p.nx + ix];
        const V b = static_cast<const V *>(p.gy)[(int64_t)pr * p.ny + iy];
        const V c = static_cast<const V *>(p.gz)[(int64_t)pr * p.nz + iz];
        const R abx = a.x * b.x - a.y * b.y, aby = a.x * b.y + a.y * b.x;
        g.x = abx * c.x - aby * c.y;
        g.y = abx * c.y + aby * c.x;
    } else {
        const double2 pxy = reinterpret_cast<const double2 *>(p.pair_geom)[2 * pr];
        const double2 pzw = reinterpret_cast<const double2 *>(p.pair_geom)[2 * pr + 1];
        const double ph = qx * pxy.x + qy * pxy.y + qz * pzw.x;
        if constexpr (sizeof(R) == 8) {
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double amp = exp(-q2 * pzw.y);
            g.x = amp * cs;
            g.y = amp * sn;
        } else {
            // FP64 range reduction to [-pi, pi], then FP32 evaluation.
            const double k = rint(ph * 0.15915494309189535);
            double r = fma(-k, 6.283185307179586, ph);
            r = fma(-k, 2.4492935982947064e-16, r);
            float sn, cs;
            sincosf((float)r, &sn, &cs);
            const float amp = expf((float)(-q2 * pzw.y));
            g.x = amp * cs;
            g.y = amp * sn;
        }
    }
    return g;
}

// Per-state accumulators.  FP32 sums pairs in short runs of kFlushPairs
// terms and folds each run into a (hi, lo) double-float pair with the
// error-free TwoSum transformation (Knuth), which keeps the sum over 10^4
// pairs at FP64-like accuracy; FP64 accumulates directly.
constexpr int kFlushPairs = 16;

template <typename R, int SB> struct Acc {
    R pr[SB], pi[SB];  // running partial sums
    R hr[SB], hi[SB], lr[SB], li[SB];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < SB; ++j) pr[j] = pi[j] = hr[j] = hi[j] = lr[j] = li[j] = R(0);
    }
    __device__ __forceinline__ static void two_sum(R &h, R &l, R x) {
        const R s = h + x;
        const R bb = s - h;
        const R err = (h - (s - bb)) + (x - bb);
        h = s;
        l += err;
    }
    __device__ __forceinline__ void flush() {
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int j = 0; j < SB; ++j) {
                two_sum(hr[j], lr[j], pr[j]);
                two_sum(hi[j], li[j], pi[j]);
                pr[j] = pi[j] = R(0);
            }
        }
    }
    __device__ __forceinline__ R re(int j) const { return sizeof(R) == 4 ? hr[j] + lr[j] : pr[j]; }
    __device__ __forceinline__ R im(int j) const { return sizeof(R) == 4 ? hi[j] + li[j] : pi[j]; }
    // starts state j from the sum (r, i) of an earlier launch
    __device__ __forceinline__ void set(int j, R r, R i) {
        if constexpr (sizeof(R) == 4) {
            hr[j] = r;
            hi[j] = i;
        } else {
            pr[j] = r;
            pi[j] = i;
        }
    }
};

// Packed FP32 pairs (Blackwell's f32x2 arithmetic): each instruction does two
// independent FP32 operations, each rounded exactly as its scalar form, so
// the packed kernels give bitwise the scalar results with half the issued
// arithmetic instructions.
using f2p = unsigned long long;  // two FP32 values in one 64-bit register pair (low word first)
__device__ __forceinline__ f2p pk(float lo, float hi) {
    f2p d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ float pk_lo(f2p v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float pk_hi(f2p v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The FP32 accumulators of Acc<float, SB> with states packed in pairs:
// state 2j in the low word and 2j + 1 in the high word of element j.  The
// same operations in the same order as Acc, so bitwise the same sums.
template <int SB> struct AccP {
    static_assert(SB % 2 == 0, "states in pairs");
    static constexpr int H = SB / 2;
    f2p pr[H], pi[H], hr[H], hi[H], lr[H], li[H];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int j = 0; j < H; ++j) pr[j] = pi[j] = hr[j] = hi[j] = lr[j] = li[j] = 0ull;
    }
    __device__ __forceinline__ static void two_sum(f2p &h, f2p &l, f2p x) {
        const f2p s = add2(h, x);
        const f2p bb = sub2(s, h);
        const f2p err = add2(sub2(h, sub2(s, bb)), sub2(x, bb));
        h = s;
        l = add2(l, err);
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int j = 0; j < H; ++j) {
            two_sum(hr[j], lr[j], pr[j]);
            two_sum(hi[j], li[j], pi[j]);
            pr[j] = pi[j] = 0ull;
        }
    }
    __device__ __forceinline__ float re(int j) const {
        return (j & 1) ? pk_hi(hr[j >> 1]) + pk_hi(lr[j >> 1]) : pk_lo(hr[j >> 1]) + pk_lo(lr[j >> 1]);
    }
    __device__ __forceinline__ float im(int j) const {
        return (j & 1) ? pk_hi(hi[j >> 1]) + pk_hi(li[j >> 1]) : pk_lo(hi[j >> 1]) + pk_lo(li[j >> 1]);
    }
    __device__ __forceinline__ void set(int j, float r, float i) {
        const int h = j >> 1;
        hr[h] = (j & 1) ? pk(pk_lo(hr[h]), r) : pk(r, pk_hi(hr[h]));
        hi[h] = (j & 1) ? pk(pk_lo(hi[h]), i) : pk(i, pk_hi(hi[h]));
    }
};

// Slots of the collapsed sums of a pair of degree L (the VEC variant): for
// w < L both parities of u + v + w occur (slots 2w and 2w + 1), for w = L only
// u = v = 0, of the parity of L (slot 2L): 2L + 1 slots.
__host__ __device__ constexpr int collapse_slot(int L, int w, int odd) { return w < L ? 2 * w + odd : 2 * L; }
__host__ __device__ constexpr int collapse_w(int L, int t) { return t < 2 * L ? t / 2 : L; }
__host__ __device__ constexpr bool collapse_odd(int L, int t) { return t < 2 * L ? (t & 1) != 0 : (L & 1) != 0; }

// VEC: the per-state coefficients of a monomial are read four per 16-byte
// shared-memory load (a pair's rows are SB floats, so each starts 16-byte
// aligned).  It pays where the block's points share (ix, iy) (10-heavy-atom
// job, 128^3: 105 -> 90 ms) and costs where three table entries per pair
// come from global memory (benzene-scale job, 64^3: 5.2 -> 5.5 ms), so the
// launcher picks it for the first case only.
// NOUNI: compiled for grids whose blocks do not share (ix, iy), without the
// shared-row branches at all (the runtime test alone, although uniform across
// the block, took the 64^3 FP32 job from 3.8 to 5.1 ms).
template <typename R, int SB, int L, bool LIST, bool VEC, bool NOUNI, typename AccT>
__device__ __forceinline__ void consume_chunk(const DirectParams &p, const R *__restrict__ cbuf,
                                              const R *__restrict__ bbuf,
                                              const typename Cplx<R>::T *__restrict__ gxy, int pr0,
                                              int np, const R (&px)[kMaxPairL + 1], const R (&py)[kMaxPairL + 1], const R (&pz)[kMaxPairL + 1],
                                              int ix, int iy, int iz, double qx, double qy, double qz,
                                              double q2, AccT &acc) {
    constexpr int mL = mono_count(L);
    using V = typename Cplx<R>::T;
    for (int i = 0; i < np; ++i) {
        V g;
        if (!LIST && !NOUNI && p.xy_uniform) {
            const V a = gxy[i];
            const V c = static_cast<const V *>(p.gz)[(int64_t)(pr0 + i) * p.nz + iz];
            g.x = a.x * c.x - a.y * c.y;
            g.y = a.x * c.y + a.y * c.x;
        } else {
            g = pair_factor<R, LIST>(p, pr0 + i, ix, iy, iz, qx, qy, qz, q2);
        }
        if constexpr (VEC) {
            // the block's x and y powers are already folded into the chunk's
            // collapsed sums (see run_class): E and O are polynomials in q_z
            // alone, 2L+1 terms per pair instead of (L+1)(L+2)(L+3)/6.  States
            // are packed in pairs (AccP): every FMA below does two states.
            static_assert(sizeof(R) == 4 && SB % 4 == 0, "four FP32 sums per load");
            constexpr int NS = 2 * L + 1, H = SB / 2;
            f2p E[H], O[H];
#pragma unroll
            for (int j = 0; j < H; ++j) E[j] = O[j] = 0ull;
            const R *bb = bbuf + (size_t)i * NS * SB;
            static_for<NS>([&](auto T) {
                constexpr int t = decltype(T)::value;
                constexpr int w = collapse_w(L, t);
                const f2p zw = pk(pz[w], pz[w]);
                const float4 *b4 = reinterpret_cast<const float4 *>(bb + t * SB);
#pragma unroll
                for (int jj = 0; jj < SB / 4; ++jj) {
                    const float4 cv = b4[jj];
                    const f2p c01 = pk(cv.x, cv.y), c23 = pk(cv.z, cv.w);
                    if constexpr (collapse_odd(L, t)) {
                        O[2 * jj] = fma2(c01, zw, O[2 * jj]);
                        O[2 * jj + 1] = fma2(c23, zw, O[2 * jj + 1]);
                    } else {
                        E[2 * jj] = fma2(c01, zw, E[2 * jj]);
                        E[2 * jj + 1] = fma2(c23, zw, E[2 * jj + 1]);
                    }
                }
            });
            const f2p gx = pk(g.x, g.x), gy = pk(g.y, g.y), ngy = pk(-g.y, -g.y);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                acc.pr[j] = fma2(gx, E[j], acc.pr[j]);
                if constexpr (L != 0) {  // s-s pairs have no odd monomial
                    acc.pr[j] = fma2(ngy, O[j], acc.pr[j]);
                    acc.pi[j] = fma2(gx, O[j], acc.pi[j]);
                }
                acc.pi[j] = fma2(gy, E[j], acc.pi[j]);
            }
        } else if constexpr (sizeof(R) == 4) {
            // every monomial of the pair, states packed in pairs (AccP)
            constexpr int H = SB / 2;
            f2p E[H], O[H];
#pragma unroll
            for (int j = 0; j < H; ++j) E[j] = O[j] = 0ull;
            const R *c = cbuf + (size_t)i * mL * SB;
            static_for<mL>([&](auto M) {
                constexpr int m = decltype(M)::value;
                constexpr int u = mono_u(m), v = mono_v(m), w = mono_w(m);
                const R mono = px[u] * py[v] * pz[w];
                const f2p mo = pk(mono, mono);
                const float2 *c2 = reinterpret_cast<const float2 *>(c + m * SB);
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    const float2 cv = c2[j];
                    if constexpr (((u + v + w) & 1) != 0)
                        O[j] = fma2(pk(cv.x, cv.y), mo, O[j]);
                    else
                        E[j] = fma2(pk(cv.x, cv.y), mo, E[j]);
                }
            });
            const f2p gx = pk(g.x, g.x), gy = pk(g.y, g.y), ngy = pk(-g.y, -g.y);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                acc.pr[j] = fma2(gx, E[j], acc.pr[j]);
                if constexpr (L != 0) {  // s-s pairs have no odd monomial
                    acc.pr[j] = fma2(ngy, O[j], acc.pr[j]);
                    acc.pi[j] = fma2(gx, O[j], acc.pi[j]);
                }
                acc.pi[j] = fma2(gy, E[j], acc.pi[j]);
            }
        } else {
            R E[SB], O[SB];
#pragma unroll
            for (int j = 0; j < SB; ++j) E[j] = O[j] = R(0);
            const R *c = cbuf + (size_t)i * mL * SB;
            static_for<mL>([&](auto M) {
                constexpr int m = decltype(M)::value;
                constexpr int u = mono_u(m), v = mono_v(m), w = mono_w(m);
                const R mono = px[u] * py[v] * pz[w];
#pragma unroll
                for (int j = 0; j < SB; ++j) {
                    if constexpr (((u + v + w) & 1) != 0)
                        O[j] = fma(c[m * SB + j], mono, O[j]);
                    else
                        E[j] = fma(c[m * SB + j], mono, E[j]);
                }
            });
            if constexpr (L == 0) {
                // s-s pairs have no odd monomial: f += g E
#pragma unroll
                for (int j = 0; j < SB; ++j) {
                    acc.pr[j] = fma(g.x, E[j], acc.pr[j]);
                    acc.pi[j] = fma(g.y, E[j], acc.pi[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < SB; ++j) {
                    acc.pr[j] = fma(g.x, E[j], acc.pr[j]);
                    acc.pr[j] = fma(-g.y, O[j], acc.pr[j]);
                    acc.pi[j] = fma(g.x, O[j], acc.pi[j]);
                    acc.pi[j] = fma(g.y, E[j], acc.pi[j]);
                }
            }
        }
        if ((i % kFlushPairs) == kFlushPairs - 1) acc.flush();
    }
    acc.flush();
}

// Runs one pair class through a double-buffered bulk-copy pipeline.  Returns
// false (uniformly across the block) when a wait timed out.
template <typename R, int SB, int L, bool LIST, bool VEC, bool NOUNI, typename AccT>
__device__ __forceinline__ bool run_class(const DirectParams &p, R *buf0, R *buf1, R *bbuf, typename Cplx<R>::T *gxy,
                                          int bx, int by, uint64_t *bars,
                                          uint32_t &phase, int sblk, const R (&px)[kMaxPairL + 1],
                                          const R (&py)[kMaxPairL + 1], const R (&pz)[kMaxPairL + 1], int ix, int iy, int iz, double qx, double qy,
                                          double qz, double q2, AccT &acc) {
    constexpr int mL = mono_count(L);
    constexpr int pair_bytes = mL * SB * (int)sizeof(R);
    static_assert(pair_bytes <= kChunkBytes, "one pair's coefficients must fit a staging buffer");
    static_assert(pair_bytes % 16 == 0, "bulk copies move multiples of 16 bytes");
    constexpr int npc = kChunkBytes / pair_bytes;
    static_assert(npc <= kMaxChunkPairs, "pair factors of a chunk must fit their shared array");
    const int pbeg = p.ps.pair_off[L], pend = p.ps.pair_off[L + 1];
    const int npairs = pend - pbeg;
    if (npairs <= 0) return true;
    const int nchunks = (npairs + npc - 1) / npc;
    const R *base = static_cast<const R *>(p.coef) +
                    ((size_t)sblk * p.ps.n_rows + (size_t)p.ps.row_off[L]) * SB;
    R *bufs[2] = {buf0, buf1};
    auto issue = [&](int c) {
        const int n = min(npc, npairs - c * npc);
        const uint32_t bytes = (uint32_t)(n * pair_bytes);
        mbar_arrive_expect_tx(&bars[c & 1], bytes);
        bulk_g2s(bufs[c & 1], base + (size_t)c * npc * mL * SB, bytes, &bars[c & 1]);
    };
    if (threadIdx.x == 0) {
        issue(0);
        if (nchunks > 1) issue(1);
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        const bool got = mbar_wait(&bars[b], (phase >> b) & 1u);
        phase ^= (1u << b);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        const int n = min(npc, npairs - c * npc);
        if (!LIST && !NOUNI && p.xy_uniform) {
            // the block's x and y factors of this chunk's pairs, once per block
            using V = typename Cplx<R>::T;
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                const int pr = pbeg + c * npc + t;
                const V a = static_cast<const V *>(p.gx)[(int64_t)pr * p.nx + bx];
                const V bb = static_cast<const V *>(p.gy)[(int64_t)pr * p.ny + by];
                V v;
                v.x = a.x * bb.x - a.y * bb.y;
                v.y = a.x * bb.y + a.y * bb.x;
                gxy[t] = v;
            }
            if constexpr (VEC) {
                // Collapsed sums of the chunk (x and y fixed for the block):
                //   B[pair][t][s] = sum_{u,v} D^s_{pair,(u,v,w)} q_x^u q_y^v over the
                // (u, v) of slot t (collapse_slot: one slot per w and parity of
                // u + v + w), so that E_s and O_s are sums of q_z^w B[t][s].
                constexpr int NS = 2 * L + 1;
                R bx_[kMaxPairL + 1], by_[kMaxPairL + 1];
                bx_[0] = by_[0] = R(1);
                const R qxb = (R)p.qax[bx], qyb = (R)p.qay[by];
#pragma unroll
                for (int k = 1; k <= kMaxPairL; ++k) {
                    bx_[k] = bx_[k - 1] * qxb;
                    by_[k] = by_[k - 1] * qyb;
                }
                // one thread per (pair, state): every slot's sum at once, each over
                // its monomials in increasing order
                const R *cb = bufs[b];
                for (int e = threadIdx.x; e < n * SB; e += blockDim.x) {
                    const int js = e % SB, i = e / SB;
                    const R *c = cb + (size_t)i * mL * SB + js;
                    R sum[NS];
#pragma unroll
                    for (int t = 0; t < NS; ++t) sum[t] = R(0);
                    static_for<mL>([&](auto M) {
                        constexpr int m = decltype(M)::value;
                        constexpr int u = mono_u(m), v = mono_v(m), w = mono_w(m);
                        constexpr int tm = collapse_slot(L, w, (u + v + w) & 1);
                        sum[tm] = fma(c[m * SB], bx_[u] * by_[v], sum[tm]);
                    });
#pragma unroll
                    for (int t = 0; t < NS; ++t) bbuf[((size_t)i * NS + t) * SB + js] = sum[t];
                }
            }
            __syncthreads();
        }
        consume_chunk<R, SB, L, LIST, VEC, NOUNI>(p, bufs[b], bbuf, gxy, pbeg + c * npc, n, px, py, pz, ix, iy, iz, qx,
                                                  qy, qz, q2, acc);
        __syncthreads();
        if (threadIdx.x == 0 && c + 2 < nchunks) issue(c + 2);
    }
    return ok;
}

// Blocks per SM the VEC variant (block-shared rows, collapsed sums) is
// compiled for: its registers allow 5 with 8 states, 4 with 12, 3 with 16.
template <int SB, bool VEC> constexpr int direct_min_blocks() { return !VEC ? 1 : SB <= 8 ? 5 : SB <= 12 ? 4 : 3; }

template <typename R, int SB, bool LIST, bool HIGH, bool VEC = false, bool NOUNI = false>
__global__ void __launch_bounds__(kDirectThreads, (direct_min_blocks<SB, VEC>())) direct_kernel(DirectParams p) {
    __shared__ __align__(128) unsigned char smem[2 * kChunkBytes];
    // (VEC) the chunk's collapsed sums: at most the size of its coefficients
    __shared__ __align__(16) unsigned char bsm[VEC ? kChunkBytes : 16];
    __shared__ __align__(16) typename Cplx<R>::T gxy[kMaxChunkPairs];
    __shared__ __align__(8) uint64_t bars[2];
    R *buf0 = reinterpret_cast<R *>(smem);
    R *buf1 = reinterpret_cast<R *>(smem + kChunkBytes);
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbarrier_init();
    }
    __syncthreads();

    const int64_t q = (int64_t)blockIdx.x * kDirectThreads + threadIdx.x;
    const bool valid = q < p.nq;
    const int64_t qq = valid ? q : 0;
    const int sblk = blockIdx.y;
    int ix = 0, iy = 0, iz = 0;
    double qx, qy, qz;
    if constexpr (LIST) {
        qx = p.qlist[3 * qq];
        qy = p.qlist[3 * qq + 1];
        qz = p.qlist[3 * qq + 2];
    } else {
        const int64_t nyz = (int64_t)p.ny * p.nz;
        ix = (int)(qq / nyz);
        iy = (int)((qq / p.nz) % p.ny);
        iz = (int)(qq % p.nz);
        qx = p.qax[ix];
        qy = p.qay[iy];
        qz = p.qaz[iz];
    }
    const double q2 = qx * qx + qy * qy + qz * qz;
    // (ix, iy) of the block's first point: the block's own when xy_uniform
    int bx = 0, by = 0;
    if constexpr (!LIST) {
        const int64_t q0 = (int64_t)blockIdx.x * kDirectThreads;
        bx = (int)(q0 / ((int64_t)p.ny * p.nz));
        by = (int)((q0 / p.nz) % p.ny);
    }
    R px[kMaxPairL + 1], py[kMaxPairL + 1], pz[kMaxPairL + 1];
    px[0] = py[0] = pz[0] = R(1);
#pragma unroll
    for (int k = 1; k <= kMaxPairL; ++k) {
        px[k] = px[k - 1] * (R)qx;
        py[k] = py[k - 1] * (R)qy;
        pz[k] = pz[k - 1] * (R)qz;
    }
    using V = typename Cplx<R>::T;
    V *f = static_cast<V *>(p.f);
    // FP32 keeps its states packed in pairs (f32x2 arithmetic)
    std::conditional_t<sizeof(R) == 4, AccP<SB>, Acc<R, SB>> acc;
    acc.zero();
    if ((p.part & kPartContinue) && valid) {
#pragma unroll
        for (int j = 0; j < SB; ++j) {
            const int s = sblk * SB + j;
            if (s < p.S) {
                const V v = f[(size_t)s * p.nq_out + q];
                acc.set(j, v.x, v.y);
            }
        }
    }

    uint32_t phase = 0;
    bool ok = true;
    auto run = [&](auto LC) {
        constexpr int L = decltype(LC)::value;
        if (ok)
            ok = run_class<R, SB, L, LIST, VEC, NOUNI>(p, buf0, buf1, reinterpret_cast<R *>(bsm), gxy, bx, by, bars, phase,
                                                       sblk, px, py, pz, ix, iy, iz,
                                           qx, qy, qz, q2, acc);
    };
    if constexpr (HIGH) {
        static_for<kMaxPairL + 1 - kHighClass>([&](auto I) {
            run(std::integral_constant<int, kHighClass + decltype(I)::value>{});
        });
    } else {
        static_for<kHighClass>([&](auto I) { run(I); });
    }
    if (!ok) {
        if (threadIdx.x == 0) flag_error(p.err, kDevErrTimeout);
        return;
    }
    if (!valid) return;
    R *f2 = static_cast<R *>(p.f2);
    const bool final_part = (p.part & kPartFinal) != 0;
    const R sc = final_part ? (R)p.scale : R(1);
#pragma unroll
    for (int j = 0; j < SB; ++j) {
        const int s = sblk * SB + j;
        if (s < p.S) {
            V v;
            v.x = sc * acc.re(j);
            v.y = sc * acc.im(j);
            f[(size_t)s * p.nq_out + q] = v;
            if (f2 && final_part) f2[(size_t)s * p.nq_out + q] = v.x * v.x + v.y * v.y;
            // f(-q) = conj(f(q)): the mirrored point of an antisymmetric grid
            const int64_t qm = p.nq_out - 1 - q;
            if (p.nq_out > p.nq && qm != q && final_part) {
                V w;
                w.x = v.x;
                w.y = -v.y;
                f[(size_t)s * p.nq_out + qm] = w;
                if (f2) f2[(size_t)s * p.nq_out + qm] = v.x * v.x + v.y * v.y;
            }
        }
    }
}

template <typename R, int SB>
static cudaError_t launch_direct_t(const DirectArgs &a, bool list, int64_t *launches, cudaStream_t st) {
    DirectParams p;
    p.ps = *a.ps;
    p.coef = a.coef;
    p.gx = a.gx;
    p.gy = a.gy;
    p.gz = a.gz;
    p.qax = a.qax;
    p.qay = a.qay;
    p.qaz = a.qaz;
    p.nx = a.nx;
    p.ny = a.ny;
    p.nz = a.nz;
    p.qlist = a.qlist;
    p.pair_geom = a.pair_geom;
    p.nq = a.nq;
    p.nq_out = a.nq_out > 0 ? a.nq_out : a.nq;
    p.S = a.S;
    p.scale = a.scale;
    p.f = a.f;
    p.f2 = a.f2;
    p.err = a.err_flag;
    p.xy_uniform = (!list && a.nz > 0 && a.nz % kDirectThreads == 0) ? 1 : 0;
    const int nsb = (a.S + SB - 1) / SB;
    dim3 grid((unsigned)((a.nq + kDirectThreads - 1) / kDirectThreads), (unsigned)nsb);
    const bool has_low = a.ps->pair_off[kHighClass] > 0;
    const bool has_high = a.ps->pair_off[kMaxPairL + 1] > a.ps->pair_off[kHighClass];
    if (has_low || !has_high) {
        p.part = has_high ? 0 : kPartFinal;
        // the collapsed sums and vector loads for FP32 blocks on block-shared
        // rows (not for the f classes, which need more registers)
        constexpr bool kVec = sizeof(R) == 4 && SB % 4 == 0;
        if (list)
            direct_kernel<R, SB, true, false><<<grid, kDirectThreads, 0, st>>>(p);
        else if (kVec && p.xy_uniform)
            direct_kernel<R, SB, false, false, kVec><<<grid, kDirectThreads, 0, st>>>(p);
        else if (!p.xy_uniform)
            direct_kernel<R, SB, false, false, false, true><<<grid, kDirectThreads, 0, st>>>(p);
        else
            direct_kernel<R, SB, false, false><<<grid, kDirectThreads, 0, st>>>(p);
        if (launches) ++*launches;
    }
    if (has_high) {
        p.part = kPartFinal | (has_low ? kPartContinue : 0);
        if (list)
            direct_kernel<R, SB, true, true><<<grid, kDirectThreads, 0, st>>>(p);
        else if (!p.xy_uniform)
            direct_kernel<R, SB, false, true, false, true><<<grid, kDirectThreads, 0, st>>>(p);
        else
            direct_kernel<R, SB, false, true><<<grid, kDirectThreads, 0, st>>>(p);
        if (launches) ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_direct(const DirectArgs &a, int fp64, int list_mode, int64_t *launches, cudaStream_t st) {
    if (a.nq == 0) return cudaSuccess;
    cudaError_t e;
    if (fp64) {
        if (a.SB == 4)
            e = launch_direct_t<double, 4>(a, list_mode != 0, launches, st);
        else if (a.SB == 8)
            e = launch_direct_t<double, 8>(a, list_mode != 0, launches, st);
        else if (a.SB == 12)
            e = launch_direct_t<double, 12>(a, list_mode != 0, launches, st);
        else
            return cudaErrorInvalidValue;
    } else {
        if (a.SB == 8)
            e = launch_direct_t<float, 8>(a, list_mode != 0, launches, st);
        else if (a.SB == 12)
            e = launch_direct_t<float, 12>(a, list_mode != 0, launches, st);
        else if (a.SB == 16)
            e = launch_direct_t<float, 16>(a, list_mode != 0, launches, st);
        else
            return cudaErrorInvalidValue;
    }
    return e;
}

}  // namespace scff

namespace scff {

// ------------------------------------------------------------------ pair screening bounds

// bound[pair][s] >= max over |q| <= qmax of |term of this pair for state s|:
// |G| = exp(-|q|^2/4p) and |q_x^u q_y^v q_z^w| <= |q|^n (n = u+v+w), so
// |term| <= sum_m |c_m| sup_{r <= qmax} r^n exp(-r^2/4p); the supremum sits at
// r = sqrt(2pn) (or at qmax when that is closer).
// Everything in FP64 from the FP64 coefficients; the result is raised by a
// relative 1e-12, far above the rounding of this short sum of positive terms.
__global__ void pair_bound_kernel(PairSetDev ps, const double *__restrict__ coef64, int SB, int S, double qmax,
                                  double *__restrict__ bound) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ps.n_pair * S) return;
    const int pr = (int)(idx / S), s = (int)(idx % S);
    int L = 0;
    while (L < kMaxPairL && pr >= ps.pair_off[L + 1]) ++L;
    const int2 rr = ps.pair_rec[pr];
    const double p = ps.rec_alpha[rr.x] + ps.rec_alpha[rr.y];
    double sup[kMaxPairL + 1];
    for (int n = 0; n <= kMaxPairL; ++n) {
        if (n == 0) {
            sup[n] = 1.0;
        } else {
            const double r = fmin(sqrt(2.0 * p * n), qmax);
            sup[n] = pow(r, n) * exp(-r * r / (4.0 * p));
        }
    }
    const int mL = mono_count(L);
    const int64_t row0 = ps.row_off[L] + (int64_t)(pr - ps.pair_off[L]) * mL;
    const double *cs = coef64 + ((size_t)(s / SB) * ps.n_rows) * SB + (s % SB);
    double b = 0.0;
    for (int m = 0; m < mL; ++m) b += fabs(cs[(size_t)(row0 + m) * SB]) * sup[mono_u(m) + mono_v(m) + mono_w(m)];
    bound[idx] = b * (1.0 + 1e-12);
}

cudaError_t launch_pair_bounds(const PairSetDev &ps, const double *coef64, int SB, int S, double qmax, double *bound,
                               cudaStream_t st) {
    const int64_t tot = (int64_t)ps.n_pair * S;
    if (tot == 0) return cudaSuccess;
    pair_bound_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ps, coef64, SB, S, qmax, bound);
    return cudaGetLastError();
}

}  // namespace scff
