// Internal interface of the spherical method (kernels_sph.cu, spherical.cpp).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "scff_internal.h"

namespace scff {

// FP64 two-table contraction (see gen_gemm64_kernel):
//   C[(s, ix), n] = scale * sum_k A[m][k] Y[kofs[k].x + iy(n)] Z[kofs[k].y + iz(n)],
// m = s * nx + ix < M, with the column rule of the tensor-core path
// (ylm = 0: iy = n / nz, iz = n % nz; ylm = 1: iz = n % nz = LM,
// iy = (n / nz) * ystride + floor(sqrt(LM))).  C is [S][nx][N], C2 = |C|^2 or null.
struct Gemm64Args {
    const double2 *A;
    int64_t lda, K;
    int M, nx;
    const double2 *Y, *Z;
    const int2 *kofs;
    int nz, ylm, ystride;
    int64_t N;
    double scale;
    double2 *C;
    double *C2;
};
cudaError_t launch_gen_gemm64(const Gemm64Args &a, cudaStream_t st);

// One parity job of the spherical contraction: the rows k = (pair, n) with
// n of parity `par`, numbered class by class and pair by pair; off[L] is the
// first k of class L (off[kNumClasses] = the job's K).
struct SphParity {
    int64_t off[kNumClasses + 1];
    int par;
};
// Rows n of parity par of a pair of class L: n = par, par + 2, ..., <= L.
__host__ __device__ inline int sph_parity_count(int L, int par) { return L >= par ? (L - par) / 2 + 1 : 0; }
// Index of (lambda, mu) among the harmonics of lambda's parity (lambda
// ascending, mu = -lambda..lambda): even lambda = 2a gives a (2a - 1) +
// lambda + mu, odd lambda = 2a + 1 gives a (2a + 1) + lambda + mu.
__host__ __device__ inline int sph_parity_sub(int lam, int mu) {
    const int a = lam / 2;
    return ((lam & 1) ? a * (2 * a + 1) : a * (2 * a - 1)) + lam + mu;
}
// Harmonics (lambda <= lam) of parity par.
__host__ __device__ inline int sph_parity_rows(int lam, int par) {
    int n = 0;
    for (int l = par; l <= lam; l += 2) n += 2 * l + 1;
    return n;
}

// Table and contraction kernels of the spherical method; `fp64` selects
// double2 (else float2) tables.
// Fills the device table of Legendre recurrence coefficients (once per device).
cudaError_t launch_sph_plm_init(cudaStream_t st);
cudaError_t launch_sph_radial(const PairSetDev &ps, const double *geom, const double *q, int nq, int NL, int fp64,
                              void *table, cudaStream_t st);
cudaError_t launch_sph_ypair(const PairSetDev &ps, const double *geom, int Lmax, int fp64, void *table,
                             cudaStream_t st);
cudaError_t launch_sph_kofs(const PairSetDev &ps, const SphParity &kp, int64_t K_pad, int nq, int NL, int NLM,
                            int2 *kofs, cudaStream_t st);
cudaError_t launch_sph_wdense(const PairSetDev &ps, const double *coef64, int SB, int S, const SphParity &kp,
                              int n_sub, const double2 *theta, int64_t K_pad, double2 *A, cudaStream_t st);
cudaError_t launch_sph_gaunt(const void *Ze, const void *Zo, int ne, int no, int fp64, int S, int nq, int NLM,
                             int NR, const int *goff, const int2 *gidx, const double *gval, double scale, double2 *R,
                             cudaStream_t st);
cudaError_t launch_sph_iso(const double2 *R, int64_t n_sq, int NR, int fp64, void *out, cudaStream_t st);
cudaError_t launch_sph_r_to_f32(const double2 *R, int64_t n, float2 *out, cudaStream_t st);
cudaError_t launch_sph_angular_tables(const double *theta, int nt, const double *phi, int np, int lmax, int fp64,
                                      void *T1, void *T2, cudaStream_t st);
cudaError_t launch_sph_angular_kofs(int NR, int64_t K_pad, int lmax, int nt, int np, int2 *kofs, cudaStream_t st);

}  // namespace scff
