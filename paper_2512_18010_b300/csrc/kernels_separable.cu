// Separable integrals of the form factor (Sec. "Cartesian Grid Method": the
// V-tensors alone suffice for integrals of f_S against a product of one-axis
// functions, at a cost linear in the longest axis).
//
//   I_s = sum_{ix,iy,iz} wx[ix] wy[iy] wz[iz] f_s(qx[ix], qy[iy], qz[iz])
//       = sum_pairs sum_uvw D^s_{pair,uvw} SX_{pair,u} SY_{pair,v} SZ_{pair,w},
//   SX_{pair,u} = sum_ix wx[ix] (i qx)^u exp(-qx^2/4p) e^{i qx P_x}   (Y, Z alike)
//
// where D is the real coefficient of the monomial form (the i^n factor is
// split over the three axis sums).  Everything runs in FP64; the sum over
// pairs is a fixed-order two-pass reduction, so the result is deterministic.
#include <math.h>

#include "scff_internal.h"
#include "device_common.cuh"

namespace scff {

// Weighted axis sums S[axrow] for one axis: thread per (pair, u) row.
__global__ void axis_sum_kernel(PairSetDev ps, const double *__restrict__ geom, const double *__restrict__ q,
                                const double *__restrict__ w, int n, int axis, double2 *__restrict__ out) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= ps.n_axrows) return;
    int L = 0;
    while (L < kMaxPairL && row >= ps.axrow_off[L + 1]) ++L;
    const int64_t local = row - ps.axrow_off[L];
    const int pr = ps.pair_off[L] + (int)(local / (L + 1));
    const int u = (int)(local % (L + 1));
    const double P = geom[4 * pr + axis], inv4p = geom[4 * pr + 3];
    double re = 0.0, im = 0.0;
    for (int i = 0; i < n; ++i) {
        const double qi = q[i];
        double sn, cs;
        sincos(qi * P, &sn, &cs);
        double amp = w[i] * exp(-qi * qi * inv4p);
        for (int t = 0; t < u; ++t) amp *= qi;
        re = fma(amp, cs, re);
        im = fma(amp, sn, im);
    }
    double xr, xi;  // times i^u
    switch (u & 3) {
    case 0: xr = re; xi = im; break;
    case 1: xr = -im; xi = re; break;
    case 2: xr = -re; xi = -im; break;
    default: xr = im; xi = -re; break;
    }
    out[row] = make_double2(xr, xi);
}

// Per-pair contribution: thread per (pair, state).
__global__ void separable_pair_kernel(PairSetDev ps, const double *__restrict__ coef64, int SB,
                                      const double2 *__restrict__ SX, const double2 *__restrict__ SY,
                                      const double2 *__restrict__ SZ, int S, double2 *__restrict__ part) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)ps.n_pair * S) return;
    const int pr = (int)(idx / S), s = (int)(idx % S);
    int L = 0;
    while (L < kMaxPairL && pr >= ps.pair_off[L + 1]) ++L;
    const int mL = mono_count(L);
    const int64_t row0 = ps.row_off[L] + (int64_t)(pr - ps.pair_off[L]) * mL;
    const int64_t ax0 = ps.axrow_off[L] + (int64_t)(pr - ps.pair_off[L]) * (L + 1);
    const double *cs = coef64 + ((size_t)(s / SB) * ps.n_rows) * SB + (s % SB);
    double re = 0.0, im = 0.0;
    for (int m = 0; m < mL; ++m) {
        const int u = mono_u(m), v = mono_v(m), w = mono_w(m);
        const int n = u + v + w;
        const double c = cs[(size_t)(row0 + m) * SB] * ((n & 2) ? -1.0 : 1.0);  // undo the folded sign of i^n
        const double2 a = SX[ax0 + u], b = SY[ax0 + v], d = SZ[ax0 + w];
        const double abr = a.x * b.x - a.y * b.y, abi = a.x * b.y + a.y * b.x;
        re = fma(c, abr * d.x - abi * d.y, re);
        im = fma(c, abr * d.y + abi * d.x, im);
    }
    part[(size_t)s * ps.n_pair + pr] = make_double2(re, im);
}

// Fixed-order reduction over pairs: one block per state.
__global__ void separable_reduce_kernel(const double2 *__restrict__ part, int n_pair, double scale,
                                        double *__restrict__ out) {
    __shared__ double sr[256], si[256];
    const int s = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int p = threadIdx.x; p < n_pair; p += blockDim.x) {
        re += part[(size_t)s * n_pair + p].x;
        im += part[(size_t)s * n_pair + p].y;
    }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sr[threadIdx.x] += sr[threadIdx.x + w];
            si[threadIdx.x] += si[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * s] = scale * sr[0];
        out[2 * s + 1] = scale * si[0];
    }
}

cudaError_t launch_separable(const PairSetDev &ps, const double *geom, const double *coef64, int SB, int S,
                             const double *const q[3], const double *const w[3], const int n[3], double2 *sums,
                             double2 *part, double scale, double *out, int64_t *launches, cudaStream_t st) {
    const int64_t rows = ps.n_axrows;
    for (int ax = 0; ax < 3; ++ax) {
        if (rows > 0)
            axis_sum_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(ps, geom, q[ax], w[ax], n[ax], ax,
                                                                            sums + ax * rows);
    }
    const int64_t tot = (int64_t)ps.n_pair * S;
    if (tot > 0)
        separable_pair_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(ps, coef64, SB, sums, sums + rows,
                                                                             sums + 2 * rows, S, part);
    separable_reduce_kernel<<<S, 256, 0, st>>>(part, ps.n_pair, scale, out);
    if (launches) *launches += 5;
    return cudaGetLastError();
}

}  // namespace scff

namespace scff {

// Exercises the bounded-wait error path: one thread waits on an mbarrier that
// no one arrives at, gives up after `tries` attempts, records the timeout in
// the context's error word and returns normally (the context stays usable).
__global__ void wait_selftest_kernel(long long tries, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbarrier_init();
        if (!mbar_wait_n(&bar, 0, tries)) flag_error(err, kDevErrTimeout);
    }
}

cudaError_t launch_wait_selftest(long long tries, int *err, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(tries, err);
    return cudaGetLastError();
}

}  // namespace scff
