// Spherical-harmonic helpers of the spherical method (host and device).
// Not part of the public ABI.
#pragma once

#include <math.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#define __device__
#endif
#endif

namespace scff {
namespace sph {

// Largest l_max of an expansion and largest L of the plane-wave expansion of
// e^{iq.P} it needs (l_max plus the highest pair degree, 6).
constexpr int kMaxLmax = 40;
constexpr int kMaxBigL = kMaxLmax + 6;

// Flattened (l, m), m = -l..l.
__host__ __device__ inline int lm_index(int l, int m) { return l * l + l + m; }
// Flattened (l, m), m = 0..l.
__host__ __device__ inline int tri_index(int l, int m) { return l * (l + 1) / 2 + m; }

// Normalised associated Legendre functions with the Condon-Shortley phase for
// m >= 0, so that Y_l^m(theta, phi) = p[tri(l, m)] e^{i m phi} with
// x = cos(theta):
//   p_00 = 1 / sqrt(4 pi)
//   p_mm = -sqrt((2m + 1) / (2m)) sqrt(1 - x^2) p_{m-1,m-1}
//   p_{m+1,m} = sqrt(2m + 3) x p_mm
//   p_lm = a_lm (x p_{l-1,m} - b_lm p_{l-2,m}),
//   a_lm = sqrt((4l^2 - 1) / (l^2 - m^2)),
//   b_lm = sqrt(((l-1)^2 - m^2) / (4 (l-1)^2 - 1)).
// The normalised three-term recurrence stays well scaled up to l ~ 100.
__host__ __device__ inline void plm_all(int lmax, double x, double *p) {
    const double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 0.28209479177387814;  // 1 / sqrt(4 pi)
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm;
        p[tri_index(m, m)] = pmm;
        if (m + 1 <= lmax) {
            double pl2 = pmm, pl1 = sqrt(2.0 * m + 3.0) * x * pmm;
            p[tri_index(m + 1, m)] = pl1;
            for (int l = m + 2; l <= lmax; ++l) {
                const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                const double b = sqrt(((double)(l - 1) * (l - 1) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
                const double pl = a * (x * pl1 - b * pl2);
                p[tri_index(l, m)] = pl;
                pl2 = pl1;
                pl1 = pl;
            }
        }
    }
}

// One column m >= 0 of the same functions: col[l - m] = p_l^m(x) for l = m..lmax.
__host__ __device__ inline void plm_column(int lmax, int m, double x, double *col) {
    const double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 0.28209479177387814;
    for (int k = 1; k <= m; ++k) pmm = -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * pmm;
    col[0] = pmm;
    if (m + 1 > lmax) return;
    double pl2 = pmm, pl1 = sqrt(2.0 * m + 3.0) * x * pmm;
    col[1] = pl1;
    for (int l = m + 2; l <= lmax; ++l) {
        const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        const double b = sqrt(((double)(l - 1) * (l - 1) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
        const double pl = a * (x * pl1 - b * pl2);
        col[l - m] = pl;
        pl2 = pl1;
        pl1 = pl;
    }
}

// Coefficients of the recurrences above, one pair per (l, m) at tri(l, m):
//   l == m:     ab[0] = -sqrt((2m + 1) / (2m))   (m >= 1; the p_mm step)
//   l == m + 1: ab[0] = sqrt(2m + 3)
//   l >= m + 2: ab[0] = a_lm, ab[1] = b_lm
__host__ __device__ inline void plm_coefficients(int l, int m, double *ab) {
    ab[0] = ab[1] = 0.0;
    if (l == m) {
        if (m >= 1) ab[0] = -sqrt((2.0 * m + 1.0) / (2.0 * m));
    } else if (l == m + 1) {
        ab[0] = sqrt(2.0 * m + 3.0);
    } else {
        ab[0] = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        ab[1] = sqrt(((double)(l - 1) * (l - 1) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
    }
}

// plm_column with the coefficients read from a table filled by
// plm_coefficients (2 doubles per tri(l, m)) instead of recomputed.
__host__ __device__ inline void plm_column_tab(int lmax, int m, double x, const double *ab, double *col) {
    const double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 0.28209479177387814;
    for (int k = 1; k <= m; ++k) pmm = ab[2 * tri_index(k, k)] * s * pmm;
    col[0] = pmm;
    if (m + 1 > lmax) return;
    double pl2 = pmm, pl1 = ab[2 * tri_index(m + 1, m)] * x * pmm;
    col[1] = pl1;
    for (int l = m + 2; l <= lmax; ++l) {
        const double *c = ab + 2 * tri_index(l, m);
        const double pl = c[0] * (x * pl1 - c[1] * pl2);
        col[l - m] = pl;
        pl2 = pl1;
        pl1 = pl;
    }
}

// p_l^m for any sign of m: Y_l^{-m} = (-1)^m conj(Y_l^m), so with
// Y_l^m = p_l^m e^{i m phi} for every m, p_l^{-m} = (-1)^m p_l^m.
__host__ __device__ inline double plm_signed(const double *p, int l, int m) {
    const int am = m < 0 ? -m : m;
    const double v = p[tri_index(l, am)];
    return (m < 0 && (am & 1)) ? -v : v;
}

// Spherical Bessel functions j_0..j_{nl-1}(x) for x >= 0.
//   x = 0: j_0 = 1, the rest 0.
//   x < 1e-3: the first two terms of the series x^L / (2L+1)!! (1 - x^2 / (2 (2L+3))).
//   otherwise Miller's downward recurrence j_{L-1} = (2L+1)/x j_L - j_{L+1}
//   from an order well above max(nl, x), normalised with the sum rule
//   sum_L (2L+1) j_L^2 = 1 and the sign of whichever of j_0 = sin x / x and
//   j_1 = sin x / x^2 - cos x / x is larger in magnitude.
__host__ __device__ inline void sph_bessel_all(int nl, double x, double *j) {
    if (x == 0.0) {
        j[0] = 1.0;
        for (int L = 1; L < nl; ++L) j[L] = 0.0;
        return;
    }
    if (x < 1e-3) {
        double t = 1.0;
        for (int L = 0; L < nl; ++L) {
            j[L] = t * (1.0 - x * x / (2.0 * (2 * L + 3)));
            t *= x / (2 * L + 3);
        }
        return;
    }
    const int start = (nl > (int)x ? nl : (int)x) + 24 + (int)(2.0 * sqrt(x + 1.0));
    const double invx = 1.0 / x;
    double fp1 = 0.0, f = 1e-30, sum = 0.0, f0 = 0.0, f1 = 0.0;
    // downward sweep; f holds the unnormalised j_L, rescaled to avoid overflow
    for (int L = start; L >= 0; --L) {
        if (L < nl) j[L] = f;
        if (L == 1) f1 = f;
        if (L == 0) f0 = f;
        sum += (2.0 * L + 1.0) * f * f;
        const double fm1 = (2.0 * L + 1.0) * invx * f - fp1;
        fp1 = f;
        f = fm1;
        if (fabs(f) > 1e140) {
            const double r = 1e-140;
            f *= r;
            fp1 *= r;
            sum *= r * r;
            f0 *= r;
            f1 *= r;
            for (int k = L; k < nl; ++k) j[k] *= r;
        }
    }
    double norm = 1.0 / sqrt(sum);
    const double j0 = sin(x) / x, j1 = sin(x) / (x * x) - cos(x) / x;
    const bool use0 = fabs(j0) >= fabs(j1);
    if ((use0 ? f0 * j0 : f1 * j1) < 0.0) norm = -norm;
    for (int L = 0; L < nl; ++L) j[L] *= norm;
}

}  // namespace sph
}  // namespace scff
