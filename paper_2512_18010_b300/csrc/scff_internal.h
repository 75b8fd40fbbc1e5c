// Internal declarations shared by the host runtime (scff_host.cpp) and the
// CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace scff {

// Highest total polynomial degree of a pair of primitive shells (f with f).
constexpr int kMaxPairL = 6;
// Cartesian functions of the widest primitive-shell record (f: 10).
constexpr int kRecW = 10;
constexpr int kNumClasses = kMaxPairL + 1;

// Number of monomials q_x^u q_y^v q_z^w with u+v+w <= L.
__host__ __device__ constexpr int mono_count(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
// Number of (v, w) with v + w <= L (the contraction index per pair in the
// tensor-core factorisation).
__host__ __device__ constexpr int vw_count(int L) { return (L + 1) * (L + 2) / 2; }

// Monomials are ordered by degree n, then u descending, then v descending.
__host__ __device__ constexpr int mono_u(int m) {
    int i = 0;
    for (int n = 0; n <= kMaxPairL; ++n)
        for (int u = n; u >= 0; --u)
            for (int v = n - u; v >= 0; --v) {
                if (i == m) return u;
                ++i;
            }
    return -1;
}
__host__ __device__ constexpr int mono_v(int m) {
    int i = 0;
    for (int n = 0; n <= kMaxPairL; ++n)
        for (int u = n; u >= 0; --u)
            for (int v = n - u; v >= 0; --v) {
                if (i == m) return v;
                ++i;
            }
    return -1;
}
__host__ __device__ constexpr int mono_w(int m) {
    int i = 0;
    for (int n = 0; n <= kMaxPairL; ++n)
        for (int u = n; u >= 0; --u)
            for (int v = n - u; v >= 0; --v) {
                if (i == m) return n - u - v;
                ++i;
            }
    return -1;
}
// Position of (u, v, w) in that order: the monomials of lower degree n = u+v+w
// come first, then those of degree n with a larger u, then larger v.
__host__ __device__ constexpr int mono_index(int u, int v, int w) {
    const int n = u + v + w;
    return n * (n + 1) * (n + 2) / 6 + (n - u) * (n - u + 1) / 2 + (n - u - v);
}

// Record types of a primitive shell.
enum RecType : int32_t { REC_S = 0, REC_P = 1, REC_D = 2, REC_SP = 3, REC_F = 4 };
__host__ __device__ constexpr int rec_nfn(int t) {
    return t == REC_S ? 1 : t == REC_P ? 3 : t == REC_D ? 6 : t == REC_F ? 10 : 4;
}
__host__ __device__ constexpr int rec_lmax(int t) { return t == REC_S ? 0 : t == REC_D ? 2 : t == REC_F ? 3 : 1; }

// Cartesian exponents of component j of a shell of angular momentum l (the
// order x^l, x^(l-1) y, x^(l-1) z, ...: x power descending, then y).
__host__ __device__ constexpr int cart_pow(int l, int j, int ax) {
    int i = 0;
    for (int a = l; a >= 0; --a)
        for (int b = l - a; b >= 0; --b) {
            if (i == j) return ax == 0 ? a : ax == 1 ? b : l - a - b;
            ++i;
        }
    return 0;
}

// Device view of one basis: primitive-shell records and the pair list sorted
// by pair class L = lmax(r1) + lmax(r2).
struct PairSetDev {
    int n_rec = 0;
    int n_pair = 0;
    int nbf = 0;
    int pair_off[kNumClasses + 1] = {0};   // pairs of class L: [pair_off[L], pair_off[L+1])
    int64_t row_off[kNumClasses + 1] = {0};// monomial rows of class L
    int64_t krow_off[kNumClasses + 1] = {0};// (v,w) rows of class L (tensor-core K index)
    int64_t n_rows = 0;                    // total monomial rows K
    int64_t n_krows = 0;                   // total (pair, v, w) rows
    int64_t n_axrows = 0;                  // total (pair, u) rows = sum (L+1)
    int64_t axrow_off[kNumClasses + 1] = {0};// (pair, u) rows of class L
    // device arrays
    double *rec_xyz = nullptr;   // [n_rec][3]
    double *rec_alpha = nullptr; // [n_rec]
    int32_t *rec_type = nullptr; // [n_rec]
    int32_t *rec_fn0 = nullptr;  // [n_rec] first function index
    double *rec_w = nullptr;     // [n_rec][kRecW] normalised weights
    int2 *pair_rec = nullptr;    // [n_pair] (r1, r2), r1 <= r2
};

// Workspace layout of one form-factor evaluation.
struct EvalBuffers {
    double *coef64 = nullptr;    // [n_sblk][n_rows][SB] signed real coefficients
    float *coef32 = nullptr;     // same, FP32
    double *pair_geom = nullptr; // [n_pair][4] = P, 1/(4p)
    void *gx = nullptr, *gy = nullptr, *gz = nullptr; // axis tables (double2 or float2)
    int *err_flag = nullptr;     // device status word
};

// State block of the direct kernels: in FP64 4, 8 or 12 (see below); in FP32
// the smallest of 8/12/16 that covers S (12 for multiples of 12 above 16,
// else 16).  Shared by every entry point so a job's arithmetic is the same
// alone and in a batch.
inline int direct_state_block(int S, bool fp64) {
    if (fp64) {
        // FP64 blocks of 4, 8 or 12 states: the fewest padded states, then the
        // largest block (the pair factors and monomials are shared by a block;
        // 12 states of the 10-heavy-atom job: 2.26 s in blocks of 4, 2.02 s in one of 12)
        if (S <= 4) return 4;
        if (S <= 8) return 8;
        int best = 12;
        for (int sb : {12, 8, 4})
            if ((S + sb - 1) / sb * sb < (S + best - 1) / best * best) best = sb;
        return best;
    }
    return S <= 8 ? 8 : (S <= 12 ? 12 : (S <= 16 ? 16 : (S % 12 == 0 ? 12 : 16)));
}

// FP64 state block for a job of nq evaluated points: blocks of 12 states
// share the pair factors and monomials best, but a small job needs more,
// smaller blocks to fill the GPU (128 points per block); the largest of
// 12, 8, 4 (fewest padded states first) that still gives two blocks per SM,
// else 4.  The results do not depend on the block size.
inline int direct_state_block_fp64(int S, int64_t nq, int sms) {
    const int64_t qb = (nq + 127) / 128;
    const int pref = direct_state_block(S, true);
    for (int sb : {12, 8, 4}) {
        if (sb > pref) continue;
        if ((S + sb - 1) / sb * sb > (S + pref - 1) / pref * pref && sb != 4) continue;
        if (qb * ((S + sb - 1) / sb) >= 2 * (int64_t)sms) return sb;
    }
    return 4;
}

// ---------------------------------------------------------------- kernels
// All launchers return the launch status and never synchronise.

cudaError_t launch_pair_geom(const PairSetDev &ps, double *pair_geom, cudaStream_t st);

// coef[(s / SB * n_rows + row) * SB + s % SB] for s < S_pad (zero beyond S).
// Kernel attributes of the pair-prep kernel on the current device (once per
// device; scff_create calls it before any capture, and launch_pairprep on a
// device where it has not run yet).
cudaError_t pairprep_init();
cudaError_t launch_pairprep(const PairSetDev &ps, const double *T, int S, int SB, int S_pad,
                            double *coef64, float *coef32, int64_t *launches, cudaStream_t st);

// Per-axis Gaussian x phase tables g[pair][i] = exp(-q_i^2/(4p)) e^{i q_i P_axis}
// computed in FP64; stored as double2 (fp64 != 0) or float2.
cudaError_t launch_axis_tables(const PairSetDev &ps, const double *pair_geom, const double *qaxis,
                               int n, int axis, void *table, int fp64, cudaStream_t st);

// bound[pair][s]: an upper bound of |pair term for state s| over |q| <= qmax,
// from the FP64 coefficients (state block SB), in FP64.
cudaError_t launch_pair_bounds(const PairSetDev &ps, const double *coef64, int SB, int S, double qmax, double *bound,
                               cudaStream_t st);

// Separable integrals I_s = sum wx wy wz f_s over a product grid (FP64).
// sums: 3 * n_axrows double2; part: S * n_pair double2; out: [S][2].
cudaError_t launch_separable(const PairSetDev &ps, const double *geom, const double *coef64, int SB, int S,
                             const double *const q[3], const double *const w[3], const int n[3], double2 *sums,
                             double2 *part, double scale, double *out, int64_t *launches, cudaStream_t st);

// Expansion of caller-basis transition matrices to the Cartesian components:
// Tc[s][a][b] = sum_e sum_f c[a][e] c[b][f] Tu[s][idx[a][e]][idx[b][f]].
constexpr int kMaxPureTerms = 3;
cudaError_t launch_pure_to_cart(int S, int ncart, int nuser, const int32_t *idx, const double *c,
                                const double *Tu, double *Tc, cudaStream_t st);

// One-thread kernel whose mbarrier wait runs out after `tries` attempts and
// sets the error word (the bounded-wait error path, for tests).
cudaError_t launch_wait_selftest(long long tries, int *err, cudaStream_t st);
// FMA-chain rate of the current device (FP32 or FP64), best of three timed
// launches after a warm-up launch; synchronous on the legacy stream.
cudaError_t measure_alu_peak(int fp64, int iters, double *tflops, double *ms);

struct DirectArgs {
    const PairSetDev *ps;
    const void *coef;        // coef64 or coef32 in [n_sblk][n_rows][SB] layout
    const void *gx, *gy, *gz;// product-grid axis tables (grid mode)
    const double *qax, *qay, *qaz; // product-grid axes
    int nx, ny, nz;
    const double *qlist;     // [n][3] (list mode)
    const double *pair_geom; // list mode
    int64_t nq;              // points computed (the first nq of the flattened grid)
    int S, SB;
    double scale;
    void *f;                 // [S][nq_out][2]
    void *f2;                // [S][nq_out] or null
    int *err_flag;
    // Hermitian half (product grids with antisymmetric axes): nq_out points in
    // all, point p also writes conj at nq_out - 1 - p (unless that is p);
    // nq_out = 0 means nq_out = nq without a mirror.
    int64_t nq_out;
};
cudaError_t launch_direct(const DirectArgs &a, int fp64, int list_mode, int64_t *launches,
                          cudaStream_t st);

}  // namespace scff
