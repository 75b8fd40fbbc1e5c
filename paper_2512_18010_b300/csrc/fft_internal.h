// Internal interface of the FFT method (kernels_fft.cu, fft_method.cpp).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "scff_internal.h"

namespace scff {

// Density tabulation: Phi_s(x_a) for the n[0] x n[1] x n[2] box points into
// out[(s / 2) * npts + p][s % 2] (two states per complex field).
struct FftDensityArgs {
    PairSetDev ps;             // records of the basis (Cartesian components)
    int nbf, nbf_pad;          // Cartesian functions; padded to a multiple of 32
    int S;
    const void *T;             // [S][nbf][nbf] Cartesian transition matrices, float or double
    void *out;                 // packed complex fields, float or double pairs
    double xmin[3], dx[3];
    int nx, ny, nz;
    int64_t npts;
    double cut;                // drop a primitive where alpha |r - A|^2 > cut (0 = never)
    double scale, vpix;
    double *parseval;          // [S][2] (real-space sums accumulated here) or null
    const void *tsym;          // [ceil(S / sbf)][kpad][sbf] symmetrised T per pair (fft_tsym)
    const int2 *pairs;         // [kpad] (mu, nu) per pair, (-1, -1) for padding
    int64_t kpad;              // pairs padded to whole chunks
    int *err;                  // set on a timed-out wait
    // FP32 tabulation only (fft_record_prep): per record, the centre's grid
    // coordinate split into an integer and a fraction, and the exponent, as
    // (ia_x, ia_y, ia_z, alpha) and (fa_x, fa_y, fa_z, 0); weights [n_rec][kRecW]
    const float4 *recg;
    const float *recw;
};

struct FftAxisArgs {
    void *data;                // complex fields (float2 or double2), in place
    int n, logn, W;            // line length, log2, lines per CTA
    int64_t es;                // element stride along the line
    int64_t inner;             // lines adjacent in memory (stride 1) per block when es > 1
    int64_t block_stride;      // distance between consecutive such blocks
};

struct FftUnpackArgs {
    const void *data;          // transformed fields
    int S;
    int n[3];
    double dq[3], xmin[3];
    double vpix;
    double dq3_over_2pi3;
    void *f, *f2;              // [S][n0][n1][n2] complex and |f|^2 (float or double), either may be null
    double *parseval;          // [S][2] (momentum-space sums accumulated here) or null
    double2 *phase;            // workspace: [n0 + n1 + n2] per-axis factors e^{i dq al x_min}
};

// Shared memory of the density kernel for sweeps of sbf states and tp points per tile.
size_t fft_density_smem(int fp64, int nbf_pad, int sbf, int tp);
cudaError_t launch_fft_density(const FftDensityArgs &a, int fp64, int sbf, int tp, cudaStream_t st);
// Per-record FP32 tabulation data (FftDensityArgs::recg, recw) of the box in a.
cudaError_t launch_fft_record_prep(const FftDensityArgs &a, float4 *recg, float *recw, cudaStream_t st);
// Pairs (mu <= nu) of nbf functions padded to whole staging chunks.
int64_t fft_pair_kpad(int nbf);
cudaError_t launch_fft_tsym(const void *T, int fp64, int nbf, int S, int sbf, void *tsym, int2 *pairs,
                            cudaStream_t st);
cudaError_t launch_fft_axis(const FftAxisArgs &a, int fp64, int64_t n_groups, cudaStream_t st);
cudaError_t launch_fft_unpack(const FftUnpackArgs &a, int fp64, cudaStream_t st);
cudaError_t launch_cast_f64_to_f32(const double *in, int64_t n, float *out, cudaStream_t st);

}  // namespace scff
