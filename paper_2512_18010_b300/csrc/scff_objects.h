// Internal object definitions of the host runtime (context and handles),
// shared by the translation units of the library.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "../../include/scff.h"
#include "scff_internal.h"

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct scff_plan_s;
struct scff_server_s;

// Evaluation configuration chosen by the autotuner (scff_host.cpp).
struct FFChoice {
    int use_tc;
    int drain;  // k-chunks per TMEM accumulation (tensor cores)
    int SB;     // states per block (direct path)
    int zs = 1; // tensor cores: the Z-staging generator variant where the grid allows it
};

struct scff_ctx {
    int device = 0;
    uint64_t budget = 0;
    int64_t launches = 0;
    int *d_err = nullptr;
    int *h_err = nullptr;  // pinned
    // workspace slots (grown on demand)
    DevBuf coef, geom, gx, gy, gz, fstage, f2stage, tc_ws;
    // stage timing (scff_set_timing): events before pair-prep, before the
    // q-evaluation, after the q-evaluation
    int timing = 0;
    int drain_every = -1;  // tensor-core TMEM accumulation length (-1 = default)
    int tc_zstage = -1;    // Z-staging generator variant: -1 automatic, 0 off, 1 on where the grid allows
    int last_path[3] = {-1, -1, -1};  // path of the last form-factor call (scff_last_path)
    int timed_valid = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::vector<struct scff_basis_s *> bases;
    std::vector<struct scff_trans_s *> transs;
    std::vector<struct scff_qgrid_s *> grids;
    std::vector<struct scff_plan_s *> plans;
    // error-bounded pair screening (0 = off) and its cached compacted pair sets
    double screen_eps = 0.0;
    std::vector<struct ScreenedSet *> screened;
    // autotuner: chosen configuration and its time per job-shape key
    int autotune = 0;
    std::map<uint64_t, struct FFChoice> tune;
    std::map<uint64_t, float> tune_ms;
    // spherical method: coefficient tables (spherical.cpp) and workspace
    struct SphCache *sph = nullptr;
    DevBuf sph_ws;
    // FFT method workspace (fft_method.cpp)
    DevBuf fft_ws;
    // Hermitian half (scff_set_hermitian): on antisymmetric product grids
    // compute half the points and fill the rest with f(-q) = conj(f(q))
    int hermitian = 1;
    // overlapped download of host outputs (scff_set_download_bands): band
    // count (0 = automatic); copy stream, events (end of launch, end of
    // copies) and host-mapped progress slots, created on first use
    int bands = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t band_ev[2] = {};
    int *progress_h = nullptr, *progress_d = nullptr;
};

// 1 when every axis of the host array pairs point i with -(point n-1-i) exactly.
int scff_axes_antisym(const double *qx, int nx, const double *qy, int ny, const double *qz, int nz);

void scff_sph_cache_free(struct SphCache *c);

struct scff_basis_s {
    scff_ctx *ctx;
    int nbf;  // functions the caller numbers (pure shells count 2l+1)
    scff::PairSetDev dev;  // Cartesian records; dev.nbf counts Cartesian components
    // Pure shells: Cartesian component a = sum over e < kMaxPureTerms of
    // cmap_c[a][e] x caller function cmap_idx[a][e] (-1 ends the list); null
    // when every shell is Cartesian.
    int32_t *cmap_idx = nullptr;
    double *cmap_c = nullptr;
};

struct scff_trans_s {
    scff_ctx *ctx;
    scff_basis_s *basis;
    int S;
    double *d_T;
};

struct scff_qgrid_s {
    scff_ctx *ctx;
    int product;
    int nx, ny, nz;
    int64_t n;
    double qmax = 0.0;           // largest |q| of the grid
    std::vector<double> hq;      // host copy of an explicit list
    double *d_qx, *d_qy, *d_qz;  // product grid axes
    double *d_q;                 // list [n][3]
    std::vector<double> hx, hy, hz;
    int antisym = 0;             // product grid with q[n-1-i] == -q[i] on every axis
};


// A pair list with the pairs whose bounded contribution is negligible
// removed (scff_set_screening); records are borrowed from the basis.
struct ScreenedSet {
    struct scff_trans_s *trans;
    double eps;
    double qmax;
    scff::PairSetDev dev;  // own pair_rec, everything else shared with the basis
    int kept, total;
};

// Whether a call in this precision asks for the Z-staging W generator variant
// of the tensor-core kernel (where the grid allows it): the context's mode,
// or the split kind's default.
int zstage_mode(const scff_ctx *c, int precision);
