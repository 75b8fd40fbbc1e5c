// Internal interface of the tensor-core (tcgen05) split-BF16 evaluation path.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "scff_internal.h"

#include <vector>

namespace scff {

struct TcArgs {
    const PairSetDev *ps;
    const float *coef32;       // [n_sblk][n_rows][SB] signed coefficients (FP32)
    int SB;
    const double *pair_geom;   // [n_pair][4]
    const double *qx, *qy, *qz;
    int nx, ny, nz;
    int S;
    double scale;
    float *f;                  // [S][nq][2]
    float *f2;                 // [S][nq] or null
    int *err;
    void *ws;                  // workspace of tc_workspace_bytes()
    size_t ws_bytes;
    cudaEvent_t ev_mark;       // if set, recorded just before the main kernel
    int kind;                  // 0: BF16 hi/lo, 1: BF16 hi/mid/lo, 2: TF32 hi/lo
    int drain_every;           // k-chunks per TMEM accumulation (0 = whole K)
};

// Device descriptor of one prepared job (read by the persistent kernel).
struct TcJobDev {
    const uint8_t *A;      // swizzled split A tiles [n_mt][nkc][stage bytes]
    const float2 *Y, *Z;   // per-axis power tables
    const int4 *kinfo;     // [nkc * BK] k -> (pair, v, w, axis row)
    const int2 *kofs;      // [nkc * BK] k -> element offsets in Y and Z
    int ny, nz, nx, nkc;
    int M, n_mt, n_nt, pad0;
    int64_t N, nq;
    float scale, pad1;
    float2 *f;             // [S][nq] complex output
    float *f2;             // [S][nq] or null
};

// Workspace of one job prepared by tc_prep_job.
size_t tc_job_bytes(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind);
// Workspace of launch_tc_form_factor (one job plus its descriptor and work list).
size_t tc_workspace_bytes(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind);
// Single job: prepare and launch.
cudaError_t launch_tc_form_factor(const TcArgs &a, int64_t *launches, cudaStream_t st);
// Batch building blocks: per-job tables/k-index/A image, the cost-sorted work
// list, and the persistent launch over a group of prepared jobs.
cudaError_t tc_prep_job(const TcArgs &a, void *ws, TcJobDev *jd, int64_t *launches, cudaStream_t st);
void tc_job_desc(const TcArgs &a, void *ws, TcJobDev *jd);
void tc_build_items(const TcJobDev *jobs, int n_jobs, std::vector<int4> &items);
cudaError_t tc_launch_persistent(int kind, const TcJobDev *d_jobs, const int4 *d_items, int n_items, int drain_every,
                                 int *err, int grid_ctas, int64_t *launches, cudaStream_t st);
int tc_num_sms();

}  // namespace scff
