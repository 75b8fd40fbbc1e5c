// Internal interface of the tensor-core (tcgen05) split-BF16 evaluation path.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "scff_internal.h"

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

size_t tc_workspace_bytes(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind);
cudaError_t launch_tc_form_factor(const TcArgs &a, int64_t *launches, cudaStream_t st);

}  // namespace scff
