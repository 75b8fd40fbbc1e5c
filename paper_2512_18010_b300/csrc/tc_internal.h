// Internal interface of the tensor-core (tcgen05) split-BF16 evaluation path.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "scff_internal.h"

#include <vector>

namespace scff {

constexpr int kMaxBands = 8;  // most launches of one job's overlapped download

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
    int kind;                  // 0: BF16 hi/lo, 1: BF16 hi/mid/lo, 2: TF32 hi/lo, 3: FP16 hi/lo
    double qabs[3];            // largest |q| of each axis (bounds of the FP16 kind's scaling)
    int drain_every;           // k-chunks per TMEM accumulation (0 = whole K)
    int zstage;                // W generator variant requested (tc_variant_resolve): 0 gather, 1 Z staging, 2 prefetch, 3 CTA pairs, 4 CTA pairs in the octant form
    // 1: the job is laid out for the CTA-pair launch (m-tiles padded to an
    // even count; set by the launchers from the resolved variant)
    int pair;
    // 1 (with pair and half): the job runs in the octant form of the CTA-pair
    // launch (see TcJobDev::oct); set by the launchers from the resolved variant
    int oct;
    // 1: the three axes are antisymmetric (q[n-1-i] = -q[i]); only the rows
    // ix < ceil(nx/2) are computed and f(-q) = conj(f(q)) fills the rest
    int half;
    // Host outputs with overlapped download (optional, f_host non-null): the
    // tiles are ordered band by band (bands of output columns) in one launch
    // that reports its progress to host-mapped slots; the host issues the
    // copy of each band's columns to f_host / f2_host on copy_st as soon as
    // every tile of the band is written, while the launch goes on.  st waits
    // for the last copy.  n_bands: 0 = chosen from the tile count, 1 = off,
    // 2..kMaxBands = that many equal bands where the grid allows.
    // *bands_used gets the band count (1: nothing was copied).
    int n_bands;
    float *f_host, *f2_host;
    cudaStream_t copy_st;
    int *progress_dev;                  // >= 8 x SMs ints, host-mapped (device address)
    volatile int *progress_host;        // the same slots (host address)
    cudaEvent_t ev_done, ev_copied;     // end of the launch, end of the copies
    int *bands_used;
    int *variant_used;         // optional: the W generator variant the launch ran
};

// Device descriptor of one prepared job (read by the persistent kernel).
struct TcJobDev {
    const uint8_t *A;      // swizzled split A tiles [n_mt][nkc][stage bytes]
    const float2 *Y, *Z;   // per-axis power tables
    const int4 *kinfo;     // [nkc * BK] k -> (pair, v, w, axis row)
    const int2 *kofs;      // [nkc * BK] k -> element offsets in Y and Z
    int ny, nz, nx, nkc;
    int M, n_mt, n_nt;
    // Column n of the output splits into (n / nz, n % nz).  ylm = 0: the Y
    // table is read at column n / nz and the Z table at n % nz (product
    // grids).  ylm = 1: Z is read at LM = n % nz and Y at
    // (n / nz) * ystride + L with L = floor(sqrt(LM)) (radial x (L, M)
    // columns of the spherical method).
    int ylm;
    int64_t N, nq;
    float scale;
    int ystride;
    // mirror = 1: row ix (of nxf) also writes conj at row nxf-1-ix, column N-1-n
    // (unless that is the row itself): f(-q) = conj(f(q)) on antisymmetric axes
    int mirror, nxf;
    float2 *f;             // [S][nq] complex output
    float *f2;             // [S][nq] or null
    // Tail split: the last split_tiles tiles of the job run as nsplit parts over
    // disjoint k ranges; parts write raw partial sums to part[slot][BM][BN] and
    // the last of the eight warp regions of a tile to arrive (counter cnt[tile][8])
    // sums the parts in order and writes the tile.  nsplit = 0: no split.
    float2 *part;
    int *cnt;
    int nsplit, split_tiles;
    // 1: laid out for the CTA-pair launch: n_mt is even and the work items'
    // m field holds the m-tile pair (tiles (2 mp, nt) and (2 mp + 1, nt))
    int pair;
    // FP16 kind: FP64 bits of the bound of the job's largest term, from which
    // the job exponent of the scaled A is derived (null for the other kinds)
    const unsigned long long *tmax;
    // 1 (pair jobs on antisymmetric grids): octant form.  The columns are the
    // Noct = nyh x nzh points (iy, iz) with iy < nyh = ceil(ny/2) and
    // iz < nzh = ceil(nz/2), 32 per tile; W is real, one row per point and
    // product (Re or Im of Y) x (Re or Im of Z), and Ar and Ai each multiply
    // it into their own accumulator.  The eight real sums of a row and point
    // give f at (ix, +-qy, +-qz) and, by f(-q) = conj(f(q)), at the mirrored
    // row: half the tensor work and half the W values per output.
    int oct, nyh, nzh;
    int64_t Noct;
};

// Split kind of a tensor-core precision (scff_precision), -1 for the others.
int tc_kind_of_precision(int precision);
// Largest |q| of each axis of a product grid, for TcArgs::qabs.
void tc_axes_abs_max(const double *qx, int nx, const double *qy, int ny, const double *qz, int nz, double out[3]);

// Work item of the persistent kernel (int4):
//   x = job | (slot + 1) << 16   (slot: part of a split tile, 0 in the high half: whole tile)
//   y = m-tile | k0 << 16        (k0: first k-chunk of the item)
//   z = n-tile, w = number of k-chunks.
__host__ __device__ inline int item_job(int x) { return x & 0xFFFF; }
__host__ __device__ inline int item_slot(int x) { return (x >> 16) - 1; }
__host__ __device__ inline int item_mt(int y) { return y & 0xFFFF; }
__host__ __device__ inline int item_k0(int y) { return y >> 16; }

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
// Most work items one job of `tiles` tiles contributes (its tail split adds
// at most 2P parts).
int64_t tc_max_items(int64_t tiles);
// progress (optional, e.g. host-mapped): progress[cta * 8 + w] = items that
// generator warp w of CTA cta has finished (its outputs written and fenced
// at system scope before the count); CTA b runs items b, b + grid, ...
// variant: the W generator variant (0 gather, 1 Z staging, 2 prefetch; see
// tc_variant_resolve), which the launch's jobs and kind must allow.  Kernel
// attributes are set on a call with n_items = 0, before any capture.
// queue (optional, device int): CTAs take their items from this shared counter
// (reset to zero on `st` before the launch) instead of the static sequence
// blockIdx.x, blockIdx.x + grid, ...; progress reporting needs the static one.
cudaError_t tc_launch_persistent(int kind, int variant, const TcJobDev *d_jobs, const int4 *d_items, int n_items,
                                 int drain_every, int *err, int grid_ctas, int64_t *launches, cudaStream_t st,
                                 int *progress = nullptr, int *queue = nullptr);
// Whether every job of a launch can use the Z-staging variant (two-piece
// kinds, product grids whose nz is a multiple of 128).
bool tc_zstage_ok(int kind, const TcJobDev *jobs, int n_jobs);
// Whether a kind has the prefetching and CTA-pair variants (the kinds that
// stage their k-offsets: FP16 hi/lo and BF16 hi/lo).
bool tc_prefetch_ok(int kind);
// Most CTA pairs (two-CTA clusters of the persistent kernel) resident at once.
int tc_num_pairs();
// The variant a launch runs for a requested one: 1 (Z staging) where the kind
// and every job's grid allow it (zstage_grid: tc_zstage_ok), 2 (prefetch) and
// 3 (CTA pairs: a two-CTA cluster shares each MMA and generates half of W per
// SM) where the kind has them, else 0 (gather).  All three form bitwise the same W
// and add the same partial sums in the same order, so the choice never
// changes a result.
int tc_variant_resolve(int kind, int requested, bool zstage_grid);
int tc_variant_for(int kind, int requested, const TcJobDev *jobs, int n_jobs);
// The automatic mode's variant for a kind (measured fastest on the
// 10-heavy-atom job): Z staging for TF32 hi/lo, CTA pairs for FP16 hi/lo and
// BF16 hi/lo, gather for BF16 hi/mid/lo.
int tc_variant_preferred(int kind);
int tc_num_sms();

// Generic two-table contraction on the tensor cores (the spherical method):
//   C[(s, ix), n] = scale * sum_k A[(s, ix), k] * Y[kofs[k].x + iy(n)] * Z[kofs[k].y + iz(n)]
// with A given as a dense complex FP64 matrix (row-major, leading dimension
// lda, K valid columns) that is split and swizzled into the tile image here,
// and (iy, iz) from the column rule of TcJobDev (ylm, ystride).  Rows are
// m = s * nx + ix, M = S * nx; C is [S][nx][N] complex FP32, C2 = |C|^2 or null.
struct TcGenericArgs {
    int kind;
    const double2 *A;
    int64_t lda, K;
    int M, nx;
    const float2 *Y, *Z;
    const int2 *kofs;      // [K_pad] (padding k must point at zero rows)
    int nz, ylm, ystride;
    int64_t N;
    float scale;
    float2 *C;
    float *C2;
    int drain_every;
    int *err;
    void *ws;              // workspace of tc_generic_bytes()
    size_t ws_bytes;
};
int64_t tc_generic_kpad(int kind, int64_t K);
size_t tc_generic_bytes(int kind, int M, int64_t K);
cudaError_t tc_run_generic(const TcGenericArgs &a, int64_t *launches, cudaStream_t st);
// Several such contractions (same kind, same workspace) in one persistent
// launch; the workspace holds their images back to back, then the
// descriptors and the work list (tc_generic_bytes summed, plus the list).
cudaError_t tc_run_generic_multi(const TcGenericArgs *jobs, int n_jobs, int64_t *launches, cudaStream_t st);

}  // namespace scff
