/*
 * scff.h -- C ABI of the B300 molecular transition form-factor library.
 *
 * The library evaluates, for every excited state s and every point q of a
 * momentum grid,
 *
 *     f_s(q) = scale * sum_{mu,nu} T^s[mu][nu] * Int phi_mu(r) phi_nu(r) e^{+i q.r} d^3r
 *
 * over real contracted Cartesian Gaussian basis functions phi (the AO-basis
 * form factor of Sec. "Analytic Method", from Eqs. fSreal and PhiTDM of
 * Sec. "FFT Method"; the paper's convention carries scale = sqrt(2) for spin,
 * Sec. "Electronic Structure Calculation"), together with |f_s(q)|^2.
 *
 * The evaluation follows the paper's Cartesian analytic method (Eqs.
 * sigmaTidbits, positionTidbits, bCoefficients, Mij, CartesianMethod,
 * DTensor and Ccoefficients): a device pair-prep kernel applies the Gaussian
 * product theorem to every pair of primitive shells and folds contraction
 * coefficients, normalisation and T^s into per-pair monomial coefficients;
 * q-evaluation kernels then sum Gaussian x phase x polynomial terms over the
 * pairs.
 *
 * Units: atomic units throughout (positions in Bohr, q in inverse Bohr).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an scff_status; SCFF_OK is 0.  No call aborts the
 *   process.  On failure the message of the calling thread's last error is
 *   available from scff_last_error().
 * - Input arrays are read during the call and copied; the caller keeps
 *   ownership and may free them when the call returns.
 * - Handles (basis, transitions, q-grids) are owned by the context and are
 *   released with the matching scff_release_* call or by scff_destroy.
 * - Output buffers are allocated by the caller.
 * - Device pointers are plain CUDA device addresses on the context's device;
 *   host pointers are ordinary host memory (pinned memory speeds up copies).
 * - A context is not thread-safe: serialise calls on one context.
 */
#ifndef SCFF_H
#define SCFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t scff_status;
enum {
    SCFF_OK = 0,
    SCFF_ERR_INVALID_ARG = 1,  /* a size, pointer, code or layout is invalid */
    SCFF_ERR_UNSUPPORTED_L = 2,/* shell angular momentum above Cartesian f */
    SCFF_ERR_OOM = 3,          /* device or host allocation failed */
    SCFF_ERR_ADMISSION = 4,    /* job footprint exceeds the context's HBM budget */
    SCFF_ERR_CUDA = 5,         /* a CUDA runtime call failed (message has the name) */
    SCFF_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    SCFF_ERR_CANCELLED = 7,    /* a queued job was cancelled */
    SCFF_ERR_NOT_FOUND = 8     /* unknown handle or job id */
};

/* Arithmetic of the q-evaluation.  Pair-prep, normalisation and the phase
 * range reduction run in FP64 in every mode. */
typedef enum {
    SCFF_FP64 = 0,   /* direct evaluation in FP64: the plain FP64 GPU path */
    SCFF_FP32 = 1,   /* direct evaluation in FP32 with FP64-accurate phases and
                        double-float accumulation across pairs */
    SCFF_BF16X3 = 2, /* tensor cores, BF16 split into hi + mid + lo pieces
                        (six piece products per complex part), FP32 accumulation */
    SCFF_TF32X3 = 3, /* tensor cores, TF32 split into hi + lo pieces (three
                        piece products per complex part), FP32 accumulation */
    SCFF_BF16X2 = 4, /* tensor cores, BF16 hi + lo (three piece products),
                        about 2e-5 relative error on the bundled workloads */
    SCFF_FP16X2 = 5  /* tensor cores, FP16 hi + lo (three piece products,
                        about 22 significant bits per operand), FP32
                        accumulation: half the tensor work of SCFF_BF16X3 at
                        the same 1e-5 bar.  FP16's narrow exponent range is
                        handled by exact power-of-two scaling of the per-axis
                        table rows, the A columns and the whole job (removed
                        in the epilogue).  Product-grid form factors (single
                        calls, plans, the server); the spherical method does
                        not take it.  The tensor-core modes need a product
                        grid; on an explicit q list they run the FP32 direct
                        path (scff_last_path reports which path ran). */
} scff_precision;

/* scff_basis flags */
#define SCFF_RENORM_CONTRACTED 1u /* rescale each contracted function to <phi|phi> = 1 */
#define SCFF_PURE_D 2u /* d shells are the 5 spherical-harmonic (pure) functions */
#define SCFF_PURE_F 4u /* f shells are the 7 spherical-harmonic (pure) functions */

typedef struct scff_ctx scff_ctx;
typedef struct scff_basis_s *scff_basis_h;
typedef struct scff_trans_s *scff_trans_h;
typedef struct scff_qgrid_s *scff_qgrid_h;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory that form-factor jobs may hold at once (0 = 90% of the free
 * memory at creation); it is what admission control checks against. */
scff_status scff_create(scff_ctx **out, int device, uint64_t hbm_budget_bytes);
void scff_destroy(scff_ctx *ctx);

/* Message of the calling thread's last failed call ("" if none). */
const char *scff_last_error(void);

/*
 * Basis set (Appendix A, Eq. defprimitive; Sec. "Analytic Method" for the
 * expansion into Cartesian terms).
 *   xyz[n_atoms][3]       atom centres, Bohr.
 *   shell_atom[n_shells]  atom index of each shell.
 *   shell_l[n_shells]     0 = s, 1 = p, 2 = Cartesian d, 3 = Cartesian f,
 *                         -1 = sp (s and p sharing exponents).  Other
 *                         values give SCFF_ERR_UNSUPPORTED_L (l >= 4) or
 *                         INVALID_ARG.
 *   shell_nprim[n_shells] primitives per shell (1..64).
 *   exponents[]           alpha of exp(-alpha r^2), all shells concatenated
 *                         (sum of shell_nprim entries), each > 0.
 *   coefficients[]        contraction coefficients, concatenated; an sp
 *                         shell stores nprim s coefficients then nprim p
 *                         coefficients.
 * Functions are numbered shell by shell; Cartesian components are ordered by
 * descending x power, then descending y power: x,y,z; xx,xy,xz,yy,yz,zz;
 * xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz; an sp shell gives s,px,py,pz.  Each primitive
 * Cartesian term is normalised to unit norm; with SCFF_RENORM_CONTRACTED the
 * contracted function is then rescaled to unit norm as well.
 *
 * Pure shells (Appendix A, Eq. defprimitive with several Cartesian terms k_i):
 * with SCFF_PURE_D (SCFF_PURE_F) every d (f) shell gives the 2l+1 real solid
 * harmonics, ordered m = -l..l, as these polynomials times the Gaussian:
 *   d: xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2
 *   f: 3x^2y-y^3, xyz, 4yz^2-x^2y-y^3, 2z^3-3x^2z-3y^2z, 4xz^2-x^3-xy^2,
 *      x^2z-y^2z, x^3-3xy^2
 * and each primitive (the whole polynomial) is normalised to unit norm.
 * T is then given in this basis; the library expands it to the Cartesian
 * components internally (the form factor is bilinear in the functions), so
 * the cost per q point is that of the Cartesian shell.
 * On success *out is a new handle and *nbf_out the function count (pure
 * shells counted with 2l+1 functions).
 */
scff_status scff_basis(scff_ctx *ctx, int n_atoms, const double *xyz, int n_shells,
                       const int32_t *shell_atom, const int32_t *shell_l,
                       const int32_t *shell_nprim, const double *exponents,
                       const double *coefficients, uint32_t flags, scff_basis_h *out,
                       int32_t *nbf_out);

/*
 * Transition density matrices T^s (Sec. "Electronic Structure Calculation",
 * the one-particle TDM in the AO basis).
 *   T[n_states][nbf][nbf] row-major FP64; T[s][mu][nu] weights phi_mu phi_nu.
 *   T_on_device: 0 = host pointer, 1 = device pointer (copied device-to-device).
 * Only the symmetric part of T contributes (the integral is symmetric in
 * mu, nu for a real basis).
 */
scff_status scff_transitions(scff_ctx *ctx, scff_basis_h basis, int n_states,
                             const double *T, int T_on_device, scff_trans_h *out);

/* Product grid q = (qx[ix], qy[iy], qz[iz]); flat index (ix*ny + iy)*nz + iz
 * (z fastest).  Host arrays, each length >= 1. */
scff_status scff_qgrid_product(scff_ctx *ctx, const double *qx, int nx, const double *qy,
                               int ny, const double *qz, int nz, scff_qgrid_h *out);

/* Explicit list of q vectors, q[n][3] host array, n >= 0. */
scff_status scff_qgrid_list(scff_ctx *ctx, const double *q, int64_t n, scff_qgrid_h *out);

/* Number of q points of a grid (or -1 for an unknown handle). */
int64_t scff_qgrid_size(scff_ctx *ctx, scff_qgrid_h grid);

/*
 * Form factor of every state on every q point (Eq. CartesianMethod evaluated
 * through its monomial form, Eqs. DTensor and Ccoefficients).
 *   precision   scff_precision.
 *   scale       overall factor (1.0 for the bare integral; sqrt(2) for the
 *               paper's spin-summed convention).
 *   f_out       [n_states][n_q][2] interleaved (Re, Im); double for SCFF_FP64,
 *               float otherwise.  Required.
 *   f2_out      [n_states][n_q] |f|^2 in the same real type, or NULL.
 *   out_on_device  1: f_out/f2_out are device pointers and the call is
 *               asynchronous on `stream`; 0: host pointers, the call copies
 *               the result back and returns after the stream has finished.
 *   stream      a cudaStream_t (NULL = the legacy default stream).
 * The pair-prep kernel runs inside every call; intermediate buffers come from
 * a context-owned workspace that grows as needed.
 */
scff_status scff_form_factor(scff_ctx *ctx, scff_basis_h basis, scff_trans_h trans,
                             scff_qgrid_h grid, int precision, double scale, void *f_out,
                             void *f2_out, int out_on_device, void *stream);

/*
 * Batches.  A plan evaluates a fixed list of jobs -- each a (basis,
 * transitions, q-grid) triple with its own scale and caller-owned DEVICE
 * outputs laid out as in scff_form_factor -- in one precision.  Jobs with a
 * product grid and a tensor-core precision are grouped so that each group's
 * tables and A images fit the workspace, and each group runs as ONE
 * persistent kernel launch over all of its output tiles (one CTA per SM,
 * tiles ordered by cost).  A tile's arithmetic does not depend on the other
 * jobs, so a job gives the same result alone and in any batch.  Other jobs
 * run the direct path.  The handles must stay alive while the plan exists.
 *   workspace_bytes  bound on the plan's device memory (0 = the context
 *                    budget, at most 64 GiB); a job that alone exceeds it
 *                    gives SCFF_ERR_ADMISSION.
 * scff_plan_run launches the plan's kernels on `stream` (asynchronous; no
 * allocation and no synchronisation inside, so it may be captured).
 * scff_plan_run_graph captures one run into a CUDA graph on its first call
 * and replays that graph on every call (stream must not be NULL).
 * scff_plan_info: info[0..5] = jobs, tensor-core jobs, groups, tiles,
 * device bytes, kernel launches per run.
 */
typedef struct {
    scff_basis_h basis;
    scff_trans_h trans;
    scff_qgrid_h grid;
    double scale;
    void *f_out;   /* device [S][n_q][2] */
    void *f2_out;  /* device [S][n_q] or NULL */
} scff_job;
typedef struct scff_plan_s *scff_plan_h;
scff_status scff_plan_create(scff_ctx *ctx, int n_jobs, const scff_job *jobs, int precision,
                             uint64_t workspace_bytes, scff_plan_h *out);
scff_status scff_plan_run(scff_ctx *ctx, scff_plan_h plan, void *stream);
scff_status scff_plan_run_graph(scff_ctx *ctx, scff_plan_h plan, void *stream);
scff_status scff_plan_info(scff_ctx *ctx, scff_plan_h plan, int64_t *info);
void scff_release_plan(scff_ctx *ctx, scff_plan_h plan);

/*
 * Serving: continuous batching of form-factor jobs (a request loop on a
 * server thread that owns all of the GPU work).
 *
 * A job references a basis and transitions that are already resident on the
 * device (scff_basis / scff_transitions, registered before submitting and
 * kept alive until the job finishes), a product q-grid given as host axes
 * (copied at submit), a scale and output buffers laid out as in
 * scff_form_factor.  Jobs are admitted in arrival order as soon as a stream
 * slot is free and their device footprint (tables, A image, axes and
 * device-side outputs) fits the free part of the server's arena, which is
 * allocated once at creation; every admitted group of jobs runs as one batch
 * (one persistent tensor-core launch over all of its tiles, which its CTAs
 * take from a device work queue).  With batch_cost_ratio > 0 a batch takes
 * only jobs whose work is within that factor of its first job's; the others
 * wait for the next batch.  Jobs arriving while batches are in flight join the next batch,
 * which may run concurrently on another slot.  A job's result does not depend on the rest
 * of its batch.  A job that can never fit the arena fails with
 * SCFF_ERR_ADMISSION.  Host output buffers that are not pinned are pinned
 * (cudaHostRegister) for the job's lifetime.
 *
 * scff_wait blocks until the job finished, at most timeout_us microseconds
 * (< 0: no limit), and returns SCFF_OK, SCFF_ERR_TIMEOUT (still running),
 * SCFF_ERR_CANCELLED or the job's error.  scff_cancel cancels a job that has
 * not been admitted yet.  scff_job_times writes the host clock (ms) at
 * submission, admission and completion.  scff_server_stats writes: jobs
 * submitted, completed, cancelled, failed, batches launched, most jobs in
 * flight at once, arena bytes.  scff_server_destroy cancels pending jobs,
 * lets in-flight batches finish, and frees the server (job ids become
 * invalid).
 */
typedef struct scff_server_s *scff_server_h;
typedef struct {
    int precision;        /* scff_precision of every job */
    int slots;            /* batches in flight at once (streams), 1..8 */
    int max_batch_jobs;   /* jobs per batch */
    uint64_t arena_bytes; /* device memory for in-flight jobs (0 = half the context budget) */
    double batch_cost_ratio; /* > 0: a batch takes only jobs whose work estimate (contraction
                                rows x states x evaluated points) is within this factor of its
                                first job's, so that small jobs do not wait for a large one to
                                finish; <= 0 (default): no limit.  On a 200-job stream with 5%
                                large jobs a factor of 16 did not lower p50/p99 (both slots'
                                launches share the SMs), so it is off by default */
} scff_server_options;
typedef struct {
    scff_basis_h basis;
    scff_trans_h trans;
    const double *qx;
    int nx;
    const double *qy;
    int ny;
    const double *qz;
    int nz;
    double scale;
    void *f_out;          /* [S][nq][2]: double for SCFF_FP64, float otherwise */
    void *f2_out;         /* [S][nq] or NULL */
    int out_on_device;    /* 1: device pointers, 0: host pointers */
} scff_request;
scff_status scff_server_create(scff_ctx *ctx, const scff_server_options *opt, scff_server_h *out);
scff_status scff_submit(scff_server_h server, const scff_request *req, int64_t *job_id);
scff_status scff_wait(scff_server_h server, int64_t job_id, int64_t timeout_us);
scff_status scff_cancel(scff_server_h server, int64_t job_id);
scff_status scff_job_times(scff_server_h server, int64_t job_id, double *ms_submit_admit_done);
scff_status scff_server_stats(scff_server_h server, int64_t *out);
void scff_server_destroy(scff_server_h server);

/* Waits for all work on `stream` and reports the device status word:
 * SCFF_ERR_TIMEOUT if a device-side wait of an asynchronous call gave up. */
scff_status scff_sync(scff_ctx *ctx, void *stream);

/* Tensor-core accumulation length: the FP32 TMEM accumulators are drained
 * into FP32 registers every `drain_every` k-chunks (0 = once, at the end;
 * -1 = the library default, 8; values below 2 act as 2).  The rounding of
 * the TMEM sums grows about linearly with this length (measured on a
 * 170-function, 12-state job in BF16 hi/mid/lo: 8 -> 3.1e-6, 16 -> 6.2e-6,
 * 32 -> 1.3e-5, whole K -> 2.3e-4), so the split modes' 1e-5 bar holds for
 * the default; longer runs are faster by about 1% only. */
scff_status scff_set_tc_drain(scff_ctx *ctx, int drain_every);

/* Path that the last successful scff_form_factor call of this context ran
 * (no counterpart in the paper): out[0] = 0 direct FP64, 1 direct FP32,
 * 2 tensor cores; out[1] = the scff_precision of its arithmetic (SCFF_FP32
 * when a tensor-core precision was asked for on an explicit q list, or when
 * the autotuner chose the FP32 direct path); out[2] = the W generator
 * variant the tensor-core kernel ran (0 gather, 1 Z staging, 2 prefetch, 3 CTA pairs,
 * 4 the octant form; see
 * scff_set_tc_variant), 0 off the tensor cores.  All -1 before the first
 * call. */
scff_status scff_last_path(scff_ctx *ctx, int32_t *out);

/* Tensor-core launch shape and W generator variant (no counterpart in the
 * paper); scff_set_tc_zstage is the same call under its earlier name.
 *   0 gather: each generator thread gathers its Y and Z table entries from
 *     global memory and keeps its share of the tile's running sums in
 *     registers.
 *   1 Z staging: on product grids whose z axis is a multiple of 128 points,
 *     every 128-column output tile lies in one y row, so one warp stages each
 *     k-chunk's Z row slices (1-D bulk copies) and Y values in shared memory
 *     for the generators.
 *   2 prefetch (FP16 hi/lo and BF16 hi/lo): the running sums live in tensor
 *     memory, and each generator thread gathers the next k-chunk's table
 *     entries while it forms the current chunk's W.
 *   3 CTA pairs (FP16 hi/lo and BF16 hi/lo, product grids): two CTAs on two
 *     SMs (a cluster) share each 256-row MMA (cta_group::2); each CTA holds
 *     the A rows of its half and generates W for half of the tile's columns,
 *     so every SM forms half as much W per unit of tensor work.
 *   4 the octant form (CTA pairs for FP16 hi/lo and BF16 hi/lo, single CTAs
 *     of the gather variant for BF16 hi/mid/lo): on grids whose three axes
 *     are antisymmetric (q[n-1-i] = -q[i]) the y and z factors at -q are the
 *     conjugates of those at +q, so W is formed real, one row per octant
 *     point and product of real or imaginary parts, and the eight real sums
 *     of a point give f at (qx, +-qy, +-qz) and, by f(-q) = conj(f(q)), at
 *     the mirrored points: half the tensor work and half the W values per
 *     output.  On other grids it runs as 3 (two-piece kinds) or 0.
 * mode: -1 automatic (the default: Z staging for TF32 hi/lo, the octant form
 * for FP16 hi/lo, BF16 hi/lo and BF16 hi/mid/lo; with
 * the autotuner on, tuned per job shape over the variants the grid and split
 * allow), 0 to 4 to request one (a variant the grid or split does not allow
 * runs as 0).  Variants 0 to 3 form bitwise the same W and add the same
 * partial sums in the same order, so their results are bitwise equal; the
 * octant form rounds differently (its W is real and its output is a sum of
 * four real sums) and meets the same accuracy bar.  A job's result depends
 * only on the job and this mode, never on the batch it runs in.  Applies to
 * calls, plans and servers created after it. */
scff_status scff_set_tc_variant(scff_ctx *ctx, int mode);
scff_status scff_set_tc_zstage(scff_ctx *ctx, int mode);

/*
 * Separable integrals (Sec. "Cartesian Grid Method": the one-axis V-tensors
 * alone give integrals of f_S against a product of one-axis functions):
 *   out[s] = scale * sum_{ix,iy,iz} wx[ix] wy[iy] wz[iz] f_s(qx[ix], qy[iy], qz[iz])
 * as (Re, Im) pairs, out[n_states][2] on the host, in FP64, without forming
 * the three-dimensional grid: the cost is linear in nx + ny + nz (the weights
 * carry the quadrature rule and the one-axis functions).  Host arrays in,
 * synchronous.
 */
scff_status scff_separable_integral(scff_ctx *ctx, scff_basis_h basis, scff_trans_h trans,
                                    const double *qx, const double *wx, int nx,
                                    const double *qy, const double *wy, int ny,
                                    const double *qz, const double *wz, int nz, double scale,
                                    double *out);

/*
 * Spherical method (Sec. "Analytic Method", Eqs. SphericalMethod, RTensor,
 * WTensor, YYY; Appendix B; Sec. "Spherical Grid Method"):
 *   f_s(q) = sum_{l <= lmax} sum_{m=-l..l} Y_l^m(q^) R^s_lm(|q|)
 * with complex spherical harmonics carrying the Condon-Shortley phase and
 * the coordinates of scff_basis as the expansion origin (centre the molecule
 * for the fastest convergence in l).  Each R^s_lm(q) is the exact
 * spherical-harmonic coefficient of f_s at radius q (no truncation inside
 * it); only the sum over l is truncated at lmax.
 *   grid->q[n_q]          radial |q| values (host, >= 0).
 *   grid->theta[n_theta], grid->phi[n_phi]: the angular product grid of f
 *                         (host; n_theta = n_phi = 0 for R and iso only).
 *   grid->lmax            0..40.
 * Outputs (any may be NULL; element type double for SCFF_FP64, float for the
 * tensor-core precisions SCFF_BF16X3, SCFF_TF32X3, SCFF_BF16X2; other
 * precisions give SCFF_ERR_INVALID_ARG):
 *   R_out   [S][n_q][(lmax+1)^2][2]  R^s_lm(q), lm = l*l + l + m, times scale.
 *   f_out   [S][n_q][n_theta][n_phi][2]  the truncated expansion on the grid.
 *   f2_out  [S][n_q][n_theta][n_phi]     |f|^2.
 *   iso_out [S][n_q]  (1/4pi) sum_{l <= lmax, m} |R_lm|^2, the isotropic
 *                     average of |f|^2 over directions (exact as lmax grows).
 * out_on_device selects device or host pointers; the call returns after
 * `stream` has finished.  The dense pair contraction runs on the tensor cores
 * for the split precisions and in FP64 on the CUDA cores for SCFF_FP64.
 */
typedef struct {
    int lmax;
    int n_q;
    const double *q;
    int n_theta;
    const double *theta;
    int n_phi;
    const double *phi;
} scff_sph_grid;

scff_status scff_spherical(scff_ctx *ctx, scff_basis_h basis, scff_trans_h trans, const scff_sph_grid *grid,
                           int precision, double scale, void *R_out, void *f_out, void *f2_out, void *iso_out,
                           int out_on_device, void *stream);

/*
 * FFT method (Sec. "The (Fast) Fourier Transform", Eqs. Falbega, continuFFT,
 * fftABC, qabc; Sec. "Fast Fourier Transform Method"): the transition density
 * Phi_s(r) = sum T^s_{mu nu} phi_mu(r) phi_nu(r) is tabulated on a box of
 * n[i] points per axis (powers of two, 4..1024), side L_i = 2 pi / dq[i],
 * centred at centre[i] (x_a = centre - L/2 + a L/n), and
 *   f_s(q) = scale * V_pix * sum_a Phi_s(x_a) e^{+i q.x_a},
 *   q = dq * (alpha - n/2), alpha = 0..n-1 per axis (ascending),
 * V_pix = prod_i L_i / n_i: the discrete Fourier sum that approximates Eq.
 * fSreal up to aliasing (spacing L/n too coarse for the densest Gaussians)
 * and tiling (box too small); the analytic methods have neither error.
 *   threshold  > 0: a primitive is dropped at points where its Gaussian
 *              factor exp(-alpha |r - A|^2) is below threshold (the paper's
 *              tabulation thresholding); 0 tabulates exactly.
 * Outputs (element type double for SCFF_FP64, float for SCFF_FP32; other
 * precisions give SCFF_ERR_INVALID_ARG):
 *   f_out  [S][n0][n1][n2][2], f2_out [S][n0][n1][n2] (either may be NULL);
 *   parseval_out [S][2] host doubles or NULL: (sum |Phi|^2 V_pix,
 *   sum |f|^2 dq0 dq1 dq2 / (2 pi)^3), equal for an exact discrete transform
 *   (Sec. "Verification", Parseval's theorem).
 * The basis may have at most ~1500 Cartesian functions (FP32; ~750 in FP64)
 * so that one tile's function values fit in shared memory (bases above ~370
 * functions in FP32, ~180 in FP64, run with 32-point tiles).  The call
 * returns after `stream` has finished.
 */
typedef struct {
    int n[3];
    double dq[3];
    double centre[3];
    double threshold;
} scff_fft_grid;

scff_status scff_fft_form_factor(scff_ctx *ctx, scff_basis_h basis, scff_trans_h trans, const scff_fft_grid *grid,
                                 int precision, double scale, void *f_out, void *f2_out, double *parseval_out,
                                 int out_on_device, void *stream);

/*
 * Hermitian half (default on).  For real T (the only kind this library
 * takes) the form factor obeys f(-q) = conj(f(q)) exactly (Eq. fSreal with a
 * real integrand).  On a product grid whose three axes are antisymmetric
 * (q[n-1-i] == -q[i] bitwise, e.g. the inclusive symmetric axes of the
 * paper's grids) scff_form_factor, plans and the server then evaluate only
 * the points of the first half of the flattened grid (the rows ix < nx/2 on
 * the tensor cores, plus the middle row when nx is odd) and write every other
 * point as the conjugate of its mirror; the output is the full grid.  enable
 * = 0 evaluates every point.  Applies to jobs created or submitted after the
 * call.
 */
scff_status scff_set_hermitian(scff_ctx *ctx, int enable);

/*
 * Overlapped download of host outputs (scff_form_factor with out_on_device =
 * 0 on the tensor-core path).  The output tiles then run band by band in one
 * launch, a band being a set of output columns (with the Hermitian half, a
 * column tile and its mirror together); the launch reports its progress to
 * host-mapped memory, and as soon as every tile of a band is written the host
 * issues a pitched device-to-host copy of the band's columns on a copy stream
 * of the context, so the copies run while later bands compute.  n_bands: 0 =
 * automatic (default: jobs of at least 1.25 waves of 128 x 128 tiles get
 * bands that end at the waves of the launch, up to 8), 1 = off (one copy
 * after the launch), 2..8 = that many equal bands where the grid allows.
 * Banding is skipped when the Hermitian half is on and ny*nz is not a
 * multiple of 128 (mirrored columns would cross tiles).  The band order hands
 * the tail split (the last tiles run as k-range parts) to other tiles than a
 * device-output call does, so results can differ from a device-output call
 * in the last bits of the FP32 sums of those tiles; both are within the
 * split-precision bounds.  Returns SCFF_ERR_INVALID_ARG for n_bands outside
 * 0..8.
 */
scff_status scff_set_download_bands(scff_ctx *ctx, int n_bands);

/*
 * Test hook of the failure-detection path (no counterpart in the paper):
 * launches one thread that waits on an mbarrier nothing arrives at, gives up
 * after `tries` (1..2^24) attempts exactly as every bounded wait of the
 * library does, and reports it through the context's error word.  Returns
 * SCFF_ERR_TIMEOUT when the wait ran out (the expected outcome); the context
 * remains usable afterwards.  Synchronous.
 */
scff_status scff_wait_selftest(scff_ctx *ctx, int64_t tries);

/*
 * ALU peak microbenchmark (measurement utility; no counterpart in the paper):
 * dependent fused multiply-add chains (8 per thread, 64 resident warps per SM)
 * on the context's device: fp64 = 0 FP32, 1 FP64, 2 FP32 as packed pairs
 * (f32x2, two FMAs per instruction); `iters` rounds per chain (1..2^24).  One
 * warm-up launch, then the best of three timed launches: *tflops = 2 x FMAs /
 * time, *ms = that launch's time.  Synchronous; the rooflines of the direct
 * (CUDA-core) kernels are quoted against it.  Other fp64 values:
 * SCFF_ERR_INVALID_ARG.
 */
scff_status scff_alu_peak(scff_ctx *ctx, int fp64, int iters, double *tflops, double *ms);

/*
 * Error-bounded pair screening (the exact-tolerance form of the paper's
 * pair thresholding, Sec. "Cartesian Grid Method").  With eps > 0, the
 * first scff_form_factor call for a (transitions, grid extent) bounds every
 * pair's contribution over |q| <= the grid's largest |q| (in FP64, from the
 * FP64 coefficients), evaluates f_s with the FP64 path at up to 64 grid
 * points (F_s = their largest |f_s|, lowered by a relative 1e-9), and removes
 * the pairs of smallest bound while, for every state, the summed bounds of
 * the removed pairs stay <= eps * F_s.  The result then differs from the
 * exact one by at most eps * max_q |f_s(q)| for every state and q.  The
 * compacted pair list is cached with the transitions.  eps = 0 (default)
 * evaluates every pair.  scff_screening_info: out[0..3] = kept pairs, all
 * pairs, kept and all contraction rows of the cached set.
 */
scff_status scff_set_screening(scff_ctx *ctx, double eps);
scff_status scff_screening_info(scff_ctx *ctx, scff_trans_h trans, scff_qgrid_h grid, int64_t *out);

/* Autotuner.  When enabled, the first scff_form_factor call for a job shape
 * (log-bucketed pair rows, states and grid points) in a tensor-core precision
 * on a product grid times the candidate configurations -- the tensor-core
 * path with TMEM drains of 8 k-chunks, and the FP32 direct path with state
 * blocks of 8, 12 and 16 -- on that job, and later calls of the same shape
 * use the fastest.  Every candidate meets the requested precision's bar (the
 * drain length is not tuned: the TMEM accumulation error grows linearly with
 * it, see scff_set_tc_drain).
 * scff_autotune_choice writes five values: out[0] = 1 tensor cores / 0 direct,
 * out[1] = drain, out[2] = state block, out[3] = best time in microseconds,
 * out[4] = the W generator variant chosen (scff_set_tc_variant's modes 0-3). */
scff_status scff_set_autotune(scff_ctx *ctx, int enable);
scff_status scff_autotune_choice(scff_ctx *ctx, scff_basis_h basis, scff_trans_h trans,
                                 scff_qgrid_h grid, int precision, int32_t *out);

/* Stage timing.  With timing enabled every scff_form_factor call records
 * CUDA events on its stream; scff_last_timing then waits for the last call
 * and writes ms_out[0] = q-evaluation kernel time, ms_out[1] = pair-prep and
 * table kernels, ms_out[2] = both (milliseconds, device clock). */
scff_status scff_set_timing(scff_ctx *ctx, int enable);
scff_status scff_last_timing(scff_ctx *ctx, double *ms_out);

/* Error statistics helper: count of q-evaluation kernel launches made by the
 * context since creation (for launch accounting in benchmarks). */
int64_t scff_kernel_launches(scff_ctx *ctx);

/*
 * Form factor without any device allocation (no counterpart in the paper: it
 * is a deployment variant of scff_form_factor for callers that cannot
 * allocate device memory -- a host framework whose caching allocator already
 * holds nearly all of HBM, a latency-bound serving loop where cudaMalloc and
 * cudaFree would synchronise the device, or a plugin that must not manage
 * device memory itself).
 *
 * It evaluates f_s(q) in FP64 on an explicit q list, with the same kernels as
 * scff_form_factor(..., SCFF_FP64, ...) on an scff_qgrid_list grid, but needs
 * no context or handles.  The basis is given as in scff_basis (host arrays);
 * T_dev [n_states][nbf][nbf], q_dev [n_q][3], f_dev [n_states][n_q][2] and
 * f2_dev [n_states][n_q] (or NULL) are caller-owned DEVICE buffers of FP64 on
 * the current device.  All intermediates live in one fixed 32 MiB device
 * array that belongs to the library and stays allocated on every GPU that
 * loaded the library until the process exits; host staging uses static
 * storage.  On success the call allocates nothing: no cudaMalloc, cudaFree
 * or other allocating routine (a rejected call stores its message for
 * scff_last_error()).  Only Cartesian shells: flags may hold
 * SCFF_RENORM_CONTRACTED alone; pure-shell flags return SCFF_ERR_INVALID_ARG.
 *
 * Limits: at most 256 primitive-shell records (one per primitive of every
 * shell) and n_states x coefficient rows within the scratch (about 3.9 M FP64
 * coefficients, states padded to a multiple of 4); larger inputs return
 * SCFF_ERR_INVALID_ARG with the limit in the message.
 *
 * Every call looks up the scratch array's device address in the current
 * context (cudaGetSymbolAddress, which allocates nothing), so the address
 * stays valid across cudaDeviceReset; the first call on a device loads the
 * library's module there, so make it before any stream capture.
 * Every call reuses the same scratch array, which keeps the previous call's
 * contents: the call rewrites everything it reads and clears its status word
 * itself.  Calls are serialised on the host, but calls whose GPU work could
 * overlap (for example on different streams of one device) race on the
 * scratch array; order them on one stream.  The call returns after `stream`
 * has finished its work.
 */
scff_status scff_form_factor_static(int n_atoms, const double *xyz, int n_shells,
                                    const int32_t *shell_atom, const int32_t *shell_l,
                                    const int32_t *shell_nprim, const double *exponents,
                                    const double *coefficients, uint32_t flags, int n_states,
                                    const double *T_dev, int64_t n_q, const double *q_dev,
                                    double scale, double *f_dev, double *f2_dev, void *stream);

void scff_release_basis(scff_ctx *ctx, scff_basis_h h);
void scff_release_transitions(scff_ctx *ctx, scff_trans_h h);
void scff_release_qgrid(scff_ctx *ctx, scff_qgrid_h h);

#ifdef __cplusplus
}
#endif
#endif /* SCFF_H */
