// Tensor-core (tcgen05) split-precision evaluation of the form factor on
// product grids.
//
// The Cartesian method factorises per axis (Eq. CartesianMethod with the
// V-tensors of Eq. CartesianVector): each pair term is
//   exp(-q^2/4p) e^{iq.P} sum_uvw i^{u+v+w} D_uvw q_x^u q_y^v q_z^w
//   = sum_uvw D_uvw X_u(q_x) Y_v(q_y) Z_w(q_z),
// with X_u(q) = (iq)^u exp(-q^2/4p) e^{i q P_x} (and Y, Z alike).  Grouping the
// x factor with the coefficients,
//   A[(s, ix), (pair, v, w)] = sum_u D^s_{pair,uvw} X_{pair,u}(q_x[ix])
//   W[(pair, v, w), (iy, iz)] = Y_{pair,v}(q_y[iy]) Z_{pair,w}(q_z[iz])
// turns the whole product-grid evaluation into one dense complex contraction
//   f[(s, ix), (iy, iz)] = sum_k A[(s,ix), k] W[k, (iy,iz)],
// which runs on the 5th-generation tensor cores:
//   * A (complex, FP32) is split into pieces (BF16 hi/mid/lo, BF16 hi/lo,
//     FP16 hi/lo or TF32 hi/lo) and stored as the SW64-swizzled K-major shared-memory image
//     of each 128 x 32-byte tile, so one 1-D bulk TMA copy lands a stage;
//   * W is generated on the fly by eight warps from FP64-accurate per-axis
//     tables (FP32 storage) and split the same way in shared memory;
//   * one thread issues tcgen05.mma (kind::f16 or kind::tf32, M = N = 128):
//     Re += Ar Wr - Ai Wi and Im += Ar Wi + Ai Wr, each product as the piece
//     products that matter for the split (six for hi/mid/lo, three for
//     hi/lo), the minus sign through the instruction's negate-A bit;
//   * two TMEM accumulator sets (Re and Im, 128 x 128 FP32 each: all 512
//     columns) alternate, and the generators drain a finished set into FP32
//     registers every `drain_every` k-chunks (bounding each TMEM sum);
//   * one persistent CTA per SM walks a cost-sorted list of (job, m-tile,
//     n-tile) items; the last (tiles mod SMs) tiles of a job run as parts over
//     disjoint k ranges whose partial sums the last part to finish adds up in
//     part order (the tail split);
//   * on antisymmetric grids only half the rows are evaluated and the
//     epilogue also writes f(-q) = conj(f(q)) at the mirrored point.
// The same kernel runs the spherical method's contractions (tc_run_generic),
// with W generated from its radial and harmonic tables.  FP64 is used only for
// the tables (range reduction of q.P) and upstream in the pair-prep.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "device_common.cuh"
#include "../../include/scff.h"
#include "scff_internal.h"
#include "tc_internal.h"
#include "tc_schedule.h"

#include <algorithm>
#include <type_traits>
#include <string.h>
#include <thread>
#include <vector>

namespace scff {
namespace tc {

constexpr int BM = 128;                              // rows (s, ix) per tile
constexpr int BN = 128;                              // columns (iy, iz) per tile
constexpr int ROW_BYTES = 64;                        // one K-chunk row (64B swizzle)
constexpr int A_ARR = BM * ROW_BYTES;                // bytes of one A array
constexpr int W_ARR = BN * ROW_BYTES;                // bytes of one W array
constexpr int GEN_WARPS = 8;                         // W generators and accumulator drains
constexpr int THREADS = 128 + GEN_WARPS * 32;        // warpgroup 0: TMA warp, MMA warp, 2 idle
constexpr int TMEM_COLS = 512;                       // two sets of (Re, Im) x 128 columns
constexpr int BAR_BYTES = 512;                       // mbarriers, TMEM slot, abort flag, item ring
constexpr int IRING = 4;                             // work items published ahead to the roles
// Register split between warpgroups (setmaxnreg): the launch provides
// THREADS x LAUNCH_REGS registers; warpgroup 0 keeps LOW_REGS per thread and
// the two generator warpgroups take HIGH_REGS.  The shares add up to the
// launch total exactly, and the host checks the compiled count before launch.
// Warpgroup 0 runs two single-thread roles (and the Z stager), which fit in
// 40; the generators' extra registers removed their spills (FP16 hi/lo on the
// 10-heavy-atom job: 7.73 ms with 72/216, 7.36 ms with 40/232).
constexpr int LAUNCH_REGS = 168;
constexpr int LOW_REGS = 40;
constexpr int HIGH_REGS = 232;
static_assert(128 * LOW_REGS + GEN_WARPS * 32 * HIGH_REGS == THREADS * LAUNCH_REGS, "register split");
static_assert(2 * BN == GEN_WARPS * 32, "two generator threads per W row");

// Split kinds.  Every value x of A and W is stored as NP pieces whose sum is x
// to about 8*NP (BF16), 22 (FP16, TF32) bits; the products kept are those whose
// piece orders add up to at most NP-1, which bounds the dropped terms by the
// precision of the split.
//   KIND_BF16X2: BF16 hi + lo,        products hh, hl, lh          (~2^-16)
//   KIND_BF16X3: BF16 hi + mid + lo,  products hh, hm, mh, hl, lh, mm (~2^-24)
//   KIND_TF32X2: TF32 hi + lo,        products hh, hl, lh          (~2^-21)
//   KIND_FP16X2: FP16 hi + lo,        products hh, hl, lh          (~2^-22)
// FP16 has 11 significant bits but only five exponent bits, so that kind
// works on scaled operands: every (pair, axis, power) row of the Y and Z
// tables is multiplied by a power of two that brings its largest possible
// magnitude on the grid to 2^6 (so |W| <= 2^12), each A column by the inverse
// of its W row's factor, and all of A by one further power of two per job
// chosen from a bound on the largest term; the epilogue removes that factor.
// Power-of-two factors are exact, so only the pieces' rounding remains.
enum { KIND_BF16X2 = 0, KIND_BF16X3 = 1, KIND_TF32X2 = 2, KIND_FP16X2 = 3 };

template <int KIND> struct Kind {
    static constexpr bool TF32 = KIND == KIND_TF32X2;
    static constexpr bool FP16 = KIND == KIND_FP16X2;
    // operand format of the instruction descriptor: 0 FP16, 1 BF16 (kind::f16), 2 TF32 (kind::tf32)
    static constexpr uint32_t FMT = TF32 ? 2u : FP16 ? 0u : 1u;
    static constexpr int NP = KIND == KIND_BF16X3 ? 3 : 2;          // pieces per value
    static constexpr int NPROD = NP == 3 ? 6 : 3;                    // piece products per complex part
    static constexpr int ELEM = TF32 ? 4 : 2;
    static constexpr int BK = ROW_BYTES / ELEM;                      // k per chunk
    static constexpr int PER_VEC = 16 / ELEM;                        // elements per 16-byte vector
    static constexpr int A_STAGE = 2 * NP * A_ARR;                   // re pieces, then im pieces
    // FUSE (two-piece kinds): each W piece is stored as three adjacent
    // 128-row arrays [-Wi | Wr | Wi], so one N = 256 MMA with B = rows
    // [Wr; Wi] adds [Ar Wr | Ar Wi] and one with B = [-Wi; Wr] adds
    // [-Ai Wi | Ai Wr] to the [Re | Im] accumulator: half the MMA
    // instructions of four N = 128 products, and a quarter fewer operand
    // bytes read from shared memory.  Otherwise the pieces are [Wr... | Wi...].
    static constexpr bool FUSE = NP == 2;
    static constexpr int W_STAGE = (FUSE ? 3 : 2) * NP * W_ARR;
    static constexpr int STAGE = A_STAGE + W_STAGE;
    static constexpr int STAGES = 2;
    // stages, then the barriers (256 B), then each generator warp's two
    // k-offset buffers (KO_BYTES).  Staging the k-offsets through shared
    // memory pays where the generators set the pace (BF16 hi/lo: -8%); where
    // the tensor pipe does (hi/mid/lo, TF32) it costs about 1%, so those read
    // them straight from global memory.
    static constexpr bool STAGE_KO = KIND == KIND_BF16X2 || KIND == KIND_FP16X2;
    static constexpr int KO_BYTES = STAGE_KO ? GEN_WARPS * 2 * (BK / 2) * 8 : 0;
    static constexpr int SMEM_BYTES = STAGES * STAGE + 1024 + BAR_BYTES + KO_BYTES;
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
};

// Launch configuration of the persistent kernel per split kind and W generator
// variant VAR:
//   VAR_GATHER: the generators gather their Y and Z table entries from global
//     memory (any product grid, the spherical method's tables) and keep the
//     tile's running sums in registers; two TMEM accumulator sets alternate.
//   VAR_ZSTAGE (two-piece kinds, grids with nz a multiple of 128): every tile
//     lies in one y row, so a chunk needs one Y value per k (shared by all
//     tile rows) and one 128-entry slice of a Z row per k; warp 2 stages both
//     into shared memory one chunk ahead (the slices by 1-D bulk copies), and
//     the generators read shared memory only.  Two stages then fit beside
//     the two Z slots.
//   VAR_PREFETCH (kinds that stage their k-offsets): the running sums live in
//     TMEM (one accumulator set for the MMAs, one for the sums, added to by
//     the generators in FP32 at every drain), which frees the registers for
//     a second set of table entries: each generator thread gathers the next
//     chunk's entries before it forms the current chunk's W, so the gather
//     latency overlaps the W work instead of preceding it.  The additions are
//     the same, in the same order, as VAR_GATHER's, so both give bitwise the
//     same tile.
//   VAR_OCT (the kinds with CTA pairs, antisymmetric grids): the CTA-pair
//     launch with the jobs in the octant form (TcJobDev::oct), which the
//     pair kernel runs per job.
enum { VAR_GATHER = 0, VAR_ZSTAGE = 1, VAR_PREFETCH = 2, VAR_PAIR = 3, VAR_OCT = 4 };
// Octant form: points per CTA-pair tile and per CTA.
constexpr int OCT_PTS = 32;
constexpr int OCT_PTH = OCT_PTS / 2;
template <int KIND, int VAR> struct Cfg {
    using KD = Kind<KIND>;
    static constexpr bool ZS = VAR == VAR_ZSTAGE;
    static constexpr bool PF = VAR == VAR_PREFETCH;
    static constexpr int STAGES = ZS ? 2 : KD::STAGES;
    static constexpr int ZSLOT = KD::BK * BN * 8;   // Z row slices of one chunk (float2)
    static constexpr int YSLOT = KD::BK * 8;        // Y values of one chunk
    // Z slots: three (the stager two chunks ahead) where shared memory allows
    static constexpr int ZSLOTS =
        STAGES * KD::STAGE + 1024 + BAR_BYTES + 3 * (ZSLOT + YSLOT) <= 232448 ? 3 : 2;
    static constexpr int ZBYTES = ZS ? ZSLOTS * (ZSLOT + YSLOT) : 0;
    static constexpr int KO_BYTES = ZS ? 0 : KD::KO_BYTES;
    static constexpr int SMEM_BYTES = STAGES * KD::STAGE + 1024 + BAR_BYTES + KO_BYTES + ZBYTES;
    static_assert(!ZS || KD::NP == 2, "Z staging is built for the two-piece kinds");
    static_assert(!PF || KD::STAGE_KO, "the prefetching generators read staged k-offsets");
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
};

// CTA-pair launch (VAR_PAIR): a cluster of two CTAs on two SMs computes a
// 256-row x 128-column tile with M = 256 MMAs (cta_group::2).  Each CTA holds
// the A rows of its own 128-row half, and the B operand (W) is split along N:
// each CTA generates W for 64 of the tile's 128 columns only, as
// [-Wi | Wr | Wi] arrays of 64 rows, so that CTA r supplies the pair's B rows
// [Wr | Wi] (and [-Wi | Wr]) of its columns.  D in each CTA's TMEM is then
// [Re | Im] of columns 0-63 followed by [Re | Im] of columns 64-127, for the
// CTA's own rows.  Per SM the MMA work per chunk is that of the single-CTA
// kernel, and the W generation half of it.
// OCTK: the build for launches whose jobs all run in the octant form (real
// W: one 64-row array per piece and CTA), whose smaller stages leave room for
// a fifth.
template <int KIND, bool OCTK = false> struct PairCfg {
    using KD = Kind<KIND>;
    static constexpr int BNH = BN / 2;                     // W rows (complex columns) per CTA
    static constexpr int W_ARRH = BNH * ROW_BYTES;         // one 64-row W array
    static constexpr int W_STAGE = (OCTK ? 1 : 3) * KD::NP * W_ARRH;
    static constexpr int STAGE = KD::A_STAGE + W_STAGE;
    static constexpr int STAGES = OCTK ? 5 : 4;
    static constexpr int KQ = KD::BK / 4;                  // k per generator thread (four per W row)
    static constexpr int KO_BYTES = GEN_WARPS * 2 * KQ * 8;
    static constexpr int SMEM_BYTES = STAGES * STAGE + 1024 + BAR_BYTES + KO_BYTES;
    static_assert(KD::FUSE && KD::STAGE_KO && !KD::TF32, "pairs are built for the 16-bit two-piece kinds");
    static_assert(KQ == KD::PER_VEC, "one 16-byte vector per generator thread and chunk");
    static_assert(4 * BNH == GEN_WARPS * 32, "four generator threads per W row");
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
    // mbarrier and flag slots (8 bytes each) in the BAR_BYTES region
    static constexpr int BO = 3 * STAGES;
    static_assert((BO + 20) * 8 <= BAR_BYTES, "barrier region");
};

// Piece orders of the kept products (A piece, W piece).
__host__ __device__ constexpr int prod_a(int i) { return i == 0 ? 0 : i == 1 ? 0 : i == 2 ? 1 : i == 3 ? 0 : i == 4 ? 2 : 1; }
__host__ __device__ constexpr int prod_w(int i) { return i == 0 ? 0 : i == 1 ? 1 : i == 2 ? 0 : i == 3 ? 2 : i == 4 ? 0 : 1; }

// Byte offset of element (row, c) in a K-major array with 64-byte rows under
// the 64B swizzle (16-byte chunk index XOR address bits 7-8).
template <int KIND>
__host__ __device__ __forceinline__ uint32_t sw64_offset(int row, int c) {
    constexpr int E = Kind<KIND>::ELEM, V = Kind<KIND>::PER_VEC;
    const int rr = row & 7;
    return (uint32_t)((row >> 3) * 512 + rr * 64 + ((((c / V) ^ ((rr >> 1) & 3))) << 4) + (c % V) * E);
}

// ------------------------------------------------------------------ FP16 operand scaling

// Exponent e with 2^e >= max_{|q| <= Q} |q|^u exp(-q^2/(4p)) (inv4p = 1/(4p)):
// the largest magnitude row u of a pair's axis table can take on an axis
// whose points satisfy |q| <= Q.  For u >= 1 the maximum sits at q^2 = 2pu,
// or at |q| = Q when the grid ends before it.  FP32 arithmetic with a margin
// of 1e-3 in the exponent, rounded up, clamped to [-60, 60].
__host__ __device__ __forceinline__ int axis_row_exp(int u, double inv4p, double Q) {
    if (u == 0) return 0;
    constexpr float kLog2e = 1.4426950408889634f;
    const float fu = (float)u, i4 = (float)inv4p, q = (float)Q;
    const float peak2 = fu / (2.f * i4);
    const float l2 = peak2 <= q * q ? 0.5f * fu * (log2f(peak2) - kLog2e) : fu * log2f(q) - q * q * i4 * kLog2e;
    return (int)fminf(60.f, fmaxf(-60.f, ceilf(l2 + 1e-3f)));
}

// Target magnitude exponents of the FP16 kind: table rows are scaled to at
// most 2^kRowExp, so |W| <= 2^(2 kRowExp); A is scaled so its largest
// possible entry is at most 2^kAExp.
constexpr int kRowExp = 6;
constexpr int kAExp = 14;

// x * 2^n for |n| <= 252, exact unless the result over- or underflows.
__device__ __forceinline__ float pow2_scale(float x, int n) {
    const int a = n / 2, b = n - a;
    return x * __int_as_float((127 + a) << 23) * __int_as_float((127 + b) << 23);
}

// Job exponent G of the FP16 kind from the bound t of its largest term
// (FP64 bits, 0 for an all-zero job): A carries 2^G so that the largest term
// maps to about 2^(kAExp + 2 kRowExp).  ceil(log2 t) is read from the bits.
__device__ __forceinline__ int fp16_job_exp(const unsigned long long *tmax) {
    const unsigned long long b = *tmax;
    if (b == 0) return 0;
    const int ex = (int)((b >> 52) & 0x7FF) - 1023;
    const int cl = ex + ((b & 0xFFFFFFFFFFFFFull) != 0 ? 1 : 0);
    return max(-100, min(100, kAExp + 2 * kRowExp - cl));
}

// ------------------------------------------------------------------ PTX wrappers

// 8-byte asynchronous global -> shared copy (LDGSTS) and its group bookkeeping.
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
    // start address >> 4, LBO unused (0), SBO = 512 B (8 rows x 64 B),
    // version 1 (bits 46-47), layout SWIZZLE_64B = 4 (bits 61-63).
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}

// Instruction descriptor: D FP32, A and B of one format (FMT: 0 FP16 or
// 1 BF16 under kind::f16, 2 TF32 under kind::tf32), both K-major, M = 128,
// N = 128; bit 13 negates A.
template <uint32_t FMT, int N = BN, int M = BM>
constexpr uint32_t idesc_mma(bool neg_a) {
    return (1u << 4) | (FMT << 7) | (FMT << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Stores one 16-byte vector of W pieces (real pr, imaginary pi) at byte
// offset off of every array of a W stage, in the kind's layout.
template <int KIND>
__device__ __forceinline__ void store_w(uint8_t *wst, uint32_t off, const uint4 (&pr)[Kind<KIND>::NP],
                                        const uint4 (&pi)[Kind<KIND>::NP]) {
    using KD = Kind<KIND>;
    constexpr int NP = KD::NP;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        if constexpr (KD::FUSE) {
            // sign bits of the pieces: 16-bit elements in pairs, TF32 one per word
            constexpr uint32_t SGN = KD::TF32 ? 0x80000000u : 0x80008000u;
            const uint4 ni = make_uint4(pi[q].x ^ SGN, pi[q].y ^ SGN, pi[q].z ^ SGN, pi[q].w ^ SGN);
            uint8_t *pb = wst + q * 3 * W_ARR + off;
            *reinterpret_cast<uint4 *>(pb) = ni;
            *reinterpret_cast<uint4 *>(pb + W_ARR) = pr[q];
            *reinterpret_cast<uint4 *>(pb + 2 * W_ARR) = pi[q];
        } else {
            *reinterpret_cast<uint4 *>(wst + q * W_ARR + off) = pr[q];
            *reinterpret_cast<uint4 *>(wst + (NP + q) * W_ARR + off) = pi[q];
        }
    }
}

template <bool TF32>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns from registers into TMEM.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 "
        "[%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- CTA pairs (a cluster of two CTAs on two SMs sharing each MMA)

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Shared-memory address of the same location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(const void *p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}

// Arrives on an mbarrier of another CTA of the cluster (release at cluster
// scope: this thread's earlier writes, shared or global, are visible to a
// thread that observes the phase with an acquiring wait).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void st_cluster_s32(uint32_t cluster_addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (as mbar_wait) acquiring at cluster scope, for barriers that
// other CTAs of the cluster arrive on; also gives up once abort_flag is set.
__device__ __forceinline__ bool mbar_wait_cl(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1; i < kWaitLimit; ++i) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((i & 15) == 0 && (*abort_flag || global_ns() - t0 > kWaitNs)) return false;
    }
    return false;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMEM allocation shared by the pair: one warp of each CTA takes part.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// One MMA over the pair (issued by the even CTA): A rows 0-127 from CTA 0's
// shared memory and 128-255 from CTA 1's at the same address, B's N rows
// 0-127 from CTA 0 and 128-255 from CTA 1; each CTA's TMEM receives its own
// 128 rows of D at tmem_d.
__device__ __forceinline__ void mma_issue_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Arrives once on the mbarrier at this address in both CTAs of the pair when
// the issuing thread's earlier MMAs have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// Splits one 16-byte vector worth of values into NP pieces (pieces[0] = hi).
//   BF16: 8 values per vector; each piece rounds the remaining residual to BF16.
//   TF32: 4 values per vector; hi = x with the 13 low mantissa bits cleared
//         (exactly a TF32 number), lo = x - hi (exact in FP32; the MMA reads
//         its top 19 bits).
template <int KIND>
__device__ __forceinline__ void split_vec(const float *x, uint4 (&pc)[Kind<KIND>::NP]) {
    constexpr int NP = Kind<KIND>::NP;
    if constexpr (Kind<KIND>::TF32) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float hf = __uint_as_float(__float_as_uint(x[i]) & 0xFFFFE000u);
            h[i] = __float_as_uint(hf);
            l[i] = __float_as_uint(x[i] - hf);
        }
        pc[0] = make_uint4(h[0], h[1], h[2], h[3]);
        pc[1] = make_uint4(l[0], l[1], l[2], l[3]);
    } else if constexpr (Kind<KIND>::FP16) {
        // hi = x rounded to FP16, lo = the remainder rounded to FP16 (the
        // operands are scaled into FP16's normal range beforehand)
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 hh = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
            const float2 hf = __half22float2(hh);
            const __half2 ll = __floats2half2_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
            h[i] = *reinterpret_cast<const uint32_t *>(&hh);
            l[i] = *reinterpret_cast<const uint32_t *>(&ll);
        }
        pc[0] = make_uint4(h[0], h[1], h[2], h[3]);
        pc[1] = make_uint4(l[0], l[1], l[2], l[3]);
    } else {
        float r[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) r[i] = x[i];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
                const float2 bf = __bfloat1622float2(b);
                r[2 * i] -= bf.x;
                r[2 * i + 1] -= bf.y;
                w[i] = *reinterpret_cast<const uint32_t *>(&b);
            }
            pc[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// One element of W: the complex product y z with each rounding explicit, so
// every generator variant forms bitwise the same value.
__device__ __forceinline__ void w_elem(float2 a, float2 b, float &re, float &im) {
    re = __fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y));
    im = __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x));
}

// ------------------------------------------------------------------ layout

struct Layout {
    int64_t n_axrows;  // zero row index of the axis tables
    int64_t K, K_pad;  // contraction length and padded length
    int nkc;           // k-chunks
    int M, M_pad, n_mt;
    int64_t N;
    int n_nt;
    int part_tiles;    // partial-sum tiles reserved for the tail split
    size_t off_X, off_Y, off_Z, off_k, off_ko, off_kexp, off_tmax, off_A, off_part, off_cnt, total;
};

using sched::tail_split;

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static Layout make_layout(const PairSetDev &ps, int S, int nx, int ny, int nz, int BK, int a_stage) {
    Layout L;
    L.n_axrows = ps.n_axrows;
    L.K = ps.n_krows;
    L.K_pad = (L.K + BK - 1) / BK * BK;
    if (L.K_pad == 0) L.K_pad = BK;
    L.nkc = (int)(L.K_pad / BK);
    L.M = S * nx;
    // sized for an even number of m-tiles, so a job can also be laid out for the CTA-pair launch
    L.M_pad = (L.M + 2 * BM - 1) / (2 * BM) * (2 * BM);
    L.n_mt = L.M_pad / BM;
    L.N = (int64_t)ny * nz;
    L.n_nt = (int)((L.N + BN - 1) / BN);
    size_t o = 0;
    L.off_X = o;
    o = align_up(o + sizeof(float2) * (size_t)(L.n_axrows + 1) * nx, 1024);
    L.off_Y = o;
    o = align_up(o + sizeof(float2) * (size_t)(L.n_axrows + 1) * ny, 1024);
    L.off_Z = o;
    o = align_up(o + sizeof(float2) * (size_t)(L.n_axrows + 1) * nz, 1024);
    L.off_k = o;
    o = align_up(o + sizeof(int4) * (size_t)L.K_pad, 1024);
    L.off_ko = o;
    o = align_up(o + sizeof(int2) * (size_t)L.K_pad, 1024);
    L.off_kexp = o;  // FP16 kind: per-k exponent of the W row factor
    o = align_up(o + sizeof(int) * (size_t)L.K_pad, 1024);
    L.off_tmax = o;  // FP16 kind: bound of the job's largest term (FP64 bits)
    o = align_up(o + 256, 1024);
    L.off_A = o;
    o = align_up(o + (size_t)L.n_mt * L.nkc * a_stage, 1024);
    // a split never needs more than 2P partial tiles (R * s <= 2P); the
    // octant form's column tiles are counted too
    const int64_t n_oct_nt = ((int64_t)((ny + 1) / 2) * ((nz + 1) / 2) + OCT_PTS - 1) / OCT_PTS;
    L.part_tiles = std::min<int64_t>(2 * (int64_t)tc_num_sms(), (int64_t)L.n_mt * std::max<int64_t>(L.n_nt, n_oct_nt) * 16);
    L.off_part = o;
    o = align_up(o + sizeof(float2) * (size_t)L.part_tiles * BM * BN, 1024);
    L.off_cnt = o;
    o = align_up(o + sizeof(int) * 8 * (size_t)L.part_tiles, 1024);
    L.total = o;
    return L;
}

template <int KIND>
static Layout make_layout_k(const PairSetDev &ps, int S, int nx, int ny, int nz) {
    return make_layout(ps, S, nx, ny, nz, Kind<KIND>::BK, Kind<KIND>::A_STAGE);
}

// ------------------------------------------------------------------ prep kernels

// X_{pair,u}(q_i) = (i q_i)^u exp(-q_i^2/(4p)) e^{i q_i P_axis}, stored in FP32:
// one thread per (pair, q_i) evaluates the Gaussian and the phase once and
// writes the rows u = 0..L of its pair; the extra row n_axrows is zero.  The
// phase q P is reduced to [-pi, pi] in FP64 (Cody-Waite with 2 pi split in
// two doubles), so the FP32 sine and cosine of the remainder and the FP32
// exponential are as accurate as the FP32 table entries; the powers of i q
// are applied in FP32 (row u carries at most u + 2 roundings of 2^-24).
// With Q >= 0 (FP16 kind) every row u is multiplied by 2^(kRowExp - e_u),
// e_u = axis_row_exp(u, 1/(4p), Q) with Q >= max |q_i| of the axis.
__global__ void axis_power_table_kernel(PairSetDev ps, const double *__restrict__ geom,
                                        const double *__restrict__ qaxis, int n, int axis, int64_t n_axrows,
                                        float2 *__restrict__ table, double Q) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((int64_t)ps.n_pair + 1) * n) return;
    const int pr = (int)(idx / n);
    const int i = (int)(idx % n);
    if (pr == ps.n_pair) {
        table[n_axrows * n + i] = make_float2(0.f, 0.f);
        return;
    }
    int L = 0;
    while (L < kMaxPairL && pr >= ps.pair_off[L + 1]) ++L;
    const int64_t row0 = ps.axrow_off[L] + (int64_t)(pr - ps.pair_off[L]) * (L + 1);
    const double q = qaxis[i];
    const double P = geom[4 * pr + axis], inv4p = geom[4 * pr + 3];
    constexpr double kTwoPiHi = 6.283185307179586, kTwoPiLo = 2.4492935982947064e-16;
    const double th = q * P;
    const double nk = rint(th * (1.0 / kTwoPiHi));
    const float r = (float)fma(-nk, kTwoPiLo, fma(-nk, kTwoPiHi, th));
    float sf, cf;
    sincosf(r, &sf, &cf);
    const float g = expf((float)(-q * q * inv4p));
    // powers of i q in FP32: each step adds one rounding of 2^-24, so row u
    // carries at most u + 2 of them (the entries are stored in FP32 anyway)
    const float qf = (float)q;
    float re = cf * g, im = sf * g;
    for (int u = 0; u <= L; ++u) {
        const int e = Q >= 0.0 ? kRowExp - axis_row_exp(u, inv4p, Q) : 0;  // exact power-of-two row scale
        table[(row0 + u) * n + i] = make_float2(ldexpf(re, e), ldexpf(im, e));
        // times i q
        const float nr = -qf * im, ni = qf * re;
        re = nr;
        im = ni;
    }
}

// k -> (pair, v, w, first axis row of the pair); padding k -> (-1, 0, 0, zero row);
// kofs[k] = element offsets of k's rows in the Y and Z tables.
__global__ void kindex_kernel(PairSetDev ps, int64_t K_pad, int64_t n_axrows, int ny, int nz, int4 *__restrict__ kinfo,
                              int2 *__restrict__ kofs) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K_pad) return;
    int4 r = make_int4(-1, 0, 0, (int)n_axrows);
    if (k < ps.n_krows) {
        int L = 0;
        while (L < kMaxPairL && k >= ps.krow_off[L + 1]) ++L;
        const int64_t local = k - ps.krow_off[L];
        const int nvw = vw_count(L);
        const int j = (int)(local % nvw);
        const int pr = ps.pair_off[L] + (int)(local / nvw);
        int v = 0, w = 0, cnt = 0;
        for (int t = 0; t <= L; ++t)
            for (int vv = t; vv >= 0; --vv) {
                if (cnt == j) {
                    v = vv;
                    w = t - vv;
                }
                ++cnt;
            }
        const int axbase = (int)(ps.axrow_off[L] + (int64_t)(pr - ps.pair_off[L]) * (L + 1));
        r = make_int4(pr, v, w, axbase);
    }
    kinfo[k] = r;
    kofs[k] = make_int2((r.w + r.y) * ny, (r.w + r.z) * nz);  // Y and Z row offsets of this k
}

// FP16 kind: per k = (pair, v, w), kexp[k] = e_v(Y) + e_w(Z), the exponent
// of the factor 2^(2 kRowExp - kexp) that the scaled tables put on W row k,
// and a bound of the term of k over the grid,
//   t_k = max_s sum_u |D^s_{pair,uvw}| 2^(e_u(X)) * 2^kexp >= |A[(s,ix),k] W[k,n]|,
// whose maximum over k (FP64 bits; positive doubles order as integers) sets
// the job exponent (fp16_job_exp).
__global__ void fp16_bound_kernel(PairSetDev ps, const float *__restrict__ coef32, int SB, int S,
                                  const double *__restrict__ geom, const int4 *__restrict__ kinfo, int64_t K_pad,
                                  double Qx, double Qy, double Qz, int *__restrict__ kexp,
                                  unsigned long long *__restrict__ tmax) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K_pad) return;
    const int4 ki = kinfo[k];
    if (ki.x < 0) {
        kexp[k] = 0;
        return;
    }
    int L = 0;
    while (L < kMaxPairL && ki.x >= ps.pair_off[L + 1]) ++L;
    const double inv4p = geom[4 * ki.x + 3];
    const int e = axis_row_exp(ki.y, inv4p, Qy) + axis_row_exp(ki.z, inv4p, Qz);
    kexp[k] = e;
    const int nu = L - ki.y - ki.z + 1;
    float xb[kMaxPairL + 1];
    for (int u = 0; u < nu; ++u) xb[u] = ldexpf(1.f, axis_row_exp(u, inv4p, Qx));
    const int64_t rowbase = ps.row_off[L] + (int64_t)(ki.x - ps.pair_off[L]) * mono_count(L);
    float best = 0.f;
    for (int s = 0; s < S; ++s) {
        const float *cs = coef32 + ((size_t)(s / SB) * ps.n_rows) * SB + (s % SB);
        float sum = 0.f;
        for (int u = 0; u < nu; ++u) sum += fabsf(cs[(size_t)(rowbase + mono_index(u, ki.y, ki.z)) * SB]) * xb[u];
        best = fmaxf(best, sum);
    }
    const double t = ldexp((double)best, e);
    if (t > 0.0) atomicMax(tmax, (unsigned long long)__double_as_longlong(t));
}

// Thread index -> (row m, 16-byte vector kv) of a tile image: consecutive
// threads take the vectors of one chunk row, then the next row of the same
// chunk, so a warp writes 512 contiguous bytes of each array of the image.
template <int KIND>
__device__ __forceinline__ void image_coords(int64_t idx, int nkc, int &m, int64_t &kv) {
    using KD = Kind<KIND>;
    constexpr int VPC = KD::BK / KD::PER_VEC;  // vectors per chunk row
    const int v = (int)(idx % VPC);
    const int r = (int)((idx / VPC) % BM);
    const int64_t tile = idx / (VPC * BM);  // mt * nkc + kc
    const int64_t kc = tile % nkc;
    m = (int)(tile / nkc) * BM + r;
    kv = kc * VPC + v;
}

// A[(s,ix), k] = sum_u D^s_{pair,(u,v,w)} X_{pair,u}(q_x[ix]), split into pieces
// and written as the swizzled shared-memory image of each tile.  One thread
// writes one 16-byte vector (PER_VEC consecutive k) of each array.
// FP16 kind: column k is multiplied by 2^(kexp[k] - 2 kRowExp + G), G the
// job exponent (the scaled W row k carries 2^(2 kRowExp - kexp[k])).
template <int KIND>
__global__ void abuild_kernel(PairSetDev ps, const float *__restrict__ coef32, int SB, int nxr, int nx,
                              const float2 *__restrict__ X, const int4 *__restrict__ kinfo, int64_t K_pad, int nkc,
                              int M, int M_pad, uint8_t *__restrict__ Abuf, const int *__restrict__ kexp,
                              const unsigned long long *__restrict__ tmax) {
    using KD = Kind<KIND>;
    constexpr int V = KD::PER_VEC, BK = KD::BK, NP = KD::NP;
    const int64_t kvn = K_pad / V;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M_pad * kvn) return;
    int m;
    int64_t kv;
    image_coords<KIND>(idx, nkc, m, kv);
    int G = 0;
    if constexpr (KD::FP16) G = fp16_job_exp(tmax) - 2 * kRowExp;
    float re[V], im[V];
    const bool mvalid = m < M;
    const int s = mvalid ? m / nxr : 0, ix = mvalid ? m % nxr : 0;  // rows (s, ix < nxr); X has nx columns
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int4 ki = kinfo[kv * V + e];
        float ar = 0.f, ai = 0.f;
        if (mvalid && ki.x >= 0) {
            int L = 0;
            while (L < kMaxPairL && ki.x >= ps.pair_off[L + 1]) ++L;
            const int64_t rowbase = ps.row_off[L] + (int64_t)(ki.x - ps.pair_off[L]) * mono_count(L);
            const float *cs = coef32 + ((size_t)(s / SB) * ps.n_rows) * SB + (s % SB);
            for (int u = 0; u <= L - ki.y - ki.z; ++u) {
                const int mi = mono_index(u, ki.y, ki.z);
                const int n = u + ki.y + ki.z;
                const float c = cs[(size_t)(rowbase + mi) * SB] * ((n & 2) ? -1.f : 1.f);
                const float2 x = X[(size_t)(ki.w + u) * nx + ix];
                ar = fmaf(c, x.x, ar);
                ai = fmaf(c, x.y, ai);
            }
            if constexpr (KD::FP16) {
                const int sh = kexp[kv * V + e] + G;
                ar = pow2_scale(ar, sh);
                ai = pow2_scale(ai, sh);
            }
        }
        re[e] = ar;
        im[e] = ai;
    }
    uint4 pr_[NP], pi_[NP];
    split_vec<KIND>(re, pr_);
    split_vec<KIND>(im, pi_);
    const int mt = m / BM, r = m % BM;
    const int64_t kc = (kv * V) / BK;
    const int c0 = (int)((kv * V) % BK);
    uint8_t *base = Abuf + ((size_t)mt * nkc + kc) * KD::A_STAGE;
    const uint32_t off = sw64_offset<KIND>(r, c0);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        *reinterpret_cast<uint4 *>(base + q * A_ARR + off) = pr_[q];
        *reinterpret_cast<uint4 *>(base + (NP + q) * A_ARR + off) = pi_[q];
    }
}

// The same A image, one block of BM x (BK / PER_VEC) threads per (m-tile,
// k-chunk): the chunk's k records are decoded once and the coefficients of
// every state the tile's rows touch (states s0..s0 + ns - 1) are staged once
// in shared memory, so each thread only reads its X entries; the sums run
// over u in the same order as abuild_kernel's, so the image is bitwise the
// same.  Dynamic shared memory: ns x BK x (kMaxPairL + 1) floats.
template <int KIND>
__global__ void __launch_bounds__(BM *Kind<KIND>::BK / Kind<KIND>::PER_VEC)
    abuild_tile_kernel(PairSetDev ps, const float *__restrict__ coef32, int SB, int nxr, int nx,
                       const float2 *__restrict__ X, const int4 *__restrict__ kinfo, int nkc, int M,
                       uint8_t *__restrict__ Abuf, const int *__restrict__ kexp,
                       const unsigned long long *__restrict__ tmax) {
    using KD = Kind<KIND>;
    constexpr int V = KD::PER_VEC, BK = KD::BK, NP = KD::NP, VPC = BK / V, NU = kMaxPairL + 1;
    extern __shared__ float csm[];           // [ns][BK][NU] signed coefficients
    __shared__ int4 kin[BK];                 // (pair or -1, v, w, axis row)
    __shared__ int kun[BK];                  // u count of k (0 for padding)
    __shared__ int ksh[BK];                  // FP16 kind: power-of-two scale of column k
    const int kc = blockIdx.x, mt = blockIdx.y;
    const int m0 = mt * BM;
    const int s0 = min(m0, M - 1) / nxr;
    const int ns = min(M - 1, m0 + BM - 1) / nxr - s0 + 1;
    int G = 0;
    if constexpr (KD::FP16) G = fp16_job_exp(tmax) - 2 * kRowExp;
    if (threadIdx.x < BK) {
        const int64_t k = (int64_t)kc * BK + threadIdx.x;
        const int4 ki = kinfo[k];
        int nu = 0;
        if (ki.x >= 0) {
            int L = 0;
            while (L < kMaxPairL && ki.x >= ps.pair_off[L + 1]) ++L;
            nu = L - ki.y - ki.z + 1;
        }
        kin[threadIdx.x] = ki;
        kun[threadIdx.x] = nu;
        if constexpr (KD::FP16) ksh[threadIdx.x] = kexp[k] + G;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ns * BK * NU; t += blockDim.x) {
        const int u = t % NU, kl = (t / NU) % BK, si = t / (NU * BK);
        const int4 ki = kin[kl];
        float c = 0.f;
        if (u < kun[kl]) {
            int L = 0;
            while (L < kMaxPairL && ki.x >= ps.pair_off[L + 1]) ++L;
            const int64_t rowbase = ps.row_off[L] + (int64_t)(ki.x - ps.pair_off[L]) * mono_count(L);
            const int s = s0 + si;
            const int n = u + ki.y + ki.z;
            c = coef32[((size_t)(s / SB) * ps.n_rows + rowbase + mono_index(u, ki.y, ki.z)) * SB + (s % SB)] *
                ((n & 2) ? -1.f : 1.f);
        }
        csm[t] = c;
    }
    __syncthreads();
    const int r = threadIdx.x / VPC, vv = threadIdx.x % VPC;
    const int m = m0 + r;
    const bool mvalid = m < M;
    const int s = mvalid ? m / nxr : s0, ix = mvalid ? m % nxr : 0;
    const float *cs = csm + (size_t)(s - s0) * BK * NU;
    float re[V], im[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int kl = vv * V + e;
        const int4 ki = kin[kl];
        const int nu = kun[kl];
        float ar = 0.f, ai = 0.f;
        if (mvalid) {
            for (int u = 0; u < nu; ++u) {
                const float c = cs[kl * NU + u];
                const float2 x = X[(size_t)(ki.w + u) * nx + ix];
                ar = fmaf(c, x.x, ar);
                ai = fmaf(c, x.y, ai);
            }
            if constexpr (KD::FP16) {
                if (nu > 0) {
                    ar = pow2_scale(ar, ksh[kl]);
                    ai = pow2_scale(ai, ksh[kl]);
                }
            }
        }
        re[e] = ar;
        im[e] = ai;
    }
    uint4 pr_[NP], pi_[NP];
    split_vec<KIND>(re, pr_);
    split_vec<KIND>(im, pi_);
    uint8_t *base = Abuf + ((size_t)mt * nkc + kc) * KD::A_STAGE;
    const uint32_t off = sw64_offset<KIND>(r, vv * V);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        *reinterpret_cast<uint4 *>(base + q * A_ARR + off) = pr_[q];
        *reinterpret_cast<uint4 *>(base + (NP + q) * A_ARR + off) = pi_[q];
    }
}

// Split-and-swizzle image of a dense complex FP64 matrix src[M][lda] (K valid
// columns; columns K..K_pad and rows M..M_pad are zero), in the same tile
// layout as abuild_kernel.  One thread writes one 16-byte vector of each array.
template <int KIND>
__global__ void dense_image_kernel(const double2 *__restrict__ src, int64_t lda, int M, int64_t K, int M_pad,
                                   int64_t K_pad, int nkc, uint8_t *__restrict__ Abuf) {
    using KD = Kind<KIND>;
    constexpr int V = KD::PER_VEC, BK = KD::BK, NP = KD::NP;
    const int64_t kvn = K_pad / V;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M_pad * kvn) return;
    int m;
    int64_t kv;
    image_coords<KIND>(idx, nkc, m, kv);
    float re[V], im[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int64_t k = kv * V + e;
        double2 v = make_double2(0.0, 0.0);
        if (m < M && k < K) v = src[(size_t)m * lda + k];
        re[e] = (float)v.x;
        im[e] = (float)v.y;
    }
    uint4 pr_[NP], pi_[NP];
    split_vec<KIND>(re, pr_);
    split_vec<KIND>(im, pi_);
    const int mt = m / BM, r = m % BM;
    const int64_t kc = (kv * V) / BK;
    const int c0 = (int)((kv * V) % BK);
    uint8_t *base = Abuf + ((size_t)mt * nkc + kc) * KD::A_STAGE;
    const uint32_t off = sw64_offset<KIND>(r, c0);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        *reinterpret_cast<uint4 *>(base + q * A_ARR + off) = pr_[q];
        *reinterpret_cast<uint4 *>(base + (NP + q) * A_ARR + off) = pi_[q];
    }
}

// ------------------------------------------------------------------ persistent main kernel

// Adds the finished accumulator group with global index gg (TMEM set gg & 1)
// into this thread's FP32 register sums: row = TMEM lane, CQ columns of Re
// and of Im.
template <int CQ>
__device__ __forceinline__ bool drain_group(int gg, uint64_t *accFull, uint64_t *accEmpty, uint32_t tmem, int lg,
                                            int lane, int colh, float (&acc_re)[CQ], float (&acc_im)[CQ]) {
    const int set = gg & 1;
    const bool got = mbar_wait(&accFull[set], (gg >> 1) & 1);
    if (__any_sync(0xffffffffu, !got)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + set * (2 * BN) + colh;
#pragma unroll
    for (int cc = 0; cc < CQ; cc += 32) {
        // two 16-column loads of Re and of Im in flight per wait
        float r0[16], r1[16], i0[16], i1[16];
        tmem_ld16(ta + cc, r0);
        tmem_ld16(ta + cc + 16, r1);
        tmem_ld16(ta + BN + cc, i0);
        tmem_ld16(ta + BN + cc + 16, i1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            acc_re[cc + j] += r0[j];
            acc_re[cc + 16 + j] += r1[j];
            acc_im[cc + j] += i0[j];
            acc_im[cc + 16 + j] += i1[j];
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&accEmpty[set]);
    return true;
}

// VAR_PREFETCH: adds the finished accumulator group with global index gg
// (the single MMA set, TMEM columns [0, 2 BN): Re then Im) to the running
// sums in columns [2 BN, 4 BN), FP32 adds in registers, 16 columns of Re and
// of Im at a time.  first: the sums start at +0 (0 + x, exactly as the
// register sums of VAR_GATHER start).  The MMA set is released once read.
template <int CQ>
__device__ __forceinline__ bool drain_to_master(int gg, bool first, uint64_t *accFull, uint64_t *accEmpty,
                                                uint32_t tmem, int lg, int lane, int colh) {
    const bool got = mbar_wait(accFull, gg & 1);
    if (__any_sync(0xffffffffu, !got)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + colh;
#pragma unroll
    for (int cc = 0; cc < CQ; cc += 16) {
        float wr[16], wi[16], mr[16], mi[16];
        tmem_ld16(ta + cc, wr);
        tmem_ld16(ta + BN + cc, wi);
        if (!first) {
            tmem_ld16(ta + 2 * BN + cc, mr);
            tmem_ld16(ta + 3 * BN + cc, mi);
        }
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            mr[j] = (first ? 0.f : mr[j]) + wr[j];
            mi[j] = (first ? 0.f : mi[j]) + wi[j];
        }
        tmem_st16(ta + 2 * BN + cc, mr);
        tmem_st16(ta + 3 * BN + cc, mi);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(accEmpty);
    tmem_wait_st();  // the sums are complete before this thread next reads them
    return true;
}

// VAR_PREFETCH, last group of a tile: running sums (if any) plus the group,
// into this thread's registers; the MMA set is released once read.
template <int CQ>
__device__ __forceinline__ bool drain_final(int gg, bool only, uint64_t *accFull, uint64_t *accEmpty, uint32_t tmem,
                                            int lg, int lane, int colh, float (&acc_re)[CQ], float (&acc_im)[CQ]) {
    const bool got = mbar_wait(accFull, gg & 1);
    if (__any_sync(0xffffffffu, !got)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + colh;
#pragma unroll
    for (int cc = 0; cc < CQ; cc += 16) {
        float wr[16], wi[16], mr[16], mi[16];
        tmem_ld16(ta + cc, wr);
        tmem_ld16(ta + BN + cc, wi);
        if (!only) {
            tmem_ld16(ta + 2 * BN + cc, mr);
            tmem_ld16(ta + 3 * BN + cc, mi);
        }
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            acc_re[cc + j] = (only ? 0.f : mr[j]) + wr[j];
            acc_im[cc + j] = (only ? 0.f : mi[j]) + wi[j];
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(accEmpty);
    return true;
}

// Octant form, one row m of a finished tile: this thread's 16 points
// (iy, iz) (columns 32 nt + 16 hs + p of the octant grid) each hold the
// eight real sums S_abc = sum_k A^a Y^b Z^c (a, b, c: real or imaginary
// part; sr[16 c' + p] = S_r and si[16 c' + p] = S_i of the W row
// c' = 2 [b = Im] + [c = Im]).  Y and Z at the mirrored axis points are the
// complex conjugates (q_y[ny-1-iy] = -q_y[iy]), so with sy, sz = +-1
//   Re f = S_rrr - sy sz S_rii - sz S_iri - sy S_iir
//   Im f = S_irr - sy sz S_iii + sz S_rri + sy S_rir
// at (ix, iy or ny-1-iy, iz or nz-1-iz), and f(-q) = conj(f(q)) at the
// mirrored row.  Points that are their own mirror are written once.
template <int CQ>
__device__ __forceinline__ void oct_write(const TcJobDev &J, const int4 &item, int m, int hs, const float (&sr)[CQ],
                                          const float (&si)[CQ]) {
    const int sidx = m / J.nx, ix = m % J.nx;
    const int ixm = J.nxf - 1 - ix;
    const bool mir = ixm != ix;
    float2 *frow = J.f + (size_t)sidx * J.nq + (size_t)ix * J.N;
    float2 *mrow = J.f + (size_t)sidx * J.nq + (size_t)ixm * J.N;
    float *f2row = J.f2 ? J.f2 + (size_t)sidx * J.nq + (size_t)ix * J.N : nullptr;
    float *m2row = J.f2 ? J.f2 + (size_t)sidx * J.nq + (size_t)ixm * J.N : nullptr;
    const float sc = J.scale;
    const int64_t n0 = (int64_t)item.z * OCT_PTS + hs * OCT_PTH;
#pragma unroll
    for (int p = 0; p < OCT_PTH; ++p) {
        const int64_t no = n0 + p;
        if (no >= J.Noct) continue;
        const int iy = (int)(no / J.nzh), iz = (int)(no % J.nzh);
        const int iy2 = J.ny - 1 - iy, iz2 = J.nz - 1 - iz;
        const float P1 = sr[p], Q3 = sr[OCT_PTH + p], Q4 = sr[2 * OCT_PTH + p], P2 = sr[3 * OCT_PTH + p];
        const float Q1 = si[p], P3 = si[OCT_PTH + p], P4 = si[2 * OCT_PTH + p], Q2 = si[3 * OCT_PTH + p];
        const float a = P1 - P2, b = P1 + P2, c = P3 + P4, d = P3 - P4;
        const float e = Q1 - Q2, g = Q1 + Q2, h = Q3 + Q4, l = Q3 - Q4;
        float2 v[4];
        v[0] = make_float2(sc * (a - c), sc * (e + h));  // (+qy, +qz)
        v[1] = make_float2(sc * (b + d), sc * (g - l));  // (+qy, -qz)
        v[2] = make_float2(sc * (b - d), sc * (g + l));  // (-qy, +qz)
        v[3] = make_float2(sc * (a + c), sc * (e - h));  // (-qy, -qz)
        const int ys[4] = {iy, iy, iy2, iy2}, zs[4] = {iz, iz2, iz, iz2};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (((r & 2) && iy2 == iy) || ((r & 1) && iz2 == iz)) continue;
            const int64_t nn = (int64_t)ys[r] * J.nz + zs[r];
            const float a2 = v[r].x * v[r].x + v[r].y * v[r].y;
            frow[nn] = v[r];
            if (f2row) f2row[nn] = a2;
            if (mir) {
                mrow[J.N - 1 - nn] = make_float2(v[r].x, -v[r].y);
                if (m2row) m2row[J.N - 1 - nn] = a2;
            }
        }
    }
}

// Writes one finished tile (this thread's row of the warp's region): a
// part of a split tile stores its raw partial sums, and the last part of a
// region to arrive sums all parts in part order; a whole tile (or the last
// part) is scaled and written, with the mirrored row on antisymmetric grids.
// pm, pr: parts and counters are indexed (tile * nsplit + part) * pm + pr and
// tile * pm + pr (pm = 2, pr = CTA rank: the two halves of a CTA pair's tile).
template <int KIND, int CQ>
__device__ __forceinline__ void tile_epilogue(const TcJobDev &J, const int4 &item, int mt, int pm, int pr, bool ok,
                                              int lg, int lane, int colh, int region, float (&acc_re)[CQ],
                                              float (&acc_im)[CQ]) {
    using KD = Kind<KIND>;
    const int m = mt * BM + lg * 32 + lane;
    const int slot = item_slot(item.x);
    bool write = ok && m < J.M;
    if (ok && slot >= 0) {
        // part of a split tile: raw partial sums of this warp's region
        const int row = lg * 32 + lane;
        const int tile = slot / J.nsplit;
        float2 *pp = J.part + ((size_t)((tile * J.nsplit + slot % J.nsplit) * pm + pr) * BM + row) * BN + colh;
#pragma unroll
        for (int j = 0; j < CQ; ++j) pp[j] = make_float2(acc_re[j], acc_im[j]);
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            int *c = J.cnt + (tile * pm + pr) * 8 + region;
            last = atomicAdd(c, 1) == J.nsplit - 1;
            if (last) *c = 0;  // ready for the next launch
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        write = write && last;
        if (last) {
            // every part of this region has landed: sum them in part order
            __threadfence();
            const int first = tile * J.nsplit;
#pragma unroll
            for (int j = 0; j < CQ; ++j) acc_re[j] = acc_im[j] = 0.f;
            for (int pt = 0; pt < J.nsplit; ++pt) {
                const float2 *src = J.part + ((size_t)((first + pt) * pm + pr) * BM + row) * BN + colh;
#pragma unroll
                for (int j = 0; j < CQ; ++j) {
                    const float2 v = __ldcg(src + j);
                    acc_re[j] += v.x;
                    acc_im[j] += v.y;
                }
            }
        }
    }
    if (write) {
        if constexpr (KD::FP16) {
            // remove the job factor 2^G of the FP16 kind's scaled A
            const int G = fp16_job_exp(J.tmax);
#pragma unroll
            for (int j = 0; j < CQ; ++j) {
                acc_re[j] = pow2_scale(acc_re[j], -G);
                acc_im[j] = pow2_scale(acc_im[j], -G);
            }
        }
        if constexpr (CQ == 4 * OCT_PTH) {
            if (J.oct) {
                oct_write(J, item, m, colh / CQ, acc_re, acc_im);
                return;
            }
        }
        const int sidx = m / J.nx, ix = m % J.nx;
        const int64_t n0 = (int64_t)item.z * BN + colh;
        float2 *frow = J.f + (size_t)sidx * J.nq + (size_t)ix * J.N;
        float *f2row = J.f2 ? J.f2 + (size_t)sidx * J.nq + (size_t)ix * J.N : nullptr;
        const float sc = J.scale;
        const int ixm = J.nxf - 1 - ix;  // mirror row (f(-q) = conj f(q))
        const bool mir = J.mirror && ixm != ix;
        float2 *mrow = J.f + (size_t)sidx * J.nq + (size_t)ixm * J.N;
        float *m2row = J.f2 ? J.f2 + (size_t)sidx * J.nq + (size_t)ixm * J.N : nullptr;
#pragma unroll
        for (int j = 0; j < CQ; ++j) {
            const int64_t nn = n0 + j;
            if (nn < J.N) {
                const float2 v = make_float2(sc * acc_re[j], sc * acc_im[j]);
                const float a2 = v.x * v.x + v.y * v.y;
                frow[nn] = v;
                if (f2row) f2row[nn] = a2;
                if (mir) {
                    mrow[J.N - 1 - nn] = make_float2(v.x, -v.y);
                    if (m2row) m2row[J.N - 1 - nn] = a2;
                }
            }
        }
    }
}

// Bounded wait that also gives up once the CTA's abort flag is set.
__device__ __forceinline__ bool mbar_wait_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 15) == 0 && (*abort_flag || global_ns() - t0 > kWaitNs)) return false;
    }
    return false;
}

// A consumer role's next work item from the item ring (ic = its count of
// items taken so far): the index, -1 when the CTA has no more, -2 if the wait
// ran out or the CTA gave up.  Called by a whole warp (lane 0 frees the slot
// once every lane has read it) or by a single thread (lane 0).  The wait polls
// the abort flag, so a producer that gave up never leaves a role waiting long.
__device__ __forceinline__ int ring_take(uint64_t *ifull, uint64_t *iempty, volatile int *iring, int ic,
                                         volatile int *abort_flag, int lane) {
    const int r = ic % IRING;
    const bool got = mbar_wait_abort(&ifull[r], (ic / IRING) & 1, abort_flag);
    const int idx = got ? iring[r] : -2;
    __syncwarp(__activemask());
    if (got && lane == 0) mbar_arrive(&iempty[r]);
    return idx;
}

// One CTA per SM walks its share of the work list: items blockIdx.x,
// blockIdx.x + gridDim.x, ... of a list sorted by cost.  An item is one
// 128 x 128 output tile of one job; its contraction runs over the job's k
// chunks.  Stage slots, mbarrier phases and the two TMEM accumulator sets
// are counted globally across items, so consecutive items pipeline without
// re-initialisation.  Each tile's reduction order depends only on its own
// job, never on the rest of the batch.
template <int KIND, int VAR>
__global__ void __launch_bounds__(THREADS, 1)
    tc_persistent_kernel(const TcJobDev *__restrict__ jobs, const int4 *__restrict__ items, int n_items,
                         int drain_every, int *err, int *progress, int *queue) {
    using KD = Kind<KIND>;
    using CF = Cfg<KIND, VAR>;
    constexpr bool ZS = CF::ZS, PF = CF::PF;
    constexpr bool TF32 = KD::TF32;
    constexpr int BK = KD::BK, V = KD::PER_VEC, NP = KD::NP, STAGES = CF::STAGES;
    constexpr int ZSLOT = CF::ZSLOT, YSLOT = CF::YSLOT, ZSLOTS = CF::ZSLOTS;
    constexpr int A_STAGE = KD::A_STAGE, STAGE = KD::STAGE;
    constexpr int KH = BK / 2;        // k per generator thread (two threads per W row)
    constexpr int KSUB = 8;           // loads in flight per sub-batch
    // octant form of the single-CTA gather kernel (BF16 hi/mid/lo, compiled as
    // VAR_OCT so the plain gather kernel keeps its registers): jobs with
    // TcJobDev::oct = 1 form a real W for 32 octant points x 4 Re/Im products
    // (rows 64 h + 16 c + p for point 16 h + p) and Ar, Ai multiply it into
    // their own accumulators (two MMAs per piece product instead of four)
    constexpr bool OCTS = !KD::FUSE && !KD::TF32 && VAR == VAR_OCT;
    constexpr int CQ = BN / 2;        // accumulator columns (of Re and of Im) per drain thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
    uint64_t *fullA = bars + 0;                  // [STAGES] A tile landed (TMA)
    uint64_t *fullW = bars + STAGES;             // [STAGES] W tile written by the generators
    uint64_t *empty = bars + 2 * STAGES;         // [STAGES] MMAs of the stage completed
    uint64_t *accFull = bars + 3 * STAGES;       // [2] accumulator set holds a finished group
    uint64_t *accEmpty = bars + 3 * STAGES + 2;  // [2] accumulator set drained
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * STAGES + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 3 * STAGES + 5);
    uint64_t *zfull = bars + 16;                 // [ZSLOTS] (ZS) Z slices landed and Y values stored
    uint64_t *zempty = bars + 20;                // [ZSLOTS] (ZS) generators done with the Z slot
    uint8_t *zbase = smem + STAGES * STAGE + BAR_BYTES;  // (ZS) [ZSLOTS][Z slices | Y values]
    uint64_t *ifull = bars + 24;                 // [IRING] item index published
    uint64_t *iempty = bars + 28;                // [IRING] every role has read it
    volatile int *iring = reinterpret_cast<volatile int *>(bars + 32);  // [IRING] item indices (-1: done)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&fullW[s], GEN_WARPS);
            mbar_init(&empty[s], 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&accFull[j], 1);
            mbar_init(&accEmpty[j], GEN_WARPS);
        }
        if constexpr (ZS) {
            for (int s = 0; s < ZSLOTS; ++s) {
                mbar_init(&zfull[s], BK);
                mbar_init(&zempty[s], GEN_WARPS);
            }
        }
        for (int r = 0; r < IRING; ++r) {
            mbar_init(&ifull[r], 1);
            mbar_init(&iempty[r], 1 + GEN_WARPS + (ZS ? 1 : 0));  // MMA thread, generators, stager
        }
        *abort_flag = 0;
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(LOW_REGS));
        if (warp == 0 && lane == 0) {
            // ---------------- TMA producer: A tile and the chunk's k-index records
            // It also takes the CTA's work items -- the next index of the
            // shared queue counter (queue != null: CTAs that finish early take
            // more items) or item blockIdx.x + ic * gridDim.x -- and publishes
            // each to the other roles through the item ring (-1: no more).
            int gc = 0;  // global chunk counter
            for (int ic = 0;; ++ic) {
                const int r = ic % IRING;
                if (ic >= IRING && !mbar_wait_abort(&iempty[r], ((ic / IRING) - 1) & 1, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                int idx = queue ? atomicAdd(queue, 1) : blockIdx.x + ic * gridDim.x;
                if (idx >= n_items || *abort_flag) idx = -1;
                iring[r] = idx;
                mbar_arrive(&ifull[r]);
                if (idx < 0) break;
                const int4 item = items[idx];
                const TcJobDev &J = jobs[item_job(item.x)];
                const uint8_t *Abase = J.A + ((size_t)item_mt(item.y) * J.nkc + item_k0(item.y)) * A_STAGE;
                for (int it = 0; it < item.w; ++it, ++gc) {
                    const int s = gc % STAGES;
                    if (gc >= STAGES && !mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t *st = smem + s * STAGE;
                    mbar_arrive_expect_tx(&fullA[s], A_STAGE);
                    bulk_g2s(st, Abase + (size_t)it * A_STAGE, A_STAGE, &fullA[s]);
                }
                if (*abort_flag) break;
            }
            // the copies of the last stages have landed before the CTA may exit
            // (consumed phases report complete at once; bounded either way)
            for (int c = max(0, gc - STAGES); c < gc; ++c) mbar_wait(&fullA[c % STAGES], (c / STAGES) & 1);
        } else if (ZS && warp == 2) {
            // ---------------- Z/Y stager (ZS): for chunk gc, lane j < BK copies
            // the tile's 128-entry slice of k's Z row (1 KB, bulk copy) and
            // stores k's Y value of the tile's y row
            int gc = 0;
            bool ok = true;
            for (int ic = 0; ok; ++ic) {
                const int idx = ring_take(ifull, iempty, iring, ic, abort_flag, lane);
                if (idx == -2) ok = false;
                if (idx < 0) break;
                const int4 item = items[idx];
                const TcJobDev &J = jobs[item_job(item.x)];
                const int64_t n0 = (int64_t)item.z * BN;
                const float2 *Yc = J.Y + (int)(n0 / J.nz);
                const float2 *Zc = J.Z + (int)(n0 % J.nz);
                const int2 *kofs = J.kofs + (size_t)item_k0(item.y) * BK;
                for (int it = 0; it < item.w; ++it, ++gc) {
                    const int s = gc % ZSLOTS;
                    // the chunk's k-offsets and Y values are read before the
                    // slot frees, so their latency overlaps the wait
                    int2 ko = make_int2(0, 0);
                    float2 y = make_float2(0.f, 0.f);
                    if (lane < BK) {
                        ko = __ldg(kofs + (size_t)it * BK + lane);
                        y = __ldg(Yc + ko.x);
                    }
                    const bool w = gc < ZSLOTS || mbar_wait(&zempty[s], ((gc / ZSLOTS) - 1) & 1);
                    if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *zb = zbase + s * (ZSLOT + YSLOT);
                    if (lane == 0) mbar_expect_tx(&zfull[s], ZSLOT);
                    __syncwarp();
                    if (lane < BK) {
                        bulk_g2s(zb + lane * (BN * 8), Zc + ko.y, BN * 8, &zfull[s]);
                        reinterpret_cast<float2 *>(zb + ZSLOT)[lane] = y;
                        mbar_arrive(&zfull[s]);
                    }
                }
            }
            if (!ok) *abort_flag = 1;
            if (lane == 0)
                for (int c = max(0, gc - ZSLOTS); c < gc; ++c) mbar_wait(&zfull[c % ZSLOTS], (c / ZSLOTS) & 1);
            __syncwarp();
        } else if (warp == 1 && lane == 0) {
            // ---------------- MMA issuer: global group gg accumulates into TMEM set gg & 1
            constexpr uint32_t ID = idesc_mma<KD::FMT>(false), IDN = idesc_mma<KD::FMT>(true);
            constexpr uint32_t ID2 = idesc_mma<KD::FMT, 2 * BN>(false);  // N = 256: [Re | Im] at once
            int gc = 0, gbase = 0;
            for (int ic = 0;; ++ic) {
                const int idx = ring_take(ifull, iempty, iring, ic, abort_flag, 0);
                if (idx == -2) *abort_flag = 1;
                if (idx < 0) break;
                const int nkc = items[idx].w;
                const bool octj = OCTS && jobs[item_job(items[idx].x)].oct != 0;
                const int G = drain_every >= 1 ? max(2, min(drain_every, nkc)) : nkc;
                bool ok = true;
                for (int it = 0; it < nkc; ++it, ++gc) {
                    const int s = gc % STAGES;
                    const uint32_t par = (gc / STAGES) & 1;
                    if (*abort_flag || !mbar_wait(&fullA[s], par) || !mbar_wait(&fullW[s], par)) {
                        ok = false;
                        break;
                    }
                    // groups alternate between the two TMEM sets; VAR_PREFETCH has
                    // one set (the other holds the running sums), freed by every drain
                    const int gg = gbase + it / G, set = PF ? 0 : gg & 1;
                    const bool first = (it % G) == 0;
                    if (first && (PF ? gg >= 1 && !mbar_wait(&accEmpty[0], (gg - 1) & 1)
                                     : gg >= 2 && !mbar_wait(&accEmpty[set], ((gg - 2) >> 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t t_re = tmem + set * (2 * BN), t_im = t_re + BN;
                    const uint32_t a0 = smem_u32(smem + s * STAGE);
                    const uint32_t w0 = a0 + A_STAGE;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint32_t ko = kk * 32;  // 32 bytes = one MMA K step
#pragma unroll
                        for (int pq = 0; pq < KD::NPROD; ++pq) {
                            const int qa = prod_a(pq), qw = prod_w(pq);
                            const uint64_t ar = smem_desc_sw64(a0 + qa * A_ARR + ko);
                            const uint64_t ai = smem_desc_sw64(a0 + (NP + qa) * A_ARR + ko);
                            const uint32_t acc = (first && kk == 0 && pq == 0) ? 0u : 1u;
                            if constexpr (KD::FUSE) {
                                const uint32_t pb = w0 + qw * 3 * W_ARR + ko;
                                mma_issue<TF32>(t_re, ar, smem_desc_sw64(pb + W_ARR), ID2, acc);  // += [Ar Wr | Ar Wi]
                                mma_issue<TF32>(t_re, ai, smem_desc_sw64(pb), ID2, 1);            // += [-Ai Wi | Ai Wr]
                            } else {
                                const uint64_t wr = smem_desc_sw64(w0 + qw * W_ARR + ko);
                                if (octj) {
                                    // real W: S_r = Ar W in the Re columns, S_i = Ai W in the Im columns
                                    mma_issue<TF32>(t_re, ar, wr, ID, acc);
                                    mma_issue<TF32>(t_im, ai, wr, ID, acc);
                                } else {
                                    const uint64_t wi = smem_desc_sw64(w0 + (NP + qw) * W_ARR + ko);
                                    mma_issue<TF32>(t_re, ar, wr, ID, acc);   // Re += Ar Wr
                                    mma_issue<TF32>(t_re, ai, wi, IDN, 1);    // Re -= Ai Wi
                                    mma_issue<TF32>(t_im, ar, wi, ID, acc);   // Im += Ar Wi
                                    mma_issue<TF32>(t_im, ai, wr, ID, 1);     // Im += Ai Wr
                                }
                            }
                        }
                    }
                    mma_commit(&empty[s]);
                    if ((it % G) == G - 1 || it == nkc - 1) mma_commit(&accFull[set]);
                }
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                gbase += (nkc + G - 1) / G;
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(HIGH_REGS));
        // ---------------- W generators (two threads per W row); they also
        // drain finished accumulator groups into FP32 registers and write the
        // finished tile.
        const int gt = threadIdx.x - 128;          // 0..255
        const int wrow = gt & (BN - 1);            // W row
        const int khalf = gt / BN;                 // which half of the chunk's k
        // drain mapping: TMEM lane group = warp % 4 (hardware rule); the two
        // warps of a lane group take column halves.
        const int lg = warp & 3;
        const int colh = ((warp - 4) >> 2) * CQ;
        // (STAGE_KO) this warp's two k-offset buffers (KH records each): the next
        // chunk's records are copied asynchronously while this chunk is generated
        int2 *kobuf = reinterpret_cast<int2 *>(smem + STAGES * STAGE + BAR_BYTES) + (warp - 4) * 2 * KH;
        int gc = 0, gbase = 0, done_items = 0;
        bool ok = true;
        for (int ic = 0; ok; ++ic) {
            const int idx = ring_take(ifull, iempty, iring, ic, abort_flag, lane);
            if (idx == -2) ok = false;
            if (idx < 0) break;
            const int4 item = items[idx];
            const TcJobDev &J = jobs[item_job(item.x)];
            const int nkc = item.w;
            const int mt = item_mt(item.y), k0 = item_k0(item.y);
            const int G = drain_every >= 1 ? max(2, min(drain_every, nkc)) : nkc;
            const int ngroups = (nkc + G - 1) / G;
            const int nz = J.nz;
            const int64_t n = (int64_t)item.z * BN + wrow;
            const bool nvalid = n < J.N;
            int iy = 0, iz = 0;
            if (nvalid) {
                iz = (int)(n % nz);
                iy = (int)(n / nz);
                if (J.ylm) {
                    int l = (int)sqrtf((float)iz);
                    while (l * l > iz) --l;
                    while ((l + 1) * (l + 1) <= iz) ++l;
                    iy = iy * J.ystride + l;
                }
            }
            // octant form: thread point op (32 per tile) and k quad kq4 (4 k) of the chunk
            const bool octj = OCTS && J.oct != 0;
            const int op = gt & 31, kq4 = gt >> 5;
            if (octj) {
                const int64_t no = (int64_t)item.z * OCT_PTS + op;
                iy = iz = 0;
                if (no < J.Noct) {
                    iz = (int)(no % J.nzh);
                    iy = (int)(no / J.nzh);
                }
            }
            const float2 *Yc = J.Y + iy;
            const float2 *Zc = J.Z + iz;
            float acc_re[CQ], acc_im[CQ];  // the tile's sums (VAR_PREFETCH: filled by the last drain)
#pragma unroll
                for (int j = 0; j < CQ; ++j) acc_re[j] = acc_im[j] = 0.f;
            const int gc0 = gc;
            int drained = 0;
            const int2 *kofs = J.kofs + (size_t)k0 * BK + khalf * KH;
            if constexpr (PF) {
                // Chunk it+1's table entries are gathered into the other
                // register set before chunk it's W is formed; the k-offsets run
                // two chunks ahead through this warp's two shared-memory buffers
                // (buffer b holds chunk c with c & 1 == b).
                float2 yv[2][KH], zv[2][KH];  // set it & 1 holds chunk it's entries
                if (lane < KH) cp_async8(kobuf + lane, kofs + lane);
                cp_async_commit();
                if (nkc > 1 && lane < KH) cp_async8(kobuf + KH + lane, kofs + BK + lane);
                cp_async_commit();
                cp_async_wait<1>();  // chunk 0's records have landed
                __syncwarp();
#pragma unroll
                for (int e = 0; e < KH; ++e) {
                    const int2 k2 = kobuf[e];
                    yv[0][e] = __ldg(Yc + k2.x);
                    zv[0][e] = __ldg(Zc + k2.y);
                }
                __syncwarp();  // every lane has read buffer 0 before chunk 2's records overwrite it
                for (int it0 = 0; it0 < nkc && ok; it0 += 2) {
                    // two chunks per pass, so each names its register sets at compile time
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const int it = it0 + p;
                        if (it < nkc && ok) {
                        const int gcc = gc0 + it, s = gcc % STAGES;
                        if (it + 2 < nkc && lane < KH)
                            cp_async8(kobuf + p * KH + lane, kofs + (size_t)(it + 2) * BK + lane);
                        cp_async_commit();
                        cp_async_wait<1>();  // chunk it+1's records have landed
                        __syncwarp();
                        if (it + 1 < nkc) {
                            const int2 *kb = kobuf + (p ^ 1) * KH;
#pragma unroll
                            for (int e = 0; e < KH; ++e) {
                                const int2 k2 = kb[e];
                                yv[p ^ 1][e] = __ldg(Yc + k2.x);
                                zv[p ^ 1][e] = __ldg(Zc + k2.y);
                            }
                        }
                        const bool w = gcc < STAGES || mbar_wait(&empty[s], ((gcc / STAGES) - 1) & 1);
                        ok = !__any_sync(0xffffffffu, !w) && !*abort_flag;
                        uint8_t *wst = smem + s * STAGE + A_STAGE;
                        if (ok) {
#pragma unroll
                        for (int jv = 0; jv < KH / V; ++jv) {
                            float re[V], im[V];
#pragma unroll
                            for (int e = 0; e < V; ++e) w_elem(yv[p][jv * V + e], zv[p][jv * V + e], re[e], im[e]);
                            uint4 pr_[NP], pi_[NP];
                            split_vec<KIND>(re, pr_);
                            split_vec<KIND>(im, pi_);
                            const uint32_t off = sw64_offset<KIND>(wrow, khalf * KH + jv * V);
                            store_w<KIND>(wst, off, pr_, pi_);
                        }
                        fence_proxy_async_smem();
                        __syncwarp();  // also: every lane has read buffer p ^ 1 before it is refilled
                        if (lane == 0) mbar_arrive(&fullW[s]);
                        // the first chunk of group gd+1 is in place: add group gd to the
                        // sums as soon as its MMAs complete (the MMAs of group gd+1 wait for it)
                        if (it > 0 && it % G == 0) {
                            const int gd = it / G - 1;
                            ok = drain_to_master<CQ>(gbase + gd, gd == 0, &accFull[0], &accEmpty[0], tmem, lg, lane,
                                                     colh);
                        }
                        }
                        }
                    }
                }
                cp_async_wait<0>();  // no copy into this warp's buffers outlives the item
                __syncwarp();
                if (ok && !drain_final<CQ>(gbase + ngroups - 1, ngroups == 1, &accFull[0], &accEmpty[0], tmem, lg,
                                           lane, colh, acc_re, acc_im))
                    ok = false;
            } else {
                // Row offsets of this warp's k (independent of the A copy, so the
                // gathers below overlap with the TMA instead of following it),
                // staged one chunk ahead by asynchronous copies into shared memory.
                if constexpr (KD::STAGE_KO && !ZS) {
                    if (lane < KH) cp_async8(kobuf + lane, kofs + lane);
                    cp_async_commit();
                }
                for (int it = 0; it < nkc && ok; ++it, ++gc) {
                    const int s = gc % STAGES;
                    if constexpr (ZS) {
                        // W from the staged Z slices and Y values of this chunk
                        const int zs = gc % ZSLOTS;
                        const bool w = mbar_wait(&zfull[zs], (gc / ZSLOTS) & 1) &&
                                       (gc < STAGES || mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1));
                        if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                            ok = false;
                            break;
                        }
                        const uint8_t *zb = zbase + zs * (ZSLOT + YSLOT);
                        const float2 *zr = reinterpret_cast<const float2 *>(zb) + (size_t)(khalf * KH) * BN + wrow;
                        const float2 *yv = reinterpret_cast<const float2 *>(zb + ZSLOT) + khalf * KH;
                        uint8_t *wst = smem + s * STAGE + A_STAGE;
#pragma unroll
                        for (int sb = 0; sb < KH; sb += KSUB) {
                            float2 y[KSUB], z[KSUB];
#pragma unroll
                            for (int e = 0; e < KSUB; ++e) {
                                y[e] = yv[sb + e];
                                z[e] = zr[(sb + e) * BN];
                            }
#pragma unroll
                            for (int jv = 0; jv < KSUB / V; ++jv) {
                                float re[V], im[V];
#pragma unroll
                                for (int e = 0; e < V; ++e) w_elem(y[jv * V + e], z[jv * V + e], re[e], im[e]);
                                uint4 pr_[NP], pi_[NP];
                                split_vec<KIND>(re, pr_);
                                split_vec<KIND>(im, pi_);
                                const uint32_t off = sw64_offset<KIND>(wrow, khalf * KH + sb + jv * V);
                                store_w<KIND>(wst, off, pr_, pi_);
                            }
                        }
                        // W visible to the tensor core; the Z slot's reads done
                        // before the stager's next bulk copy overwrites it
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&fullW[s]);
                            mbar_arrive(&zempty[zs]);
                        }
                    } else if constexpr (KD::STAGE_KO) {
                    // all KH table pairs of this chunk are requested at once (the
                    // k-offsets come from this warp's shared-memory buffer, staged
                    // one chunk ahead), before the wait for the stage
                    if (it + 1 < nkc && lane < KH)
                        cp_async8(kobuf + ((it + 1) & 1) * KH + lane, kofs + (size_t)(it + 1) * BK + lane);
                    cp_async_commit();
                    cp_async_wait<1>();  // this chunk's records have landed
                    __syncwarp();
                    const int2 *kb = kobuf + (it & 1) * KH;
                    float2 y[KH], z[KH];
#pragma unroll
                    for (int e = 0; e < KH; ++e) {
                        const int2 k2 = kb[e];
                        y[e] = __ldg(Yc + k2.x);
                        z[e] = __ldg(Zc + k2.y);
                    }
                    const bool w = gc < STAGES || mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1);
                    if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *wst = smem + s * STAGE + A_STAGE;
#pragma unroll
                    for (int jv = 0; jv < KH / V; ++jv) {
                        float re[V], im[V];
#pragma unroll
                        for (int e = 0; e < V; ++e) w_elem(y[jv * V + e], z[jv * V + e], re[e], im[e]);
                        uint4 pr_[NP], pi_[NP];
                        split_vec<KIND>(re, pr_);
                        split_vec<KIND>(im, pi_);
                        const uint32_t off = sw64_offset<KIND>(wrow, khalf * KH + jv * V);
                        store_w<KIND>(wst, off, pr_, pi_);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&fullW[s]);
                    } else if (octj) {
                    // four Re/Im products of the point at four k from one gather each;
                    // split word pairs hold a product at two k (8-byte stores)
                    const int2 *ko4 = J.kofs + (size_t)(k0 + it) * BK + kq4 * 4;
                    float2 y[4], z[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int2 k2 = __ldg(ko4 + e);
                        y[e] = __ldg(Yc + k2.x);
                        z[e] = __ldg(Zc + k2.y);
                    }
                    const bool w = gc < STAGES || mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1);
                    if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *wst = smem + s * STAGE + A_STAGE;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // products 2h (Re or Im of Y by Re of Z) and 2h + 1 (by Im of Z)
                        float v[8];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float yc = h ? y[e].y : y[e].x;
                            v[e] = __fmul_rn(yc, z[e].x);
                            v[4 + e] = __fmul_rn(yc, z[e].y);
                        }
                        uint4 pc_[NP];
                        split_vec<KIND>(v, pc_);
                        const int rbase = (op >> 4) * 64 + (op & 15);
                        const uint32_t o0 = sw64_offset<KIND>(rbase + (2 * h) * OCT_PTH, kq4 * 4);
                        const uint32_t o1 = sw64_offset<KIND>(rbase + (2 * h + 1) * OCT_PTH, kq4 * 4);
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            *reinterpret_cast<uint2 *>(wst + q * W_ARR + o0) = make_uint2(pc_[q].x, pc_[q].y);
                            *reinterpret_cast<uint2 *>(wst + q * W_ARR + o1) = make_uint2(pc_[q].z, pc_[q].w);
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&fullW[s]);
                    } else {
                    int2 ko[KH];
#pragma unroll
                    for (int e = 0; e < KH; ++e) ko[e] = __ldg(kofs + (size_t)it * BK + e);
                    const bool w = gc < STAGES || mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1);
                    if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *wst = smem + s * STAGE + A_STAGE;
#pragma unroll
                    for (int sb = 0; sb < KH; sb += KSUB) {
                        float2 y[KSUB], z[KSUB];
#pragma unroll
                        for (int e = 0; e < KSUB; ++e) {
                            y[e] = __ldg(Yc + ko[sb + e].x);
                            z[e] = __ldg(Zc + ko[sb + e].y);
                        }
#pragma unroll
                        for (int jv = 0; jv < KSUB / V; ++jv) {
                            float re[V], im[V];
#pragma unroll
                            for (int e = 0; e < V; ++e) w_elem(y[jv * V + e], z[jv * V + e], re[e], im[e]);
                            uint4 pr_[NP], pi_[NP];
                            split_vec<KIND>(re, pr_);
                            split_vec<KIND>(im, pi_);
                            const uint32_t off = sw64_offset<KIND>(wrow, khalf * KH + sb + jv * V);
                            store_w<KIND>(wst, off, pr_, pi_);
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&fullW[s]);
                    }
                    // Local group gd is complete once the MMAs of its last chunk
                    // are; that is guaranteed STAGES chunks later, so drain it then
                    // without stalling the tensor pipe.
                    while (drained < ngroups && (drained + 1) * G - 1 + STAGES <= it) {
                        if (!drain_group<CQ>(gbase + drained, accFull, accEmpty, tmem, lg, lane, colh, acc_re, acc_im)) {
                            ok = false;
                            break;
                        }
                        ++drained;
                    }
                }
                if constexpr (KD::STAGE_KO && !ZS) {
                    cp_async_wait<0>();  // no copy into this warp's buffers outlives the item
                    __syncwarp();
                }
                while (ok && drained < ngroups) {
                    if (!drain_group<CQ>(gbase + drained, accFull, accEmpty, tmem, lg, lane, colh, acc_re, acc_im))
                        ok = false;
                    ++drained;
                }
            }
            gbase += ngroups;
            gc = gc0 + nkc;
            tile_epilogue<KIND, CQ>(J, item, mt, 1, 0, ok, lg, lane, colh, warp - 4, acc_re, acc_im);
            if (progress && ok) {
                // publish how many items this warp has finished: its writes
                // above reach memory (system scope) before the count does
                __threadfence_system();
                __syncwarp();
                ++done_items;
                if (lane == 0)
                    *reinterpret_cast<volatile int *>(progress + blockIdx.x * GEN_WARPS + (warp - 4)) = done_items;
            }
        }
        if (!ok) *abort_flag = 1;
    }
    if (threadIdx.x == 0 && *abort_flag) flag_error(err, kDevErrTimeout);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ------------------------------------------------------------------ CTA-pair kernel

// A pair role's next work item (ring_take for clusters): the ring slot is
// written and published by the even CTA; every consumer of either CTA frees
// it on the even CTA's iempty barrier.
__device__ __forceinline__ int ring_take_pair(uint64_t *ifull, uint64_t *iempty, volatile int *iring, int ic,
                                              volatile int *abort_flag, int lane) {
    const int r = ic % IRING;
    const bool got = mbar_wait_cl(&ifull[r], (ic / IRING) & 1, abort_flag);
    const int idx = got ? iring[r] : -2;
    __syncwarp(__activemask());
    if (got && lane == 0) mbar_arrive_cluster(mapa_shared(&iempty[r], 0));
    return idx;
}

// Adds finished accumulator group gg (TMEM set gg & 1) into this thread's
// register sums: row = TMEM lane, CQ columns of Re at column re0 of the set
// and of Im at re0 + im_off; frees the set on the even CTA's accEmpty.
// local (optional): the set's local barrier this warp arrives on instead
// (the octant-only build: the even CTA's accEmpty, or the odd CTA's
// accDrained, which one thread relays to the even CTA per group).
template <int CQ>
__device__ __forceinline__ bool drain_group_pair(int gg, uint64_t *accFull, uint64_t *accEmpty, uint32_t tmem,
                                                 int lg, int lane, int re0, int im_off, float (&acc_re)[CQ],
                                                 float (&acc_im)[CQ], volatile int *abort_flag,
                                                 uint64_t *local = nullptr) {
    const int set = gg & 1;
    const bool got = mbar_wait_abort(&accFull[set], (gg >> 1) & 1, abort_flag);
    if (__any_sync(0xffffffffu, !got)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + set * (2 * BN) + re0;
#pragma unroll
    for (int cc = 0; cc < CQ; cc += 32) {
        float r0[16], r1[16], i0[16], i1[16];
        tmem_ld16(ta + cc, r0);
        tmem_ld16(ta + cc + 16, r1);
        tmem_ld16(ta + im_off + cc, i0);
        tmem_ld16(ta + im_off + cc + 16, i1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            acc_re[cc + j] += r0[j];
            acc_re[cc + 16 + j] += r1[j];
            acc_im[cc + j] += i0[j];
            acc_im[cc + 16 + j] += i1[j];
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
        if (local) mbar_arrive(&local[set]);
        else mbar_arrive_cluster(mapa_shared(&accEmpty[set], 0));
    }
    return true;
}

// Persistent kernel over CTA pairs (PairCfg).  Items are (job, m-tile pair,
// n-tile) as for the single-CTA kernel, with the m field holding the pair
// index mp: CTA r of the cluster computes rows of m-tile 2 mp + r.  Roles:
//   even CTA: warp 0 lane 0 takes the items (queue counter or the static
//     sequence cluster, cluster + clusters, ...), publishes each to both
//     CTAs' item rings and bulk-copies its own A stages; warp 1 lane 0 issues
//     the pair's MMAs once both CTAs' A and W stages have landed and commits
//     to the stage and accumulator barriers of both CTAs;
//   odd CTA: warp 0 lane 0 bulk-copies its A stages; warp 1 lane 0 relays
//     each landed stage to the even CTA's fullA barrier;
//   both: eight generator warps write the CTA's half of W (arriving on the
//     even CTA's fullW) and drain the CTA's TMEM rows into registers (freeing
//     a set on the even CTA's accEmpty), then write the CTA's half tile.
// The per-tile arithmetic (W elements, MMA order, drain groups, sums) is the
// single-CTA kernel's, so the two launches give bitwise the same results.
template <int KIND, bool OCTK>
__global__ void __launch_bounds__(THREADS, 1)
    tc_pair_kernel(const TcJobDev *__restrict__ jobs, const int4 *__restrict__ items, int n_items, int drain_every,
                   int *err, int *progress, int *queue) {
    using KD = Kind<KIND>;
    using PC = PairCfg<KIND, OCTK>;
    constexpr int BK = KD::BK, V = KD::PER_VEC, NP = KD::NP, STAGES = PC::STAGES, KQ = PC::KQ;
    constexpr int A_STAGE = KD::A_STAGE, STAGE = PC::STAGE, W_ARRH = PC::W_ARRH, BNH = PC::BNH;
    constexpr int CQ = BN / 2;  // accumulator columns (of Re and of Im) per drain thread
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
    constexpr int BO = PC::BO;
    uint64_t *fullA = bars + 0;            // [STAGES] A stage landed (even CTA: both CTAs' stages)
    uint64_t *fullW = bars + STAGES;       // [STAGES] (even CTA) W stage written by both CTAs' generators
    uint64_t *empty = bars + 2 * STAGES;   // [STAGES] MMAs of the stage completed (both CTAs)
    uint64_t *accFull = bars + BO;         // [2] accumulator set holds a finished group (both CTAs)
    uint64_t *accEmpty = bars + BO + 2;    // [2] (even CTA) accumulator set drained in both CTAs
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + BO + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + BO + 5);
    uint64_t *ifull = bars + BO + 8;       // [IRING] item published
    uint64_t *iempty = bars + BO + 12;     // [IRING] (even CTA) every role of both CTAs has read it
    volatile int *iring = reinterpret_cast<volatile int *>(bars + BO + 16);
    uint64_t *accDrained = bars + BO + 18;  // [2] (odd CTA, octant-only build) set drained by its warps
    int2 *kobuf_all = reinterpret_cast<int2 *>(smem + STAGES * STAGE + BAR_BYTES);

    const uint32_t rank = cluster_rank();
    const bool lead = rank == 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t cid, ncl;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(ncl));

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&fullA[s], 1);
            // even CTA: its generator warps and the odd CTA's relay (A and W of the odd CTA landed)
            // (the octant-only build: the four generator warps of the chunk's parity)
            mbar_init(&fullW[s], (OCTK ? GEN_WARPS / 2 : GEN_WARPS) + (lead ? 1 : 0));
            mbar_init(&empty[s], 1);
        }
        for (int j = 0; j < 2; ++j) {
            mbar_init(&accFull[j], 1);
            // octant-only build: the even CTA's warps arrive locally and one relay
            // arrival covers the odd CTA's (accDrained)
            mbar_init(&accEmpty[j], OCTK ? GEN_WARPS + 1 : 2 * GEN_WARPS);
            mbar_init(&accDrained[j], GEN_WARPS);
        }
        for (int r = 0; r < IRING; ++r) {
            mbar_init(&ifull[r], 1);
            // consumers: even CTA MMA thread + generators, odd CTA copier + relay(s) + generators
            mbar_init(&iempty[r], (1 + GEN_WARPS) + ((OCTK ? 4 : 2) + GEN_WARPS));
        }
        *abort_flag = 0;
        fence_mbarrier_init();
    }
    if (warp == 0) tmem_alloc_pair(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // barriers of both CTAs initialised and TMEM allocated before any remote access
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(LOW_REGS));
        if (warp == 0 && lane == 0) {
            // ---------------- items (even CTA) and this CTA's A stages
            int gc = 0;
            for (int ic = 0;; ++ic) {
                int idx;
                if (lead) {
                    const int r = ic % IRING;
                    if (ic >= IRING && !mbar_wait_cl(&iempty[r], ((ic / IRING) - 1) & 1, abort_flag)) {
                        *abort_flag = 1;
                        break;
                    }
                    idx = queue ? atomicAdd(queue, 1) : (int)(cid + (uint32_t)ic * ncl);
                    if (idx >= n_items || *abort_flag) idx = -1;
                    iring[r] = idx;
                    st_cluster_s32(mapa_shared((const void *)&iring[r], 1), idx);
                    mbar_arrive(&ifull[r]);
                    mbar_arrive_cluster(mapa_shared(&ifull[r], 1));
                } else {
                    idx = ring_take_pair(ifull, iempty, iring, ic, abort_flag, 0);
                    if (idx == -2) *abort_flag = 1;
                }
                if (idx < 0) break;
                const int4 item = items[idx];
                const TcJobDev &J = jobs[item_job(item.x)];
                const int mt = 2 * item_mt(item.y) + (int)rank;
                const uint8_t *Abase = J.A + ((size_t)mt * J.nkc + item_k0(item.y)) * A_STAGE;
                for (int it = 0; it < item.w; ++it, ++gc) {
                    const int s = gc % STAGES;
                    if (gc >= STAGES && !mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                    mbar_arrive_expect_tx(&fullA[s], A_STAGE);
                    bulk_g2s(smem + s * STAGE, Abase + (size_t)it * A_STAGE, A_STAGE, &fullA[s]);
                }
                if (*abort_flag) break;
            }
            // the copies of the last stages have landed before the CTA may exit
            for (int c = max(0, gc - STAGES); c < gc; ++c)
                mbar_wait_n(&fullA[c % STAGES], (c / STAGES) & 1, kWaitLimit);
        } else if (OCTK && warp == 3 && lane == 0 && !lead) {
            // ---------------- odd CTA (octant-only build): once all its generator
            // warps have drained an accumulator group, one release arrival at
            // cluster scope frees the set on the even CTA's accEmpty
            int gbase = 0;
            bool ok = true;
            for (int ic = 0; ok; ++ic) {
                const int idx = ring_take_pair(ifull, iempty, iring, ic, abort_flag, 0);
                if (idx == -2) ok = false;
                if (idx < 0) break;
                const int nkc = items[idx].w;
                const int G = drain_every >= 1 ? max(2, min(drain_every, nkc)) : nkc;
                const int ngroups = (nkc + G - 1) / G;
                for (int i = 0; i < ngroups; ++i) {
                    const int gg = gbase + i;
                    if (*abort_flag || !mbar_wait_abort(&accDrained[gg & 1], (gg >> 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(&accEmpty[gg & 1], 0));
                }
                gbase += ngroups;
            }
            if (!ok) *abort_flag = 1;
        } else if ((warp == 1 || (OCTK && warp == 2)) && lane == 0 && !lead) {
            // ---------------- odd CTA: once a stage's A has landed and its W is
            // written, one release arrival on the even CTA's fullW covers both.
            // The octant-only build relays from two threads (warp 1 the even
            // chunks, warp 2 the odd ones), so two release arrivals at cluster
            // scope can be in flight at once.
            const int rpar = warp - 1;
            int gc = 0;
            bool ok = true;
            for (int ic = 0; ok; ++ic) {
                const int idx = ring_take_pair(ifull, iempty, iring, ic, abort_flag, 0);
                if (idx == -2) ok = false;
                if (idx < 0) break;
                const int nkc = items[idx].w;
                for (int it = 0; it < nkc; ++it, ++gc) {
                    if (OCTK && (gc & 1) != rpar) continue;
                    const int s = gc % STAGES;
                    const uint32_t par = (gc / STAGES) & 1;
                    if (*abort_flag || !mbar_wait_abort(&fullA[s], par, abort_flag) ||
                        !mbar_wait_abort(&fullW[s], par, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(&fullW[s], 0));
                }
            }
            if (!ok) *abort_flag = 1;
        } else if (warp == 1 && lane == 0) {
            // ---------------- even CTA: MMA issuer for the pair
            constexpr uint32_t ID2 = idesc_mma<KD::FMT, 2 * BN, 2 * BM>(false);  // M = 256, N = 256
            constexpr uint32_t IDO = idesc_mma<KD::FMT, BN, 2 * BM>(false);      // octant form: M = 256, N = 128
            int gc = 0, gbase = 0;
            for (int ic = 0;; ++ic) {
                const int idx = ring_take_pair(ifull, iempty, iring, ic, abort_flag, 0);
                if (idx == -2) *abort_flag = 1;
                if (idx < 0) break;
                const int4 itm = items[idx];
                const int nkc = itm.w;
                const bool oct = OCTK || jobs[item_job(itm.x)].oct != 0;
                const int G = drain_every >= 1 ? max(2, min(drain_every, nkc)) : nkc;
                bool ok = true;
                for (int it = 0; it < nkc; ++it, ++gc) {
                    const int s = gc % STAGES;
                    const uint32_t par = (gc / STAGES) & 1;
                    if (*abort_flag || !mbar_wait_abort(&fullA[s], par, abort_flag) ||
                        !mbar_wait_cl(&fullW[s], par, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int gg = gbase + it / G, set = gg & 1;
                    const bool first = (it % G) == 0;
                    if (first && gg >= 2 && !mbar_wait_cl(&accEmpty[set], ((gg - 2) >> 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t t_d = tmem + set * (2 * BN);
                    const uint32_t a0 = smem_u32(smem + s * STAGE);
                    const uint32_t w0 = a0 + A_STAGE;
                    if (oct) {
                        // real W (NP arrays of 64 rows per CTA): S_r = Ar W in columns
                        // [0, BN) of the set, S_i = Ai W in [BN, 2 BN)
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t ko = kk * 32;
#pragma unroll
                            for (int pq = 0; pq < KD::NPROD; ++pq) {
                                const int qa = prod_a(pq), qw = prod_w(pq);
                                const uint64_t ar = smem_desc_sw64(a0 + qa * A_ARR + ko);
                                const uint64_t ai = smem_desc_sw64(a0 + (NP + qa) * A_ARR + ko);
                                const uint64_t wb = smem_desc_sw64(w0 + qw * W_ARRH + ko);
                                const uint32_t acc = (first && kk == 0 && pq == 0) ? 0u : 1u;
                                mma_issue_pair(t_d, ar, wb, IDO, acc);
                                mma_issue_pair(t_d + BN, ai, wb, IDO, acc);
                            }
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t ko = kk * 32;  // 32 bytes = one MMA K step
#pragma unroll
                            for (int pq = 0; pq < KD::NPROD; ++pq) {
                                const int qa = prod_a(pq), qw = prod_w(pq);
                                const uint64_t ar = smem_desc_sw64(a0 + qa * A_ARR + ko);
                                const uint64_t ai = smem_desc_sw64(a0 + (NP + qa) * A_ARR + ko);
                                const uint32_t acc = (first && kk == 0 && pq == 0) ? 0u : 1u;
                                const uint32_t pb = w0 + qw * 3 * W_ARRH + ko;
                                mma_issue_pair(t_d, ar, smem_desc_sw64(pb + W_ARRH), ID2, acc);  // += [Ar Wr | Ar Wi] per half
                                mma_issue_pair(t_d, ai, smem_desc_sw64(pb), ID2, 1);             // += [-Ai Wi | Ai Wr]
                            }
                        }
                    }
                    mma_commit_pair(&empty[s]);
                    if ((it % G) == G - 1 || it == nkc - 1) mma_commit_pair(&accFull[set]);
                }
                if (!ok) {
                    *abort_flag = 1;
                    break;
                }
                gbase += (nkc + G - 1) / G;
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(HIGH_REGS));
        // ---------------- W generators (four threads per W row of this CTA's
        // half), accumulator drains and the half tile's epilogue
        const int gt = threadIdx.x - 128;   // 0..255
        const int wrow = gt & (BNH - 1);    // W row: column n0 + rank * BNH + wrow
        const int kq = gt / BNH;            // quarter of the chunk's k (one per warp)
        const int lg = warp & 3;            // TMEM lane group of the drains
        const int hsel = (warp - 4) >> 2;   // column half of the drains
        int2 *kobuf = kobuf_all + (warp - 4) * 2 * KQ;
        int gc = 0, gbase = 0, done_items = 0;
        bool ok = true;
        // where the drains arrive (the octant-only build: locally, see accDrained)
        uint64_t *dloc = OCTK ? (lead ? accEmpty : accDrained) : nullptr;
        for (int ic = 0; ok; ++ic) {
            const int idx = ring_take_pair(ifull, iempty, iring, ic, abort_flag, lane);
            if (idx == -2) ok = false;
            if (idx < 0) break;
            const int4 item = items[idx];
            const TcJobDev &J = jobs[item_job(item.x)];
            const int nkc = item.w;
            const int mp = item_mt(item.y), k0 = item_k0(item.y);
            const int G = drain_every >= 1 ? max(2, min(drain_every, nkc)) : nkc;
            const int ngroups = (nkc + G - 1) / G;
            // octant form: this thread's point opt (16 per CTA) and pair of k (kp) in
            // its warp's quarter of the chunk; it forms the four W rows of the point
            // (16 c + opt for the product c = 2 [Im Y] + [Im Z]) at both k.  A warp
            // covers 8 points x 4 k pairs, so its 4-byte shared stores hit 32
            // distinct banks.
            const bool oct = OCTK || J.oct != 0;
            const int opt = ((gt >> 5) & 1) * 8 + (gt & 7), kp = (gt >> 3) & 3;
            int iy = 0, iz = 0;
            if (oct) {
                const int64_t no = (int64_t)item.z * OCT_PTS + rank * OCT_PTH + opt;
                if (no < J.Noct) {
                    iz = (int)(no % J.nzh);
                    iy = (int)(no / J.nzh);
                }
            } else {
                const int64_t n = (int64_t)item.z * BN + rank * BNH + wrow;
                if (n < J.N) {
                    iz = (int)(n % J.nz);
                    iy = (int)(n / J.nz);
                }
            }
            // drains: columns of Re and Im (or of S_r and S_i) of this thread's half
            const int dre0 = oct ? hsel * BNH : hsel * 2 * BNH, dim_off = oct ? BN : BNH;
            const float2 *Yc = J.Y + iy;
            const float2 *Zc = J.Z + iz;
            float acc_re[CQ], acc_im[CQ];
#pragma unroll
            for (int j = 0; j < CQ; ++j) acc_re[j] = acc_im[j] = 0.f;
            const int gc0 = gc;
            int drained = 0;
            if constexpr (OCTK) {
                // Octant-only build: warps 4-7 write the W stages of the item's even
                // chunks and warps 8-11 those of its odd chunks, so the latency chains
                // (k-offsets, gathers, stores, proxy fence) of two chunks run at once.
                // Warp (4 + 4 grp + wq) covers quarter wq of its chunks' k; a thread
                // forms points pl and pl + 8 of the CTA's 16 (four Re/Im products
                // each, W rows 16 c + point) at the two k of its pair kpa.
                const int grp = (warp - 4) >> 2, wq = (warp - 4) & 3, kpa = lane >> 3, pl = lane & 7;
                const float2 *Yu[2], *Zu[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int64_t no = (int64_t)item.z * OCT_PTS + rank * OCT_PTH + u * 8 + pl;
                    int ya = 0, za = 0;
                    if (no < J.Noct) {
                        za = (int)(no % J.nzh);
                        ya = (int)(no / J.nzh);
                    }
                    Yu[u] = J.Y + ya;
                    Zu[u] = J.Z + za;
                }
                const int4 *ko4 = reinterpret_cast<const int4 *>(J.kofs + (size_t)k0 * BK + wq * KQ + 2 * kpa);
                int4 kn = make_int4(0, 0, 0, 0);
                if (grp < nkc) kn = __ldg(ko4 + (size_t)grp * (BK / 2));
                for (int it = grp; it < nkc && ok; it += 2) {
                    const int g2 = gc0 + it, s = g2 % STAGES;
                    const int4 kc = kn;
                    if (it + 2 < nkc) kn = __ldg(ko4 + (size_t)(it + 2) * (BK / 2));
                    float2 yy[2][2], zz[2][2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        yy[u][0] = __ldg(Yu[u] + kc.x);
                        zz[u][0] = __ldg(Zu[u] + kc.y);
                        yy[u][1] = __ldg(Yu[u] + kc.z);
                        zz[u][1] = __ldg(Zu[u] + kc.w);
                    }
                    const bool w = g2 < STAGES || mbar_wait(&empty[s], ((g2 / STAGES) - 1) & 1);
                    if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    uint8_t *wst = smem + s * STAGE + A_STAGE;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const float2 *y2 = yy[u], *z2 = zz[u];
                        const float v[V] = {__fmul_rn(y2[0].x, z2[0].x), __fmul_rn(y2[1].x, z2[1].x),
                                            __fmul_rn(y2[0].x, z2[0].y), __fmul_rn(y2[1].x, z2[1].y),
                                            __fmul_rn(y2[0].y, z2[0].x), __fmul_rn(y2[1].y, z2[1].x),
                                            __fmul_rn(y2[0].y, z2[0].y), __fmul_rn(y2[1].y, z2[1].y)};
                        uint4 pc_[NP];
                        split_vec<KIND>(v, pc_);
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const uint32_t wd[4] = {pc_[q].x, pc_[q].y, pc_[q].z, pc_[q].w};
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                *reinterpret_cast<uint32_t *>(
                                    wst + q * W_ARRH + sw64_offset<KIND>(c * OCT_PTH + u * 8 + pl, wq * KQ + 2 * kpa)) =
                                    wd[c];
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&fullW[s]);  // the odd CTA's relay forwards it
                    while (drained < ngroups && (drained + 1) * G - 1 + STAGES <= it) {
                        if (!drain_group_pair<CQ>(gbase + drained, accFull, accEmpty, tmem, lg, lane, dre0, dim_off,
                                                  acc_re, acc_im, abort_flag, dloc)) {
                            ok = false;
                            break;
                        }
                        ++drained;
                    }
                }
            } else {
            const int2 *kofs = J.kofs + (size_t)k0 * BK + kq * KQ;
            // octant form: each thread's two k-offsets (16 aligned bytes), read one
            // chunk ahead into registers; the other form stages the warp's eight
            // through shared memory
            const int4 *kofs4 = reinterpret_cast<const int4 *>(kofs + 2 * kp);
            int4 kn = make_int4(0, 0, 0, 0);
            if (oct) {
                kn = __ldg(kofs4);
            } else {
                if (lane < KQ) cp_async8(kobuf + lane, kofs + lane);
                cp_async_commit();
            }
            for (int it = 0; it < nkc && ok; ++it, ++gc) {
                const int s = gc % STAGES;
                const int2 *kb = kobuf + (it & 1) * KQ;
                float2 y[KQ], z[KQ];
                if (oct) {
                    const int4 kc = kn;
                    if (it + 1 < nkc) kn = __ldg(kofs4 + (size_t)(it + 1) * (BK / 2));
                    y[0] = __ldg(Yc + kc.x);
                    z[0] = __ldg(Zc + kc.y);
                    y[1] = __ldg(Yc + kc.z);
                    z[1] = __ldg(Zc + kc.w);
                } else {
                    if (it + 1 < nkc && lane < KQ)
                        cp_async8(kobuf + ((it + 1) & 1) * KQ + lane, kofs + (size_t)(it + 1) * BK + lane);
                    cp_async_commit();
                    cp_async_wait<1>();  // this chunk's records have landed
                    __syncwarp();
#pragma unroll
                    for (int e = 0; e < KQ; ++e) {
                        const int2 k2 = kb[e];
                        y[e] = __ldg(Yc + k2.x);
                        z[e] = __ldg(Zc + k2.y);
                    }
                }
                const bool w = gc < STAGES || mbar_wait(&empty[s], ((gc / STAGES) - 1) & 1);
                if (__any_sync(0xffffffffu, !w) || *abort_flag) {
                    ok = false;
                    break;
                }
                uint8_t *wst = smem + s * STAGE + A_STAGE;
                if (oct) {
                    // real W: (Re or Im of Y) x (Re or Im of Z) at the two k, one 64-row
                    // array per piece; split word c holds row 16 c + opt at both k
                    const float v[V] = {__fmul_rn(y[0].x, z[0].x), __fmul_rn(y[1].x, z[1].x),
                                        __fmul_rn(y[0].x, z[0].y), __fmul_rn(y[1].x, z[1].y),
                                        __fmul_rn(y[0].y, z[0].x), __fmul_rn(y[1].y, z[1].x),
                                        __fmul_rn(y[0].y, z[0].y), __fmul_rn(y[1].y, z[1].y)};
                    uint4 pc_[NP];
                    split_vec<KIND>(v, pc_);
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const uint32_t wd[4] = {pc_[q].x, pc_[q].y, pc_[q].z, pc_[q].w};
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            *reinterpret_cast<uint32_t *>(wst + q * W_ARRH +
                                                          sw64_offset<KIND>(c * OCT_PTH + opt, kq * KQ + 2 * kp)) = wd[c];
                    }
                } else {
                    float re[V], im[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) w_elem(y[e], z[e], re[e], im[e]);
                    uint4 pr_[NP], pi_[NP];
                    split_vec<KIND>(re, pr_);
                    split_vec<KIND>(im, pi_);
                    const uint32_t off = sw64_offset<KIND>(wrow, kq * KQ);
                    constexpr uint32_t SGN = 0x80008000u;
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        uint8_t *pb = wst + q * 3 * W_ARRH + off;
                        *reinterpret_cast<uint4 *>(pb) =
                            make_uint4(pi_[q].x ^ SGN, pi_[q].y ^ SGN, pi_[q].z ^ SGN, pi_[q].w ^ SGN);
                        *reinterpret_cast<uint4 *>(pb + W_ARRH) = pr_[q];
                        *reinterpret_cast<uint4 *>(pb + 2 * W_ARRH) = pi_[q];
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&fullW[s]);  // the odd CTA's relay forwards it
                while (drained < ngroups && (drained + 1) * G - 1 + STAGES <= it) {
                    if (!drain_group_pair<CQ>(gbase + drained, accFull, accEmpty, tmem, lg, lane, dre0, dim_off, acc_re,
                                              acc_im, abort_flag)) {
                        ok = false;
                        break;
                    }
                    ++drained;
                }
            }
            }
            cp_async_wait<0>();  // no copy into this warp's buffers outlives the item
            __syncwarp();
            while (ok && drained < ngroups) {
                if (!drain_group_pair<CQ>(gbase + drained, accFull, accEmpty, tmem, lg, lane, dre0, dim_off, acc_re,
                                          acc_im, abort_flag, dloc))
                    ok = false;
                ++drained;
            }
            gbase += ngroups;
            gc = gc0 + nkc;
            tile_epilogue<KIND, CQ>(J, item, 2 * mp + (int)rank, 2, (int)rank, ok, lg, lane, hsel * CQ, warp - 4,
                                    acc_re, acc_im);
            if (progress && ok) {
                // items this warp has finished (static schedule: cluster c runs c, c + clusters, ...),
                // its writes above visible at system scope before the count
                __threadfence_system();
                __syncwarp();
                ++done_items;
                if (lane == 0)
                    *reinterpret_cast<volatile int *>(progress + blockIdx.x * GEN_WARPS + (warp - 4)) = done_items;
            }
        }
        if (!ok) *abort_flag = 1;
    }
    if (threadIdx.x == 0 && *abort_flag) flag_error(err, kDevErrTimeout);
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // no CTA leaves while the other may still reach its shared memory or TMEM
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, TMEM_COLS);
    }
}

}  // namespace tc

// ------------------------------------------------------------------ host side

// Calls f(std::integral_constant<int, KIND>) for the run-time split kind.
template <typename F>
static auto with_kind(int kind, F &&f) {
    switch (kind) {
    case tc::KIND_BF16X2: return f(std::integral_constant<int, tc::KIND_BF16X2>{});
    case tc::KIND_BF16X3: return f(std::integral_constant<int, tc::KIND_BF16X3>{});
    case tc::KIND_FP16X2: return f(std::integral_constant<int, tc::KIND_FP16X2>{});
    default: return f(std::integral_constant<int, tc::KIND_TF32X2>{});
    }
}

static tc::Layout layout_of(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind) {
    return with_kind(kind, [&](auto K) { return tc::make_layout_k<decltype(K)::value>(ps, S, nx, ny, nz); });
}

size_t tc_job_bytes(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind) {
    return layout_of(ps, S, nx, ny, nz, kind).total;
}

size_t tc_workspace_bytes(const PairSetDev &ps, int S, int nx, int ny, int nz, int kind) {
    const tc::Layout L = layout_of(ps, S, nx, ny, nz, kind);
    const int64_t n_oct_nt = ((int64_t)((ny + 1) / 2) * ((nz + 1) / 2) + tc::OCT_PTS - 1) / tc::OCT_PTS;
    // descriptors (one per band) and work items: the tiles plus at most 2P
    // parts of the tail split per band
    return L.total + 1024 + 256 + (sizeof(TcJobDev) * kMaxBands + 255) / 256 * 256 +
           sizeof(int4) * (size_t)tc_max_items((int64_t)L.n_mt * std::max<int64_t>(L.n_nt, n_oct_nt) +
                                               (int64_t)(kMaxBands - 1) * 2 * tc_num_sms());
}

// Descriptor of one job whose tables and A image live in `ws`.
// Layout of one job with the rows actually computed: all (s, ix), or with
// `half` the rows ix < ceil(nx/2) (the sizes stay those of the full job).
template <int KIND>
static tc::Layout job_layout(const TcArgs &a) {
    using namespace tc;
    Layout L = make_layout_k<KIND>(*a.ps, a.S, a.nx, a.ny, a.nz);
    const int nxr = a.half ? (a.nx + 1) / 2 : a.nx;
    const int mq = a.pair ? 2 * BM : BM;  // pairs: an even number of m-tiles (the last may be all padding)
    L.M = a.S * nxr;
    L.M_pad = (L.M + mq - 1) / mq * mq;
    L.n_mt = L.M_pad / BM;
    if (a.oct) L.n_nt = (int)(((int64_t)((a.ny + 1) / 2) * ((a.nz + 1) / 2) + OCT_PTS - 1) / OCT_PTS);
    return L;
}

template <int KIND>
static void job_desc_t(const TcArgs &a, void *ws, TcJobDev *jd) {
    using namespace tc;
    const Layout L = job_layout<KIND>(a);
    uint8_t *w = static_cast<uint8_t *>(ws);
    jd->A = w + L.off_A;
    jd->Y = reinterpret_cast<float2 *>(w + L.off_Y);
    jd->Z = reinterpret_cast<float2 *>(w + L.off_Z);
    jd->kinfo = reinterpret_cast<int4 *>(w + L.off_k);
    jd->kofs = reinterpret_cast<int2 *>(w + L.off_ko);
    jd->ny = a.ny;
    jd->nz = a.nz;
    jd->nx = a.half ? (a.nx + 1) / 2 : a.nx;  // rows per state
    jd->nkc = L.nkc;
    jd->M = L.M;
    jd->n_mt = L.n_mt;
    jd->n_nt = L.n_nt;
    jd->N = L.N;
    jd->nq = (int64_t)a.nx * L.N;  // the full grid: state stride
    jd->scale = (float)a.scale;
    jd->f = reinterpret_cast<float2 *>(a.f);
    jd->f2 = a.f2;
    jd->mirror = a.half;
    jd->nxf = a.nx;
    int R = 0, sp = 0;
    if (a.pair) tail_split((L.n_mt / 2) * L.n_nt, L.nkc, tc_num_pairs(), &R, &sp);
    else tail_split(L.n_mt * L.n_nt, L.nkc, tc_num_sms(), &R, &sp);
    jd->pair = a.pair ? 1 : 0;
    jd->part = reinterpret_cast<float2 *>(w + L.off_part);
    jd->cnt = reinterpret_cast<int *>(w + L.off_cnt);
    jd->nsplit = sp;
    jd->split_tiles = sp ? R : 0;
    jd->tmax = Kind<KIND>::FP16 ? reinterpret_cast<const unsigned long long *>(w + L.off_tmax) : nullptr;
    // octant form: CTA pairs (two-piece kinds) or the single-CTA gather kernel (hi/mid/lo)
    jd->oct = a.oct && a.half && (a.pair || !Kind<KIND>::FUSE) ? 1 : 0;
    jd->nyh = (a.ny + 1) / 2;
    jd->nzh = (a.nz + 1) / 2;
    jd->Noct = (int64_t)jd->nyh * jd->nzh;
}

// Tables, k-index and the A image of one job in `ws` (tc_job_bytes bytes).
template <int KIND>
static cudaError_t prep_job_t(const TcArgs &a, void *ws, TcJobDev *jd, int64_t *launches, cudaStream_t st) {
    using namespace tc;
    using KD = Kind<KIND>;
    const PairSetDev &ps = *a.ps;
    const Layout L = job_layout<KIND>(a);
    if (L.n_mt > (1 << 24)) return cudaErrorInvalidConfiguration;
    if (a.oct && !(a.half && (a.pair || !KD::FUSE))) return cudaErrorInvalidValue;
    uint8_t *w = static_cast<uint8_t *>(ws);
    float2 *X = reinterpret_cast<float2 *>(w + L.off_X);
    float2 *Y = reinterpret_cast<float2 *>(w + L.off_Y);
    float2 *Z = reinterpret_cast<float2 *>(w + L.off_Z);
    int4 *kinfo = reinterpret_cast<int4 *>(w + L.off_k);
    uint8_t *Abuf = w + L.off_A;
    const double *qa[3] = {a.qx, a.qy, a.qz};
    float2 *tab[3] = {X, Y, Z};
    const int na[3] = {a.nx, a.ny, a.nz};
    for (int ax = 0; ax < 3; ++ax) {
        const int64_t tot = ((int64_t)ps.n_pair + 1) * na[ax];
        // FP16 kind: the Y and Z rows are scaled (X only enters A in FP32)
        const double Q = KD::FP16 && ax > 0 ? a.qabs[ax] : -1.0;
        axis_power_table_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(ps, a.pair_geom, qa[ax], na[ax], ax,
                                                                               L.n_axrows, tab[ax], Q);
    }
    int2 *kofs = reinterpret_cast<int2 *>(w + L.off_ko);
    kindex_kernel<<<(unsigned)((L.K_pad + 255) / 256), 256, 0, st>>>(ps, L.K_pad, L.n_axrows, a.ny, a.nz, kinfo, kofs);
    int *kexp = reinterpret_cast<int *>(w + L.off_kexp);
    unsigned long long *tmax = reinterpret_cast<unsigned long long *>(w + L.off_tmax);
    if constexpr (KD::FP16) {
        cudaError_t e = cudaMemsetAsync(tmax, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        fp16_bound_kernel<<<(unsigned)((L.K_pad + 255) / 256), 256, 0, st>>>(
            ps, a.coef32, a.SB, a.S, a.pair_geom, kinfo, L.K_pad, a.qabs[0], a.qabs[1], a.qabs[2], kexp, tmax);
        if (launches) *launches += 1;
    }
    {
        const int nxr = a.half ? (a.nx + 1) / 2 : a.nx;
        // states one m-tile's rows can touch, and their staged coefficients
        const int ns_max = std::min(a.S, (BM + nxr - 1) / nxr + 1);
        const size_t csm = sizeof(float) * (size_t)ns_max * KD::BK * (kMaxPairL + 1);
        if (csm <= 48 * 1024 && L.M > 0) {
            abuild_tile_kernel<KIND><<<dim3((unsigned)L.nkc, (unsigned)L.n_mt), BM * KD::BK / KD::PER_VEC, csm, st>>>(
                ps, a.coef32, a.SB, nxr, a.nx, X, kinfo, L.nkc, L.M, Abuf, kexp, tmax);
        } else {
            const int64_t tot = (int64_t)L.M_pad * (L.K_pad / KD::PER_VEC);
            abuild_kernel<KIND><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
                ps, a.coef32, a.SB, nxr, a.nx, X, kinfo, L.K_pad, L.nkc, L.M, L.M_pad, Abuf, kexp, tmax);
        }
    }
    if (launches) *launches += 5;
    cudaError_t e = cudaMemsetAsync(w + L.off_cnt, 0, sizeof(int) * 8 * (size_t)L.part_tiles, st);
    if (e != cudaSuccess) return e;
    if (jd) job_desc_t<KIND>(a, ws, jd);
    return cudaGetLastError();
}

void tc_job_desc(const TcArgs &a, void *ws, TcJobDev *jd) {
    with_kind(a.kind, [&](auto K) { job_desc_t<decltype(K)::value>(a, ws, jd); });
}

cudaError_t tc_prep_job(const TcArgs &a, void *ws, TcJobDev *jd, int64_t *launches, cudaStream_t st) {
    return with_kind(a.kind, [&](auto K) { return prep_job_t<decltype(K)::value>(a, ws, jd, launches, st); });
}

// Items of the tiles (mt, nt) of descriptor j, in the given order; the last
// J.split_tiles of them run as J.nsplit parts.
static void append_items(const TcJobDev &J, int j, const std::vector<int2> &tiles, std::vector<int4> &items) {
    const int n = (int)tiles.size();
    const int first_split = J.nsplit ? n - J.split_tiles : n;
    for (int i = 0; i < n; ++i) {
        const int mt = tiles[i].x, nt = tiles[i].y;
        if (i < first_split) {
            items.push_back(make_int4(j, mt, nt, J.nkc));
            continue;
        }
        for (int p = 0; p < J.nsplit; ++p) {
            const int k0 = (int)((int64_t)p * J.nkc / J.nsplit), k1 = (int)((int64_t)(p + 1) * J.nkc / J.nsplit);
            const int slot = (i - first_split) * J.nsplit + p;
            items.push_back(make_int4(j | ((slot + 1) << 16), mt | (k0 << 16), nt, k1 - k0));
        }
    }
}

// Work list of a group of prepared jobs: every (job, m-tile, n-tile), most
// expensive first (longest k loop), so the static round-robin assignment of
// items to CTAs balances well.
void tc_build_items(const TcJobDev *jobs, int n_jobs, std::vector<int4> &items) {
    items.clear();
    std::vector<int2> tiles;
    for (int j = 0; j < n_jobs; ++j) {
        const TcJobDev &J = jobs[j];
        tiles.clear();
        const int n_rows = J.pair ? J.n_mt / 2 : J.n_mt;  // m-tiles, or m-tile pairs
        for (int i = 0; i < n_rows * J.n_nt; ++i) tiles.push_back(make_int2(i / J.n_nt, i % J.n_nt));
        append_items(J, j, tiles, items);
    }
    // longest first; the stable order keeps each job's tiles row-major and its parts last
    std::stable_sort(items.begin(), items.end(), [](const int4 &x, const int4 &y) { return x.w > y.w; });
}

using sched::band_runs;

// Per-device slots of the launchers' one-time set-up (kernel attributes, SM
// and cluster counts): the current device's index, folded into the table.
constexpr int kAttrDevices = 64;
static int current_device_slot() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    return dev % kAttrDevices;
}


template <int KIND, int VAR>
static cudaError_t persistent_t(const TcJobDev *d_jobs, const int4 *d_items, int n_items, int drain_every, int *err,
                                int grid_ctas, int64_t *launches, cudaStream_t st, int *progress, int *queue) {
    using namespace tc;
    using CF = Cfg<KIND, VAR>;
    static bool attr_set[kAttrDevices] = {};  // kernel attributes are per device
    const int dev = current_device_slot();
    cudaError_t e;
    if (!attr_set[dev]) {
        // The register split inside the kernel assumes exactly LAUNCH_REGS
        // registers per thread at launch; anything else could leave the
        // increasing warpgroups waiting, so refuse to launch.
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, tc_persistent_kernel<KIND, VAR>);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != LAUNCH_REGS) return cudaErrorInvalidDeviceFunction;
        e = cudaFuncSetAttribute(tc_persistent_kernel<KIND, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 CF::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    if (n_items <= 0) return cudaSuccess;
    const int grid = std::max(1, std::min(grid_ctas, n_items));
    tc_persistent_kernel<KIND, VAR><<<grid, THREADS, CF::SMEM_BYTES, st>>>(d_jobs, d_items, n_items, drain_every, err,
                                                                         progress, queue);
    if (launches) ++*launches;
    return cudaGetLastError();
}

// CTA-pair launch: grid = 2 x pairs, clusters of two CTAs.  OCTK: the build
// for launches whose jobs all run in the octant form.
template <int KIND, bool OCTK>
static cudaError_t pair_t(const TcJobDev *d_jobs, const int4 *d_items, int n_items, int drain_every, int *err,
                          int grid_ctas, int64_t *launches, cudaStream_t st, int *progress, int *queue) {
    using namespace tc;
    using PC = PairCfg<KIND, OCTK>;
    static bool attr_set[kAttrDevices] = {};  // kernel attributes are per device
    const int dev = current_device_slot();
    cudaError_t e;
    if (!attr_set[dev]) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, tc_pair_kernel<KIND, OCTK>);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != LAUNCH_REGS) return cudaErrorInvalidDeviceFunction;
        e = cudaFuncSetAttribute(tc_pair_kernel<KIND, OCTK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PC::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    if (n_items <= 0) return cudaSuccess;
    const int pairs = std::max(1, std::min(std::min(grid_ctas / 2, tc_num_pairs()), n_items));
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(2 * pairs, 1, 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = PC::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tc_pair_kernel<KIND, OCTK>, d_jobs, d_items, n_items, drain_every, err, progress,
                           queue);
    if (launches) ++*launches;
    return e != cudaSuccess ? e : cudaGetLastError();
}

int tc_num_pairs() {
    static int cnt[kAttrDevices] = {};
    const int slot = current_device_slot();
    int &n = cnt[slot];
    if (!n) {
        // the pair kernels of both kinds have the same footprint (one CTA per SM)
        using PC = tc::PairCfg<tc::KIND_FP16X2>;
        cudaFuncSetAttribute(tc::tc_pair_kernel<tc::KIND_FP16X2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PC::SMEM_BYTES);
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(2 * 1024, 1, 1);
        cfg.blockDim = dim3(tc::THREADS, 1, 1);
        cfg.dynamicSmemBytes = PC::SMEM_BYTES;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, tc::tc_pair_kernel<tc::KIND_FP16X2, false>, &cfg) != cudaSuccess ||
            c <= 0) {
            cudaGetLastError();
            c = tc_num_sms() / 2;
        }
        n = std::min(c, tc_num_sms() / 2);
    }
    return n;
}

int tc_variant_preferred(int kind) {
    return kind == tc::KIND_TF32X2 ? tc::VAR_ZSTAGE : tc::VAR_OCT;
}

bool tc_prefetch_ok(int kind) { return kind == tc::KIND_FP16X2 || kind == tc::KIND_BF16X2; }

bool tc_zstage_ok(int kind, const TcJobDev *jobs, int n_jobs) {
    if (kind == tc::KIND_BF16X3 || n_jobs <= 0) return false;
    for (int j = 0; j < n_jobs; ++j)
        if (jobs[j].ylm || jobs[j].nz % tc::BN != 0) return false;
    return true;
}

int tc_variant_resolve(int kind, int requested, bool zstage_grid) {
    if (requested == tc::VAR_ZSTAGE) return kind != tc::KIND_BF16X3 && zstage_grid ? tc::VAR_ZSTAGE : tc::VAR_GATHER;
    if (requested == tc::VAR_PREFETCH) return tc_prefetch_ok(kind) ? tc::VAR_PREFETCH : tc::VAR_GATHER;
    if (requested == tc::VAR_PAIR) return tc_prefetch_ok(kind) ? tc::VAR_PAIR : tc::VAR_GATHER;
    if (requested == tc::VAR_OCT)
        return tc_prefetch_ok(kind) || kind == tc::KIND_BF16X3 ? tc::VAR_OCT : tc::VAR_GATHER;
    return tc::VAR_GATHER;
}

int tc_variant_for(int kind, int requested, const TcJobDev *jobs, int n_jobs) {
    // jobs laid out for pairs run the pair launch; others never do
    // (VAR_OCT: every job in the octant form, the five-stage build; jobs of both
    // forms share the four-stage build, which takes the form per job)
    bool pair = n_jobs > 0, oct = n_jobs > 0;
    for (int j = 0; j < n_jobs; ++j) {
        pair = pair && jobs[j].pair && !jobs[j].ylm;
        oct = oct && jobs[j].oct;
    }
    if (pair) return oct ? tc::VAR_OCT : tc::VAR_PAIR;
    // single CTAs: jobs in the octant form run in the gather kernel's octant
    // build, which also takes jobs in the Re/Im form
    bool any_oct = false;
    for (int j = 0; j < n_jobs; ++j) any_oct = any_oct || jobs[j].oct;
    if (any_oct && kind == tc::KIND_BF16X3) return tc::VAR_OCT;
    const int v = tc_variant_resolve(kind, requested, tc_zstage_ok(kind, jobs, n_jobs));
    return v == tc::VAR_PAIR || v == tc::VAR_OCT ? tc::VAR_GATHER : v;
}

cudaError_t tc_launch_persistent(int kind, int variant, const TcJobDev *d_jobs, const int4 *d_items, int n_items,
                                 int drain_every, int *err, int grid_ctas, int64_t *launches, cudaStream_t st,
                                 int *progress, int *queue) {
    if (queue && n_items > 0) {
        // the queue counter starts at zero for every launch (a memset node in a captured graph)
        const cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
    }
    return with_kind(kind, [&](auto K) {
        constexpr int KIND = decltype(K)::value;
        if constexpr (KIND != tc::KIND_BF16X3) {
            if (variant == tc::VAR_ZSTAGE)
                return persistent_t<KIND, tc::VAR_ZSTAGE>(d_jobs, d_items, n_items, drain_every, err, grid_ctas,
                                                          launches, st, progress, queue);
        }
        if constexpr (tc::Kind<KIND>::STAGE_KO && !tc::Kind<KIND>::TF32) {
            if (variant == tc::VAR_OCT)
                return pair_t<KIND, true>(d_jobs, d_items, n_items, drain_every, err, grid_ctas, launches, st,
                                          progress, queue);
            if (variant == tc::VAR_PAIR)
                return pair_t<KIND, false>(d_jobs, d_items, n_items, drain_every, err, grid_ctas, launches, st,
                                           progress, queue);
        }
        if constexpr (!tc::Kind<KIND>::FUSE && !tc::Kind<KIND>::TF32) {
            if (variant == tc::VAR_OCT)
                return persistent_t<KIND, tc::VAR_OCT>(d_jobs, d_items, n_items, drain_every, err, grid_ctas,
                                                       launches, st, progress, queue);
        }
        if constexpr (tc::Kind<KIND>::STAGE_KO) {
            if (variant == tc::VAR_PREFETCH)
                return persistent_t<KIND, tc::VAR_PREFETCH>(d_jobs, d_items, n_items, drain_every, err, grid_ctas,
                                                            launches, st, progress, queue);
        }
        return persistent_t<KIND, tc::VAR_GATHER>(d_jobs, d_items, n_items, drain_every, err, grid_ctas, launches,
                                                  st, progress, queue);
    });
}

int tc_kind_of_precision(int precision) {
    switch (precision) {
    case SCFF_BF16X2: return tc::KIND_BF16X2;
    case SCFF_BF16X3: return tc::KIND_BF16X3;
    case SCFF_TF32X3: return tc::KIND_TF32X2;
    case SCFF_FP16X2: return tc::KIND_FP16X2;
    default: return -1;
    }
}

void tc_axes_abs_max(const double *qx, int nx, const double *qy, int ny, const double *qz, int nz, double out[3]) {
    const double *q[3] = {qx, qy, qz};
    const int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        double m = 0.0;
        for (int i = 0; i < n[a]; ++i) m = std::max(m, fabs(q[a][i]));
        out[a] = m;
    }
}

int64_t tc_max_items(int64_t tiles) { return tiles + 2 * (int64_t)tc_num_sms(); }

int tc_num_sms() {
    static int cnt[kAttrDevices] = {};
    const int slot = current_device_slot();
    if (!cnt[slot]) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cnt[slot] = n > 0 ? n : 148;
    }
    return cnt[slot];
}

// Single job: prepare it in the workspace, then one persistent launch over
// its tiles.  The descriptor and work list go to the end of the workspace.
// With host outputs and bands, the tiles are ordered band by band, the launch
// reports its progress, and each band's columns are copied to the host while
// later bands compute (see TcArgs).
cudaError_t launch_tc_form_factor(const TcArgs &args, int64_t *launches, cudaStream_t st) {
    using tc::BN;
    const bool can_band =
        args.f_host && args.copy_st && args.progress_dev && args.progress_host && args.ev_done && args.ev_copied;
    TcArgs a = args;
    {
        const int v = tc_variant_resolve(a.kind, a.zstage, false);
        a.pair = tc_prefetch_ok(a.kind) && (v == tc::VAR_PAIR || v == tc::VAR_OCT) ? 1 : 0;
        a.oct = v == tc::VAR_OCT && a.half ? 1 : 0;
    }
    const size_t jb = tc_job_bytes(*a.ps, a.S, a.nx, a.ny, a.nz, a.kind);
    if (jb + 1024 + sizeof(TcJobDev) > a.ws_bytes) return cudaErrorInvalidValue;
    TcJobDev jd;
    memset(&jd, 0, sizeof(jd));
    cudaError_t e = tc_prep_job(a, a.ws, &jd, launches, st);
    if (e != cudaSuccess) return e;
    // the job's tail split (job_desc_t) covers its last split_tiles tiles in any order
    const int64_t n_tiles = (int64_t)(jd.pair ? jd.n_mt / 2 : jd.n_mt) * jd.n_nt;
    const int64_t first_split = jd.nsplit ? n_tiles - jd.split_tiles : n_tiles;
    const int64_t n_items_all = first_split + (n_tiles - first_split) * (jd.nsplit ? jd.nsplit : 1);
    // units that take items in turn: CTAs, or CTA pairs (two CTAs per unit)
    const int per = a.pair ? 2 : 1;
    const int units = (int)std::max<int64_t>(1, std::min<int64_t>(a.pair ? tc_num_pairs() : tc_num_sms(), n_items_all));
    const int grid = per * units;
    const int n_rows = jd.n_mt / per;  // m-tiles, or m-tile pairs
    int bounds[kMaxBands + 1];
    // Bands are ranges of column tiles (d = min(nt, n_nt-1-nt) with the
    // mirror).  In the octant form they are ranges of octant y rows iy (each
    // band also covers the mirrored rows ny-1-iy), banded only when a y row
    // is a whole number of tiles.
    const bool oct = jd.oct != 0;
    const int oct_row_tiles = jd.nzh / tc::OCT_PTS;
    int G = 1;
    if (can_band && !oct)
        G = sched::band_bounds(n_rows, jd.n_nt, jd.mirror != 0, jd.N, BN, a.n_bands, units, first_split, jd.nsplit,
                               kMaxBands, bounds);
    else if (can_band && oct && jd.nzh % tc::OCT_PTS == 0)
        G = sched::band_bounds(n_rows, a.ny, true, jd.N, a.nz, a.n_bands, units, first_split, jd.nsplit, kMaxBands,
                               bounds);
    const int64_t unit_cols = oct ? a.nz : BN;  // output columns per band unit
    std::vector<int4> items;
    int runs[kMaxBands][2][2], nruns[kMaxBands];
    int64_t band_end[kMaxBands];
    if (G == 1) {
        tc_build_items(&jd, 1, items);
    } else {
        // tiles band by band; band g ends after the items of its tiles
        std::vector<int2> tiles;
        for (int g = 0; g < G; ++g) {
            if (oct) {
                // octant y rows [b_g, b_g+1): their tiles, and the output rows they fill
                nruns[g] = band_runs(a.ny, true, bounds[g], bounds[g + 1], runs[g]);
                for (int mt = 0; mt < n_rows; ++mt)
                    for (int iy = bounds[g]; iy < bounds[g + 1]; ++iy)
                        for (int t = 0; t < oct_row_tiles; ++t) tiles.push_back(make_int2(mt, iy * oct_row_tiles + t));
            } else {
                nruns[g] = band_runs(jd.n_nt, jd.mirror != 0, bounds[g], bounds[g + 1], runs[g]);
                for (int mt = 0; mt < n_rows; ++mt)
                    for (int r = 0; r < nruns[g]; ++r)
                        for (int nt = runs[g][r][0]; nt < runs[g][r][1]; ++nt) tiles.push_back(make_int2(mt, nt));
            }
            const int64_t t = (int64_t)tiles.size();
            band_end[g] = t <= first_split ? t : first_split + (t - first_split) * jd.nsplit;
        }
        append_items(jd, 0, tiles, items);
    }
    uint8_t *tail = static_cast<uint8_t *>(a.ws) + (jb + 255) / 256 * 256;
    TcJobDev *d_job = reinterpret_cast<TcJobDev *>(tail);
    int4 *d_items = reinterpret_cast<int4 *>(tail + 256);
    if ((size_t)(tail + 256 - static_cast<uint8_t *>(a.ws)) + sizeof(int4) * items.size() > a.ws_bytes)
        return cudaErrorInvalidValue;
    e = cudaMemcpyAsync(d_job, &jd, sizeof(jd), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    const int n_items = (int)items.size();
    if (n_items != n_items_all) return cudaErrorInvalidValue;
    if (G > 1) {
        // the previous banded launch (if any) has ended, even if its call
        // returned early, before its slots are reused
        if ((e = cudaEventSynchronize(a.ev_done)) != cudaSuccess) return e;
        for (int i = 0; i < grid * tc::GEN_WARPS; ++i) a.progress_host[i] = 0;
    }
    if (a.ev_mark) cudaEventRecord(a.ev_mark, st);
    const int variant = tc_variant_for(a.kind, a.zstage, &jd, 1);
    if (a.variant_used) *a.variant_used = variant;
    e = tc_launch_persistent(a.kind, variant, d_job, d_items, n_items,
                             a.drain_every, a.err, grid, launches, st, G > 1 ? a.progress_dev : nullptr);
    if (a.bands_used) *a.bands_used = G;
    if (e != cudaSuccess || G == 1) return e;
    if ((e = cudaEventRecord(a.ev_done, st)) != cudaSuccess) return e;
    // unit b (a CTA, or the CTA pair 2b, 2b + 1) runs items b, b + units, ...:
    // items [0, E) are written once each generator warp of the unit has
    // finished ceil((E - b) / units) items (a split tile's last part writes
    // the tile before it counts itself)
    auto written = [&](int64_t E) {
        for (int b = 0; b < units && b < E; ++b) {
            const int need = (int)((E - b + units - 1) / units);
            for (int c = per * b; c < per * (b + 1); ++c)
                for (int w = 0; w < tc::GEN_WARPS; ++w)
                    if (a.progress_host[c * tc::GEN_WARPS + w] < need) return false;
        }
        return true;
    };
    const size_t rows = (size_t)a.S * a.nx;  // output rows (s, ix) of N columns
    // on an error after some copies were queued, wait for them before returning:
    // they write into the caller's buffers
    auto fail_after_copies = [&](cudaError_t err) {
        cudaStreamSynchronize(a.copy_st);
        return err;
    };
    bool launch_over = false;
    for (int g = 0; g < G; ++g) {
        // the launch ends in any case (every device wait is bounded), and
        // then every band is final
        while (!launch_over && !written(band_end[g])) {
            const cudaError_t q = cudaEventQuery(a.ev_done);
            if (q == cudaSuccess) launch_over = true;
            else if (q != cudaErrorNotReady) return fail_after_copies(q);
            else std::this_thread::yield();
        }
        for (int r = 0; r < nruns[g]; ++r) {
            const int64_t c0 = (int64_t)runs[g][r][0] * unit_cols,
                          c1 = std::min<int64_t>(jd.N, (int64_t)runs[g][r][1] * unit_cols);
            if (c1 <= c0) continue;
            e = cudaMemcpy2DAsync(a.f_host + 2 * c0, 8 * jd.N, a.f + 2 * c0, 8 * jd.N, 8 * (c1 - c0), rows,
                                  cudaMemcpyDeviceToHost, a.copy_st);
            if (e == cudaSuccess && a.f2_host && a.f2)
                e = cudaMemcpy2DAsync(a.f2_host + c0, 4 * jd.N, a.f2 + c0, 4 * jd.N, 4 * (c1 - c0), rows,
                                      cudaMemcpyDeviceToHost, a.copy_st);
            if (e != cudaSuccess) return fail_after_copies(e);
        }
    }
    if ((e = cudaEventRecord(a.ev_copied, a.copy_st)) != cudaSuccess) return fail_after_copies(e);
    e = cudaStreamWaitEvent(st, a.ev_copied, 0);
    return e == cudaSuccess ? e : fail_after_copies(e);
}

// ------------------------------------------------------------------ generic two-table contraction

template <int KIND> static int bk_of() { return tc::Kind<KIND>::BK; }

int64_t tc_generic_kpad(int kind, int64_t K) {
    const int BK = kind == tc::KIND_TF32X2 ? bk_of<tc::KIND_TF32X2>() : bk_of<tc::KIND_BF16X3>();
    int64_t kp = (K + BK - 1) / BK * BK;
    return kp > 0 ? kp : BK;
}

static size_t a_stage_of(int kind) {
    switch (kind) {
    case tc::KIND_BF16X2: return tc::Kind<tc::KIND_BF16X2>::A_STAGE;
    case tc::KIND_BF16X3: return tc::Kind<tc::KIND_BF16X3>::A_STAGE;
    default: return tc::Kind<tc::KIND_TF32X2>::A_STAGE;
    }
}

size_t tc_generic_bytes(int kind, int M, int64_t K) {
    const int64_t K_pad = tc_generic_kpad(kind, K);
    const int BK = kind == tc::KIND_TF32X2 ? bk_of<tc::KIND_TF32X2>() : bk_of<tc::KIND_BF16X3>();
    const int n_mt = (M + tc::BM - 1) / tc::BM;
    const size_t img = (size_t)n_mt * (size_t)(K_pad / BK) * a_stage_of(kind);
    return (img + 1023) / 1024 * 1024 + 1024;
}

template <int KIND>
static void dense_image_t(const TcGenericArgs &a, int M_pad, int64_t K_pad, int nkc, uint8_t *img, cudaStream_t st) {
    using KD = tc::Kind<KIND>;
    const int64_t tot = (int64_t)M_pad * (K_pad / KD::PER_VEC);
    tc::dense_image_kernel<KIND><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a.A, a.lda, a.M, a.K, M_pad, K_pad,
                                                                                 nkc, img);
}

cudaError_t tc_run_generic_multi(const TcGenericArgs *jobs, int n_jobs, int64_t *launches, cudaStream_t st) {
    using namespace tc;
    if (n_jobs <= 0) return cudaSuccess;
    const TcGenericArgs &a0 = jobs[0];
    const int BK = a0.kind == KIND_TF32X2 ? bk_of<KIND_TF32X2>() : bk_of<KIND_BF16X3>();
    std::vector<TcJobDev> descs;
    std::vector<size_t> img_off;
    size_t off = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const TcGenericArgs &a = jobs[j];
        if (a.kind != a0.kind || a.ws != a0.ws) return cudaErrorInvalidValue;
        if (a.M <= 0 || a.N <= 0) continue;
        const int64_t K_pad = tc_generic_kpad(a.kind, a.K);
        const int nkc = (int)(K_pad / BK);
        const int n_mt = (a.M + BM - 1) / BM;
        const int n_nt = (int)((a.N + BN - 1) / BN);
        TcJobDev jd;
        memset(&jd, 0, sizeof(jd));
        jd.A = static_cast<uint8_t *>(a0.ws) + off;
        jd.Y = a.Y;
        jd.Z = a.Z;
        jd.kofs = a.kofs;
        jd.nz = a.nz;
        jd.nx = a.nx;
        jd.nkc = nkc;
        jd.M = a.M;
        jd.n_mt = n_mt;
        jd.n_nt = n_nt;
        jd.ylm = a.ylm;
        jd.ystride = a.ystride;
        jd.N = a.N;
        jd.nq = (int64_t)a.nx * a.N;
        jd.scale = a.scale;
        jd.f = a.C;
        jd.f2 = a.C2;
        img_off.push_back(off);
        descs.push_back(jd);
        off += ((size_t)n_mt * nkc * a_stage_of(a.kind) + 1023) / 1024 * 1024;
        // split-and-swizzle image of this job's A
        const int M_pad = n_mt * BM;
        uint8_t *img = static_cast<uint8_t *>(a0.ws) + img_off.back();
        switch (a.kind) {
        case KIND_BF16X2: dense_image_t<KIND_BF16X2>(a, M_pad, K_pad, nkc, img, st); break;
        case KIND_BF16X3: dense_image_t<KIND_BF16X3>(a, M_pad, K_pad, nkc, img, st); break;
        default: dense_image_t<KIND_TF32X2>(a, M_pad, K_pad, nkc, img, st); break;
        }
        if (launches) ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (descs.empty()) return cudaSuccess;
    std::vector<int4> items;
    tc_build_items(descs.data(), (int)descs.size(), items);
    uint8_t *tail = static_cast<uint8_t *>(a0.ws) + off;
    const size_t dbytes = (sizeof(TcJobDev) * descs.size() + 255) / 256 * 256;
    if (off + dbytes + sizeof(int4) * items.size() > a0.ws_bytes) return cudaErrorInvalidValue;
    TcJobDev *d_jobs = reinterpret_cast<TcJobDev *>(tail);
    int4 *d_items = reinterpret_cast<int4 *>(tail + dbytes);
    cudaError_t e = cudaMemcpyAsync(d_jobs, descs.data(), sizeof(TcJobDev) * descs.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return tc_launch_persistent(a0.kind, tc::VAR_GATHER, d_jobs, d_items, (int)items.size(), a0.drain_every, a0.err,
                                tc_num_sms(), launches, st);
}

cudaError_t tc_run_generic(const TcGenericArgs &a, int64_t *launches, cudaStream_t st) {
    return tc_run_generic_multi(&a, 1, launches, st);
}

}  // namespace scff
