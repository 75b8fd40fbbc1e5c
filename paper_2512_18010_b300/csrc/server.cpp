// Serving runtime: continuous batching of form-factor jobs on one GPU.
//
// Clients submit jobs (a basis and transitions already resident on the
// device, a product q-grid, output buffers) from any thread.  One server
// thread owns all CUDA work.  On every pass it
//   1. retires batches whose completion event has fired (frees their device
//      memory, records the completion time, wakes waiters);
//   2. if a stream slot is free, admits pending jobs in arrival order while
//      their device footprint fits the free part of the arena (first-fit
//      allocator over one pre-allocated block: no cudaMalloc per job), and
//      launches them as one batch -- per-job pair-prep and tables, then ONE
//      persistent tensor-core launch over all tiles of the batch -- on the
//      slot's stream, followed by the output copies and a completion event.
// Jobs that arrive while earlier batches run are admitted into the next
// batch as soon as a slot and memory free up, so their work overlaps on the
// device with the batches already in flight.  A job that waited past eight
// admissions of later jobs blocks further skipping until it fits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/scff.h"
#include "scff_internal.h"
#include "scff_objects.h"
#include "tc_internal.h"

namespace scff {
scff_status set_last_error(scff_status code, const char *msg);
}
using namespace scff;

namespace {

scff_status serr(scff_status code, const char *fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t up1k(size_t x) { return (x + 1023) / 1024 * 1024; }

// First-fit allocator over [0, size).
class Arena {
  public:
    void init(size_t size) {
        free_.clear();
        free_[0] = size;
        size_ = size;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = up1k(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up1k(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

enum JobState { PENDING = 0, RUNNING = 1, DONE = 2, CANCELLED = 3, FAILED = 4 };

struct SJob {
    int64_t id;
    scff_request req;
    std::vector<double> ax[3];
    int S = 0, S_pad = 0;
    int64_t nq = 0;
    int half = 0;            // Hermitian half of an antisymmetric grid (fixed at submit)
    size_t footprint = 0;    // bytes of the job's arena block
    size_t off = 0;          // arena offset
    size_t scratch_need = 0; // pair geometry + coefficients of this job
    double cost = 0;         // work estimate: contraction rows x states x evaluated points
    int skipped = 0;
    int state = PENDING;
    scff_status status = SCFF_OK;
    bool registered = false; // host output pinned by the server
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Batch {
    std::vector<SJob *> jobs;
    size_t scratch_off = 0, scratch_bytes = 0;
    cudaEvent_t ev = nullptr;
};

}  // namespace

struct scff_server_s {
    scff_ctx *ctx = nullptr;
    int precision = SCFF_TF32X3;
    int variant = 0;                 // W generator variant requested (the context's mode when created)
    int slots = 2;
    int max_batch = 64;
    double cost_ratio = 0.0;         // batch members' work within this factor of the first one's (<= 0: any)
    std::vector<cudaStream_t> streams;
    std::vector<Batch *> busy;       // per slot, null when free
    std::vector<void *> h_stage;     // pinned staging for descriptors and work lists, per slot
    std::vector<int *> h_err;        // pinned status words, per slot
    size_t stage_bytes = 8u << 20;
    void *arena_ptr = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<SJob *> pending;
    std::unordered_map<int64_t, SJob *> jobs;
    int64_t next_id = 1;
    bool stop = false;
    std::thread th;
    int64_t n_submitted = 0, n_done = 0, n_cancel = 0, n_failed = 0, n_batches = 0, max_inflight = 0;
    int64_t inflight = 0;
};

namespace {

bool tc_precision(int p) { return tc_kind_of_precision(p) >= 0; }
int tc_kind_of(int p) { return tc_kind_of_precision(p); }

// Device bytes of one job: q axes, tables + A image (tensor cores) or axis
// tables (direct path), and device outputs when the client's are on the host.
void size_job(scff_server_s *sv, SJob *j) {
    const PairSetDev &ps = j->req.basis->dev;
    const bool fp64 = sv->precision == SCFF_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const int nx = j->req.nx, ny = j->req.ny, nz = j->req.nz;
    size_t b = up1k(sizeof(double) * (size_t)(nx + ny + nz));
    if (tc_precision(sv->precision))
        b += up1k(tc_job_bytes(ps, j->S, nx, ny, nz, tc_kind_of(sv->precision)));
    else
        b += up1k((size_t)ps.n_pair * (nx + ny + nz) * 2 * rsz);
    if (!j->req.out_on_device) b += up1k((size_t)j->S * j->nq * 3 * rsz);
    j->footprint = b;
    const int SB = tc_precision(sv->precision) ? 8 : direct_state_block(j->S, fp64);
    j->S_pad = (j->S + SB - 1) / SB * SB;
    const double rows = tc_precision(sv->precision) ? (double)ps.n_krows : (double)ps.n_rows;
    j->cost = rows * j->S * (double)(j->half ? (j->nq + 1) / 2 : j->nq);
    j->scratch_need = up1k((size_t)ps.n_pair * 4 * sizeof(double)) + up1k((size_t)j->S_pad * ps.n_rows * rsz);
}

void finish_job(scff_server_s *sv, SJob *j, int state, scff_status st) {
    j->state = state;
    j->status = st;
    j->t_done = now_ms();
    if (j->registered) {
        cudaHostUnregister(j->req.f_out);
        if (j->req.f2_out) cudaHostUnregister(j->req.f2_out);
        j->registered = false;
    }
    if (state == DONE) ++sv->n_done;
    if (state == FAILED) ++sv->n_failed;
    if (state == CANCELLED) ++sv->n_cancel;
}

// Launches one batch on slot k.  Runs on the server thread without the lock.
scff_status launch_batch(scff_server_s *sv, int k, Batch *B) {
    cudaStream_t st = sv->streams[k];
    scff_ctx *c = sv->ctx;
    uint8_t *arena = static_cast<uint8_t *>(sv->arena_ptr);
    const bool fp64 = sv->precision == SCFF_FP64;
    const bool tc = tc_precision(sv->precision);
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    int *d_err = reinterpret_cast<int *>(arena + B->scratch_off);
    double *geom = reinterpret_cast<double *>(arena + B->scratch_off + 1024);
    size_t geom_max = 0;
    for (SJob *j : B->jobs) geom_max = std::max(geom_max, up1k((size_t)j->req.basis->dev.n_pair * 4 * sizeof(double)));
    void *coef = arena + B->scratch_off + 1024 + geom_max;
    uint8_t *desc_dev = arena + B->scratch_off + B->scratch_bytes - sv->stage_bytes;
    if (cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) return SCFF_ERR_CUDA;
    std::vector<TcJobDev> descs;
    for (SJob *j : B->jobs) {
        const PairSetDev &ps = j->req.basis->dev;
        uint8_t *base = arena + j->off;
        double *qd[3];
        size_t o = 0;
        for (int a = 0; a < 3; ++a) {
            qd[a] = reinterpret_cast<double *>(base + o);
            o += sizeof(double) * j->ax[a].size();
        }
        o = up1k(o);
        for (int a = 0; a < 3; ++a)
            if (cudaMemcpyAsync(qd[a], j->ax[a].data(), sizeof(double) * j->ax[a].size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
                return SCFF_ERR_CUDA;
        uint8_t *work = base + o;
        size_t work_bytes = tc ? up1k(tc_job_bytes(ps, j->S, j->req.nx, j->req.ny, j->req.nz, tc_kind_of(sv->precision)))
                               : up1k((size_t)ps.n_pair * (j->req.nx + j->req.ny + j->req.nz) * 2 * rsz);
        void *fdev = j->req.f_out, *f2dev = j->req.f2_out;
        if (!j->req.out_on_device) {
            fdev = work + work_bytes;
            f2dev = j->req.f2_out ? static_cast<uint8_t *>(fdev) + (size_t)j->S * j->nq * 2 * rsz : nullptr;
        }
        const int SB = tc ? 8 : direct_state_block(j->S, fp64);
        if (launch_pair_geom(ps, geom, st) != cudaSuccess) return SCFF_ERR_CUDA;
        int64_t launches = 1;
        if (launch_pairprep(ps, j->req.trans->d_T, j->S, SB, j->S_pad, fp64 ? (double *)coef : nullptr,
                            fp64 ? nullptr : (float *)coef, &launches, st) != cudaSuccess)
            return SCFF_ERR_CUDA;
        if (tc) {
            TcArgs ta;
            memset(&ta, 0, sizeof(ta));
            ta.ps = &ps;
            ta.coef32 = (const float *)coef;
            ta.SB = SB;
            ta.pair_geom = geom;
            ta.qx = qd[0];
            ta.qy = qd[1];
            ta.qz = qd[2];
            ta.nx = j->req.nx;
            ta.ny = j->req.ny;
            ta.nz = j->req.nz;
            ta.S = j->S;
            ta.scale = j->req.scale;
            ta.f = (float *)fdev;
            ta.f2 = (float *)f2dev;
            ta.kind = tc_kind_of(sv->precision);
            ta.half = j->half;
            {
                const int v = tc_variant_resolve(ta.kind, sv->variant, false);
                ta.pair = tc_prefetch_ok(ta.kind) && (v == 3 || v == 4) ? 1 : 0;
                ta.oct = v == 4 && j->half ? 1 : 0;
            }
            tc_axes_abs_max(j->ax[0].data(), j->req.nx, j->ax[1].data(), j->req.ny, j->ax[2].data(), j->req.nz,
                            ta.qabs);
            TcJobDev jd;
            memset(&jd, 0, sizeof(jd));
            if (tc_prep_job(ta, work, &jd, &launches, st) != cudaSuccess) return SCFF_ERR_CUDA;
            descs.push_back(jd);
        } else {
            DirectArgs a;
            memset(&a, 0, sizeof(a));
            a.ps = &ps;
            a.coef = coef;
            a.nq = j->half ? (j->nq + 1) / 2 : j->nq;
            a.nq_out = j->nq;
            a.S = j->S;
            a.SB = SB;
            a.scale = j->req.scale;
            a.f = fdev;
            a.f2 = f2dev;
            a.err_flag = d_err;
            const size_t stride = (size_t)ps.n_pair * 2 * rsz;
            void *t0 = work, *t1 = work + stride * j->req.nx, *t2 = work + stride * (j->req.nx + j->req.ny);
            if (launch_axis_tables(ps, geom, qd[0], j->req.nx, 0, t0, fp64, st) != cudaSuccess ||
                launch_axis_tables(ps, geom, qd[1], j->req.ny, 1, t1, fp64, st) != cudaSuccess ||
                launch_axis_tables(ps, geom, qd[2], j->req.nz, 2, t2, fp64, st) != cudaSuccess)
                return SCFF_ERR_CUDA;
            a.gx = t0;
            a.gy = t1;
            a.gz = t2;
            a.qax = qd[0];
            a.qay = qd[1];
            a.qaz = qd[2];
            a.nx = j->req.nx;
            a.ny = j->req.ny;
            a.nz = j->req.nz;
            if (launch_direct(a, fp64 ? 1 : 0, 0, &launches, st) != cudaSuccess) return SCFF_ERR_CUDA;
        }
        c->launches += launches;
    }
    if (tc && !descs.empty()) {
        std::vector<int4> items;
        tc_build_items(descs.data(), (int)descs.size(), items);
        const size_t need = up1k(sizeof(TcJobDev) * descs.size()) + sizeof(int4) * items.size();
        if (need > sv->stage_bytes) return SCFF_ERR_ADMISSION;
        uint8_t *hs = static_cast<uint8_t *>(sv->h_stage[k]);
        memcpy(hs, descs.data(), sizeof(TcJobDev) * descs.size());
        memcpy(hs + up1k(sizeof(TcJobDev) * descs.size()), items.data(), sizeof(int4) * items.size());
        if (cudaMemcpyAsync(desc_dev, hs, need, cudaMemcpyHostToDevice, st) != cudaSuccess) return SCFF_ERR_CUDA;
        const int drain = c->drain_every >= 0 ? c->drain_every : 8;
        int64_t launches = 0;
        if (tc_launch_persistent(tc_kind_of(sv->precision),
                                 tc_variant_for(tc_kind_of(sv->precision), sv->variant, descs.data(),
                                                (int)descs.size()),
                                 reinterpret_cast<const TcJobDev *>(desc_dev),
                                 reinterpret_cast<const int4 *>(desc_dev + up1k(sizeof(TcJobDev) * descs.size())),
                                 (int)items.size(), drain, d_err, tc_num_sms(), &launches, st, nullptr,
                                 reinterpret_cast<int *>(arena + B->scratch_off + 256)) != cudaSuccess)
            return SCFF_ERR_CUDA;
        c->launches += launches;
    }
    // outputs to host buffers
    for (SJob *j : B->jobs) {
        if (j->req.out_on_device) continue;
        const PairSetDev &ps = j->req.basis->dev;
        uint8_t *base = arena + j->off;
        size_t o = up1k(sizeof(double) * (j->ax[0].size() + j->ax[1].size() + j->ax[2].size()));
        size_t work_bytes = tc ? up1k(tc_job_bytes(ps, j->S, j->req.nx, j->req.ny, j->req.nz, tc_kind_of(sv->precision)))
                               : up1k((size_t)ps.n_pair * (j->req.nx + j->req.ny + j->req.nz) * 2 * rsz);
        uint8_t *fdev = base + o + work_bytes;
        if (cudaMemcpyAsync(j->req.f_out, fdev, (size_t)j->S * j->nq * 2 * rsz, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return SCFF_ERR_CUDA;
        if (j->req.f2_out &&
            cudaMemcpyAsync(j->req.f2_out, fdev + (size_t)j->S * j->nq * 2 * rsz, (size_t)j->S * j->nq * rsz,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SCFF_ERR_CUDA;
    }
    if (cudaMemcpyAsync(sv->h_err[k], d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SCFF_ERR_CUDA;
    if (cudaEventRecord(B->ev, st) != cudaSuccess) return SCFF_ERR_CUDA;
    return SCFF_OK;
}

void server_loop(scff_server_s *sv) {
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progress = false;
        // 1. retire finished batches
        for (int k = 0; k < sv->slots; ++k) {
            Batch *B = sv->busy[k];
            if (!B) continue;
            if (cudaEventQuery(B->ev) == cudaErrorNotReady) continue;
            const int herr = *sv->h_err[k];
            for (SJob *j : B->jobs) {
                sv->arena.release(j->off, j->footprint);
                finish_job(sv, j, herr ? FAILED : DONE, herr ? SCFF_ERR_TIMEOUT : SCFF_OK);
                --sv->inflight;
            }
            sv->arena.release(B->scratch_off, B->scratch_bytes);
            cudaEventDestroy(B->ev);
            delete B;
            sv->busy[k] = nullptr;
            progress = true;
        }
        if (progress) sv->cv_done.notify_all();
        // 2. admit and launch
        int slot = -1;
        for (int k = 0; k < sv->slots; ++k)
            if (!sv->busy[k]) {
                slot = k;
                break;
            }
        if (slot >= 0 && !sv->pending.empty()) {
            Batch *B = new Batch();
            size_t geom_max = 0, coef_max = 0;
            bool blocked = false;
            for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)B->jobs.size() < sv->max_batch;) {
                SJob *j = *it;
                if (j->state == CANCELLED) {
                    it = sv->pending.erase(it);
                    continue;
                }
                const PairSetDev &jps = j->req.basis->dev;
                const size_t jgeom = up1k((size_t)jps.n_pair * 4 * sizeof(double));
                // the job alone with the batch scratch it needs (the form of sbytes below)
                if (j->footprint + up1k(1024 + jgeom + j->scratch_need + sv->stage_bytes) > sv->arena.size()) {
                    it = sv->pending.erase(it);
                    finish_job(sv, j, FAILED, SCFF_ERR_ADMISSION);
                    progress = true;
                    continue;
                }
                if (blocked) break;
                // Jobs of very different cost go to different batches: every job of a
                // batch completes when the batch's launch ends, so a small job batched
                // with a large one would wait for it.  Skipping for this reason does not
                // count as starving (the first pending job always opens the next batch).
                if (!B->jobs.empty() && sv->cost_ratio > 0 &&
                    (j->cost > sv->cost_ratio * B->jobs[0]->cost || B->jobs[0]->cost > sv->cost_ratio * j->cost)) {
                    ++it;
                    continue;
                }
                // Admitted only if its block and the batch scratch grown to cover it
                // both fit (a trial allocation of the scratch, given back at once), so
                // the scratch allocation after the loop always succeeds: an empty arena
                // always takes the first job, and batches cannot be put back forever.
                const size_t g2 = std::max(geom_max, jgeom), c2 = std::max(coef_max, j->scratch_need);
                size_t off, toff;
                bool fit = sv->arena.alloc(j->footprint, &off);
                if (fit) {
                    if (sv->arena.alloc(up1k(1024 + g2 + c2 + sv->stage_bytes), &toff)) {
                        sv->arena.release(toff, up1k(1024 + g2 + c2 + sv->stage_bytes));
                    } else {
                        sv->arena.release(off, j->footprint);
                        fit = false;
                    }
                }
                if (fit) {
                    j->off = off;
                    j->state = RUNNING;
                    j->t_admit = now_ms();
                    B->jobs.push_back(j);
                    geom_max = g2;
                    coef_max = c2;
                    it = sv->pending.erase(it);
                } else {
                    if (++j->skipped > 8) blocked = true;  // starving: stop admitting jobs behind it
                    ++it;
                }
            }
            size_t soff = 0;
            const size_t sbytes = up1k(1024 + geom_max + coef_max + sv->stage_bytes);
            if (!B->jobs.empty() && !sv->arena.alloc(sbytes, &soff)) {
                // (not reached: admission reserved room for the scratch) put the jobs
                // back (front, in order) and retry after a retirement
                for (auto r = B->jobs.rbegin(); r != B->jobs.rend(); ++r) {
                    sv->arena.release((*r)->off, (*r)->footprint);
                    (*r)->state = PENDING;
                    sv->pending.push_front(*r);
                }
                B->jobs.clear();
            }
            if (!B->jobs.empty()) {
                B->scratch_off = soff;
                B->scratch_bytes = sbytes;
                cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming);
                sv->busy[slot] = B;
                sv->inflight += (int64_t)B->jobs.size();
                sv->max_inflight = std::max(sv->max_inflight, sv->inflight);
                ++sv->n_batches;
                lk.unlock();
                scff_status st = launch_batch(sv, slot, B);
                lk.lock();
                if (st != SCFF_OK) {
                    // the stream may hold partial work: wait for it, then fail the batch
                    cudaStreamSynchronize(sv->streams[slot]);
                    for (SJob *j : B->jobs) {
                        sv->arena.release(j->off, j->footprint);
                        finish_job(sv, j, FAILED, st);
                        --sv->inflight;
                    }
                    sv->arena.release(B->scratch_off, B->scratch_bytes);
                    cudaEventDestroy(B->ev);
                    delete B;
                    sv->busy[slot] = nullptr;
                    sv->cv_done.notify_all();
                }
                progress = true;
            } else {
                delete B;
            }
        }
        const bool any_busy = std::any_of(sv->busy.begin(), sv->busy.end(), [](Batch *b) { return b != nullptr; });
        if (sv->stop && sv->pending.empty() && !any_busy) break;
        if (!progress) {
            if (any_busy)
                sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" scff_status scff_server_create(scff_ctx *c, const scff_server_options *opt, scff_server_h *out) {
    if (!c || !out) return serr(SCFF_ERR_INVALID_ARG, "scff_server_create: NULL context or output");
    *out = nullptr;
    scff_server_options o = opt ? *opt : scff_server_options{SCFF_TF32X3, 2, 64, 0, 0.0};
    if (o.precision < SCFF_FP64 || o.precision > SCFF_FP16X2 || o.slots < 1 || o.slots > 8 || o.max_batch_jobs < 1)
        return serr(SCFF_ERR_INVALID_ARG, "scff_server_create: invalid options");
    cudaSetDevice(c->device);
    scff_server_s *sv = new scff_server_s();
    sv->ctx = c;
    sv->precision = o.precision;
    sv->variant = zstage_mode(c, o.precision);
    sv->slots = o.slots;
    sv->max_batch = o.max_batch_jobs;
    sv->cost_ratio = o.batch_cost_ratio;
    size_t arena = o.arena_bytes ? o.arena_bytes : (size_t)(c->budget / 2);
    if (cudaMalloc(&sv->arena_ptr, arena) != cudaSuccess) {
        delete sv;
        return serr(SCFF_ERR_OOM, "scff_server_create: cannot allocate a %zu-byte arena", arena);
    }
    sv->arena.init(arena);
    for (int k = 0; k < sv->slots; ++k) {
        cudaStream_t s;
        void *hs = nullptr;
        int *he = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&hs, sv->stage_bytes) != cudaSuccess || cudaMallocHost((void **)&he, sizeof(int)) != cudaSuccess) {
            for (auto x : sv->streams) cudaStreamDestroy(x);
            for (auto x : sv->h_stage) cudaFreeHost(x);
            cudaFree(sv->arena_ptr);
            delete sv;
            return serr(SCFF_ERR_OOM, "scff_server_create: stream or pinned staging allocation failed");
        }
        *he = 0;
        sv->streams.push_back(s);
        sv->h_stage.push_back(hs);
        sv->h_err.push_back(he);
        sv->busy.push_back(nullptr);
    }
    // tensor-core kernel attributes are set once, outside the server thread's launches
    if (tc_precision(sv->precision))
        for (int v : {0, 1, 2, 3})
            tc_launch_persistent(tc_kind_of(sv->precision), v, nullptr, nullptr, 0, 0, nullptr, 0, nullptr, 0);
    sv->th = std::thread(server_loop, sv);
    *out = sv;
    return SCFF_OK;
}

extern "C" scff_status scff_submit(scff_server_h sv, const scff_request *r, int64_t *job_id) {
    if (!sv || !r || !job_id) return serr(SCFF_ERR_INVALID_ARG, "scff_submit: NULL argument");
    scff_ctx *c = sv->ctx;
    if (!r->basis || !r->trans || r->trans->basis != r->basis || !r->f_out || r->nx < 1 || r->ny < 1 || r->nz < 1 ||
        !r->qx || !r->qy || !r->qz || !isfinite(r->scale))
        return serr(SCFF_ERR_INVALID_ARG, "scff_submit: invalid request");
    SJob *j = new SJob();
    j->req = *r;
    j->ax[0].assign(r->qx, r->qx + r->nx);
    j->ax[1].assign(r->qy, r->qy + r->ny);
    j->ax[2].assign(r->qz, r->qz + r->nz);
    j->half = (sv->ctx->hermitian && scff_axes_antisym(r->qx, r->nx, r->qy, r->ny, r->qz, r->nz) &&
               (int64_t)r->nx * r->ny * r->nz > 1) ? 1 : 0;
    j->S = r->trans->S;
    j->nq = (int64_t)r->nx * r->ny * r->nz;
    j->t_submit = now_ms();
    size_job(sv, j);
    if (!r->out_on_device) {
        // Pageable host outputs are pinned for the job so that the copies stay asynchronous.
        cudaPointerAttributes at;
        const size_t rsz = sv->precision == SCFF_FP64 ? 8 : 4;
        if (cudaPointerGetAttributes(&at, r->f_out) == cudaSuccess && at.type == cudaMemoryTypeUnregistered) {
            cudaSetDevice(c->device);
            if (cudaHostRegister(r->f_out, (size_t)j->S * j->nq * 2 * rsz, cudaHostRegisterDefault) == cudaSuccess &&
                (!r->f2_out || cudaHostRegister(r->f2_out, (size_t)j->S * j->nq * rsz, cudaHostRegisterDefault) ==
                                   cudaSuccess))
                j->registered = true;
        }
        cudaGetLastError();
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j->id = sv->next_id++;
        sv->jobs[j->id] = j;
        sv->pending.push_back(j);
        ++sv->n_submitted;
        *job_id = j->id;
    }
    sv->cv_work.notify_one();
    return SCFF_OK;
}

extern "C" scff_status scff_wait(scff_server_h sv, int64_t id, int64_t timeout_us) {
    if (!sv) return serr(SCFF_ERR_INVALID_ARG, "scff_wait: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return serr(SCFF_ERR_NOT_FOUND, "scff_wait: unknown job %lld", (long long)id);
    SJob *j = it->second;
    auto done = [&] { return j->state >= DONE; };
    if (timeout_us < 0)
        sv->cv_done.wait(lk, done);
    else if (!sv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return serr(SCFF_ERR_TIMEOUT, "scff_wait: job %lld not finished within %lld us", (long long)id,
                    (long long)timeout_us);
    if (j->state == CANCELLED) return serr(SCFF_ERR_CANCELLED, "scff_wait: job %lld was cancelled", (long long)id);
    if (j->state == FAILED) return serr(j->status, "scff_wait: job %lld failed (status %d)", (long long)id, j->status);
    return SCFF_OK;
}

extern "C" scff_status scff_cancel(scff_server_h sv, int64_t id) {
    if (!sv) return serr(SCFF_ERR_INVALID_ARG, "scff_cancel: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return serr(SCFF_ERR_NOT_FOUND, "scff_cancel: unknown job %lld", (long long)id);
    SJob *j = it->second;
    if (j->state != PENDING) return serr(SCFF_ERR_INVALID_ARG, "scff_cancel: job %lld is no longer pending", (long long)id);
    finish_job(sv, j, CANCELLED, SCFF_ERR_CANCELLED);
    sv->cv_done.notify_all();
    return SCFF_OK;
}

extern "C" scff_status scff_job_times(scff_server_h sv, int64_t id, double *ms) {
    if (!sv || !ms) return serr(SCFF_ERR_INVALID_ARG, "scff_job_times: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return serr(SCFF_ERR_NOT_FOUND, "scff_job_times: unknown job %lld", (long long)id);
    SJob *j = it->second;
    ms[0] = j->t_submit;
    ms[1] = j->t_admit;
    ms[2] = j->t_done;
    return SCFF_OK;
}

extern "C" scff_status scff_server_stats(scff_server_h sv, int64_t *out) {
    if (!sv || !out) return serr(SCFF_ERR_INVALID_ARG, "scff_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out[0] = sv->n_submitted;
    out[1] = sv->n_done;
    out[2] = sv->n_cancel;
    out[3] = sv->n_failed;
    out[4] = sv->n_batches;
    out[5] = sv->max_inflight;
    out[6] = (int64_t)sv->arena.size();
    return SCFF_OK;
}

extern "C" void scff_server_destroy(scff_server_h sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        // pending jobs are cancelled; in-flight batches finish
        for (SJob *j : sv->pending)
            if (j->state == PENDING) finish_job(sv, j, CANCELLED, SCFF_ERR_CANCELLED);
        sv->pending.clear();
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    if (sv->th.joinable()) sv->th.join();
    cudaSetDevice(sv->ctx->device);
    for (auto s : sv->streams) cudaStreamDestroy(s);
    for (auto h : sv->h_stage) cudaFreeHost(h);
    for (auto h : sv->h_err) cudaFreeHost(h);
    cudaFree(sv->arena_ptr);
    for (auto &kv : sv->jobs) delete kv.second;
    delete sv;
}
