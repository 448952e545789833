// Serving loop: continuous batching of foreground-estimation jobs on one GPU, scheduled
// by level pass.
//
// Callers submit jobs (I and alpha, F and B to fill; host or device memory) at any time. A
// scheduler thread admits queued jobs in arrival order while a slot is free and the job's
// device bytes fit in the server's HBM budget and in the device's free memory read at
// that moment. An admitted job gets its device buffers from the server's stream-ordered
// memory pool (no device-wide synchronisation): I and alpha with rows padded to the 16-byte
// grid (host inputs are copied up into them; device inputs on the grid are read in place),
// its two intermediate-level buffers, and F and B. Its pyramid plan (the level passes of
// Algorithm 1 with their tensor maps) is built once, at admission.
//
// Host copies go through one stream per direction in pieces of at most 8 MB, issued by the
// scheduler a few at a time, the job with the fewest bytes left first: a small job's copies
// wait behind at most a few pieces of a large one, never behind its whole transfer.
//
// Each scheduler step takes, in admission order, the next level passes of every admitted
// job whose inputs are on the device and that no running launch holds, up to a budget of
// pixel-sweeps per launch (a single larger pass runs alone), and runs them as one work
// list on an idle compute stream: the coarse levels of the jobs that start, then the
// passes, each job's passes in dependency order. A large job therefore advances level by
// level across launches while the jobs that arrive meanwhile join the next launch on
// another stream; it never holds a stream for its whole solve. When the launch that held
// a job's last pass is done, its outputs are copied back (or, in device memory, complete)
// and the job completes. Buffers and budget are released as jobs complete, and each job's
// submit and completion times are kept for latency statistics. The scheduler thread polls
// its events without sleeping while any work is in flight (one host core), and sleeps on a
// condition variable when idle.
//
// Parameter sets the work list does not run (red-black order, levels without sweeps) are
// served whole jobs per launch through fg_estimate_batch.
#include "fgml.h"
#include "fgml_internal.h"
#include "serve_internal.h"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

thread_local std::string s_err;

fg_status sfail(fg_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s_err = buf;
    return st;
}

int esize(fg_dtype d) { return d == FG_F32 ? 4 : 2; }
long long round16(long long bytes) { return (bytes + 15) & ~15LL; }
bool on_grid(const void *p, long long pitch_bytes) { return ((uintptr_t)p & 15) == 0 && (pitch_bytes & 15) == 0; }

constexpr long long kDefaultStepWork = 16LL << 20;   // pixel-sweeps of level passes per launch
constexpr size_t kWorklistReserve = 2u << 20;        // work-list bytes reserved per compute stream
constexpr size_t kPiece = 8u << 20;                  // bytes of one host copy piece at most
constexpr size_t kPiecesInFlight = 6;                // pieces queued per direction at most

// One piece of a job's copy: a contiguous copy of `bytes`, or (stage > 0) the launch that
// copies rows onto the 16-byte grid. Host copies are always contiguous: a pitched
// (row-by-row) copy from host memory runs at a fraction of the link's bandwidth when rows
// are a few KB (measured: 30 GB/s at 1.2 KB rows, 100 GB/s at 6 KB, 210 GB/s contiguous).
struct Piece {
    void *dst = nullptr;
    const void *src = nullptr;
    size_t bytes = 0;
    cudaMemcpyKind kind = cudaMemcpyHostToDevice;
    int stage = 0;
    fgml::StageJob jobs[2];
    long long rows = 0;
};

void add_pieces(std::vector<Piece> &v, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
    for (size_t o = 0; o < bytes; o += kPiece) {
        Piece p;
        p.dst = static_cast<char *>(dst) + o;
        p.src = static_cast<const char *>(src) + o;
        p.bytes = std::min(kPiece, bytes - o);
        p.kind = kind;
        v.push_back(p);
    }
}

struct Job {
    uint64_t ticket;
    fg_request req;
    size_t bytes;            // device bytes reserved for the job
    size_t level_bytes;      // each of its two intermediate-level buffers
    bool copy_in;            // I and alpha are copied into server buffers
    bool via_raw;            // host rows off the 16-byte grid: copied up packed into dRaw first
    Clock::time_point t_submit, t_done;
    void *dI = nullptr, *dA = nullptr, *dF = nullptr, *dB = nullptr, *dL0 = nullptr, *dL1 = nullptr;
    void *dRaw = nullptr;
    long long pI = 0, pA = 0;             // row pitches of dI and dA (elements)
    fgml::ServePlan *plan = nullptr;
    int next_pass = 0, passes = 0;        // level passes launched so far, and in all
    bool coarse_done = false, in_flight = false;
    std::vector<Piece> pieces;            // the copy under way (inputs up, then outputs down)
    size_t next_piece = 0, left = 0;      // first piece not issued, bytes not issued
    bool inputs_issued = false;           // every input copy issued and inputs_ready recorded
    cudaEvent_t allocated = nullptr;      // its buffers exist (recorded on the pool's stream)
    cudaEvent_t inputs_ready = nullptr;   // the job's inputs are on the device
    cudaEvent_t finished = nullptr;       // its outputs are back in host memory
    int state = 0;           // 0 queued, 1 in progress, 3 done, 4 failed
    fg_status status = FG_OK;
    std::string error;
};

// One launch: the jobs with passes (or coarse levels) in it, and its completion event.
struct Step {
    std::vector<std::shared_ptr<Job>> jobs;
    cudaEvent_t done = nullptr;
    int stream = -1;
};

}  // namespace

struct fg_server {
    fg_server_cfg cfg;
    int device = 0;
    bool levels = true;                  // level-granular launches (else whole jobs)
    std::vector<cudaStream_t> streams;   // compute streams
    cudaStream_t up = nullptr, down = nullptr;   // host copies, one stream per direction
    cudaStream_t mem = nullptr;          // allocations and frees of the pool (nothing else)
    cudaMemPool_t pool = nullptr;
    size_t free_headroom = 0;            // device memory free beyond the reserve, last read
    Clock::time_point free_at{};         // when it was read
    std::vector<bool> busy;
    int *errors = nullptr;               // pinned: the device error words after each stream's launch
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> admitted;    // passes still to launch, admission order
    std::vector<std::shared_ptr<Job>> uploading;   // input copies not all issued
    std::vector<std::shared_ptr<Job>> downloading; // output copies not all issued
    std::vector<std::shared_ptr<Job>> finishing;   // output copies issued, not yet complete
    std::deque<cudaEvent_t> up_pieces, down_pieces;   // issued pieces, oldest first
    std::vector<cudaEvent_t> spare_events;
    std::vector<Step> running;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    size_t used = 0;
    int inflight = 0;
    bool stop = false;
    std::thread worker;
    fg_server_stats stats;
    Clock::time_point t0 = Clock::now();
};

namespace {

// Device bytes a job holds while admitted: copies of I and alpha with padded rows (host
// inputs, or device inputs off the 16-byte grid), its two intermediate-level buffers,
// F and B for host outputs, and slack.
size_t job_bytes(const Job &j) {
    const fg_request &r = j.req;
    const size_t n = (size_t)r.w * r.h, es = esize(r.dtype);
    size_t b = 2 * j.level_bytes + (1u << 20);
    if (j.copy_in) b += (size_t)r.h * (round16(3LL * r.w * es) + round16((long long)r.w * es));
    if (j.via_raw) b += n * es * 4 + 256;
    if (!(r.flags & FG_REQ_DEVICE_OUTPUT)) b += n * es * (3 + 3);
    return b;
}

// Device memory admission keeps free: 2 % of the device, at least 256 MiB.
size_t reserve_bytes(size_t total) { return std::max<size_t>(total / 50, 256ull << 20); }

void fail_job(fg_server *s, Job &j, fg_status st, const std::string &msg) {
    j.status = st;
    j.error = msg;
    j.state = 4;
    j.t_done = Clock::now();
    s->stats.failed += 1;
}

// Returns a job's buffers, events and plan (its device work is complete or was never
// launched) and its share of the budget.
void release(fg_server *s, Job &j) {
    const bool dout = j.req.flags & FG_REQ_DEVICE_OUTPUT;
    cudaStream_t st = s->mem;   // where every buffer was allocated
    if (j.copy_in) {
        if (j.dI) cudaFreeAsync(j.dI, st);
        if (j.dA) cudaFreeAsync(j.dA, st);
    }
    if (!dout) {
        if (j.dF) cudaFreeAsync(j.dF, st);
        if (j.dB) cudaFreeAsync(j.dB, st);
    }
    if (j.dL0) cudaFreeAsync(j.dL0, st);
    if (j.dL1) cudaFreeAsync(j.dL1, st);
    if (j.dRaw) cudaFreeAsync(j.dRaw, st);
    j.dI = j.dA = j.dF = j.dB = j.dL0 = j.dL1 = j.dRaw = nullptr;
    if (j.allocated) cudaEventDestroy(j.allocated);
    if (j.inputs_ready) cudaEventDestroy(j.inputs_ready);
    if (j.finished) cudaEventDestroy(j.finished);
    j.allocated = j.inputs_ready = j.finished = nullptr;
    if (j.plan) fgml::serve_plan_destroy(j.plan);
    j.plan = nullptr;
    s->used -= j.bytes;
    s->inflight -= 1;
}

// Device memory free for new jobs: what the device reports, plus what the server's pool
// holds unused, less the reserve.
bool read_headroom(fg_server *s) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    uint64_t reserved = 0, in_use = 0;
    cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(s->pool, cudaMemPoolAttrUsedMemCurrent, &in_use);
    const size_t avail = free_b + (reserved > in_use ? (size_t)(reserved - in_use) : 0);
    const size_t reserve = reserve_bytes(total_b);
    s->free_headroom = avail > reserve ? avail - reserve : 0;
    return true;
}

cudaError_t alloc(fg_server *s, void **p, size_t bytes, cudaStream_t st) {
    return cudaMallocFromPoolAsync(p, bytes, s->pool, st);
}

// Buffers, input copy pieces and plan of one admitted job; false (and the reason) on
// failure.
bool stage_job(fg_server *s, Job &j, std::string &why) {
    const fg_request &r = j.req;
    const int es = esize(r.dtype);
    const size_t npx = (size_t)r.w * r.h;
    cudaStream_t up = s->mem;   // allocations go on the pool's own stream
    const bool din = r.flags & FG_REQ_DEVICE_INPUT, dout = r.flags & FG_REQ_DEVICE_OUTPUT;
    cudaError_t e = cudaSuccess;
    if (j.copy_in) {
        j.pI = round16(3LL * r.w * es) / es;
        j.pA = round16((long long)r.w * es) / es;
        e = alloc(s, &j.dI, (size_t)j.pI * es * r.h, up);
        if (e == cudaSuccess) e = alloc(s, &j.dA, (size_t)j.pA * es * r.h, up);
        if (e == cudaSuccess && j.via_raw) e = alloc(s, &j.dRaw, npx * es * 4 + 256, up);
    } else {
        j.dI = const_cast<void *>(r.I);
        j.dA = const_cast<void *>(r.alpha);
        j.pI = 3LL * r.w;
        j.pA = r.w;
    }
    if (dout) {
        j.dF = r.F;
        j.dB = r.B;
    } else {
        if (e == cudaSuccess) e = alloc(s, &j.dF, npx * 3 * es, up);
        if (e == cudaSuccess) e = alloc(s, &j.dB, npx * 3 * es, up);
    }
    if (j.level_bytes) {
        if (e == cudaSuccess) e = alloc(s, &j.dL0, j.level_bytes, up);
        if (e == cudaSuccess) e = alloc(s, &j.dL1, j.level_bytes, up);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j.allocated, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j.inputs_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j.finished, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j.allocated, up);
    if (e == cudaSuccess && !j.copy_in) {
        // nothing to copy: the inputs are ready once the buffers are (and the caller's event)
        e = cudaEventRecord(j.inputs_ready, up);
        j.inputs_issued = true;
    }
    if (e != cudaSuccess) {
        why = std::string("admission: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    if (j.copy_in) {
        const size_t bI = npx * 3 * es, bA = npx * es;
        if (din || j.via_raw) {
            // rows onto the 16-byte grid by one launch: from the caller's device buffers, or
            // from the packed copy the host pieces put in dRaw
            const void *sI = din ? r.I : j.dRaw;
            const void *sA = din ? r.alpha : static_cast<char *>(j.dRaw) + ((bI + 255) & ~(size_t)255);
            if (!din) {
                add_pieces(j.pieces, j.dRaw, r.I, bI, cudaMemcpyHostToDevice);
                add_pieces(j.pieces, const_cast<void *>(sA), r.alpha, bA, cudaMemcpyHostToDevice);
            }
            Piece p;
            p.stage = 2;
            p.jobs[0] = fgml::StageJob{sI, j.dI, 3LL * r.w * es, j.pI * es, 3LL * r.w * es, r.h, 0};
            p.jobs[1] = fgml::StageJob{sA, j.dA, (long long)r.w * es, j.pA * es, (long long)r.w * es, r.h, r.h};
            p.rows = 2LL * r.h;
            j.pieces.push_back(p);
        } else {
            // host rows already on the grid: straight into place
            add_pieces(j.pieces, j.dI, r.I, bI, cudaMemcpyHostToDevice);
            add_pieces(j.pieces, j.dA, r.alpha, bA, cudaMemcpyHostToDevice);
        }
        j.left = din ? 0 : bI + bA;
    }
    if (s->levels) {
        if (fgml::serve_plan_create((int)r.dtype, s->cfg.params, j.dI, j.pI, j.dA, j.pA, j.copy_in, r.w,
                                    r.h, j.dF, j.dB, 3LL * r.w, j.dL0, j.dL1, &j.plan) != FG_OK) {
            why = std::string("admission: ") + fg_last_error();
            return false;
        }
        j.passes = fgml::serve_plan_passes(j.plan);
    }
    return true;
}

// Whether the caller's event for device inputs (if any) has fired.
bool caller_ready(const Job &j) {
    if (!(j.req.flags & FG_REQ_DEVICE_INPUT) || !j.req.ready_event) return true;
    const cudaError_t q = cudaEventQuery(static_cast<cudaEvent_t>(j.req.ready_event));
    if (q == cudaErrorNotReady) return false;
    cudaGetLastError();
    return true;
}

cudaEvent_t take_event(fg_server *s) {
    cudaEvent_t ev = nullptr;
    if (!s->spare_events.empty()) {
        ev = s->spare_events.back();
        s->spare_events.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ev = nullptr;
    }
    return ev;
}

// Issues copy pieces on one direction's stream, the job with the fewest bytes left first,
// keeping at most kPiecesInFlight pieces queued. A job whose last input piece is issued
// records inputs_ready; one whose last output piece is issued records `finished` and
// moves to the finishing list.
void pump(fg_server *s, bool upward) {
    std::vector<std::shared_ptr<Job>> &list = upward ? s->uploading : s->downloading;
    std::deque<cudaEvent_t> &queued = upward ? s->up_pieces : s->down_pieces;
    cudaStream_t st = upward ? s->up : s->down;
    while (!queued.empty() && cudaEventQuery(queued.front()) != cudaErrorNotReady) {
        cudaGetLastError();
        s->spare_events.push_back(queued.front());
        queued.pop_front();
    }
    while (queued.size() < kPiecesInFlight) {
        std::shared_ptr<Job> pick;
        for (auto &j : list)
            if ((!pick || j->left < pick->left) && (!upward || caller_ready(*j))) pick = j;
        if (!pick) break;
        Job &j = *pick;
        if (j.next_piece == 0) cudaStreamWaitEvent(st, j.allocated, 0);   // its buffers exist
        const Piece &p = j.pieces[j.next_piece++];
        cudaError_t e;
        if (p.stage) {
            fgml::StageList L;
            std::memset(&L, 0, sizeof L);
            L.local[0] = p.jobs[0];
            L.local[1] = p.jobs[1];
            e = fgml::launch_stage_rows((int)j.req.dtype, L, p.stage, p.rows, st);
        } else {
            e = cudaMemcpyAsync(p.dst, p.src, p.bytes, p.kind, st);
        }
        j.left -= p.bytes;
        if (e != cudaSuccess && j.status == FG_OK) {
            j.status = FG_ERR_CUDA;
            j.error = std::string(upward ? "copy of the inputs: " : "copy of the outputs: ") + cudaGetErrorString(e);
            cudaGetLastError();
        }
        if (cudaEvent_t ev = take_event(s)) {
            cudaEventRecord(ev, st);
            queued.push_back(ev);
        }
        if (j.next_piece == j.pieces.size()) {
            j.pieces.clear();
            j.next_piece = 0;
            if (upward) {
                cudaEventRecord(j.inputs_ready, st);
                j.inputs_issued = true;
            } else {
                cudaEventRecord(j.finished, st);
                s->finishing.push_back(pick);
            }
            list.erase(std::find(list.begin(), list.end(), pick));
        }
    }
}

// Admit queued jobs while a slot, the budget and the device's free memory allow; returns
// how many were admitted.
int admit(fg_server *s) {
    int n = 0;
    if (s->queue.empty()) return 0;
    // the device's free memory, read again at most once a millisecond; what this server
    // admitted since the last read is taken off it
    const Clock::time_point now = Clock::now();
    if (s->free_at == Clock::time_point() || now - s->free_at > std::chrono::milliseconds(1)) {
        if (!read_headroom(s)) return 0;
        s->free_at = now;
    }
    size_t &headroom = s->free_headroom;
    // nothing in flight that could free memory, and the next job does not fit what the
    // device has free: fail it rather than wait for memory other users may never release
    while (!s->queue.empty() && s->inflight == 0 && s->queue.front()->bytes > headroom) {
        std::shared_ptr<Job> j = s->queue.front();
        s->queue.pop_front();
        fail_job(s, *j, FG_ERR_OOM, "job needs " + std::to_string(j->bytes) + " device bytes, " +
                                        std::to_string(headroom) + " are free beyond the reserve");
        s->cv_done.notify_all();
    }
    while (!s->queue.empty() && s->inflight < s->cfg.max_inflight_jobs &&
           s->used + s->queue.front()->bytes <= (size_t)s->cfg.hbm_budget_bytes &&
           s->queue.front()->bytes <= headroom) {
        std::shared_ptr<Job> j = s->queue.front();
        s->queue.pop_front();
        headroom -= j->bytes;
        s->used += j->bytes;
        s->inflight += 1;
        std::string why;
        if (!stage_job(s, *j, why)) {
            release(s, *j);
            fail_job(s, *j, FG_ERR_OOM, why);
            s->cv_done.notify_all();
            continue;
        }
        j->state = 1;
        s->admitted.push_back(j);
        if (!j->pieces.empty()) s->uploading.push_back(j);
        s->stats.max_inflight = std::max<long long>(s->stats.max_inflight, s->inflight);
        s->stats.max_bytes = std::max<long long>(s->stats.max_bytes, (long long)s->used);
        ++n;
    }
    return n;
}

// A job joins a launch once its inputs are on the device, so that no launch (and none of
// the other jobs in it) waits behind an upload.
bool inputs_on_device(Job &j) {
    if (j.coarse_done) return true;
    if (!j.inputs_issued || !caller_ready(j)) return false;
    const cudaError_t q = cudaEventQuery(j.inputs_ready);
    if (q == cudaErrorNotReady) return false;
    cudaGetLastError();   // an upload error surfaces again in the launch
    return true;
}

// One launch on an idle compute stream: the ready passes of the admitted jobs of one dtype
// (level mode), or whole jobs through fg_estimate_batch. Returns whether it launched.
bool launch_step(fg_server *s) {
    int k = -1;
    for (size_t i = 0; i < s->busy.size(); ++i)
        if (!s->busy[i]) {
            k = (int)i;
            break;
        }
    if (k < 0) return false;
    fg_dtype dt = FG_F32;
    bool found = false;
    for (auto &j : s->admitted)
        if (!j->in_flight && j->status == FG_OK && inputs_on_device(*j)) {
            dt = j->req.dtype;
            found = true;
            break;
        }
    if (!found) return false;
    const long long budget = s->cfg.step_work > 0 ? s->cfg.step_work : kDefaultStepWork;
    Step step;
    step.stream = k;
    std::vector<fgml::ServePart> parts;
    std::vector<int> upto;   // pass each job of the step runs to
    long long work = 0;
    for (auto &j : s->admitted) {
        if (j->in_flight || j->req.dtype != dt || j->status != FG_OK || !inputs_on_device(*j)) continue;
        if ((int)step.jobs.size() >= s->cfg.max_batch) break;
        int last = j->next_pass;
        if (s->levels) {
            // passes in order while they fit the budget; the first pass of a launch always
            // goes in, so a pass larger than the budget runs alone
            while (last < j->passes) {
                const long long w = fgml::serve_plan_work(j->plan, last);
                if (work > 0 && work + w > budget) break;
                work += w;
                ++last;
            }
            // nothing of the job fits: it waits for a later launch (a job whose levels are all
            // coarse has nothing but its coarse launch)
            if (last == j->next_pass && (j->coarse_done || j->passes > 0)) continue;
            parts.push_back(fgml::ServePart{j->plan, j->coarse_done ? 0 : 1, j->next_pass, last});
        } else {
            last = j->passes;
        }
        step.jobs.push_back(j);
        upto.push_back(last);
        if (s->levels && work >= budget) break;
    }
    if (step.jobs.empty()) return false;
    cudaStream_t st = s->streams[k];
    // complete already: orders the pool's allocations and the copies up before the launch
    for (auto &j : step.jobs)
        if (!j->coarse_done) cudaStreamWaitEvent(st, j->inputs_ready, 0);
    fg_status status;
    if (s->levels) {
        status = fgml::serve_launch((int)dt, s->cfg.params, parts.data(), (int)parts.size(), st);
    } else {
        const int n = (int)step.jobs.size();
        std::vector<fg_image> I(n), A(n), F(n), B(n);
        for (int i = 0; i < n; ++i) {
            const Job &j = *step.jobs[i];
            const fg_request &r = j.req;
            const long long es = esize(r.dtype);
            I[i] = fg_image{j.dI, r.w, r.h, j.pI * es, r.dtype};
            A[i] = fg_image{j.dA, r.w, r.h, j.pA * es, r.dtype};
            F[i] = fg_image{j.dF, r.w, r.h, 3 * r.w * es, r.dtype};
            B[i] = fg_image{j.dB, r.w, r.h, 3 * r.w * es, r.dtype};
        }
        status = fg_estimate_batch(n, I.data(), A.data(), &s->cfg.params, F.data(), B.data(), st);
    }
    if (status != FG_OK) {
        const std::string err = fg_last_error();
        cudaStreamSynchronize(st);
        for (auto &j : step.jobs) {
            s->admitted.erase(std::find(s->admitted.begin(), s->admitted.end(), j));
            release(s, *j);
            fail_job(s, *j, status, err);
        }
        s->cv_done.notify_all();
        return true;
    }
    // the device error words as the launch leaves them, read back without a synchronisation
    s->errors[2 * k] = s->errors[2 * k + 1] = 0;
    fgml::enqueue_device_error_read(&s->errors[2 * k], st);
    cudaEventCreateWithFlags(&step.done, cudaEventDisableTiming);
    cudaEventRecord(step.done, st);
    for (size_t i = 0; i < step.jobs.size(); ++i) {
        Job &j = *step.jobs[i];
        j.next_pass = upto[i];
        j.coarse_done = true;
        j.in_flight = true;
    }
    s->busy[k] = true;
    s->running.push_back(std::move(step));
    s->stats.batches += 1;
    return true;
}

// Retire finished launches: their jobs are free for the next one, and jobs with every
// pass done move on to their copy back. A launch that failed, or whose bounded device
// waits gave up, fails its jobs.
void retire_steps(fg_server *s) {
    for (size_t i = 0; i < s->running.size();) {
        Step &b = s->running[i];
        const cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        fg_status dev = FG_OK;
        std::string derr;
        int code = 0;
        if (q != cudaSuccess) {
            dev = FG_ERR_CUDA;
            derr = cudaGetErrorString(q);
            cudaGetLastError();
        } else if ((s->errors[2 * b.stream] || s->errors[2 * b.stream + 1]) &&
                   fgml::read_and_clear_device_error(&code, s->streams[b.stream]) == cudaSuccess) {
            // a launch (this one or a concurrent one) set an error word: clear it and fail
            // this launch's jobs
            dev = FG_ERR_TIMEOUT;
            derr = "a bounded device-side wait gave up";
        }
        for (auto &jp : b.jobs) {
            Job &j = *jp;
            j.in_flight = false;
            if (dev != FG_OK && j.status == FG_OK) {
                j.status = dev;
                j.error = derr;
            }
            if (j.status != FG_OK || j.next_pass < j.passes) continue;
            // every pass done: outputs in device memory are complete; host outputs go
            // back in pieces
            s->admitted.erase(std::find(s->admitted.begin(), s->admitted.end(), jp));
            if (j.req.flags & FG_REQ_DEVICE_OUTPUT) {
                s->finishing.push_back(jp);   // `finished` was never recorded: complete
                continue;
            }
            const size_t bytes = (size_t)j.req.w * j.req.h * 3 * esize(j.req.dtype);
            add_pieces(j.pieces, j.req.F, j.dF, bytes, cudaMemcpyDeviceToHost);
            add_pieces(j.pieces, j.req.B, j.dB, bytes, cudaMemcpyDeviceToHost);
            j.left = 2 * bytes;
            s->downloading.push_back(jp);
        }
        cudaEventDestroy(b.done);
        s->busy[b.stream] = false;
        s->running.erase(s->running.begin() + i);
    }
    // jobs that failed (a launch, or a copy up) with passes still to run end here, once
    // nothing queued reads or writes their buffers
    for (size_t i = 0; i < s->admitted.size();) {
        Job &j = *s->admitted[i];
        if (j.status == FG_OK || j.in_flight || !j.inputs_issued ||
            cudaEventQuery(j.inputs_ready) == cudaErrorNotReady) {
            ++i;
            continue;
        }
        release(s, j);
        const fg_status st = j.status;
        const std::string msg = j.error;
        fail_job(s, j, st, msg);
        s->admitted.erase(s->admitted.begin() + i);
        s->cv_done.notify_all();
    }
}

// Complete the jobs whose outputs are in place; returns how many completed.
int retire_jobs(fg_server *s) {
    int n = 0;
    for (size_t i = 0; i < s->finishing.size();) {
        Job &j = *s->finishing[i];
        const cudaError_t q = cudaEventQuery(j.finished);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        if (q != cudaSuccess && j.status == FG_OK) {
            j.status = FG_ERR_CUDA;
            j.error = cudaGetErrorString(q);
            cudaGetLastError();
        }
        release(s, j);
        if (j.status == FG_OK) {
            j.t_done = Clock::now();
            j.state = 3;
            s->stats.completed += 1;
            s->stats.pixels += (long long)j.req.w * j.req.h;
        } else {
            const fg_status st = j.status;
            const std::string msg = j.error;
            fail_job(s, j, st, msg);
        }
        s->finishing.erase(s->finishing.begin() + i);
        ++n;
    }
    return n;
}

void worker_main(fg_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        retire_steps(s);
        pump(s, false);
        if (retire_jobs(s)) s->cv_done.notify_all();
        admit(s);
        pump(s, true);
        while (launch_step(s)) {
        }
        const bool active = !s->running.empty() || !s->finishing.empty() || !s->admitted.empty() ||
                            !s->downloading.empty() || !s->up_pieces.empty() || !s->down_pieces.empty();
        if (s->stop && s->queue.empty() && !active) break;
        if (active) {
            // work in flight: poll its events again at once, letting submitters in
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            // idle: sleep until a submission (or a long poll interval)
            s->cv_work.wait_for(lk, std::chrono::microseconds(2000));
        }
    }
}

double secs(const fg_server *s, Clock::time_point t) {
    return std::chrono::duration<double>(t - s->t0).count();
}

void destroy_streams(fg_server *s) {
    for (cudaStream_t x : s->streams) {
        cudaStreamSynchronize(x);
        fg_release_workspace(x);
        cudaStreamDestroy(x);
    }
    for (cudaStream_t *x : {&s->up, &s->down, &s->mem})
        if (*x) {
            cudaStreamSynchronize(*x);
            cudaStreamDestroy(*x);
            *x = nullptr;
        }
    for (cudaEvent_t ev : s->spare_events) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->up_pieces) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->down_pieces) cudaEventDestroy(ev);
    s->spare_events.clear();
    s->up_pieces.clear();
    s->down_pieces.clear();
    s->streams.clear();
    if (s->pool) cudaMemPoolDestroy(s->pool);
    s->pool = nullptr;
    if (s->errors) cudaFreeHost(s->errors);
    s->errors = nullptr;
}

}  // namespace

extern "C" {

void fg_server_cfg_default(fg_server_cfg *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->max_inflight_jobs = 256;
    c->hbm_budget_bytes = 0;
    c->streams = 2;
    c->max_batch = 64;
    fg_params_default(&c->params);
    c->step_work = kDefaultStepWork;
}

fg_status fg_server_create(const fg_server_cfg *cfg, fg_server **out) {
    s_err.clear();
    if (!out) return sfail(FG_ERR_INVALID_ARG, "out is NULL");
    fg_server_cfg c;
    fg_server_cfg_default(&c);
    if (cfg) c = *cfg;
    if (c.max_inflight_jobs < 1 || c.streams < 1 || c.streams > 16 || c.max_batch < 1)
        return sfail(FG_ERR_INVALID_ARG, "invalid server configuration");
    std::unique_ptr<fg_server> s(new fg_server());
    cudaGetDevice(&s->device);
    if (c.hbm_budget_bytes <= 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            return sfail(FG_ERR_CUDA, "cudaMemGetInfo failed");
        }
        c.hbm_budget_bytes = (long long)(free_b / 2);
    }
    s->cfg = c;
    s->levels = fgml::serve_supported(c.params);
    std::memset(&s->stats, 0, sizeof s->stats);
    // the server's own pool keeps what jobs return (no release to the system between
    // jobs), so admission and completion never wait on the driver's page mapping
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return sfail(FG_ERR_CUDA, "memory pool creation failed");
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    bool ok = cudaMallocHost((void **)&s->errors, 2 * sizeof(int) * c.streams) == cudaSuccess;
    if (ok) std::memset(s->errors, 0, 2 * sizeof(int) * c.streams);
    for (int i = 0; i < c.streams && ok; ++i) {
        cudaStream_t a = nullptr;
        ok = cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking) == cudaSuccess;
        if (a) s->streams.push_back(a);
        s->busy.push_back(false);
        if (ok && s->levels) ok = fgml::serve_reserve(a, kWorklistReserve) == FG_OK;
    }
    ok = ok && cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->down, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->mem, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy_streams(s.get());
        return sfail(FG_ERR_CUDA, "stream or workspace creation failed");
    }
    // the pool takes its memory now (half the budget, at most 32 GiB, returned to the pool
    // at once and kept there), so that jobs do not wait for the driver to map pages when
    // a burst raises the memory in use
    {
        const size_t warm = std::min<size_t>((size_t)c.hbm_budget_bytes / 2, 32ull << 30);
        void *p = nullptr;
        if (warm && cudaMallocFromPoolAsync(&p, warm, s->pool, s->mem) == cudaSuccess) {
            cudaFreeAsync(p, s->mem);
            cudaStreamSynchronize(s->mem);
        }
        cudaGetLastError();
    }
    fg_server *raw = s.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return FG_OK;
}

fg_status fg_server_submit(fg_server *s, const fg_request *r, uint64_t *ticket) {
    s_err.clear();
    if (!s || !r || !ticket) return sfail(FG_ERR_INVALID_ARG, "NULL argument");
    if (!r->I || !r->alpha || !r->F || !r->B) return sfail(FG_ERR_INVALID_ARG, "NULL buffer");
    if (r->w < 1 || r->h < 1 || r->w > 32767 || r->h > 32767)
        return sfail(FG_ERR_INVALID_ARG, "size %dx%d outside [1, 32767]", r->w, r->h);
    if (r->dtype != FG_F32 && r->dtype != FG_BF16 && r->dtype != FG_F16)
        return sfail(FG_ERR_INVALID_ARG, "unknown dtype");
    if (r->flags & ~(FG_REQ_DEVICE_INPUT | FG_REQ_DEVICE_OUTPUT))
        return sfail(FG_ERR_INVALID_ARG, "unknown request flags 0x%x", r->flags);
    const int es = esize(r->dtype);
    if ((r->flags & FG_REQ_DEVICE_INPUT) && ((uintptr_t)r->I % es || (uintptr_t)r->alpha % es))
        return sfail(FG_ERR_INVALID_ARG, "device inputs are misaligned");
    if ((r->flags & FG_REQ_DEVICE_OUTPUT) && ((uintptr_t)r->F % es || (uintptr_t)r->B % es))
        return sfail(FG_ERR_INVALID_ARG, "device outputs are misaligned");
    auto j = std::make_shared<Job>();
    j->req = *r;
    j->level_bytes = s->levels ? fgml::serve_level_bytes(r->w, r->h, (int)r->dtype, s->cfg.params) : 0;
    j->copy_in = !(r->flags & FG_REQ_DEVICE_INPUT) ||
                 !(on_grid(r->I, 3LL * r->w * es) && on_grid(r->alpha, (long long)r->w * es));
    j->via_raw = !(r->flags & FG_REQ_DEVICE_INPUT) && ((long long)r->w * es) % 16 != 0;
    j->bytes = job_bytes(*j);
    if ((long long)j->bytes > s->cfg.hbm_budget_bytes)
        return sfail(FG_ERR_INVALID_ARG, "job needs %zu device bytes, above the budget of %lld",
                     j->bytes, s->cfg.hbm_budget_bytes);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return sfail(FG_ERR_BUSY, "server is shutting down");
        j->ticket = s->next_ticket++;
        j->t_submit = Clock::now();
        s->jobs[j->ticket] = j;
        s->queue.push_back(j);
        s->stats.submitted += 1;
        *ticket = j->ticket;
    }
    s->cv_work.notify_one();
    return FG_OK;
}

fg_status fg_server_poll(fg_server *s, uint64_t ticket, int *done) {
    s_err.clear();
    if (!s || !done) return sfail(FG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(FG_ERR_INVALID_ARG, "unknown ticket");
    const Job &j = *it->second;
    *done = j.state >= 3 ? 1 : 0;
    if (j.state == 4) return sfail(j.status, "%s", j.error.c_str());
    return FG_OK;
}

fg_status fg_server_wait(fg_server *s, uint64_t ticket, int timeout_ms) {
    s_err.clear();
    if (!s) return sfail(FG_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(FG_ERR_INVALID_ARG, "unknown ticket");
    std::shared_ptr<Job> j = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 1LL << 40 : timeout_ms),
                                        [&] { return j->state >= 3; });
    if (!ok) return sfail(FG_ERR_TIMEOUT, "job %llu not done within %d ms",
                          (unsigned long long)ticket, timeout_ms);
    if (j->state == 4) return sfail(j->status, "%s", j->error.c_str());
    return FG_OK;
}

fg_status fg_server_times(fg_server *s, uint64_t ticket, double *submit_s, double *done_s) {
    s_err.clear();
    if (!s || !submit_s || !done_s) return sfail(FG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(FG_ERR_INVALID_ARG, "unknown ticket");
    const Job &j = *it->second;
    if (j.state < 3) return sfail(FG_ERR_BUSY, "job not finished");
    *submit_s = secs(s, j.t_submit);
    *done_s = secs(s, j.t_done);
    return FG_OK;
}

fg_status fg_server_release(fg_server *s, uint64_t ticket) {
    s_err.clear();
    if (!s) return sfail(FG_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return sfail(FG_ERR_INVALID_ARG, "unknown ticket");
    if (it->second->state < 3) return sfail(FG_ERR_BUSY, "job not finished");
    s->jobs.erase(it);
    return FG_OK;
}

fg_status fg_server_get_stats(fg_server *s, fg_server_stats *out) {
    s_err.clear();
    if (!s || !out) return sfail(FG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->budget_bytes = s->cfg.hbm_budget_bytes;
    return FG_OK;
}

void fg_server_destroy(fg_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy_streams(s);
    delete s;
}

const char *fg_server_last_error(void) { return s_err.c_str(); }

}  // extern "C"
