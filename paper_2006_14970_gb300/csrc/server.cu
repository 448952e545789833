// Serving loop: continuous batching of foreground-estimation jobs on one GPU.
//
// Callers submit jobs (I and alpha, F and B to fill; host or device memory) at any time. A
// scheduler thread admits queued jobs in arrival order while a slot is free and the job's
// device bytes fit in the server's HBM budget and in the device's free memory read at
// that moment; admitted jobs get device buffers from the stream-ordered allocator (no
// device-wide synchronisation), host inputs are copied up (device inputs read in place),
// and every admitted job not yet launched is merged with the others of its dtype into
// one fg_estimate_batch launch on the next idle compute stream. Jobs that arrive while
// earlier batches run are admitted as soon as slots and memory free up and join the
// next batch, whose work overlaps the running ones on the device. Completion is
// detected with events; results are copied back, buffers and budget released, and the
// job's submit and completion times kept for latency statistics.
#include "fgml.h"
#include "fgml_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
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

struct Job {
    uint64_t ticket;
    fg_request req;
    size_t bytes;            // device bytes reserved for the job
    Clock::time_point t_submit, t_done;
    void *dI = nullptr, *dA = nullptr, *dF = nullptr, *dB = nullptr;
    cudaEvent_t inputs_ready = nullptr;   // the job's inputs are on the device
    int state = 0;           // 0 queued, 1 admitted, 2 launched, 3 done, 4 failed
    fg_status status = FG_OK;
    std::string error;
};

struct Batch {
    std::vector<std::shared_ptr<Job>> jobs;
    cudaEvent_t done = nullptr;
    int stream = -1;
};

}  // namespace

struct fg_server {
    fg_server_cfg cfg;
    int device = 0;
    std::vector<cudaStream_t> streams;
    cudaStream_t up = nullptr;        // uploads of every job, in admission order
    size_t free_headroom = 0;          // device memory free beyond the reserve, last read
    Clock::time_point free_at{};       // when it was read
    std::vector<bool> busy;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> queue;
    std::vector<std::shared_ptr<Job>> admitted;
    std::vector<Batch> running;
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

// Device bytes a job holds while admitted: the copies of host inputs and outputs it
// needs (I and alpha, F and B), its share of the intermediate levels (two buffers of the
// largest intermediate level, a quarter of the image each for the paper's schedule) and
// slack for the work list.
size_t job_bytes(const fg_request &r) {
    const size_t n = (size_t)r.w * r.h, es = esize(r.dtype);
    size_t b = n * es * 3 + (1u << 20);
    if (!(r.flags & FG_REQ_DEVICE_INPUT)) b += n * es * (3 + 1);
    if (!(r.flags & FG_REQ_DEVICE_OUTPUT)) b += n * es * (3 + 3);
    return b;
}

// Device memory admission keeps free: 2 % of the device, at least 256 MiB.
size_t reserve_bytes(size_t total) { return std::max<size_t>(total / 50, 256ull << 20); }

void fail_job(Job &j, fg_status st, const std::string &msg) {
    j.status = st;
    j.error = msg;
    j.state = 4;
    j.t_done = Clock::now();
}

void release(fg_server *s, Job &j, cudaStream_t st) {
    const bool din = j.req.flags & FG_REQ_DEVICE_INPUT, dout = j.req.flags & FG_REQ_DEVICE_OUTPUT;
    if (j.inputs_ready) {
        cudaEventDestroy(j.inputs_ready);
        j.inputs_ready = nullptr;
    }
    if (j.dI && !din) cudaFreeAsync(j.dI, st);
    if (j.dA && !din) cudaFreeAsync(j.dA, st);
    if (j.dF && !dout) cudaFreeAsync(j.dF, st);
    if (j.dB && !dout) cudaFreeAsync(j.dB, st);
    j.dI = j.dA = j.dF = j.dB = nullptr;
    s->used -= j.bytes;
    s->inflight -= 1;
}

// Admit queued jobs while a slot, the budget and the device's free memory allow; returns
// how many were admitted. Free memory is read again for every admission round, so memory
// taken or released by other users of the device counts.
int admit(fg_server *s) {
    int n = 0;
    if (s->queue.empty()) return 0;
    // the device's free memory, read again at most once a millisecond; what this server
    // allocated since the last read is taken off it
    const Clock::time_point now = Clock::now();
    if (s->free_at == Clock::time_point() || now - s->free_at > std::chrono::milliseconds(1)) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const size_t reserve = reserve_bytes(total_b);
        s->free_headroom = free_b > reserve ? free_b - reserve : 0;
        s->free_at = now;
    }
    size_t &headroom = s->free_headroom;   // for new allocations
    // nothing in flight that could free memory, and the next job does not fit what the
    // device has free: fail it rather than wait for memory other users may never release
    while (!s->queue.empty() && s->inflight == 0 && s->queue.front()->bytes > headroom) {
        std::shared_ptr<Job> j = s->queue.front();
        s->queue.pop_front();
        fail_job(*j, FG_ERR_OOM, "job needs " + std::to_string(j->bytes) + " device bytes, " +
                                     std::to_string(headroom) + " are free beyond the reserve");
        s->stats.failed += 1;
        s->cv_done.notify_all();
    }
    while (!s->queue.empty() && s->inflight < s->cfg.max_inflight_jobs &&
           s->used + s->queue.front()->bytes <= (size_t)s->cfg.hbm_budget_bytes &&
           s->queue.front()->bytes <= headroom) {
        std::shared_ptr<Job> j = s->queue.front();
        s->queue.pop_front();
        headroom -= j->bytes;
        cudaStream_t up = s->up;
        const size_t npx = (size_t)j->req.w * j->req.h, es = esize(j->req.dtype);
        const bool din = j->req.flags & FG_REQ_DEVICE_INPUT, dout = j->req.flags & FG_REQ_DEVICE_OUTPUT;
        cudaError_t e = cudaSuccess;
        if (din) {
            j->dI = const_cast<void *>(j->req.I);
            j->dA = const_cast<void *>(j->req.alpha);
        } else {
            e = cudaMallocAsync(&j->dI, npx * 3 * es, up);
            if (e == cudaSuccess) e = cudaMallocAsync(&j->dA, npx * es, up);
        }
        if (dout) {
            j->dF = j->req.F;
            j->dB = j->req.B;
        } else {
            if (e == cudaSuccess) e = cudaMallocAsync(&j->dF, npx * 3 * es, up);
            if (e == cudaSuccess) e = cudaMallocAsync(&j->dB, npx * 3 * es, up);
        }
        if (e == cudaSuccess && !din) e = cudaMemcpyAsync(j->dI, j->req.I, npx * 3 * es, cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess && !din) e = cudaMemcpyAsync(j->dA, j->req.alpha, npx * es, cudaMemcpyHostToDevice, up);
        // device inputs still being written elsewhere: the upload stream (which every
        // batch waits for) waits for the caller's event
        if (e == cudaSuccess && din && j->req.ready_event)
            e = cudaStreamWaitEvent(up, static_cast<cudaEvent_t>(j->req.ready_event), 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->inputs_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(j->inputs_ready, up);
        s->used += j->bytes;
        s->inflight += 1;
        if (e != cudaSuccess) {
            cudaGetLastError();
            release(s, *j, up);
            fail_job(*j, FG_ERR_OOM, std::string("admission: ") + cudaGetErrorString(e));
            s->stats.failed += 1;
            s->cv_done.notify_all();
            continue;
        }
        j->state = 1;
        s->admitted.push_back(j);
        s->stats.max_inflight = std::max<long long>(s->stats.max_inflight, s->inflight);
        s->stats.max_bytes = std::max<long long>(s->stats.max_bytes, (long long)s->used);
        ++n;
    }
    return n;
}

// Launch the admitted jobs of one dtype as one batch on an idle stream.
bool launch_batch(fg_server *s) {
    if (s->admitted.empty()) return false;
    int k = -1;
    for (size_t i = 0; i < s->busy.size(); ++i)
        if (!s->busy[i]) {
            k = (int)i;
            break;
        }
    if (k < 0) return false;
    const fg_dtype dt = s->admitted.front()->req.dtype;
    Batch b;
    b.stream = k;
    std::vector<std::shared_ptr<Job>> rest;
    for (auto &j : s->admitted) {
        if (j->req.dtype == dt && (int)b.jobs.size() < s->cfg.max_batch)
            b.jobs.push_back(j);
        else
            rest.push_back(j);
    }
    s->admitted.swap(rest);
    cudaStream_t st = s->streams[k];
    // the batch runs once its own jobs' inputs are on the device
    for (auto &j : b.jobs) cudaStreamWaitEvent(st, j->inputs_ready, 0);
    const int n = (int)b.jobs.size();
    std::vector<fg_image> I(n), A(n), F(n), B(n);
    for (int i = 0; i < n; ++i) {
        const fg_request &r = b.jobs[i]->req;
        const long long es = esize(r.dtype);
        I[i] = fg_image{b.jobs[i]->dI, r.w, r.h, 3 * r.w * es, r.dtype};
        A[i] = fg_image{b.jobs[i]->dA, r.w, r.h, r.w * es, r.dtype};
        F[i] = fg_image{b.jobs[i]->dF, r.w, r.h, 3 * r.w * es, r.dtype};
        B[i] = fg_image{b.jobs[i]->dB, r.w, r.h, 3 * r.w * es, r.dtype};
    }
    fg_status status = fg_estimate_batch(n, I.data(), A.data(), &s->cfg.params, F.data(), B.data(), st);
    const std::string err = status == FG_OK ? std::string() : std::string(fg_last_error());
    for (int i = 0; i < n; ++i) {
        Job &j = *b.jobs[i];
        const size_t npx = (size_t)j.req.w * j.req.h, es = esize(j.req.dtype);
        if (status == FG_OK) {
            if (!(j.req.flags & FG_REQ_DEVICE_OUTPUT)) {
                cudaMemcpyAsync(j.req.F, j.dF, npx * 3 * es, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(j.req.B, j.dB, npx * 3 * es, cudaMemcpyDeviceToHost, st);
            }
            j.state = 2;
        } else {
            j.status = status;
            j.error = err;
        }
    }
    cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    cudaEventRecord(b.done, st);
    s->busy[k] = true;
    s->running.push_back(std::move(b));
    s->stats.batches += 1;
    return true;
}

// Retire finished batches; returns how many jobs completed.
int retire(fg_server *s) {
    int n = 0;
    for (size_t i = 0; i < s->running.size();) {
        Batch &b = s->running[i];
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
        } else if (fgml::read_and_clear_device_error(&code, s->streams[b.stream]) == cudaSuccess && code) {
            dev = FG_ERR_TIMEOUT;
            derr = "a bounded device-side wait gave up";
        }
        const Clock::time_point now = Clock::now();
        for (auto &jp : b.jobs) {
            Job &j = *jp;
            release(s, j, s->streams[b.stream]);
            j.t_done = now;
            if (j.status == FG_OK && dev != FG_OK) {
                j.status = dev;
                j.error = derr;
            }
            j.state = j.status == FG_OK ? 3 : 4;
            if (j.status == FG_OK) {
                s->stats.completed += 1;
                s->stats.pixels += (long long)j.req.w * j.req.h;
            } else {
                s->stats.failed += 1;
            }
            ++n;
        }
        cudaEventDestroy(b.done);
        s->busy[b.stream] = false;
        s->running.erase(s->running.begin() + i);
    }
    return n;
}

void worker_main(fg_server *s) {
    cudaSetDevice(s->device);
    cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        const int done = retire(s);
        if (done) s->cv_done.notify_all();
        admit(s);
        while (launch_batch(s)) {
        }
        if (s->stop && s->queue.empty() && s->admitted.empty() && s->running.empty()) break;
        // nothing to launch: sleep until a submission or a short poll interval passes
        s->cv_work.wait_for(lk, std::chrono::microseconds(s->running.empty() ? 2000 : 20));
    }
    lk.unlock();
    cudaStreamSynchronize(s->up);
    cudaStreamDestroy(s->up);
}

double secs(const fg_server *s, Clock::time_point t) {
    return std::chrono::duration<double>(t - s->t0).count();
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
    std::memset(&s->stats, 0, sizeof s->stats);
    for (int i = 0; i < c.streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            return sfail(FG_ERR_CUDA, "stream creation failed");
        }
        s->streams.push_back(st);
        s->busy.push_back(false);
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
    if ((r->flags & FG_REQ_DEVICE_INPUT) && ((uintptr_t)r->I % esize(r->dtype) || (uintptr_t)r->alpha % esize(r->dtype)))
        return sfail(FG_ERR_INVALID_ARG, "device inputs are misaligned");
    auto j = std::make_shared<Job>();
    j->req = *r;
    j->bytes = job_bytes(*r);
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
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        fg_release_workspace(st);
        cudaStreamDestroy(st);
    }
    delete s;
}

const char *fg_server_last_error(void) { return s_err.c_str(); }

}  // extern "C"
