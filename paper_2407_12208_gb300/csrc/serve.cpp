// serve.cpp -- serving engine: continuous batching of k-means jobs on one GPU.
//
// Jobs (Lloyd runs or single nearest-centre assignments of uneven n, d, k)
// are queued at km_submit.  A job is admitted as soon as (a) its memory --
// data, centres, labels and its workspace -- fits in the caller's arena
// (first-fit allocator, 256-byte blocks) and (b) one of the worker streams is
// free (16 by default); queued jobs are scanned in arrival order on every
// change, so a small job can start while a large one waits for memory.  Each
// worker thread drives its jobs on its own CUDA stream, so the kernels of
// concurrently admitted jobs overlap on the device (launched directly: a
// graph recorded here would make a device-wide synchronisation in the
// caller's threads fail while it is being recorded).  Jobs whose data is
// resident on the device (KM_JOB_DEVICE_DATA) are read in place.  Results
// stay resident in the arena until km_release.  Every device wait inside the
// kernels is bounded; a job whose kernels time out finishes with KM_ETIMEOUT
// instead of hanging.
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "serve.h"

size_t km_internal_ws_bytes(int64_t n, int d, int k, const km_params* p);

namespace {

using Clock = std::chrono::steady_clock;

enum class JobState { Queued, Running, Done, Failed, Cancelled };

struct Job {
    uint64_t id = 0;
    km_job spec{};
    std::vector<float> X, C;
    size_t bytes = 0, off = 0;
    bool has_mem = false;
    JobState state = JobState::Queued;
    volatile int cancel = 0;
    km_status status = KM_OK;
    std::string err;
    double sse = 0, eta = 0;
    int iters = 0;
    Clock::time_point t_submit, t_admit, t_done;
    float* dX = nullptr;
    float* dC0 = nullptr;
    float* dC = nullptr;
    int32_t* dlab = nullptr;
    void* dws = nullptr;
    size_t ws_bytes = 0;
};

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct km_serve {
    int device = 0, num_sms = 148;
    km_tune* tune = nullptr;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    size_t arena_usable = 0;  // the aligned part of the arena: no job larger than this ever fits
    std::mutex mu;
    std::condition_variable cv;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    std::deque<Job*> pending;
    std::deque<Job*> ready;
    std::unordered_map<uint64_t, Job*> jobs;
    std::vector<std::thread> workers;
    int n_workers = 16;
    int busy = 0;
    bool stop = false;
    uint64_t next_id = 1;

    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t o = it->first;
                free_blocks.erase(it);
                if (rest) free_blocks[o + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release_mem(size_t off, size_t bytes) {
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
    // Caller holds mu.  Admits queued jobs in arrival order while workers are free.
    void try_admit() {
        for (auto it = pending.begin(); it != pending.end() && busy + (int)ready.size() < n_workers;) {
            Job* j = *it;
            size_t off = 0;
            if (alloc(j->bytes, &off)) {
                j->off = off;
                j->has_mem = true;
                j->t_admit = Clock::now();
                it = pending.erase(it);
                ready.push_back(j);
                cv.notify_all();
            } else {
                ++it;
            }
        }
    }
    void worker_loop();
};

void km_serve::worker_loop() {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    km_ctx_view view{device, num_sms, tune};
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !ready.empty(); });
            if (stop && ready.empty()) break;
            j = ready.front();
            ready.pop_front();
            busy++;
            j->state = JobState::Running;
        }
        const km_job& s = j->spec;
        char* base = arena + j->off;
        size_t o = 0;
        auto take = [&](size_t b) { char* p = base + o; o = up256(o + b); return p; };
        const bool resident = (s.flags & KM_JOB_DEVICE_DATA) != 0;
        j->dX = resident ? const_cast<float*>(s.X) : (float*)take(sizeof(float) * (size_t)s.n * s.d);
        j->dC0 = (float*)take(sizeof(float) * (size_t)s.k * s.d);
        j->dC = (float*)take(sizeof(float) * (size_t)s.k * s.d);
        j->dlab = (int32_t*)take(sizeof(int32_t) * (size_t)s.n);
        j->ws_bytes = j->bytes - o;
        j->dws = take(0);
        km_status rc = KM_OK;
        std::string err;
        cudaError_t ce = cudaSuccess;
        if (!j->cancel) {
            if (resident) {
                ce = cudaMemcpyAsync(j->dC0, s.C_init, sizeof(float) * (size_t)s.k * s.d, cudaMemcpyDeviceToDevice, st);
            } else {
                ce = cudaMemcpyAsync(j->dX, j->X.data(), sizeof(float) * j->X.size(), cudaMemcpyHostToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(j->dC0, j->C.data(), sizeof(float) * j->C.size(), cudaMemcpyHostToDevice, st);
            }
        }
        if (j->cancel) {
            rc = KM_ECANCELLED;
        } else if (ce != cudaSuccess) {
            rc = KM_ECUDA;
            err = "copy into the arena failed";
        } else {
            rc = km_internal_run_job(&view, j->dX, s.n, s.d, s.k, j->dC0, &s.p, s.kind, j->dC, j->dlab, j->dws,
                                     j->ws_bytes, st, &j->sse, &j->eta, &j->iters, &err, &j->cancel);
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            j->status = rc;
            j->err = err;
            j->t_done = Clock::now();
            j->state = rc == KM_OK ? JobState::Done : (rc == KM_ECANCELLED ? JobState::Cancelled : JobState::Failed);
            std::vector<float>().swap(j->X);
            std::vector<float>().swap(j->C);
            busy--;
            if (j->state != JobState::Done && j->has_mem) {  // failed jobs hold no results
                release_mem(j->off, j->bytes);
                j->has_mem = false;
            }
            try_admit();
        }
    }
    cudaStreamDestroy(st);
}

km_status serve_create(km_serve** out, int device, int num_sms, km_tune* tune, void* arena, size_t arena_bytes) {
    km_serve* s = new km_serve();
    s->device = device;
    s->num_sms = num_sms;
    s->tune = tune;
    s->arena = (char*)arena;
    s->arena_bytes = arena_bytes;
    const uintptr_t a0 = (uintptr_t)arena, a1 = up256(a0);
    if (arena_bytes <= (a1 - a0) + 256) { delete s; return KM_EINVAL; }
    s->free_blocks[a1 - a0] = (arena_bytes - (a1 - a0)) & ~(size_t)255;
    s->arena_usable = (arena_bytes - (a1 - a0)) & ~(size_t)255;
    if (const char* e = std::getenv("MPKM_SERVE_WORKERS")) {
        int v = std::atoi(e);
        if (v >= 1 && v <= 64) s->n_workers = v;
    }
    for (int i = 0; i < s->n_workers; i++) s->workers.emplace_back([s] { s->worker_loop(); });
    *out = s;
    return KM_OK;
}

void serve_destroy(km_serve* s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Job* j : s->pending) j->cancel = 1;
        for (Job* j : s->ready) j->cancel = 1;
        for (auto& kv : s->jobs) kv.second->cancel = 1;
        s->cv.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
}

km_status serve_submit(km_serve* s, const km_job* job, uint64_t* job_id, std::string* err) {
    const bool resident = (job->flags & KM_JOB_DEVICE_DATA) != 0;
    const size_t data = (resident ? 0 : up256(sizeof(float) * (size_t)job->n * job->d)) +
                        2 * up256(sizeof(float) * (size_t)job->k * job->d) + up256(sizeof(int32_t) * (size_t)job->n);
    const size_t ws = km_internal_ws_bytes(job->n, job->d, job->k, &job->p);
    const size_t bytes = up256(data + ws);
    // a job larger than the whole arena can never be admitted (checked before
    // the host arrays are copied)
    if (bytes > s->arena_usable) {
        if (err) *err = "job needs more memory than the arena holds";
        return KM_ENOMEM;
    }
    Job* j = new Job();
    j->spec = *job;
    j->bytes = bytes;
    if (!resident) {
        j->X.assign(job->X, job->X + (size_t)job->n * job->d);
        j->C.assign(job->C_init, job->C_init + (size_t)job->k * job->d);
    }
    j->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    j->id = s->next_id++;
    s->jobs[j->id] = j;
    s->pending.push_back(j);
    s->try_admit();
    *job_id = j->id;
    return KM_OK;
}

km_status serve_poll(km_serve* s, uint64_t job_id, km_result* out) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return KM_EINVAL;
    Job* j = it->second;
    if (j->state == JobState::Queued || j->state == JobState::Running) return KM_ENOTREADY;
    std::memset(out, 0, sizeof *out);
    out->status = j->status;
    out->message = j->err.c_str();
    out->iters = j->iters;
    out->sse = j->sse;
    out->eta = j->eta;
    out->latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    out->queue_ms = j->has_mem || j->state == JobState::Done
                        ? std::chrono::duration<double, std::milli>(j->t_admit - j->t_submit).count()
                        : out->latency_ms;
    if (j->state == JobState::Done) {
        out->C = j->dC;
        out->labels = j->dlab;
        return KM_OK;
    }
    return j->state == JobState::Cancelled ? KM_ECANCELLED : j->status;
}

km_status serve_release(km_serve* s, uint64_t job_id) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return KM_EINVAL;
    Job* j = it->second;
    if (j->state == JobState::Queued || j->state == JobState::Running) return KM_ENOTREADY;
    if (j->has_mem) s->release_mem(j->off, j->bytes);
    s->jobs.erase(it);
    delete j;
    s->try_admit();
    return KM_OK;
}

km_status serve_cancel(km_serve* s, uint64_t job_id) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return KM_EINVAL;
    Job* j = it->second;
    j->cancel = 1;
    if (j->state == JobState::Queued) {
        for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
            if (*p == j) { s->pending.erase(p); break; }
        j->state = JobState::Cancelled;
        j->status = KM_ECANCELLED;
        j->t_done = Clock::now();
    }
    return KM_OK;
}
