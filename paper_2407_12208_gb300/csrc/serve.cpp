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

#include "group.h"
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
    int busy = 0;         // workers running a job or a group of jobs
    int ready_group = 0;  // ready jobs that can run grouped
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
    // Caller holds mu.  Admits queued jobs in arrival order while workers are
    // free; small jobs that run grouped (up to GROUP_MAX per launch) take a
    // worker per group, so more of them may wait ready.
    bool has_room(bool group_next) const {
        const int rg = ready_group + (group_next ? 1 : 0);
        const int rn = (int)ready.size() - ready_group + (group_next ? 0 : 1);
        return busy + rn + (rg + km::GROUP_MAX - 1) / km::GROUP_MAX <= n_workers;
    }
    void try_admit() {
        for (auto it = pending.begin(); it != pending.end();) {
            Job* j = *it;
            const bool g = km_internal_groupable(j->spec);
            if (!has_room(g)) break;
            size_t off = 0;
            if (alloc(j->bytes, &off)) {
                j->off = off;
                j->has_mem = true;
                j->t_admit = Clock::now();
                it = pending.erase(it);
                ready.push_back(j);
                ready_group += g ? 1 : 0;
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
        // one job, or a group of small jobs with the same loop parameters
        std::vector<Job*> group;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [&] { return stop || !ready.empty(); });
            if (stop && ready.empty()) break;
            Job* j = ready.front();
            ready.pop_front();
            group.push_back(j);
            if (km_internal_groupable(j->spec)) {
                ready_group--;
                const km_params& p0 = j->spec.p;
                for (auto it = ready.begin(); it != ready.end() && (int)group.size() < km::GROUP_MAX;) {
                    const km_job& o = (*it)->spec;
                    if (km_internal_groupable(o) && o.p.max_iter == p0.max_iter && o.p.empty == p0.empty &&
                        o.p.tau == p0.tau) {
                        group.push_back(*it);
                        it = ready.erase(it);
                        ready_group--;
                    } else {
                        ++it;
                    }
                }
            }
            busy++;
            for (Job* g : group) g->state = JobState::Running;
        }
        // each job's place in the arena and its inputs
        std::vector<km_status> rc(group.size(), KM_OK);
        std::vector<std::string> err(group.size());
        for (size_t q = 0; q < group.size(); q++) {
            Job* j = group[q];
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
            cudaError_t ce = cudaSuccess;
            if (j->cancel) {
                rc[q] = KM_ECANCELLED;
                continue;
            }
            if (resident) {
                ce = cudaMemcpyAsync(j->dC0, s.C_init, sizeof(float) * (size_t)s.k * s.d, cudaMemcpyDeviceToDevice, st);
            } else {
                ce = cudaMemcpyAsync(j->dX, j->X.data(), sizeof(float) * j->X.size(), cudaMemcpyHostToDevice, st);
                if (ce == cudaSuccess)
                    ce = cudaMemcpyAsync(j->dC0, j->C.data(), sizeof(float) * j->C.size(), cudaMemcpyHostToDevice, st);
            }
            if (ce != cudaSuccess) {
                rc[q] = KM_ECUDA;
                err[q] = "copy into the arena failed";
            }
        }
        if (group.size() == 1 && !km_internal_groupable(group[0]->spec)) {
            Job* j = group[0];
            const km_job& s = j->spec;
            if (rc[0] == KM_OK)
                rc[0] = km_internal_run_job(&view, j->dX, s.n, s.d, s.k, j->dC0, &s.p, s.kind, j->dC, j->dlab, j->dws,
                                            j->ws_bytes, st, &j->sse, &j->eta, &j->iters, &err[0], &j->cancel);
        } else {
            // grouped: one launch for the jobs still to run; their scratch, SSE
            // trajectory and iteration count sit in each job's workspace
            std::vector<km_batch_job> bj;
            std::vector<size_t> which;
            std::vector<double> sse_last(group.size(), 0.0);
            for (size_t q = 0; q < group.size(); q++) {
                if (rc[q] != KM_OK) continue;
                Job* j = group[q];
                const km_job& s = j->spec;
                char* w = (char*)j->dws;
                const size_t need = up256(sizeof(double) * (size_t)s.n) + up256(sizeof(double) * (size_t)(s.p.max_iter + 1)) + 256;
                if (need > j->ws_bytes) {
                    rc[q] = KM_ENOMEM;
                    err[q] = "workspace too small for the grouped run";
                    continue;
                }
                km_batch_job b{};
                b.X = j->dX; b.n = s.n; b.d = s.d; b.k = s.k; b.C_init = j->dC0; b.C_out = j->dC; b.labels = j->dlab;
                b.scratch = (double*)w;
                b.sse_per_iter = (double*)(w + up256(sizeof(double) * (size_t)s.n));
                b.iters = (int32_t*)(w + up256(sizeof(double) * (size_t)s.n) + up256(sizeof(double) * (size_t)(s.p.max_iter + 1)));
                bj.push_back(b);
                which.push_back(q);
            }
            if (!bj.empty()) {
                std::string e;
                const km_status r = km_internal_run_batch(&view, bj.data(), (int)bj.size(), &group[which[0]]->spec.p, st, &e);
                // each job's trajectory and iteration count back on the worker's stream
                const int T = group[which[0]]->spec.p.max_iter + 1;
                std::vector<double> sse((size_t)T * which.size());
                std::vector<int32_t> its(which.size());
                cudaError_t ce = cudaSuccess;
                for (size_t m = 0; m < which.size() && r == KM_OK && ce == cudaSuccess; m++) {
                    ce = cudaMemcpyAsync(sse.data() + (size_t)T * m, bj[m].sse_per_iter, sizeof(double) * T,
                                         cudaMemcpyDeviceToHost, st);
                    if (ce == cudaSuccess)
                        ce = cudaMemcpyAsync(&its[m], bj[m].iters, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
                }
                if (r == KM_OK && ce == cudaSuccess) ce = cudaStreamSynchronize(st);
                for (size_t m = 0; m < which.size(); m++) {
                    Job* j = group[which[m]];
                    if (r != KM_OK || ce != cudaSuccess) {
                        rc[which[m]] = r != KM_OK ? r : KM_ECUDA;
                        err[which[m]] = r != KM_OK ? e : std::string(cudaGetErrorString(ce));
                        continue;
                    }
                    j->iters = its[m];
                    j->sse = sse[(size_t)T * m + (size_t)its[m]];
                    j->eta = 0.0;  // the FP32 direct path flags no pair
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            const Clock::time_point now = Clock::now();
            for (size_t q = 0; q < group.size(); q++) {
                Job* j = group[q];
                j->status = rc[q];
                j->err = err[q];
                j->t_done = now;
                j->state = rc[q] == KM_OK ? JobState::Done
                                          : (rc[q] == KM_ECANCELLED ? JobState::Cancelled : JobState::Failed);
                std::vector<float>().swap(j->X);
                std::vector<float>().swap(j->C);
                if (j->state != JobState::Done && j->has_mem) {  // failed jobs hold no results
                    release_mem(j->off, j->bytes);
                    j->has_mem = false;
                }
            }
            busy--;
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
