// serve.h -- internal interface of the serving engine (serve.cpp) used by the
// C-ABI layer.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mpkm.h"

struct km_serve;
struct km_tune;  // the owning context's table of screening-kernel variants (api.cu)
struct km_ctx_view {
    int device;
    int num_sms;
    km_tune* tune;
};

km_status serve_create(km_serve** out, int device, int num_sms, km_tune* tune, void* arena, size_t arena_bytes);
void serve_destroy(km_serve* s);
km_status serve_submit(km_serve* s, const km_job* job, uint64_t* job_id, std::string* err);
km_status serve_poll(km_serve* s, uint64_t job_id, km_result* out);
km_status serve_release(km_serve* s, uint64_t job_id);
km_status serve_cancel(km_serve* s, uint64_t job_id);

// Runs one job to completion on `st` (defined in api.cu).  `cancel` is polled
// between Lloyd iterations.
// Whether a job can run inside a grouped launch (km_lloyd_run_batch's limits),
// and the grouped run of such jobs on `st` (waits for it to finish).
bool km_internal_groupable(const km_job& job);
km_status km_internal_run_batch(km_ctx_view* v, const km_batch_job* jobs, int njobs, const km_params* p,
                                cudaStream_t st, std::string* err);
km_status km_internal_run_job(km_ctx_view* v, const float* X, int64_t n, int d, int k, const float* C_init,
                              const km_params* p, int kind, float* C_out, int32_t* labels, void* ws,
                              size_t ws_bytes, cudaStream_t st, double* sse, double* eta, int* iters,
                              std::string* err, const volatile int* cancel);
