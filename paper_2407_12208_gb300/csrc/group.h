// group.h -- grouped Lloyd runs of small jobs (k_group.cu), used by the C-ABI
// layer and the serving engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace km {

constexpr int GROUP_MAX = 32;        // jobs per launch
constexpr int GROUP_MAX_K = 64;      // centres per job
constexpr int GROUP_MAX_D = 8;       // coordinates per row
constexpr int64_t GROUP_MAX_N = 16384;  // rows per job

struct GroupJob {
    const float* X;         // n x d
    const float* C_init;    // k x d
    float* C_out;           // k x d
    int32_t* labels;        // n
    double* md;             // n doubles of scratch (the rows' distances)
    double* sse;            // max_iter + 1: SSE of every assignment
    int32_t* iters;         // iterations done
    int n, k;
};

struct GroupArgs {
    GroupJob job[GROUP_MAX];
    int max_iter;
    int empty_farthest;
    double tau;
    float gamma32;  // Theorem 4.1's relative bound of the fp32 distances, as the library uses it
};

// One CTA per job, all of dimension d (1..8).
cudaError_t launch_group_lloyd(const GroupArgs& a, int njobs, int d, cudaStream_t st);

}  // namespace km
