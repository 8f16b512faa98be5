// seed.h -- D^2-sampling seeding (k_seed.cu), used by the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace km {

// Chunks of D^2 the pick sums (the size of csum / clast below).
size_t seed_chunk_count(int64_t n);
// The k picks into idx (device) and their rows into C_out (k x d); D2: n
// doubles of scratch; csum / clast: seed_chunk_count(n) doubles / int64 of
// scratch; u_dev: the k draws in [0, 1).
cudaError_t launch_seed_pp(const float* X, int64_t n, int d, int k, const double* u_dev, double* D2, int64_t* idx,
                           double* csum, int64_t* clast, float* C_out, int num_sms, cudaStream_t st, int* nlaunch);

}  // namespace km
