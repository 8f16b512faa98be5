// internal.h -- declarations shared between the C-ABI layer and the kernel
// translation units of libmpkm.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace km {

// Epilogue groups of the screening kernel (four warps each; tile t goes to
// group t mod TC_GROUPS) and candidate-list entries per row and group (48 per
// row in all).
constexpr int TC_GROUPS = 3;
constexpr int TC_LIST = 48 / TC_GROUPS;
// Candidate pairs reserved per row in the workspace; rows past the capacity
// are recomputed by the full-row kernel.
constexpr int TC_PAIRS_PER_ROW = 8;

// Per-call device counters (lives in the workspace, zeroed per call).
struct DevCounters {
    unsigned long long pairs;
    unsigned long long flagged;
    unsigned long long fp32_evals;
    unsigned long long fp64_evals;
    unsigned long long amb_rows;
    unsigned long long ovf_rows;
    unsigned status;     // KM_DEVERR_* bits
    int amb_count;       // length of the ambiguous-row list
    int ovf_count;       // length of the overflow-row list
    int pad;
    unsigned long long npairs;  // candidate pairs written by the screening kernel
};

// Column-side constants of the reliability bound: maxima over centres.
struct ColMax {
    float nc;    // max ||c_j||
    float nrc;   // max ||c~_j - c_j||
    float ncq;   // max ||c~_j||
    float q;     // max ||c_j||^2
    float ncq2;  // max ||c~_j||^2
    float pad[3];
    // minima of the same statistics: a lower bound of every pair's threshold
    float nc_min, nrc_min, ncq_min, q_min, ncq2_min;
    float pad2[3];
};

// Parameters of the reliability test / candidate window, host-computed.
struct TestParams {
    int test;        // 0 tc, 1 paper, 2 off
    float rho;
    float kacc;      // accumulation coefficient of B (2 gamma_d(u_acc) + 4 u32)
    float kn;        // norm/rounding coefficient of B
    float paper_coef;  // rho * c_A * gamma^l_{d+2} (paper test)
    float bsafe;     // relative safety factor applied to B evaluated in fp32
    float gamma32;   // gamma_{d+2}(2^-24) with safety, for fp32 direct certification
};

// Lets `func` take all the dynamic shared memory a block can have (the
// per-block maximum less the kernel's static shared memory).  Every call sets
// the same value: jobs of different shapes launched from several host threads
// (the serving workers) cannot lower the limit under one another's launches;
// the launch itself states the bytes it uses.
constexpr int kMaxBlockSmem = 227 * 1024;
template <typename F>
inline cudaError_t allow_max_smem(F* func) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(func));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reinterpret_cast<const void*>(func), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxBlockSmem - (int)fa.sharedSizeBytes);
}

// ---- kernels (launch wrappers; all asynchronous on `st`) -----------------
// quantise rows of A (m x d fp32) to fmt (0 fp16, 1 bf16, 2 e4m3) with row
// stride ldq elements; stat[i] = (||a||^2 fp32, ||a||, ||a~||, ||a~ - a||);
// rscale[i] = the row's power-of-two scale (e4m3; fp16/bf16 write 1).
// absmax_out (nullable): max |a| over A folded in with atomicMax on its bits
// (the caller zeroes it first).
cudaError_t launch_quantize(const float* A, int64_t m, int d, int fmt, int ldq, void* Aq, float4* stat,
                            float* rscale, cudaStream_t st, unsigned* absmax_out = nullptr);
// column maxima of the centre statistics, q_j padded with +inf to kpad
// entries and the centres' scales (cscale, nullable: all 1) padded with 1
cudaError_t launch_colmax(const float4* cstat, int k, const float* cscale, ColMax* out, float* qpad, float* spad,
                          int kpad, cudaStream_t st);

// candidates per sampled row under the format's certification window (the
// choice of the low format): acc[0] += candidates, acc[1] += rows above one
// list's capacity; nsample rows at a stride of n / nsample
cudaError_t launch_predict_candidates(const float* X, int64_t n, int d, const float* C, int k, int fmt,
                                      const ColMax* cmx, const TestParams& tp, int nsample,
                                      unsigned long long* acc, int num_sms, cudaStream_t st);

// direct-formula assignment (thread per row).  acc64: binary64 accumulation
// (the plain FP64 path) else fp32 with certification; rows = all n, or the
// device list row_list[0 .. *row_count).  Uncertified fp32 rows are appended
// to amb_list / cnt->amb_count.
// absmax_out (nullable, zeroed by the caller): max |x| over the rows read.
cudaError_t launch_direct_assign(bool acc64, const float* X, int64_t n, const float* C, int k, int d,
                                 const int32_t* row_list, const int* row_count, int32_t* labels,
                                 double* min_dist, int32_t* amb_list, DevCounters* cnt, float gamma32,
                                 int num_sms, cudaStream_t st, unsigned* absmax_out = nullptr);
// exact argmin of the rows of a device list, one block per row: fp32 direct
// values of all centres, certified, binary64 where still open (fp32_first),
// or binary64 for all centres.
cudaError_t launch_rows_full(bool fp32_first, const float* X, const float* C, int k, int d, const int32_t* row_list,
                             const int* row_count, int32_t* labels, double* min_dist, DevCounters* cnt,
                             float gamma32, int num_sms, cudaStream_t st);

// tensor-core screening kernel (tcgen05).  mode 0: candidates; mode 1: distance matrix.
// Epilogue variants of mode 0 when K fits two 128-byte atoms (they give the same
// results; which is fastest depends on the shape): 64-column steps with all 16
// quads staged (FULL) or 8 at a time (HALF, which leaves shared memory for a
// second A stage), or 32-column steps (C32).  Wider K: REG only.
constexpr int TC_SV_FULL = 0, TC_SV_HALF = 1, TC_SV_C32 = 2, TC_SV_REG = 3;
struct TcArgs {
    int64_t n;
    int k, d, fmt, kchunks;   // kchunks = number of 128-byte K atoms
    const float4* xstat;
    const float* xscale;
    const float4* cstat;
    const float* qpad;        // q_j = ||c_j||^2 for j < k, +inf up to the padded tile width
    const float* spad;        // the centres' E4M3 scales s_j for j < k, 1 up to the padded tile width
    const ColMax* colmax;
    TestParams tp;
    int mode;
    int variant;              // mode 0 epilogue variant TC_SV_FULL / HALF / C32
    uint32_t* cand;           // mode 0: TC_GROUPS x TC_LIST x n quad entries (group, slot, row), common.cuh
    int ebits;                // low bits of an entry holding the quad index and mask: ceil(log2 ceil(k / 4)) + 4
    int4* rowinfo;            // n x TC_GROUPS: (count, overflow, window W bits, d^min bits) per epilogue group
    int2* pairs;              // refinement: candidate pairs (row, j), each row's pairs contiguous
    int64_t pair_cap;         // capacity of pairs / v32
    float* v32;               // fp32 direct value of each pair
    int2* rowpair;            // n: (offset, count) of the row's pairs, count -1: whole-row recompute
    float* D;                 // mode 1: n x k
    uint32_t* flag_bits;      // mode 1 (nullable)
    int2* flag_queue;         // mode 1: flagged pairs for the fp64 patch (bounded; D holds -1 marks)
    int64_t flag_queue_cap;
    unsigned long long* flag_queue_len;
    DevCounters* cnt;
};
cudaError_t launch_tc(const void* Xq, const void* Cq, int ldq, const TcArgs& a, int num_sms,
                      cudaStream_t st);
size_t tc_smem_bytes(int fmt, int d, int k);

// candidate refinement: fp32 direct values of the pairs, then certified
// argmin + min_dist per row; rows left open are appended to full_list
// (cnt->ovf_count) for the full-row kernel
cudaError_t launch_refine(const float* X, const float* C, const TcArgs& a, int32_t* labels,
                          double* min_dist, int32_t* full_list, int32_t* amb_list, int num_sms, cudaStream_t st,
                          int* nlaunch);
// the fallback's direct values for the flagged pairs of the distance matrix
// (marked -1 in D): fb 0 binary64, 1 binary32, 2 the low format fmt (0
// fp16, 1 bf16) itself; from the queue, or by a scan of D when it overflowed
cudaError_t launch_patch_flagged(int fb, int fmt, const float* X, const float* C, int64_t n, int k, int d,
                                 const int2* queue, const unsigned long long* qlen, int64_t cap, float* D,
                                 DevCounters* cnt, int num_sms, cudaStream_t st);
// out[i] = sum_l fl(a_il^2) in binary32, recursive summation (Alg. 2's d_xx)
cudaError_t launch_rowdot_fp32(const float* A, int64_t m, int d, float* out, int num_sms, cudaStream_t st);
// the distance matrix on CUDA cores, rounded operations in order: mode 0 Alg. 2
// in binary32 (dxx, dyy from launch_rowdot_fp32; test 1 paper: coef = fl(rho
// c_A gamma_{d+2}(2^-24)); test 0 tc: kacc, kn; 2 off), flagged pairs marked
// -1, queued and set in flag_bits (nullable); mode 1 direct formula in
// binary64, mode 2 in binary32
cudaError_t launch_matrix(int mode, const float* X, int64_t n, const float* C, int k, int d, const float* dxx,
                          const float* dyy, int test, float rho, float coef, float kacc, float kn, float* D,
                          uint32_t* flag_bits, int2* queue, int64_t qcap, unsigned long long* qlen, DevCounters* cnt,
                          int num_sms, cudaStream_t st);

// centre update
cudaError_t launch_absmax(const float* X, int64_t count, unsigned* out_bits, cudaStream_t st);
// per-cluster exact sums: iscratch holds 4k + 2 ints, perm n ints.
// md_out (nullable): each row's ||x_i - C_wd[labels[i]]||^2 to binary64
// accuracy (the winner distances of launch_winner_dist, bit for bit), fused
// into the pass over X where the kernel allows.  *nlaunch: kernels launched.
// nscale (0: n): the row count that, with max |x|, fixes the fixed-point
// scale (all shards' rows when the sums of several shards are added).
cudaError_t launch_accumulate(const float* X, int64_t n, int d, const int32_t* labels, int k,
                              const unsigned* absmax_bits, long long* sums, long long* counts, int* iscratch,
                              int32_t* perm, int num_sms, cudaStream_t st, const float* C_wd, double* md_out,
                              int* nlaunch, int64_t nscale = 0);
// md[i] = ||x_i - C[labels[i]]||^2, Eq. (dist-direct), to binary64 accuracy
// on the fp32 pipe (double-float arithmetic of df.cuh)
cudaError_t launch_winner_dist(const float* X, int64_t n, int d, const float* C, const int32_t* labels, double* md,
                               int num_sms, cudaStream_t st);
// bytes of scratch the empty-cluster selection needs (launch_finalize's esel)
size_t empty_select_bytes(int k);
// means (binary64 division, fp32 store), empty clusters (KM_EMPTY_FARTHEST:
// the rows of largest min_dist, one cooperative launch), shift.
// esel: empty_select_bytes(k) bytes, 256-byte aligned; status: the device
// status word (a bounded wait that runs out sets its timeout bit).
cudaError_t launch_finalize(const long long* sums, const long long* counts, const unsigned* absmax_bits,
                            int64_t n, int k, int d, const float* C_old, int empty_policy, const float* X,
                            const double* min_dist, float* C_new, int64_t* counts_out, double* shift,
                            void* esel, unsigned* status, int num_sms, cudaStream_t st, int* nlaunch,
                            int64_t nscale = 0);
// the e rows of largest min_dist (ties: lowest index), in that order, into
// rows_out / vals_out; esel: empty_select_bytes(e) bytes
cudaError_t launch_farthest_rows(const double* min_dist, int64_t n, int e, long long* rows_out, double* vals_out,
                                 void* esel, unsigned* status, int num_sms, cudaStream_t st);
// deterministic sum of n doubles (fixed two-level order)
cudaError_t launch_sum_f64(const double* v, int64_t n, double* partials, int nparts, double* out,
                           cudaStream_t st);

}  // namespace km
