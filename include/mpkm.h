/*
 * mpkm.h -- C-ABI of libmpkm: mixed-precision Lloyd's k-means on GB300.
 *
 * Method: E. Carson, X. Chen, X. Liu, "Computing k-means in Mixed Precision"
 * (arXiv 2407.12208).  Distances are formed by the expanded formula
 * Eq. (dist-expanded) with the cross term on tensor cores in a low format,
 * screened by the reliability test of Section 4.3 (Alg. 2), and the pairs
 * that fail it (or that could still be a row's nearest centre) are
 * recomputed by the direct formula Eq. (dist-direct) from the original fp32
 * data.  The centre update is Eq. (center); Lloyd's loop is Alg. 1 / Alg. 3.
 *
 * Conventions for every entry point:
 *  - X is n x d, C is k x d, both row-major fp32 (points as rows, the layout
 *    of Eq. (dist-blas3)).  Unless stated otherwise every array argument is a
 *    DEVICE pointer owned by the caller; the library never frees it.
 *  - The library allocates no device memory on the synchronous paths: the
 *    caller passes a workspace `ws` of at least km_workspace_size() bytes
 *    (256-byte aligned).  The serving calls draw from the arena given to
 *    km_init().
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    ordered on it; outputs whose name ends in `_host` are host pointers and
 *    imply a synchronisation of `stream` before the call returns.
 *  - Every call returns a km_status; no exception crosses the ABI.  On
 *    failure km_last_error() returns a message.  Argument errors are found
 *    before any launch.  A device-side wait that runs out of its iteration
 *    budget makes the kernel stop and the next synchronising call return
 *    KM_ETIMEOUT.
 *  - There is no CPU fallback: an unsupported combination returns
 *    KM_EUNSUPPORTED.
 *  - A context serves one calling thread at a time (its last-call record,
 *    profiling events and host-step copy streams are unsynchronised state);
 *    concurrent callers use one context each, or the serving calls, which
 *    are thread-safe.
 */
#ifndef MPKM_H
#define MPKM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct km_ctx km_ctx;

typedef enum {
    KM_OK = 0,
    KM_EINVAL = 1,        /* bad argument (null pointer, n<1, d<1, k<1, k>n, rho out of range) */
    KM_ENOMEM = 2,        /* workspace / arena too small; a job that can never be admitted */
    KM_ECUDA = 3,         /* a CUDA runtime or driver call failed */
    KM_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
    KM_ENOTREADY = 5,     /* km_poll: job still running */
    KM_ECANCELLED = 6,    /* km_poll: job was cancelled */
    KM_EUNSUPPORTED = 7   /* combination not implemented (e.g. E4M3 with d < 16) */
} km_status;

/* Low precision u_l of the cross term (Section 4.3).  The two *_DIRECT modes
 * skip the expanded formula and evaluate Eq. (dist-direct) on CUDA cores. */
typedef enum {
    KM_FP64_DIRECT = 0,   /* the plain FP64 path: Eq. (dist-direct) in binary64 */
    KM_FP32_DIRECT = 1,   /* Eq. (dist-direct) in fp32, certified, fp64 where ambiguous */
    KM_FP16 = 2,          /* binary16 cross term (Table 1.1), FP32 accumulation */
    KM_BF16 = 3,          /* bfloat16 cross term (Table 1.1), FP32 accumulation */
    KM_E4M3 = 4,          /* FP8 E4M3 cross term with power-of-two per-row scales */
    KM_FP32 = 5           /* km_distances only: Alg. 2 with binary32 as the low precision, on CUDA
                             cores, every operation rounded in the order Alg. 2 states it */
} km_low;

/* Precision of the fallback (Eq. (fallback-rule)): the direct formula that
 * km_distances evaluates for the pairs failing the reliability test.  The
 * assignment calls always certify their argmin in fp32 and binary64 and take
 * only KM_FB_FP64. */
typedef enum {
    KM_FB_FP64 = 0,       /* binary64 (Alg. 2) */
    KM_FB_FP32 = 1,       /* binary32 */
    KM_FB_LOW = 2         /* the low format itself, every operation rounded to it (the same-precision
                             fallback of Section 4.2; fp16 / bf16, and binary32 for KM_FP32) */
} km_fallback;

/* Reliability test of Section 4.3. */
typedef enum {
    KM_TEST_TC = 0,       /* Theorem 4.2 + Eq. (quantis-convert-error) instantiated for
                             tensor-core arithmetic: flag iff d^ <= rho * B(x, c) */
    KM_TEST_PAPER = 1,    /* Alg. 2: flag iff d^ <= rho * c_A * gamma^l_{r+2} (||x~||^2 + ||c~||^2) */
    KM_TEST_OFF = 2       /* no flags (uniform low precision); argmin still certified */
} km_test;

typedef enum {
    KM_EMPTY_KEEP = 0,     /* an empty cluster keeps its previous centre */
    KM_EMPTY_FARTHEST = 1  /* empty clusters (ascending j) take the points with the largest
                              current min_dist, ties to the lowest index, each point once */
} km_empty;

typedef struct {
    int32_t low;          /* km_low */
    int32_t test;         /* km_test */
    double rho;           /* safety factor, > 1 for KM_TEST_TC, > 2 for KM_TEST_PAPER (Eq. (quantis-reliability-test)); default 5 */
    double paper_factor;  /* c_A in {1, 2}: 1 = Alg. 2 as printed, 2 = E^l of Section 4.3 (default 2) */
    int32_t max_iter;     /* Lloyd iterations t_max (Alg. 1) */
    int32_t empty;        /* km_empty */
    double tau;           /* stop when max_j ||c_j^(t) - c_j^(t-1)|| < tau; tau <= 0 runs max_iter iterations */
    int32_t fallback;     /* km_fallback (km_distances; default KM_FB_FP64) */
} km_params;

/* Counters of the last assign / distances / lloyd call on a context. */
typedef struct {
    uint64_t pairs;           /* point-centre pairs screened (n*k per assignment) */
    uint64_t flagged;         /* pairs failing the reliability test: eta = flagged / pairs (Eq. (eta)) */
    uint64_t fp32_evals;      /* direct-formula evaluations in fp32 (certification of the argmin) */
    uint64_t fp64_evals;      /* direct-formula evaluations in binary64 */
    uint64_t ambiguous_rows;  /* rows whose low-precision argmin could not be certified */
    uint64_t overflow_rows;   /* rows whose candidate list overflowed (re-scanned over all centres) */
    double sse;               /* sum of min_dist of the last assignment (Eq. (sse)) */
} km_stats;

/* Fills the defaults: BF16, KM_TEST_TC, rho 5, c_A 2, max_iter 20, tau 0, FARTHEST, KM_FB_FP64. */
void km_default_params(km_params* p);

/* Creates a context on `device`.  `arena` (device memory, caller-owned, may
 * be NULL with arena_bytes 0) backs the serving calls only; it must stay
 * valid until km_destroy. */
km_status km_init(km_ctx** out, int device, void* arena, size_t arena_bytes);
km_status km_destroy(km_ctx* ctx);
const char* km_last_error(const km_ctx* ctx);

/* Bytes of workspace the synchronous calls (km_distances, km_assign,
 * km_update_centroids, km_lloyd_step, km_lloyd_run with p->max_iter) need for
 * these sizes: the largest of their layouts, all O(n (d + k_slots)) -- about
 * 0.66 GB at n = 1e6, d = 128, k = 1024 with a 16-bit low format. */
km_status km_workspace_size(const km_ctx* ctx, int64_t n, int d, int k, const km_params* p,
                            size_t* bytes);

/* The quantisation of Alg. 2's first line (Section 4.3: x~ = fl_l(x)) as the
 * tensor-core paths perform it, with the row statistics they use.
 *  - Xq: n rows of ldq elements of the low format, ldq = d rounded up to a
 *    multiple of 8 (fp16, bf16: 2 bytes each) or 16 (E4M3: 1 byte each),
 *    padding zero.  E4M3 holds fl(x / s) (saturating), fp16/bf16 fl(x).
 *  - stats: n x 4 floats (16-byte aligned): ||x||^2 (formed to about 2^-44
 *    and rounded to fp32), then ||x||, ||x~|| and ||x~ - x|| with
 *    x~ = s fl(x / s), each inflated by (1 + 2^-12) so that it bounds the
 *    exact norm from above; an element that overflowed the low format makes
 *    the last two +inf.
 *  - scale: n floats, the row's scale s.  E4M3: the smallest power of two
 *    with max_l |x_l| / s <= 448 (so the row maximum lands in (224, 448]),
 *    at least 2^-126, and 1 for an all-zero row; fp16/bf16: 1.
 * low must be KM_FP16, KM_BF16 or KM_E4M3 (else KM_EUNSUPPORTED).  Device
 * pointers, asynchronous on `stream`. */
km_status km_quantize(km_ctx* ctx, const float* X, int64_t n, int d, int32_t low, void* Xq, float* stats,
                      float* scale, void* stream);

/* Which low format pays for this data (no counterpart in the paper, which
 * fixes the format per experiment).  The cost of the screening path grows
 * with the candidates it keeps per row: the centres whose d^ lies within
 * 2 B_max of the row minimum, B the error bound behind the reliability test
 * (Theorem 4.2 + Eq. (quantis-convert-error)), and a row whose candidates
 * overflow its list is recomputed over all centres.  On a strided sample of
 * 2048 rows this call counts, from fp32 direct distances, the candidates
 * each row would keep under BF16 and under E4M3 (per-row scales) and the
 * share of rows above one list's capacity, and returns *low_host = KM_E4M3
 * when d >= 16, its predicted overflow share is at most max_overflow_share
 * and it keeps at most two candidates per row more than BF16; else KM_BF16.
 * stats_host (nullable, host, 4 doubles): BF16 mean candidates per row and
 * overflow share, then the same for E4M3 (+inf and 1 when d < 16).  ws: as
 * km_workspace_size.  Synchronises `stream`.  KM_EUNSUPPORTED where no
 * tensor-core path exists (k > 65535, d too large for the BF16 tiles). */
km_status km_choose_low(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                        double max_overflow_share, int32_t* low_host, double* stats_host, void* ws, size_t ws_bytes,
                        void* stream);

/* Alg. 2 for all pairs (Section 4.3; the distance-matrix experiments of
 * Section 6.1).  D (n x k fp32, row-major) receives, per pair, the expanded
 * low-precision value where the reliability test passes and the direct
 * value in the fallback's precision (p->fallback; rounded to fp32, the
 * working precision) where it fails.  flag_bits (nullable; ceil(n*k/32)
 * words, bit (i*k+j) of the row-major pair index) marks the pairs that fell
 * back.  n_flagged_host (nullable, host) receives the number of flagged
 * pairs.  low: FP16/BF16/E4M3 (tensor cores, the cross term accumulated in
 * fp32), KM_FP32 (Alg. 2 in binary32), or KM_FP64_DIRECT / KM_FP32_DIRECT
 * (the direct formula for every pair in that precision, no test).
 * KM_FB_LOW with E4M3 is KM_EUNSUPPORTED (no E4M3 arithmetic). */
km_status km_distances(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                       const km_params* p, float* D, uint32_t* flag_bits,
                       uint64_t* n_flagged_host, void* ws, size_t ws_bytes, void* stream);

/* Assignment step of Alg. 3: labels[i] = argmin_j d(x_i, c_j)^2 (lowest j on
 * ties).  The argmin is certified: it equals the binary64 direct-formula
 * argmin wherever that row's best/second-best gap exceeds the proved error
 * bounds (in practice: relative gaps above ~1e-7).  min_dist (nullable,
 * n doubles) receives ||x_i - c_label||^2 by the direct formula (Eq.
 * (dist-direct)) from the fp32 data to binary64 accuracy: relative error
 * below 2^-40 (exactly the binary64 sum in coordinate order on the FP64
 * path).  n_flagged_host (nullable, host): number of pairs that failed the
 * reliability test. */
km_status km_assign(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                    const km_params* p, int32_t* labels, double* min_dist,
                    uint64_t* n_flagged_host, void* ws, size_t ws_bytes, void* stream);

/* Tuning of the screening kernel (no counterpart in the paper).  When K fits
 * two 128-byte atoms (d <= 128 for FP16/BF16, d <= 256 for E4M3) the
 * tensor-core kernel's epilogue comes in three variants that give the same
 * labels, distances and counts: 64-column steps staging all 16 quads of a
 * step in shared memory (KM_SV_FULL), 64-column steps staging 8 at a time,
 * which leaves room for a second operand stage (KM_SV_HALF), and 32-column
 * steps (KM_SV_C32).  Which is fastest depends on d, k and the data.  The
 * context keeps one variant per shape class (format, ceil(d) in 128-byte
 * atoms, ceil(k / 128), and whether n has fewer 128-row blocks than the GPU
 * has SMs); its serving jobs use the same table.  Untuned classes take HALF
 * when K is two atoms, else FULL. */
enum { KM_SV_AUTO = -1, KM_SV_FULL = 0, KM_SV_HALF = 1, KM_SV_C32 = 2, KM_SV_REG = 3 };

/* Times km_assign on the first min(n, 2^20) rows of X with each variant
 * (one warm-up and three timed calls each, CUDA events on `stream`), keeps
 * the fastest for this shape class and returns it in *variant_host
 * (KM_SV_REG when K is wider than two atoms and nothing was timed; -1 for
 * the direct formats).  ms_host (nullable, host, 3 floats): mean ms per call
 * of FULL, HALF, C32.  labels: n int32 of device scratch.  ws: as km_assign.
 * Synchronises `stream`. */
km_status km_autotune(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d, const km_params* p,
                      int32_t* labels, int32_t* variant_host, float* ms_host, void* ws, size_t ws_bytes,
                      void* stream);
/* Sets the variant of the shape class of (n, d, k, low) to `variant`
 * (KM_SV_FULL / HALF / C32), or with KM_SV_AUTO returns it to the default.
 * KM_EUNSUPPORTED for a direct format or (unless KM_SV_AUTO) K wider than
 * two atoms. */
km_status km_set_screen_variant(km_ctx* ctx, int64_t n, int d, int k, int32_t low, int32_t variant);

/* Centre update, Eq. (center), in precision higher than the working one
 * (Section 4.4): per-cluster sums are formed exactly in 64-bit fixed point
 * (order-independent, hence deterministic), divided in binary64 and stored
 * in fp32.  counts (k int64), C_new (k x d fp32).  min_dist (nullable, n
 * doubles) is needed only for KM_EMPTY_FARTHEST.  shift_host (nullable,
 * host): max_j ||c_new_j - c_old_j||; with NULL the shift is not computed
 * (here and in km_lloyd_step / km_lloyd_step_host). */
km_status km_update_centroids(km_ctx* ctx, const float* X, int64_t n, int d,
                              const int32_t* labels, int k, const float* C_old,
                              const km_params* p, const double* min_dist, float* C_new,
                              int64_t* counts, double* shift_host, void* ws, size_t ws_bytes,
                              void* stream);

/* One iteration of Alg. 3's loop: the assignment of X to C_old (as
 * km_assign: labels, min_dist (nullable)) followed by the centre update of
 * Eq. (center) on those labels (as km_update_centroids: C_new, counts
 * (nullable), shift_host (nullable, host)).  The two share one pass where
 * they can: the largest |x|, which fixes the scale of the exact centre
 * sums, comes out of the quantisation pass.  The results equal km_assign
 * followed by km_update_centroids bit for bit.  Workspace: as km_lloyd_run
 * (km_workspace_size). */
km_status km_lloyd_step(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_old,
                        const km_params* p, int32_t* labels, double* min_dist, float* C_new,
                        int64_t* counts, double* shift_host, void* ws, size_t ws_bytes,
                        void* stream);

/* ---- row-sharded updates: the exchange of a data-parallel Lloyd iteration --
 * Eq. (center) is a sum over points, so with the rows of X split over
 * several processes (one GPU each, C replicated) an iteration needs one
 * exchange: the per-cluster sums and counts.  The library forms them as
 * exact 64-bit fixed-point integers, so adding the shards' integers (an
 * all-reduce of k (d + 1) int64, in any order) gives exactly the sums of the
 * whole data and every process then finalises the same centres, bit for bit
 * equal to one process holding all rows.  The fixed-point scale follows from
 * the largest |x| over ALL shards and their total row count, agreed on first
 * (a max- and a sum-reduction).  Empty clusters: each shard proposes its rows
 * of largest min_dist (km_farthest_rows); the caller merges the candidates
 * (largest min_dist first, ties to the lowest global row index). */

/* max |x| over count floats as its binary32 bit pattern (non-negative floats
 * order like their bits, so shards' values reduce with an integer maximum).
 * ws: 256 bytes.  Synchronises `stream`. */
km_status km_absmax(km_ctx* ctx, const float* X, int64_t count, uint32_t* bits_host, void* ws, size_t ws_bytes,
                    void* stream);
/* The shard's per-cluster fixed-point sums (k x d int64) and counts (k int64)
 * of its rows (labels: n int32 in [0, k)), at the scale of absmax_bits (all
 * shards' max |x|) and n_total (all shards' rows).  Device outputs; ws as
 * km_workspace_size for the shard. */
km_status km_update_partial(km_ctx* ctx, const float* X, int64_t n, int d, const int32_t* labels, int k,
                            uint32_t absmax_bits, int64_t n_total, int64_t* sums, int64_t* counts, void* ws,
                            size_t ws_bytes, void* stream);
/* Centres from the summed integers: c_j = sum_j 2^-S / count_j in binary64,
 * stored in fp32 (as km_update_centroids); an empty cluster keeps C_old's
 * row (re-seed it afterwards); shift_host (nullable): max_j ||c_j - c_old_j||. */
km_status km_update_finalize(km_ctx* ctx, const int64_t* sums, const int64_t* counts, int k, int d,
                             uint32_t absmax_bits, int64_t n_total, const float* C_old, float* C_new,
                             double* shift_host, void* ws, size_t ws_bytes, void* stream);
/* The e rows of largest min_dist (ties to the lowest index), in that order:
 * rows (e int64, device) and their min_dist (e doubles, device); 1 <= e <= n
 * and e at most the k the workspace was sized for.  Synchronises `stream`. */
km_status km_farthest_rows(km_ctx* ctx, const double* min_dist, int64_t n, int e, int64_t* rows, double* vals,
                           void* ws, size_t ws_bytes, void* stream);

/* Alg. 3 for many small jobs at once (no counterpart in the paper): one
 * launch runs every job's whole Lloyd loop, one thread block per job, instead
 * of about ten launches per iteration each.  For low = KM_FP32_DIRECT and jobs
 * with d <= 8, 1 <= k <= 64, k <= n <= 16384; all jobs share p (max_iter,
 * tau, empty).  Every job's centres, labels, SSE per iteration and iteration
 * count equal km_lloyd_run's on that job alone, bit for bit.  All pointers of
 * a job are device pointers: sse_per_iter (max_iter + 1 doubles), iters (one
 * int32), scratch (n doubles).  Asynchronous on `stream`; errors in the
 * arguments return before any launch. */
typedef struct {
    const float* X;
    int64_t n;
    int d;
    int k;
    const float* C_init;
    float* C_out;
    int32_t* labels;
    double* sse_per_iter;
    int32_t* iters;
    double* scratch;
} km_batch_job;
km_status km_lloyd_run_batch(km_ctx* ctx, const km_batch_job* jobs, int njobs, const km_params* p, void* stream);

/* Initial centres by D^2 sampling (k-means++; Section 2 names it beside
 * uniformly drawn initial centres and leaves it outside the method).  The
 * random draws are inputs: u_host, k doubles in [0, 1) (host).
 *   i_0 = min(floor(u_0 n), n - 1); D^2_i = d(x_i, x_{i_0})^2;
 *   for t = 1..k-1: T = sum_i D^2_i; i_t = the first row whose prefix sum of
 *   D^2 exceeds u_t T (the last row with D^2 > 0 when rounding leaves none;
 *   min(floor(u_t n), n - 1) when T = 0); D^2_i = min(D^2_i, d(x_i, x_{i_t})^2).
 * Distances by the direct formula to binary64 accuracy (relative error below
 * 2^-40), sums in binary64 in a fixed order, so the picks do not depend on
 * the launch; they equal the binary64 sequence except where a draw lies
 * within rounding of a boundary between two rows.  C_out (k x d fp32,
 * device) receives the picked rows, idx_host (nullable, host, k int64) their
 * indices.  1 <= k <= n, d <= 512.  ws: device memory of at least
 * 8 n + 16 k + 16 min(n, 16384) + 1280 bytes, 256-byte aligned.
 * Synchronises `stream`. */
km_status km_seed_pp(km_ctx* ctx, const float* X, int64_t n, int d, int k, const double* u_host, float* C_out,
                     int64_t* idx_host, void* ws, size_t ws_bytes, void* stream);

/* Failure-path check (no paper counterpart): launches one warp that waits on
 * an mbarrier no thread arrives at.  The wait is the same bounded wait every
 * kernel of the library uses: after its budget (about a second) it sets the
 * timeout bit of the device status word and returns, so the call returns
 * KM_ETIMEOUT and the context (and device) stay usable.  ws: at least 256
 * bytes of device memory, 256-byte aligned. */
km_status km_selftest_timeout(km_ctx* ctx, void* ws, size_t ws_bytes, void* stream);

/* km_lloyd_step on HOST buffers (no paper counterpart: the transfer around
 * one iteration of Alg. 3's loop body, for callers whose data lives in host
 * memory).  X_host (n x d fp32), C_host (k x d) are read, and labels_host
 * (n int32), min_dist_host (nullable, n doubles), C_new_host (k x d),
 * counts_host (nullable, k int64) and shift_host (nullable) written, all in
 * host memory; the call returns when they are there (it synchronises
 * `stream`).  The rows travel in up to four chunks of whole 128-row blocks,
 * each about half the size of the one before, on a copy stream owned by the
 * context (a second one carries the results back): each chunk is assigned
 * (labels and min_dist) as soon as it has arrived and its results go back
 * while the next chunk is assigned; the centre update follows the last
 * chunk.  With pinned (page-locked) host
 * buffers the copies overlap the kernels; pageable ones still give the same
 * results.  The results equal km_lloyd_step on device copies of the same
 * inputs bit for bit.  ws: device memory of km_host_workspace_size bytes
 * (256-byte aligned), holding the device copies and the step's workspace.
 * Errors as km_lloyd_step. */
km_status km_host_workspace_size(const km_ctx* ctx, int64_t n, int d, int k, const km_params* p,
                                 size_t* bytes);
km_status km_lloyd_step_host(km_ctx* ctx, const float* X_host, int64_t n, int d, int k,
                             const float* C_host, const km_params* p, int32_t* labels_host,
                             double* min_dist_host, float* C_new_host, int64_t* counts_host,
                             double* shift_host, void* ws, size_t ws_bytes, void* stream);

/* Alg. 3: Lloyd's loop with the mixed-precision assignment.  C_out (k x d)
 * receives the final centres, labels (n) the final reassignment.
 * sse_per_iter and eta_per_iter (nullable, host, max_iter + 1 doubles):
 * SSE and flagged fraction of every assignment, the last one being the
 * final reassignment.  iters_done (nullable, host).
 * The iterations are recorded once as two CUDA graphs (even and odd
 * iterations) and replayed, one launch per iteration; with phase timing on
 * (km_set_profiling) they are launched kernel by kernel, with the same
 * results.  While the call records, another thread of the process must not
 * synchronise the whole device (cudaDeviceSynchronize fails while any stream
 * is being recorded); a stream the runtime refuses to record falls back to
 * the direct launches.  With a legacy default stream the replays run on a
 * stream of the context, ordered after and before the caller's work. */
km_status km_lloyd_run(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_init,
                       const km_params* p, float* C_out, int32_t* labels, double* sse_per_iter,
                       double* eta_per_iter, int* iters_done, void* ws, size_t ws_bytes,
                       void* stream);

/* Counters of the last assign / distances / lloyd call (synchronises that
 * call's stream).  Returns KM_ETIMEOUT if a device-side wait ran out. */
km_status km_get_stats(km_ctx* ctx, km_stats* out);

/* Phase timing.  While on, every call on this context records a pair of
 * CUDA events on its stream around each phase below (no device memory is
 * allocated; the events are host-side driver objects). */
enum {
    KM_PHASE_QUANTISE = 0,   /* low-precision copies of X and C + norms (Alg. 2 line 1) */
    KM_PHASE_SCREEN = 1,     /* tensor-core cross term + reliability test + candidates */
    KM_PHASE_REFINE = 2,     /* direct-formula recompute of candidates, certified argmin */
    KM_PHASE_FULLROW = 3,    /* rows re-scanned over all centres */
    KM_PHASE_UPDATE = 4,     /* centre update (Eq. (center)) */
    KM_PHASE_DIRECT = 5,     /* direct-formula assignment (FP64 / FP32 paths) */
    KM_NUM_PHASES = 6
};
km_status km_set_profiling(km_ctx* ctx, int on);
/* Sum of each phase's duration (ms, ms[KM_NUM_PHASES]) and number of timed
 * occurrences (counts, nullable) since the previous read; synchronises. */
km_status km_get_phase_times(km_ctx* ctx, double* ms, int64_t* counts);
/* Number of kernels this context has launched since km_init. */
km_status km_get_launch_count(const km_ctx* ctx, uint64_t* launches);

/* ---- assignment without allocation -------------------------------------- */

/* The paper has no counterpart to this call.  It is km_assign with
 * low = KM_FP32_DIRECT (the same kernels and the same results) for callers
 * that cannot allocate device memory when they assign: a process whose
 * device memory is all held by a caching pool or by another framework,
 * where a cudaMalloc would fail, and latency-bound loops
 * that must not call cudaMalloc/cudaFree (cudaFree can synchronise the whole
 * device).  It takes no workspace.  Its scratch (the device counters and the
 * list of rows left open, one int32 per row) is a file-scope device array of
 * the library sized for KM_STATIC_MAX_ROWS rows: 4 MiB + 256 B per device.
 *  - n > KM_STATIC_MAX_ROWS returns KM_ENOMEM before any launch; the other
 *    argument errors are km_assign's (d <= 256 as on every direct path).
 *  - labels (n int32) and min_dist (n doubles) are required device outputs.
 *  - On success the call allocates nothing, host or device.  A rejected call
 *    stores its message for km_last_error, as every call does.
 *  - The first call on each device does one-time set-up: it resolves the
 *    scratch address with cudaGetSymbolAddress, which may load the
 *    library's device code.  Make that first call before any stream
 *    capture begins.
 *  - Each call clears the scratch counters on `stream` before its kernels.
 *  - There is one scratch per device and process.  Calls whose work overlaps
 *    in time on one device (other streams, threads or contexts) race on it
 *    and give wrong results: order them on one stream or with events.
 *  - km_get_stats and the phase timers do not report on this call. */
#define KM_STATIC_MAX_ROWS 1048576
km_status km_assign_static(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                           int32_t* labels, double* min_dist, void* stream);

/* ---- serving (continuous batching on one GPU) ---------------------------- */

/* A job: X (n x d) and C_init (k x d).  kind 0 = Lloyd (Alg. 3, p.max_iter
 * iterations), kind 1 = one nearest-centre assignment against C_init.
 * flags 0: X and C_init are HOST pointers, copied before km_submit returns
 * and into the arena at admission.  flags KM_JOB_DEVICE_DATA: they are
 * DEVICE pointers on the context's device that stay valid and unchanged
 * until km_poll reports the job finished; X is read in place (resident
 * points take no arena memory), C_init is copied into the arena at
 * admission. */
#define KM_JOB_DEVICE_DATA 1
typedef struct {
    const float* X;
    int64_t n;
    int32_t d;
    int32_t k;
    const float* C_init;
    km_params p;
    int32_t kind;
    int32_t flags;
} km_job;

typedef struct {
    km_status status;     /* KM_OK when finished */
    int32_t iters;
    double sse;
    double eta;           /* flagged fraction over all assignments of the job */
    double latency_ms;    /* submit -> completion */
    double queue_ms;      /* submit -> admission */
    const float* C;       /* device pointer into the arena (k x d), valid until km_release */
    const int32_t* labels;/* device pointer into the arena (n), valid until km_release */
    const char* message;  /* why the job failed ("" when it did not), valid until km_release */
} km_result;

/* Queues a job; it is admitted as soon as its memory (centres, labels and
 * workspace; the points too for host data) fits in the arena, up to 16 jobs
 * running at once, each on its own stream so that their kernels overlap on
 * the device (launched directly: no graph is recorded beside the caller's
 * work); queued jobs are considered in arrival order on every change,
 * so a small job can start while a large one waits for memory.  Host arrays
 * are copied before the call returns.  KM_ENOMEM if the job could never fit
 * in the arena. */
km_status km_submit(km_ctx* ctx, const km_job* job, uint64_t* job_id);
/* KM_ENOTREADY until the job is done; then fills *out. */
km_status km_poll(km_ctx* ctx, uint64_t job_id, km_result* out);
/* Frees a finished job's arena memory (its result pointers become invalid). */
km_status km_release(km_ctx* ctx, uint64_t job_id);
/* Cancels a queued or running job (a running job stops between iterations). */
km_status km_cancel(km_ctx* ctx, uint64_t job_id);

#ifdef __cplusplus
}
#endif
#endif /* MPKM_H */
