/*
 * bs.h -- C ABI of the GB300 boson-sampling permanent library (libbs.so).
 *
 * Hot path of "High performance Boson Sampling simulation via data-flow
 * engines" (Morse et al., arXiv 2309.07027): the generalized
 * Balasubramanian-Bax-Franklin-Glynn permanent with row and column
 * multiplicities (Sec. 2.2, Eq. bbfgrepeated) walked in n-ary reflected Gray
 * order, its Laplace minors, and Clifford & Clifford sampling built on them
 * (Sec. 4).  All arithmetic runs in CUDA kernels for sm_103a; there is no CPU
 * fallback: without a usable GPU every compute call returns BS_ENODEV.
 *
 * Conventions
 *   - Complex numbers are bs_c128 {re, im} (two IEEE doubles).
 *   - Matrices are row-major with a leading dimension `ld` counted in complex
 *     elements (ld >= cols).  Rows are output modes, columns input modes
 *     (Sec. 2: column sums of the unitary, rows carry the output
 *     multiplicities).
 *   - Host-pointer calls are synchronous: inputs are copied in, outputs are
 *     written to caller memory before the call returns.  The caller owns every
 *     buffer it passes; the library never keeps a caller pointer.
 *   - `*_dev` calls take device pointers, enqueue work on the context's stream
 *     and return without waiting; bs_ctx_sync() waits and reports kernel
 *     status (for example a deadline that expired).
 *   - Return value: BS_OK (0) or a negative BS_E* code; bs_last_error() gives a
 *     message for the calling thread.
 *   - Limits: n = sum of multiplicities <= BS_MAX_N (48); weights
 *     prod C(M_k, Delta_k) < 2^48 are exact in FP64.
 */
#ifndef BS_H
#define BS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BS_MAX_N 48

enum {
    BS_OK = 0,
    BS_EINVAL = -1,    /* bad argument (sizes, multiplicities, sums, limits) */
    BS_ENOMEM = -2,    /* device memory budget or allocation exhausted */
    BS_ECUDA = -3,     /* CUDA runtime error (message in bs_last_error) */
    BS_ETIMEOUT = -4,  /* a kernel deadline expired (status word) */
    BS_ENODEV = -5,    /* no usable CUDA device */
    BS_ECANCELED = -6  /* a served request was cancelled (bs_server_cancel) */
};

typedef struct {
    double re, im;
} bs_c128;

/* Arithmetic of the walk.
 *   BS_FP64:  column sums, products, weights and sums in double precision;
 *             partial sums combined in double-double.
 *   BS_MIXED: column sums and products in single precision (column sums
 *             re-seeded from the matrix every chunk, and every 2^8 steps
 *             inside it for jobs whose error would otherwise drift past the
 *             tolerance; columns scaled by powers of two), addends summed in
 *             float-float runs, partial sums in double-double (Sec. 3.2
 *             discusses the accuracy trade-off), for every job whose
 *             predicted FP32 error meets the MIXED tolerance
 *             (bs_ctx_set_mixed_tolerance); other jobs run in the double-float
 *             kernels of BS_DF64 (FP64-class, the cancellation-prone jobs).
 *   BS_DF64:  double-float: every quantity an unevaluated pair of floats
 *             (about 48 significant bits) on the single-precision pipe --
 *             column sums exact in fixed point (no drift), products by
 *             FMA-based exact multiplication, compensated sums, partial sums
 *             in double-double; results within the FP64 tolerance at several
 *             times the FP64 kernels' speed on this part, whose FP64 rate is
 *             1/64 of its FP32 rate. */
typedef enum { BS_FP64 = 0, BS_MIXED = 1, BS_DF64 = 2 } bs_mode;

typedef struct bs_ctx bs_ctx;

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the
 * device memory the context may allocate (0 = no cap).  On success *out owns
 * a stream and grow-only device buffers; release with bs_ctx_destroy.
 * Errors: BS_EINVAL (out == NULL), BS_ENODEV, BS_ECUDA. */
int bs_ctx_create(bs_ctx** out, int device, size_t mem_budget_bytes);

/* Free every resource of the context (NULL is accepted). */
void bs_ctx_destroy(bs_ctx* ctx);

/* Message of the last failed call made by this thread (never NULL). */
const char* bs_last_error(const bs_ctx* ctx);

/* Use an external cudaStream_t (passed as void*) for all later work; any
 * handle is taken as is, 0 meaning the legacy default stream.  The caller
 * keeps the stream alive.  bs_ctx_use_own_stream() returns to the context's
 * own stream. */
int bs_ctx_set_stream(bs_ctx* ctx, void* stream);
int bs_ctx_use_own_stream(bs_ctx* ctx);

/* Wait for all work enqueued on the context's stream and report the kernel
 * status word: BS_OK or BS_ETIMEOUT (a deadline expired), or BS_ECUDA. */
int bs_ctx_sync(bs_ctx* ctx);

/* Relative deadline (seconds) for every later walk launch: warps stop taking
 * work once the device clock passes launch time + seconds, and the call
 * returns BS_ETIMEOUT.  0 disables the deadline. */
int bs_ctx_set_deadline(bs_ctx* ctx, double seconds);

/* Chunk-length knob: log2_chunk_max caps the chunk length (= the re-seed
 * interval of the column sums) of the given mode (default 11, 12 for
 * BS_DF64); values
 * outside [4, 20] are rejected with BS_EINVAL. */
int bs_ctx_set_chunk_log2(bs_ctx* ctx, bs_mode mode, int log2_chunk_max);
int bs_ctx_get_chunk_log2(const bs_ctx* ctx, bs_mode mode);

/* Accuracy target of BS_MIXED: a job runs in the FP32 kernels when the
 * precision rule predicts an FP32 error of at most tol * prod_j ||a_j||^{N_j}
 * (column norms over the rows repeated by their multiplicities) -- with its
 * column sums re-seeded every 2^8 steps when only their drift over longer
 * chunks breaks that -- else in the double-float kernels.  Default 1e-6.  Larger values keep more jobs in FP32; a value
 * >= 1e300 sends every MIXED job to FP32 (to measure the FP32 error itself).
 * Errors: BS_EINVAL (tol <= 0 or NaN). */
int bs_ctx_set_mixed_tolerance(bs_ctx* ctx, double tol);

/* Autotuner: times a synthetic problem of the given kind (0 permanent,
 * 1 minors), mode and K product columns (4..48) with chunk-length caps
 * 2^8, 2^10, 2^12, 2^14 (the chunk length is the re-seed interval of the
 * column sums and sets how many warps share one job) and keeps the fastest
 * for the mode in this context.  *best_log2 (nullable) receives the cap,
 * *best_addends_per_s (nullable) the measured rate. */
int bs_tune(bs_ctx* ctx, bs_mode mode, int kind, int K, int* best_log2, double* best_addends_per_s);

/* ------------------------------------------------------------------ */
/* Permanents                                                          */
/* ------------------------------------------------------------------ */

/* perm(A, M, N) of Eq. bbfgrepeated (Sec. 2.2): the permanent of the
 * n x n matrix obtained by repeating row r row_mult[r] times and column c
 * col_mult[c] times, n = sum(row_mult) = sum(col_mult) (Sec. 4, U_ST).
 *   A        rows x cols, row-major, leading dimension ld (host memory).
 *   row_mult rows non-negative ints; col_mult cols non-negative ints.
 *   out      result rounded to double; out_lo (nullable) receives the low
 *            part of the double-double sum (out + out_lo ~ 106 bits of the
 *            computed value).
 * n = 0 gives 1 (the empty permanent).  The orientation (A or A^T) with
 * fewer addends is chosen automatically (perm(A) = perm(A^T)).
 * Errors: BS_EINVAL (negative multiplicity, sums differ, n > BS_MAX_N,
 * ld < cols, NULL pointers), BS_ENOMEM, BS_ECUDA, BS_ETIMEOUT. */
int bs_perm(bs_ctx* ctx, const bs_c128* A, int rows, int cols, int ld, const int* row_mult,
            const int* col_mult, bs_mode mode, bs_c128* out, bs_c128* out_lo);

/* Batch of `count` independent permanents of uneven sizes in one persistent
 * launch per column bucket (Appendix A.4 batches equal-size matrices; here
 * sizes may differ).  Item b: matrix rows[b] x cols[b], row-major with
 * ld = cols[b], at A_packed + a_offset[b]; multiplicities at
 * mult_packed + row_mult_off[b] (rows[b] ints) and + col_mult_off[b]
 * (cols[b] ints).  out[b] receives item b (host memory).  An invalid item
 * fails the whole call with BS_EINVAL before any work is queued. */
int bs_perm_batch(bs_ctx* ctx, int count, const bs_c128* A_packed, const int64_t* a_offset, const int* rows,
                  const int* cols, const int* mult_packed, const int64_t* row_mult_off,
                  const int64_t* col_mult_off, bs_mode mode, bs_c128* out);

/* Device-pointer batch: A_packed_dev and out_dev are device pointers; the
 * offsets, sizes and multiplicities are host arrays (they drive the host
 * plan).  Enqueued on the context stream; out_dev is valid after
 * bs_ctx_sync().  A_packed_dev must stay valid until then. */
int bs_perm_batch_dev(bs_ctx* ctx, int count, const bs_c128* A_packed_dev, const int64_t* a_offset,
                      const int* rows, const int* cols, const int* mult_packed, const int64_t* row_mult_off,
                      const int64_t* col_mult_off, bs_mode mode, bs_c128* out_dev);

/* Laplace minors used by a Clifford & Clifford step (Sec. 4, Clifford &
 * Clifford's algorithm; the paper batches such permanents "with identical
 * row selections but different column selections", Appendix A.4).
 * Requires sum(row_mult) = sum(col_mult) - 1.  minors[c] (cols entries) is
 * the permanent of the expanded matrix with one copy of column c removed,
 * 0 when col_mult[c] == 0.  All minors come from one shared Gray walk over
 * the rows.  For any row vector v,  sum_c col_mult[c] v[c] minors[c] is the
 * permanent of A with v appended as one more row.
 * Errors as bs_perm. */
int bs_laplace_minors(bs_ctx* ctx, const bs_c128* A, int rows, int cols, int ld, const int* row_mult,
                      const int* col_mult, bs_mode mode, bs_c128* minors);

/* Formula of a plain permanent for bs_perm_formula (Sec. 2): the
 * generalized walk of this library in its binary case, or one of the two
 * Gray-coded formulas the paper compares it with.
 *   BS_FORMULA_BBFG   Eq. bbfg: delta_1 = +1, 2^(n-1) addends, prefactor
 *                     2^(1-n); the same path as bs_perm with unit
 *                     multiplicities.
 *   BS_FORMULA_RYSER  Eq. ryser: column subsets S in Gray order, row sums
 *                     sum_{j in S} a_ij updated by one column per step,
 *                     2^n addends, prefactor (-1)^n.
 *   BS_FORMULA_NW     Nijenhuis-Wilf form of Eq. ryser: row sums start at
 *                     x_i = a_in - (a_i1 + ... + a_in) / 2 and walk subsets
 *                     of the first n-1 columns, 2^(n-1) addends, prefactor
 *                     (-1)^(n-1) 2. */
typedef enum { BS_FORMULA_BBFG = 0, BS_FORMULA_RYSER = 1, BS_FORMULA_NW = 2 } bs_formula;

/* Permanent of the n x n matrix A (row-major, leading dimension ld >= n) by
 * `formula`, walked by the FP64 permanent kernel in double precision with
 * double-double partial sums: the accuracy and speed comparison of Sec. 3.2
 * (Fig. accuracy) on this GPU.  Only the packing of the start sums and the
 * rows added per step, and the prefactor, differ between formulas.  n = 0
 * gives 1.  out_lo (nullable) receives the double-double tail.
 * Errors: BS_EINVAL (n < 0, n > BS_MAX_N, ld < n, NULL pointers, unknown
 * formula), BS_ENOMEM, BS_ECUDA, BS_ETIMEOUT. */
int bs_perm_formula(bs_ctx* ctx, const bs_c128* A, int n, int ld, bs_formula formula, bs_c128* out,
                    bs_c128* out_lo);

/* Allocation-free permanent, for callers that may not allocate device
 * memory when they need a result: hosts whose memory manager owns a fixed
 * device budget and forbids allocations outside it, and real-time loops that
 * must not enter the CUDA allocator (cudaMalloc / cudaFree may synchronise the
 * device and have no latency bound).  Computes the same permanent as bs_perm
 * (same kernels, any mode) without any device or host heap allocation:
 * all device scratch is one file-scope __device__ array of 8 MiB that every
 * GPU loading the library holds until the process exits.  The paper has no
 * counterpart of this call.
 *   A, row_mult, col_mult, out, out_lo: host memory as in bs_perm (no
 *   context); stream: a cudaStream_t as void* (0 = legacy default stream);
 *   the inputs are staged from the caller's stack and the call synchronises
 *   the stream before it returns.  There is no deadline: the walk runs to
 *   the end of the job.
 * Limit: the job's warp tasks must fit the fixed scratch (about 2.6e5 tasks,
 * e.g. every permanent with up to 2^34 addends); larger jobs return
 * BS_EINVAL with a message naming the limit.  The first call on a device looks
 * up the array's device address.  Calls share the array: calls that overlap
 * on the GPU race and must be serialised by the caller. */
int bs_perm_noalloc(const bs_c128* A, int rows, int cols, int ld, const int* row_mult, const int* col_mult,
                    bs_mode mode, void* stream, bs_c128* out, bs_c128* out_lo);

/* ------------------------------------------------------------------ */
/* Clifford & Clifford sampling (Sec. 4)                               */
/* ------------------------------------------------------------------ */

/* Draw n_samples output patterns of ideal boson sampling with interferometer
 * U (m x m, row-major, host) and input occupation input_occupation[m]
 * (n = sum <= BS_MAX_N photons), Clifford & Clifford's algorithm: a random
 * permutation of the input photons, then for k = 1..n the row r_k drawn with
 * probability proportional to |sum_l U[r, col_l] minor_l|^2 using the minors
 * of the (k-1) x k matrix of rows drawn so far (Eq. bs_p gives the output
 * distribution).  Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed
 * by (seed low, seed high) with counter (sample low, sample high, purpose,
 * index): purpose 0 / index j drives the Fisher-Yates swap of position j
 * (j = n-1..1) with position floor(w0 (j+1) / 2^32); purpose 1 / index k gives
 * u = ((w0 << 32 | w1) >> 11) 2^-53 for step k, and r_k is the first row whose
 * running FP64 weight sum (row order) exceeds u times the total.  Sample s of a
 * seed does not depend on n_samples.
 * out: n_samples x m occupation counts (host).  All samples advance together,
 * one batched minors launch per step. */
int bs_sample(bs_ctx* ctx, const bs_c128* U, int m, const int* input_occupation, int n_samples, uint64_t seed,
              bs_mode mode, int* out);

/* General form: U is m_rows x m_cols (row-major, leading dimension ld), one
 * input occupation per column, and only output rows < m_detected are counted
 * in out (n_samples x m_detected); rows >= m_detected model loss modes (Sec. 4,
 * lossy simulation by extra modes).  m_detected <= 0 means m_rows. */
int bs_sample_ex(bs_ctx* ctx, const bs_c128* U, int m_rows, int m_cols, int ld, const int* input_occupation,
                 int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out);

/* bs_sample_ex that also returns each chain's drawn rows: rows_out
 * (n_samples x n, host, n = sum of input_occupation) receives r_1, ..., r_n
 * of every sample in draw order (step k of Clifford & Clifford's algorithm
 * draws r_k; the occupation counts in out are their histogram over rows <
 * m_detected).  The draws are the same as bs_sample_ex's for the same
 * arguments.  Errors as bs_sample_ex, and BS_EINVAL when rows_out is NULL. */
int bs_sample_trace(bs_ctx* ctx, const bs_c128* U, int m_rows, int m_cols, int ld, const int* input_occupation,
                    int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out, int* rows_out);

/* Device-pointer form of bs_sample_ex: U_dev and out_dev on the device,
 * input_occupation on the host.  Enqueued; valid after bs_ctx_sync(). */
int bs_sample_dev(bs_ctx* ctx, const bs_c128* U_dev, int m_rows, int m_cols, int ld, const int* input_occupation,
                  int n_samples, uint64_t seed, int m_detected, bs_mode mode, int* out_dev);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of requests from many clients          */
/* ------------------------------------------------------------------ */

/* A server owns one device memory block of mem_budget_bytes (the admission
 * budget), a stream and a scheduler thread.  Requests (permanents or Laplace
 * minors, as bs_perm / bs_laplace_minors, and whole Clifford & Clifford
 * samples, bs_server_submit_sample) are admitted in arrival order while
 * one of max_active slots is free and their device memory fits the budget;
 * every scheduling tick walks a share of tick_tasks warp tasks of every
 * resident request in one launch per kernel group, so requests arriving
 * while others run are admitted at the next tick and their work overlaps on
 * the device (iteration-level scheduling).  Results are bit-identical to
 * running each request alone.  mode: BS_FP64, BS_DF64 or BS_MIXED (per-job
 * precision rule as for bs_perm).  Every entry point may be called from any
 * host thread.  Errors: BS_EINVAL, BS_ENODEV, BS_ENOMEM. */
typedef struct bs_server bs_server;
int bs_server_create(bs_server** out, int device, size_t mem_budget_bytes, int max_active, int tick_tasks,
                     bs_mode mode);
/* Stops the scheduler (after its current tick) and frees everything; pending
 * requests are dropped.  No other call on this server may be in progress or
 * follow (a thread blocked in a wait must have returned). */
void bs_server_destroy(bs_server* server);

/* Submits a request (kind 0: permanent, 1: minors; host arrays, copied
 * before returning).  Returns a ticket >= 0, or a negative BS_E* code. */
int64_t bs_server_submit(bs_server* server, int kind, const bs_c128* A, int rows, int cols, int ld,
                         const int* row_mult, const int* col_mult);

/* bs_server_poll: 1 and the result (1 value, or cols minors) when the request
 * is done, 0 while pending, negative on error.  bs_server_wait blocks until
 * done and returns BS_OK.  Either releases the ticket once it returns a
 * result.  latency_s (nullable): submit-to-completion time. */
int bs_server_poll(bs_server* server, int64_t ticket, bs_c128* out, int out_len, double* latency_s);
int bs_server_wait(bs_server* server, int64_t ticket, bs_c128* out, int out_len, double* latency_s);

/* A sampling request: one Clifford & Clifford chain (one sample, Sec. 4)
 * served by the engine.  U is m_rows x m_cols (row-major, leading dimension
 * ld, copied before returning), one input occupation per column; rows >=
 * m_detected are loss modes (m_detected <= 0: all rows counted).  The
 * chain's interferometer, permuted inputs and drawn rows stay on the device;
 * each step's minors job (planned on the device) joins the shared walk
 * launches of the next tick, and the row r_k is drawn on the device with the
 * random numbers of bs_sample: sample `sample` of `seed` gives exactly the
 * counts of sample `sample` of bs_sample / bs_sample_ex with that seed and the
 * server's mode.  Returns a ticket >= 0, or a negative BS_E* code. */
int64_t bs_server_submit_sample(bs_server* server, const bs_c128* U, int m_rows, int m_cols, int ld,
                                const int* input_occupation, uint64_t seed, uint64_t sample, int m_detected);
/* 1 and the occupation counts (m_detected ints) when the chain is done, 0
 * while pending, negative on error (BS_ECANCELED after bs_server_cancel);
 * the wait form blocks.  Either releases the ticket once it returns a
 * result. */
int bs_server_poll_sample(bs_server* server, int64_t ticket, int* counts, int len, double* latency_s);
int bs_server_wait_sample(bs_server* server, int64_t ticket, int* counts, int len, double* latency_s);

/* Cancels a pending request (any kind).  A request still waiting for
 * admission is dropped at once; an admitted one is released after the
 * current tick, when none of its kernels is in flight.  Its waiter then
 * receives BS_ECANCELED.  Errors: BS_EINVAL (unknown or finished ticket). */
int bs_server_cancel(bs_server* server, int64_t ticket);

typedef struct {
    uint64_t submitted, completed, ticks, walk_launches;
    double busy_s;            /* time spent in ticks */
    double p50_ms, p99_ms, max_ms;  /* submit-to-completion latency of completed requests */
    int max_resident;         /* largest number of requests resident at once */
    size_t mem_peak_bytes;    /* peak bytes of the budget in use */
    size_t mem_in_use_bytes;  /* bytes of the budget in use now (requests and a tick's descriptors) */
    int resident, waiting;    /* requests admitted / waiting for admission now */
    uint64_t cancelled;       /* requests ended by bs_server_cancel */
} bs_server_stats;
int bs_server_get_stats(bs_server* server, bs_server_stats* out);

/* ------------------------------------------------------------------ */
/* Measurement and diagnostics                                         */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t walk_launches;     /* walk kernels launched */
    uint64_t kernel_launches;   /* all kernels this context launched */
    uint64_t addends[3];        /* Gray-walk addends evaluated: [FP64, FP32, double-float kernels] */
    uint64_t addend_flops[3];   /* algorithmic flops of those addends */
    double walk_ms[3];          /* summed walk-kernel time (profiling on) */
    uint64_t timed_launches[3]; /* walk launches included in walk_ms */
} bs_stats;

/* Sampling and batches replay their kernel sequence from a captured CUDA
 * graph (re-captured when shapes, buffers, deadline, stream or the profiling
 * switch change) when on != 0 (the default); 0 launches every kernel
 * directly.  With profiling on, a sampling graph carries the walk timing
 * events (read before its next replay); batches then launch directly. */
int bs_ctx_set_graphs(bs_ctx* ctx, int on);

/* Record CUDA events around every walk launch (on its stream) when on != 0;
 * bs_ctx_get_stats() then reports their summed durations.  A profiled
 * sampling graph replay waits for the previous replay's events before it is
 * launched. */
int bs_ctx_set_profiling(bs_ctx* ctx, int on);

/* Durations (ms) of the walk launches timed since the last call, oldest
 * first; at most max_entries are written, the number available is returned
 * (or a negative error).  Waits for the context's stream. */
int bs_ctx_get_walk_times(bs_ctx* ctx, double* ms_out, int max_entries);
int bs_ctx_get_stats(bs_ctx* ctx, bs_stats* out);
int bs_ctx_reset_stats(bs_ctx* ctx);

/* Measured lane-FMA issue rates of the FP64 and FP32 pipes of this device
 * (operations per second, 1 FMA = 2 flops), from a timed microbenchmark. */
int bs_measure_fma_rates(bs_ctx* ctx, double* fp64_fma_per_s, double* fp32_fma_per_s);

/* Host-only check of the n-ary reflected Gray counter the kernels use: walks
 * `steps` moves from index `start` over digits with the given radices (the
 * first nbin must be 2) and writes the Delta vector after every move to
 * deltas (steps x ndigits), the moved digit to moved (steps), and the binomial
 * weight to weights (steps).  Returns BS_EINVAL on bad radices. */
int bs_debug_gray_walk(int ndigits, int nbin, const int* radix, uint64_t start, int steps, int* deltas,
                       int* moved, uint64_t* weights);

/* Host-only planner summary for a permanent (kind 0) or minors (kind 1)
 * problem (info holds 8 entries): info[0] = addends C, info[1] = digit rows,
 * info[2] = binary digits, info[3] = product columns, info[4] = 1 if
 * transposed, info[5] = pinned source row, info[6] = log2 of the chunk length
 * and info[7] = warp tasks when the job runs alone in FP64 mode.  Returns
 * BS_EINVAL on invalid multiplicities. */
int bs_debug_plan(int rows, int cols, const int* row_mult, const int* col_mult, int kind, int64_t* info);

/* Host-only view of the BS_MIXED precision rule for a permanent (kind 0) or
 * minors (kind 1) problem: *log2_err receives the predicted log2 of the
 * FP32 walk's error relative to prod_j ||a_j||^{N_j} for FP32 chunks of
 * 2^chunk_log2 addends (chunk_log2 <= 0: the chunk length of the problem
 * planned alone), *log2L (nullable) that chunk exponent, *plan (nullable)
 * the decision at the default tolerance 1e-6: 1 FP32, 2 FP32 with the column
 * sums re-seeded from the matrix every 2^8 steps inside each chunk (the
 * prediction without its drift term meets the tolerance), 0 the fallback
 * kernels.  Returns BS_EINVAL on invalid multiplicities. */
int bs_debug_mixed_error(int rows, int cols, const int* row_mult, const int* col_mult, int kind, int chunk_log2,
                         double* log2_err, int* log2L, int* plan);

#ifdef __cplusplus
}
#endif

#endif /* BS_H */
