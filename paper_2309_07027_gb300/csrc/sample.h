// Shared rules of the host planner, the device planner and the sampler.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "bs_job.h"
#include "gray.h"
#include <math.h>

// Chunk length exponent of a job with C addends whose warp tasks cover `cpt`
// chunks: aim at about `target` tasks per job, never below 2^log2min addends
// per chunk (decode cost) nor above 2^log2max (the re-seed interval).
// Depends only on (C, cpt, log2min, log2max, target), so a job is cut the
// same way alone or inside any batch that uses the same rule.  Jobs planned
// one call at a time use BS_TARGET_TASKS_SINGLE (several tasks per resident
// warp, so one job fills the GPU without a ragged tail) and chunks of at
// least 2^6, shorter only for jobs too small to give 256 tasks
// (bs_choose_log2L_single).  The sampler and the server, which always run many jobs
// together, use BS_TARGET_TASKS_MANY (longer chunks, fewer tasks) with a
// floor of 2^3: their small jobs (early steps, heavy-collision chains sent to
// FP64) are latency-bound, and short chunks spread them over more warps.
#define BS_TARGET_TASKS_SINGLE 32768
// FP32 jobs planned one call at a time aim at fewer, longer chunks: the FP32
// walks are bound by the L1 delivery of rows, and every chunk start re-reads
// about half the rows (4096-item batch: 3.6 % faster than with 32768).
#define BS_TARGET_TASKS_SINGLE_FP32 8192
#define BS_TARGET_TASKS_MANY 64
#define BS_LOG2L_MIN_SINGLE 6
#define BS_LOG2L_MIN_MANY 3
// Floor for the tiniest jobs planned alone (at most BS_FILL_TINY_C
// addends): chunks of 2 addends.  Such a job's walk time is one warp's FP64
// instruction stream (one instruction per 64 cycles per scheduler on this
// part), and more, shorter chunks spread it over more warps; a chunk start
// decodes its index and seeds the column sums (about the work of one or two
// addends), so shorter chunks would only add work.  Larger small jobs keep
// the 2^3 floor: batches of them are throughput-bound, and there the extra
// seeding of 2-addend chunks cost more than it saved (a 64-item batch of
// k = 10..16 ran 19 % slower with the lower floor for every job).
#define BS_LOG2L_MIN_FILL 1
#define BS_FILL_TINY_C 1024
// Warp tasks below which a job planned alone is latency-bound (its walk
// time is one lane's chunk); see bs_choose_log2L_single.
#define BS_TARGET_TASKS_FILL 256
// Default cap of the chunk length (the re-seed interval) by precision:
// 2^11 addends for the FP64 and FP32 kernels, 2^12 for double-float.  The
// sampler's FP64 steps run about 1 % faster with 2^11 than with 2^12 (twice
// the tasks of its largest jobs, a shorter last wave per launch; 2^9..2^11
// measured alike), its MIXED steps 1.4 % (2^10: 7 % slower), while its
// double-float steps showed no difference between 2^11 and 2^13.  Jobs
// planned one call at a time rarely reach the cap.
BS_HD int bs_default_log2max(int prec) { return prec == BS_PREC_DF ? 12 : 11; }
BS_HD int bs_floor_log2(uint64_t x) {  // floor(log2(x)) for x >= 1, 0 for x = 0
    int l = 0;
    while ((2ull << l) <= x) ++l;
    return l;
}
BS_HD int bs_choose_log2L(uint64_t C, int cpt, int log2min, int log2max, int target) {
    const uint64_t per = C / ((uint64_t)cpt * (uint64_t)target);
    int l = bs_floor_log2(per);
    if (l < log2min) l = log2min;
    if (l > log2max) l = log2max;
    return l;
}
// The rule for jobs planned one call at a time: bs_choose_log2L with the
// single-call target and floor 2^6, except that a job too small to give
// BS_TARGET_TASKS_FILL tasks at that floor gets shorter chunks (down to 2^3,
// or 2^BS_LOG2L_MIN_FILL for the tiniest) until it does: such a job is
// latency-bound, and
// its walk time is one lane's chunk, not the total work (a 576-addend FP64
// job in one warp of 9 chunks of 64 runs at one scheduler's FP64 rate).
// 256 tasks keeps the re-seeding of mid-size jobs as it was: with 2048 (one
// resident wave) jobs of 2^19 to 2^21 addends also got shorter chunks and the
// 4096-item batch ran 5 % slower, for no gain on small calls.
BS_HD int bs_choose_log2L_single(uint64_t C, int cpt, int log2max, int target) {
    const int big = bs_choose_log2L(C, cpt, BS_LOG2L_MIN_SINGLE, log2max, target);
    if (big > BS_LOG2L_MIN_SINGLE) return big;
    int fill = bs_floor_log2(C / ((uint64_t)cpt * (uint64_t)BS_TARGET_TASKS_FILL));
    if (fill > BS_LOG2L_MIN_SINGLE) fill = BS_LOG2L_MIN_SINGLE;
    const int floor = C <= BS_FILL_TINY_C ? BS_LOG2L_MIN_FILL : BS_LOG2L_MIN_MANY;
    if (fill < floor) fill = floor;
    return fill > log2max ? log2max : fill;
}

// Lanes that walk one chunk together in the FP32 fused-minor kernel (each
// owns a contiguous group of the bucket's column pairs, so G divides KB / 2):
// 4 at widths 24 and 48, else 2.  Two lanes do less redundant exchange work
// per addend (one shuffle round instead of two, each lane's product chains
// twice as long) and measured faster wherever their registers allow 2-3
// CTAs per SM: widths 32 and 40 by 6-12 %; at 24 four lanes at 5 CTAs per SM
// are faster, and at 48 two lanes would spill.  A warp task of that kernel
// covers 32 / G chunks, one of the FP64 fused-minor kernel 16 (lane pairs);
// the permanent kernels give each lane its own chunk (32 per task).
#define BS_MINORS_FP32_GROUP_KB(KB) (((KB) == 24 || (KB) == 48) ? 4 : 2)
BS_HD int bs_minors_fp32_group(int K) { return BS_MINORS_FP32_GROUP_KB((K + 3) & ~3); }
// Lanes per chunk of the double-float kernels (permanent and minors), by
// 8-column bucket width KB: each lane owns KB / (2G) column pairs
// (8 -> 1 x 4, 16 -> 2 x 4, 24 -> 4 x 3, 32 -> 4 x 4, 40 -> 4 x 5,
// 48 -> 8 x 3), so a lane's double-float state fits its registers.
#define BS_DF_GROUP_KB(KB) ((KB) <= 8 ? 1 : (KB) <= 16 ? 2 : (KB) <= 40 ? 4 : 8)
BS_HD int bs_df_group(int K) { return BS_DF_GROUP_KB((K + 7) & ~7); }
BS_HD int bs_chunks_per_task(int kind, int prec, int K) {
    if (prec == BS_PREC_DF) return 32 / bs_df_group(K);
    if (kind != BS_KIND_MINORS) return 32;
    return prec == BS_PREC_FP32 ? 32 / bs_minors_fp32_group(K) : 16;  // FP64 minors: lane pairs
}

// Algorithmic flops of one addend (the roofline numerator):
//   permanent: column update 2K + product 6(K-1) + weighted accumulate 4
//   minors:    column update 2K + suffix and prefix products 12(K-2) + 2
//              + per-column product-accumulate 8K
BS_HD int64_t bs_flops_per_addend(int K, int kind) {
    if (kind == BS_KIND_PERM) return 8 * (int64_t)K - 2;
    int64_t kk = K < 2 ? 2 : K;
    return 2 * (int64_t)K + 12 * (kk - 2) + 2 + 8 * (int64_t)K;
}

// MIXED-mode precision rule: the predicted log2 of the FP32 walk's error
// relative to the MIXED tolerance scale prod_j ||a_j||^{N_j} (column norms
// over the rows repeated by their multiplicities).
//
// Model.  With the entries of a column of comparable magnitude
// (|a_kj|^2 ~ ||a_j||^2 / n), the column sum of the addend with Delta vector D
// has |c_j(D)|^2 ~ ||a_j||^2 Q(D) / n, Q(D) = sum over rows of (M_k - 2 D_k)^2,
// so the root-sum-square of the weighted addends is
//   RSS / prod_j ||a_j|| = 2^(1-n) sqrt( sum_D prod_k C(M_k, D_k)^2 (Q(D)/n)^K )
// (the pinned row: coefficient M_p - 2D for D in [0, M_p), weight
// C(M_p - 1, D)).  A heavily repeated row enters through its extreme D,
// whose coefficients +-M make those addends large though their weights are
// small.  Each addend carries a relative rounding error of about
// sqrt(K) 2^-24, and the incremental column sums drift like sqrt(steps)
// within a chunk of 2^log2L addends, so
//   log2 err ~ log2(RSS / prod ||a_j||) + log2(K)/2
//              + max(0, log2L - 8)/2 + c,
// c = -22.02 being the largest residual of that form over 724 measured FP32
// jobs (K = 10..40, multiplicities 1..8, chunks 2^3..2^12, errors against
// the FP64 kernels on Haar-random inputs), plus one bit of margin.  The sum
// over D is a dynamic program over Q: binary rows add 1 to Q with weight 2
// (two values of D); every other row adds (top - 2D)^2 with weight C(.,D)^2.
// The model assumes unstructured inputs; matrices with many exact zeros
// (block structure) cancel far more than it predicts and belong in FP64.
#define BS_MIXED_LOG2_TOL_DEFAULT (-19.93f)  // log2(1e-6)
// Kernels of the MIXED jobs that fail the FP32 rule: the double-float
// kernels (errors about 2^-46 relative, far inside the MIXED tolerance, at
// about 5x the FP64 kernels' speed on this part).
#define BS_MIXED_FALLBACK_PREC BS_PREC_DF
#define BS_MIXED_QMAX (BS_MAX_PHOTONS * BS_MAX_PHOTONS)  // Q <= sum M_k^2 <= n^2
#define BS_MIXED_RESIDUAL (-21.02)
// Chunks up to 2^8 addends show no drift term in the measured errors; FP32
// jobs that need it re-seed their column sums from the matrix every 2^8
// steps inside a chunk, which keeps them within that length.
#define BS_FP32_RESEED_LOG2 8

// x^K by repeated squaring (K >= 0): plain multiplications, so host and
// device compute the same value, far cheaper than pow() on the FP64 pipe.
BS_HD double bs_ipow(double x, int K) {
    double r = 1.0;
    while (K > 0) {
        if (K & 1) r *= x;
        x *= x;
        K >>= 1;
    }
    return r;
}

// q_work: BS_MIXED_QMAX + 1 doubles of scratch.  radix / nrows: the job's
// digits; pinned_m: multiplicity of the pinned row (its other pinned_m - 1
// copies are the digit of radix pinned_m when pinned_m > 1); log2L: the
// chunk length the FP32 kernel would use for the job.
BS_HD float bs_mixed_log2_error(const int* radix, int nrows, int pinned_m, int K, int n, int log2L,
                                double* q_work) {
    if (n <= 0) return -1000.0f;
    double* f = q_work;
    f[0] = 1.0;
    int qmax = 0, nb = 0;
    int off = pinned_m <= 1 ? 1 : 0;  // a lone pinned copy: coefficient 1
    bool pin_seen = pinned_m <= 1;
    for (int j = 0; j < nrows; ++j) {
        const int M = radix[j] - 1;
        const bool pin = !pin_seen && radix[j] == pinned_m;
        if (pin) pin_seen = true;
        if (!pin && M == 1) {
            ++nb;
            continue;
        }
        const int top = pin ? pinned_m : M;  // largest |coefficient|
        const int dmax = pin ? pinned_m - 1 : M;
        const int add = top * top;
        if (qmax + add > BS_MIXED_QMAX) return 1000.0f;  // outside the model: FP64
        // the row's squared weights C(dmax, d)^2 and squared coefficients,
        // once per row (dmax <= 48; exact integers below 2^53)
        double w2[BS_MAX_PHOTONS + 1];
        int sq[BS_MAX_PHOTONS + 1];
        uint64_t b = 1;
        for (int d = 0; d <= dmax; ++d) {
            if (d > 0) b = b * (uint64_t)(dmax - d + 1) / (uint64_t)d;
            w2[d] = (double)b * (double)b;
            sq[d] = (top - 2 * d) * (top - 2 * d);
        }
        for (int q = qmax + add; q >= 0; --q) {
            double acc = 0.0;
            for (int d = 0; d <= dmax; ++d) {
                const int src = q - sq[d];
                if (src < 0 || src > qmax) continue;
                acc += f[src] * w2[d];
            }
            f[q] = acc;
        }
        qmax += add;
    }
    double total = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (int q = 0; q <= qmax; ++q)
        if (f[q] != 0.0) total += f[q] * bs_ipow((double)(q + off + nb) * inv_n, K);
    if (!(total > 0.0)) return -1000.0f;
    const double lrss = (1.0 - (double)n) + 0.5 * (log2(total) + (double)nb);
    const double drift = log2L > BS_FP32_RESEED_LOG2 ? 0.5 * (double)(log2L - BS_FP32_RESEED_LOG2) : 0.0;
    return (float)(lrss + 0.5 * log2((double)(K > 1 ? K : 1)) + drift + BS_MIXED_RESIDUAL);
}

// The MIXED decision for a job the FP32 kernels would walk in chunks of
// 2^log2L addends, against log2_tol (default log2(1e-6)):
//   1  FP32 (predicted error <= log2_tol), column sums seeded at chunk starts;
//   2  FP32 with the column sums also re-seeded every 2^BS_FP32_RESEED_LOG2
//      steps (the prediction without the drift term is <= log2_tol) -- the
//      re-seeding bounds the drift of the incremental FP32 sums, at the cost
//      of one seed (about half the rows) per 2^8 steps;
//   0  neither: FP64-class arithmetic (BS_MIXED_FALLBACK_PREC: where
//      cancellation demands it, the column sums, products and sums keep
//      about 48 bits).
// Depends only on the multiplicities, K, n and the FP32 chunk length, so
// every planner with the same chunk rule decides alike.
BS_HD int bs_mixed_fp32_plan(const int* radix, int nrows, int pinned_m, int K, int n, int log2L, float log2_tol,
                             double* q_work) {
    const float e = bs_mixed_log2_error(radix, nrows, pinned_m, K, n, log2L, q_work);
    if (e <= log2_tol) return 1;
    if (log2L > BS_FP32_RESEED_LOG2 && e - 0.5f * (float)(log2L - BS_FP32_RESEED_LOG2) <= log2_tol) return 2;
    return 0;
}

namespace bs {

// The precision choice of a sampling step: bs_mode, the MIXED threshold and
// fallback, and the chunk-length caps by precision.
struct StepRule {
    int mode;
    float mixed_log2_tol;
    int mixed_fallback;
    int log2max[BS_NPREC];
};

struct CcArgs {
    int S;                        // chains (samples) in this batch
    int n;                        // photons
    int m_rows, m_det, ld;        // U rows, counted rows, leading dimension
    uint64_t seed;
    uint64_t sample_base;         // index of the first sample (RNG counter)
    const double2* U;             // device, m_rows x ld
    const int* inputs;            // device, n expanded input columns
    int* cols;                    // device, S x n permuted columns
    int* rows;                    // device, S x n drawn rows
    bs_job* jobs;                 // device, S
    int* meta;                    // device, S x meta_stride
    void* data;                   // device arena (double or float complex)
    bs_zdd* partials;             // device, S x tasks_stride x n
    double2* minors;              // device, S x n
    unsigned long long* total;    // device task totals, one per precision (BS_PREC_*)
    unsigned long long* counter;  // device work counters, one per precision
    unsigned long long* stats;    // device [addends, flops] per precision
    int* lists;                   // device job lists, S per precision
    int* list_len;                // device list lengths, one per precision
    int* out;                     // device, S x m_det
    int* trace;                   // device, S x n drawn rows in draw order (nullable)
    int64_t meta_stride, data_stride, tasks_stride;
    int mode;                     // bs_mode: FP64, MIXED (per-chain rule) or DF64
    float mixed_log2_tol;         // the rule's threshold, log2 of the MIXED tolerance
    int mixed_fallback;           // MIXED: precision of the jobs that fail the rule
    int log2max64, log2max32, log2maxdf;
};

// One served Clifford & Clifford chain (one sample) resident in a server's
// device arena.  Offsets count from the arena base.
struct ChainDesc {
    const double2* U;       // m_rows x m_cols, leading dimension m_cols
    int m_rows, m_cols, m_det, n;
    uint64_t seed, sample;  // the Philox key and counter of the sample
    const int* inputs;      // n expanded input columns
    int* cols;              // n permuted columns
    int* rows;              // n drawn rows
    int* counts;            // m_det occupation counts (written after step n)
    bs_job* job;            // the chain's job descriptor
    int64_t meta_off;       // int units
    int64_t data_byte_off;  // bytes (16-byte aligned)
    int64_t partial_off;    // bs_zdd units
    int out_index;          // minors slot in the server's output block (double2 units)
    int k;                  // the step whose row is drawn now (1 = the first)
    StepRule rule;
};

// Fisher-Yates permutation of every chain's input columns (as cc_init).
cudaError_t launch_chain_init(const ChainDesc* d, int count, cudaStream_t st);
// For every chain: draw r_k from the step-k minors in minors_base +
// out_index (k >= 2), then plan and pack its step k + 1 minors job, or,
// after step n, write its occupation counts.  One CTA per chain.
cudaError_t launch_chain_advance(const ChainDesc* d, int count, int max_m_rows, void* arena,
                                 const double2* minors_base, cudaStream_t st);

cudaError_t launch_cc_init(const CcArgs& a, const CcArgs* da, cudaStream_t st);
cudaError_t launch_cc_plan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_scan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_draw(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_counts(const CcArgs& a, const CcArgs* da, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int count, cudaStream_t s);

}  // namespace bs
