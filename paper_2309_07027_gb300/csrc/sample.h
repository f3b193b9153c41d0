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
// Warp tasks below which a job planned alone is latency-bound (its walk
// time is one lane's chunk); see bs_choose_log2L_single.
#define BS_TARGET_TASKS_FILL 256
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
// BS_TARGET_TASKS_FILL tasks at that floor gets shorter chunks (down to the
// 2^3 floor of the sampler) until it does: such a job is latency-bound, and
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
    if (fill < BS_LOG2L_MIN_MANY) fill = BS_LOG2L_MIN_MANY;
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
BS_HD int bs_chunks_per_task(int kind, int fp32, int K) {
    if (kind != BS_KIND_MINORS) return 32;
    return fp32 ? 32 / bs_minors_fp32_group(K) : 16;  // FP64 minors: lane pairs
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

// MIXED-mode precision rule.  FP32 rounding gives each addend a relative
// error of about K 2^-24, amplified by up to sqrt(M) where a column sum of a
// repeated row cancels; the addends' root-sum-square is about
// 2^(1-n) sqrt(prod_j C(2 M_j, M_j)) times prod_col ||a_col|| (Vandermonde:
// sum_D C(M, D)^2 = C(2M, M)), so the predicted error relative to the MIXED
// tolerance scale prod_col ||a_col|| is
//   log2 K + log2(2n)/2 + log2(max M)/2 - 24 + (1 - n)
//     + sum_j log2 C(2 M_j, M_j) / 2 + 2        (safety factor 4).
// The job runs in FP32 when that is <= log2(1e-6), else in FP64 ("FP64 ...
// at large k, where cancellation demands it").  Depends only on the
// multiplicities, K and n, so every planner decides alike.
BS_HD int bs_mixed_uses_fp32(const int* radix, int nrows, int K, int n) {
    float lg = log2f((float)(K > 1 ? K : 1)) + 0.5f * log2f(2.0f * (float)(n > 1 ? n : 1)) - 24.0f +
               (1.0f - (float)n) + 2.0f;
    int mmax = 1;
    for (int j = 0; j < nrows; ++j) {
        const int M = radix[j] - 1;
        if (M > mmax) mmax = M;
        for (int t = 1; t <= M; ++t) lg += 0.5f * log2f((float)(M + t) / (float)t);
    }
    lg += 0.5f * log2f((float)mmax);
    return lg <= -19.93f;
}

namespace bs {

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
    unsigned long long* total;    // device task totals [FP64, FP32]
    unsigned long long* counter;  // device work counters [FP64, FP32]
    unsigned long long* stats;    // device [addends64, flops64, addends32, flops32]
    int* lists;                   // device job lists: [FP64: S][FP32: S]
    int* list_len;                // device list lengths [FP64, FP32]
    int* out;                     // device, S x m_det
    int64_t meta_stride, data_stride, tasks_stride;
    int mixed;                    // 1: MIXED mode (per-chain FP32 / FP64 rule)
    int log2max64, log2max32;
};

cudaError_t launch_cc_init(const CcArgs& a, const CcArgs* da, cudaStream_t st);
cudaError_t launch_cc_plan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_scan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_draw(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st);
cudaError_t launch_cc_counts(const CcArgs& a, const CcArgs* da, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int count, cudaStream_t s);

}  // namespace bs
