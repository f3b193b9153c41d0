// Clifford & Clifford sampling on the device (Sec. 4; algorithm B of
// Clifford & Clifford, "The classical complexity of boson sampling", 2018).
//
// All n_samples chains advance in lockstep.  For step k = 1..n:
//   plan   (one CTA per chain) distinct rows drawn so far and their counts
//          become the row multiplicities of a minors job over the chain's
//          first k permuted input columns; pinned row = a row of smallest
//          count, binary digits first (Sec. 2.2); then the job is packed
//          from U (same packing as the permanent path);
//   scan   task offsets of all chains, task total, counter reset;
//   walk   one persistent fused-minors launch for every chain (walk.cuh);
//   reduce minors of every chain (fixed-order double-double);
//   draw   w_i = |sum_l U[i, col_l] minor_l|^2 for every output row i, and
//          r_k = the smallest i whose running FP64 sum (row order) exceeds
//          u * total, u uniform in [0, 1).
// Random numbers come from Philox4x32-10 (Salmon et al., SC'11) with key
// (seed low, seed high) and counter (sample low, sample high, purpose, index):
//   purpose 0, index j: Fisher-Yates swap of position j (j = n-1 .. 1) with
//            position floor(w0 (j + 1) / 2^32);
//   purpose 1, index k: u = ((w0 << 32 | w1) >> 11) 2^-53 for step k.
#include <cuda_runtime.h>
#include "kernels.h"
#include "pack.cuh"
#include "sample.h"
#include "walk.cuh"

namespace bs {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t x0 = hi1 ^ c[1] ^ k0;
        const uint32_t x2 = hi0 ^ c[3] ^ k1;
        c[0] = x0;
        c[1] = lo1;
        c[2] = x2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ void rng_words(uint64_t seed, uint64_t sample, uint32_t purpose, uint32_t index,
                                          uint32_t w[4]) {
    w[0] = (uint32_t)sample;
    w[1] = (uint32_t)(sample >> 32);
    w[2] = purpose;
    w[3] = index;
    philox4x32_10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__global__ void philox_kernel(const uint32_t* in, uint32_t* out, int count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint32_t c[4] = {in[6 * i], in[6 * i + 1], in[6 * i + 2], in[6 * i + 3]};
    philox4x32_10(c, in[6 * i + 4], in[6 * i + 5]);
    for (int t = 0; t < 4; ++t) out[4 * i + t] = c[t];
}

cudaError_t launch_philox(const uint32_t* in, uint32_t* out, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    philox_kernel<<<(count + 127) / 128, 128, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

// cols[s][0..n) = Fisher-Yates permutation of the expanded input columns.
__global__ void cc_init_kernel(const CcArgs* __restrict__ pa) {
    const CcArgs& a = *pa;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    int* cols = a.cols + (size_t)s * a.n;
    for (int j = 0; j < a.n; ++j) cols[j] = a.inputs[j];
    for (int j = a.n - 1; j >= 1; --j) {
        uint32_t w[4];
        rng_words(a.seed, a.sample_base + (uint64_t)s, 0u, (uint32_t)j, w);
        int t = (int)(((uint64_t)w[0] * (uint64_t)(j + 1)) >> 32);
        int tmp = cols[j];
        cols[j] = cols[t];
        cols[t] = tmp;
    }
}

// The step-k minors job of one chain, planned by one thread: the distinct
// rows drawn so far (rows[0..k-2]) and their counts become the row
// multiplicities of a minors job over the chain's first k permuted input
// columns; pinned row = a row of smallest count, binary digits first
// (Sec. 2.2); precision by the mode (MIXED: the FP32 rule with the chunk
// length the FP32 kernel would use).  Fills every job field but the offsets
// (set by the caller, except data_off, which depends on the precision and is
// left to the caller too) and writes the metadata at meta (= base +
// jb.meta_off).  Returns the precision.  Scratch arrays: BS_MAX_PHOTONS ints
// each, q_work BS_MIXED_QMAX + 1 doubles.
__device__ int plan_minors_step(const int* __restrict__ rows, const int* __restrict__ cols, int k, const StepRule& rule,
                                bs_job& jb, int* __restrict__ meta, int* urow, int* ucnt, int* drad, int* dsrc,
                                double* q_work) {
    int nu = 0;
    for (int t = 0; t < k - 1; ++t) {
        int r = rows[t], f = -1;
        for (int u = 0; u < nu; ++u)
            if (urow[u] == r) f = u;
        if (f >= 0)
            ucnt[f]++;
        else {
            urow[nu] = r;
            ucnt[nu] = 1;
            ++nu;
        }
    }
    int p = 0;
    for (int u = 1; u < nu; ++u)
        if (ucnt[u] < ucnt[p]) p = u;
    jb.kind = BS_KIND_MINORS;
    jb.K = k;
    jb.n = k - 1;
    jb.src_trans = 0;
    // digits: binary rows (count 1) in order of first appearance, then
    // repeated rows by increasing count (insertion sort)
    int nrows = 0;
    for (int u = 0; u < nu; ++u)
        if (u != p && ucnt[u] == 1) {
            drad[nrows] = 2;
            dsrc[nrows] = urow[u];
            ++nrows;
        }
    const int nbin = nrows;
    for (int u = 0; u <= nu; ++u) {
        int src, m;
        if (u < nu) {
            if (u == p || ucnt[u] == 1) continue;
            src = urow[u];
            m = ucnt[u];
        } else {
            if (ucnt[p] < 2) continue;
            src = urow[p];
            m = ucnt[p] - 1;
        }
        int pos = nrows;
        while (pos > nbin && drad[pos - 1] > m + 1) {
            drad[pos] = drad[pos - 1];
            dsrc[pos] = dsrc[pos - 1];
            --pos;
        }
        drad[pos] = m + 1;
        dsrc[pos] = src;
        ++nrows;
    }
    jb.nrows = nrows;
    jb.nbin = nbin;
    uint64_t C = 1;
    for (int j = 0; j < nrows; ++j) C *= (uint64_t)drad[j];
    int prec = rule.mode == 2 ? BS_PREC_DF : BS_PREC_FP64;
    jb.reseed_log2 = 0;
    if (rule.mode == 1) {
        const int l32 = bs_choose_log2L(C, bs_chunks_per_task(BS_KIND_MINORS, BS_PREC_FP32, k), BS_LOG2L_MIN_MANY,
                                        rule.log2max[BS_PREC_FP32], BS_TARGET_TASKS_MANY);
        const int plan = bs_mixed_fp32_plan(drad, nrows, ucnt[p], k, k - 1, l32, rule.mixed_log2_tol, q_work);
        prec = plan ? BS_PREC_FP32 : rule.mixed_fallback;
        jb.reseed_log2 = plan == 2 ? BS_FP32_RESEED_LOG2 : 0;
    }
    jb.prec = prec;
    jb.normalize = prec != BS_PREC_FP64 ? 1 : 0;
    const int cpt = bs_chunks_per_task(BS_KIND_MINORS, prec, k);
    for (int j = 0; j < nrows; ++j) {
        meta[j] = drad[j];
        meta[nrows + j] = dsrc[j];
    }
    for (int c = 0; c < k; ++c) meta[2 * nrows + c] = cols[c];
    meta[2 * nrows + 2 * k] = urow[p];
    jb.C = C;
    jb.log2L = bs_choose_log2L(C, cpt, BS_LOG2L_MIN_MANY, rule.log2max[prec], BS_TARGET_TASKS_MANY);
    jb.ntasks = (uint32_t)((C + ((uint64_t)cpt << jb.log2L) - 1) / ((uint64_t)cpt << jb.log2L));
    jb.task_begin = 0;
    return prec;
}

// Plan + pack the step-k minors job of every chain (one CTA per chain).
__global__ void cc_plan_kernel(const CcArgs* __restrict__ pa, int k) {
    const CcArgs& a = *pa;
    __shared__ int urow[BS_MAX_PHOTONS], ucnt[BS_MAX_PHOTONS];
    __shared__ int drad[BS_MAX_PHOTONS], dsrc[BS_MAX_PHOTONS];
    __shared__ bs_job sjb;
    __shared__ double q_work[BS_MIXED_QMAX + 1];  // the MIXED rule's scratch (thread 0)
    const int s = blockIdx.x;
    if (threadIdx.x == 0) {
        bs_job jb = {};  // every field not set here or by the planner is zero
        jb.meta_off = (int64_t)s * a.meta_stride;
        jb.partial_off = (int64_t)s * a.tasks_stride * a.n;
        jb.out_index = s * a.n;
        jb.src_off = 0;
        jb.src_ld = a.ld;
        const StepRule rule = {a.mode, a.mixed_log2_tol, a.mixed_fallback, {a.log2max64, a.log2max32, a.log2maxdf}};
        const int prec = plan_minors_step(a.rows + (size_t)s * a.n, a.cols + (size_t)s * a.n, k, rule, jb,
                                          a.meta + jb.meta_off, urow, ucnt, drad, dsrc, q_work);
        // the chain's data slot holds data_stride complex doubles; an FP32
        // job indexes it in complex floats (twice as many, same bytes), a DF
        // job in 16-byte units
        jb.data_off = (int64_t)s * a.data_stride * (prec == BS_PREC_FP32 ? 2 : 1);
        a.jobs[s] = jb;
        sjb = jb;
    }
    __syncthreads();
    pack_job(sjb, a.U, a.meta, a.data, sjb.prec, threadIdx.x, blockDim.x);
}

// Inclusive block scan of 64-bit values (Hillis-Steele, blockDim <= 1024).
__device__ unsigned long long block_scan(unsigned long long v, unsigned long long* buf) {
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        unsigned long long x = threadIdx.x >= (unsigned)off ? buf[threadIdx.x - off] : 0ull;
        __syncthreads();
        buf[threadIdx.x] += x;
        __syncthreads();
    }
    unsigned long long r = buf[threadIdx.x];
    __syncthreads();
    return r;
}

// One CTA: for each precision p (BS_PREC_*) the compacted list of
// chains walked by that kernel, their task offsets (exclusive scan of ntasks
// in list order), the task total, a zeroed work counter, and the addend /
// flop counters used for the roofline.
__global__ void cc_scan_kernel(const CcArgs* __restrict__ pa, int k) {
    const CcArgs& a = *pa;
    __shared__ unsigned long long buf[1024];
    __shared__ unsigned long long carry_t, carry_n, adds;
    for (int p = 0; p < BS_NPREC; ++p) {
        if (threadIdx.x == 0) {
            carry_t = 0;
            carry_n = 0;
            adds = 0;
        }
        __syncthreads();
        for (int base = 0; base < a.S; base += blockDim.x) {
            const int s = base + threadIdx.x;
            const bool mine = s < a.S && a.jobs[s].prec == p;
            const unsigned long long nt = mine ? a.jobs[s].ntasks : 0ull;
            if (mine) atomicAdd(&adds, (unsigned long long)a.jobs[s].C);
            const unsigned long long pos = block_scan(mine ? 1ull : 0ull, buf);
            const unsigned long long tsk = block_scan(nt, buf);
            if (mine) {
                a.lists[p * a.S + (int)(carry_n + pos - 1)] = s;
                a.jobs[s].task_begin = carry_t + tsk - nt;
            }
            __syncthreads();  // every thread has used the carries
            if (threadIdx.x == blockDim.x - 1) {
                carry_n += pos;
                carry_t += tsk;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            a.total[p] = carry_t;
            a.counter[p] = 0ull;
            a.list_len[p] = (int)carry_n;
            a.stats[2 * p] += adds;
            a.stats[2 * p + 1] += adds * (unsigned long long)bs_flops_per_addend(k, BS_KIND_MINORS);
        }
        __syncthreads();
    }
}

// r_k of one chain (the whole CTA; wts: m_rows doubles of shared memory):
// w_i = |sum_l U[i, col_l] minor_l|^2 for every output row i (minor = 1 at
// k = 1), then the smallest i whose running FP64 sum (row order) exceeds
// u * total, u from Philox (seed, sample, purpose 1, index k).  Thread 0
// returns the row (other threads return -1).
__device__ int draw_row(const double2* __restrict__ U, int ld, int m_rows, const int* __restrict__ cols, int k,
                        const double2* __restrict__ mn, uint64_t seed, uint64_t sample, double* wts) {
    for (int i = threadIdx.x; i < m_rows; i += blockDim.x) {
        double re = 0.0, im = 0.0;
        const double2* urow = U + (size_t)i * ld;
        for (int l = 0; l < k; ++l) {
            const double2 u = urow[cols[l]];
            const double2 m = (k == 1) ? make_double2(1.0, 0.0) : mn[l];
            re = __fma_rn(u.x, m.x, re);
            re = __fma_rn(-u.y, m.y, re);
            im = __fma_rn(u.x, m.y, im);
            im = __fma_rn(u.y, m.x, im);
        }
        wts[i] = __fma_rn(re, re, im * im);
    }
    __syncthreads();
    int pick = -1;
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (int i = 0; i < m_rows; ++i) total += wts[i];
        uint32_t w[4];
        rng_words(seed, sample, 1u, (uint32_t)k, w);
        const double u = (double)((((uint64_t)w[0] << 32) | (uint64_t)w[1]) >> 11) * 0x1.0p-53;
        const double target = u * total;
        double cdf = 0.0;
        for (int i = 0; i < m_rows; ++i) {
            cdf += wts[i];
            if (cdf > target) {
                pick = i;
                break;
            }
        }
        if (pick < 0)
            for (int i = m_rows - 1; i >= 0; --i)
                if (wts[i] > 0.0) {
                    pick = i;
                    break;
                }
        if (pick < 0) pick = 0;
    }
    return pick;
}

// Draw r_k for every chain (one CTA per chain).
__global__ void cc_draw_kernel(const CcArgs* __restrict__ pa, int k) {
    const CcArgs& a = *pa;
    extern __shared__ double wts[];
    const int s = blockIdx.x;
    const int pick = draw_row(a.U, a.ld, a.m_rows, a.cols + (size_t)s * a.n, k, a.minors + (size_t)s * a.n, a.seed,
                              a.sample_base + (uint64_t)s, wts);
    if (threadIdx.x == 0) a.rows[(size_t)s * a.n + (k - 1)] = pick;
}

// Occupation counts of every chain; with a trace buffer, also the drawn
// rows r_1..r_n in draw order.
__global__ void cc_counts_kernel(const CcArgs* __restrict__ pa) {
    const CcArgs& a = *pa;
    const int s = blockIdx.x;
    const int* rows = a.rows + (size_t)s * a.n;
    for (int i = threadIdx.x; i < a.m_det; i += blockDim.x) {
        int c = 0;
        for (int t = 0; t < a.n; ++t) c += rows[t] == i;
        a.out[(size_t)s * a.m_det + i] = c;
    }
    if (a.trace)
        for (int t = threadIdx.x; t < a.n; t += blockDim.x) a.trace[(size_t)s * a.n + t] = rows[t];
}

// ------------------------------------------------------------------ served chains
__global__ void chain_init_kernel(const ChainDesc* __restrict__ list, int count) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= count) return;
    const ChainDesc& d = list[c];
    for (int j = 0; j < d.n; ++j) d.cols[j] = d.inputs[j];
    for (int j = d.n - 1; j >= 1; --j) {
        uint32_t w[4];
        rng_words(d.seed, d.sample, 0u, (uint32_t)j, w);
        const int t = (int)(((uint64_t)w[0] * (uint64_t)(j + 1)) >> 32);
        const int tmp = d.cols[j];
        d.cols[j] = d.cols[t];
        d.cols[t] = tmp;
    }
}

__global__ void chain_advance_kernel(const ChainDesc* __restrict__ list, void* __restrict__ arena,
                                     const double2* __restrict__ minors_base) {
    extern __shared__ double wts[];
    __shared__ int urow[BS_MAX_PHOTONS], ucnt[BS_MAX_PHOTONS];
    __shared__ int drad[BS_MAX_PHOTONS], dsrc[BS_MAX_PHOTONS];
    __shared__ bs_job sjb;
    __shared__ double q_work[BS_MIXED_QMAX + 1];
    const ChainDesc& d = list[blockIdx.x];
    const int k = d.k;
    const int pick = draw_row(d.U, d.m_cols, d.m_rows, d.cols, k, minors_base + d.out_index, d.seed, d.sample, wts);
    if (threadIdx.x == 0) d.rows[k - 1] = pick;
    __syncthreads();
    if (k >= d.n) {
        for (int i = threadIdx.x; i < d.m_det; i += blockDim.x) {
            int cnt = 0;
            for (int t = 0; t < d.n; ++t) cnt += d.rows[t] == i;
            d.counts[i] = cnt;
        }
        return;
    }
    if (threadIdx.x == 0) {
        bs_job jb = {};
        jb.meta_off = d.meta_off;
        jb.partial_off = d.partial_off;
        jb.out_index = d.out_index;
        jb.src_off = 0;
        jb.src_ld = d.m_cols;
        const int prec = plan_minors_step(d.rows, d.cols, k + 1, d.rule, jb, static_cast<int*>(arena) + d.meta_off,
                                          urow, ucnt, drad, dsrc, q_work);
        jb.data_off = d.data_byte_off / (prec == BS_PREC_FP32 ? 8 : 16);
        *d.job = jb;
        sjb = jb;
    }
    __syncthreads();
    pack_job(sjb, d.U, static_cast<int*>(arena), arena, sjb.prec, threadIdx.x, blockDim.x);
}

cudaError_t launch_chain_init(const ChainDesc* d, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    chain_init_kernel<<<(count + 63) / 64, 64, 0, st>>>(d, count);
    return cudaGetLastError();
}

cudaError_t launch_chain_advance(const ChainDesc* d, int count, int max_m_rows, void* arena,
                                 const double2* minors_base, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_m_rows * sizeof(double);
    // static shared memory: the MIXED rule's scratch and the planner's arrays
    const size_t stat = (BS_MIXED_QMAX + 1) * sizeof(double) + 4 * BS_MAX_PHOTONS * sizeof(int) + sizeof(bs_job);
    if (smem + stat > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(chain_advance_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    chain_advance_kernel<<<count, 128, smem, st>>>(d, arena, minors_base);
    return cudaGetLastError();
}

// `a` is the host copy (launch shapes); `da` the same struct in device
// memory, which the kernels read (so a captured graph can be replayed with
// new seeds / offsets by rewriting *da).
cudaError_t launch_cc_init(const CcArgs& a, const CcArgs* da, cudaStream_t st) {
    if (a.S <= 0) return cudaSuccess;
    cc_init_kernel<<<(a.S + 127) / 128, 128, 0, st>>>(da);
    return cudaGetLastError();
}

cudaError_t launch_cc_plan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st) {
    cc_plan_kernel<<<a.S, 64, 0, st>>>(da, k);
    return cudaGetLastError();
}

cudaError_t launch_cc_scan(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st) {
    (void)a;
    cc_scan_kernel<<<1, 1024, 0, st>>>(da, k);
    return cudaGetLastError();
}

cudaError_t launch_cc_draw(const CcArgs& a, const CcArgs* da, int k, cudaStream_t st) {
    size_t smem = (size_t)a.m_rows * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(cc_draw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cc_draw_kernel<<<a.S, 128, smem, st>>>(da, k);
    return cudaGetLastError();
}

cudaError_t launch_cc_counts(const CcArgs& a, const CcArgs* da, cudaStream_t st) {
    cc_counts_kernel<<<a.S, 64, 0, st>>>(da);
    return cudaGetLastError();
}

}  // namespace bs
