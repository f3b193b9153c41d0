// FP32 ("mixed") walk kernels: column sums and products in single precision,
// re-seeded from the matrix at every chunk start; addends summed in short
// single-precision runs folded into float-float, chunk totals combined in
// double-double.  Column sums are packed pairs (walk_fp32.cuh).  Minors split
// each chunk's column pairs over 2 or 4 lanes (16 or 8 chunks per warp task).
// One instantiation per column bucket.
#include "kernels.h"
#include "walk_fp32.cuh"

namespace bs {

constexpr int kPermBlock = 128;
constexpr int kMinorsBlock = 128;


// CTAs per SM the permanent kernel is compiled for, by bucket width (the
// register budgets the measured kernels ran at: 96 registers at widths 20
// and 24, 128 at 28..40, 168 above; 80 and less below 20).
template <int KB>
struct PermMinBlocks {
    static constexpr int value = KB <= 8 ? 8 : KB <= 12 ? 7 : KB <= 16 ? 6 : KB <= 24 ? 5 : KB <= 40 ? 4 : 3;
};

template <int KB>
__global__ void __launch_bounds__(kPermBlock, PermMinBlocks<KB>::value) walk_fp32_perm_kernel(WalkArgs a) {
    const int lane = threadIdx.x & 31;
    const bs_job* __restrict__ jobs = a.jobs;
    const unsigned long long total = task_total(a);
    const int njobs = job_count(a);
    const unsigned long long deadline = warp_deadline(a.deadline_rel_ns);
    for (;;) {
        unsigned long long t = next_task(a.counter, total, a.status, deadline, lane);
        if (t >= total) break;
        const bs_job jb = jobs[find_job(jobs, a.job_list, njobs, t)];
        if (((jb.K + 3) >> 2) != KB / 4 || jb.kind != BS_KIND_PERM) {
            if (lane == 0) atomicExch(a.status, BS_STATUS_BADJOB);
            continue;
        }
        walk_task_perm_fp32<KB>(jb, a.data, a.meta + BS_META_RADIX(jb), a.partials, (uint32_t)(t - jb.task_begin) + jb.task_offset,
                                  lane);
    }
}

// Resident CTAs per SM the fused-minor kernel is compiled for: the count
// that measured fastest.  4-lane groups: width 24 at 96 registers, 5 CTAs;
// width 48 left to the compiler (232 registers, 2 CTAs).  2-lane groups: up
// to 20 columns 128 registers, 4 CTAs; 28 and 32 columns 168 registers, 3
// CTAs (8 and 132 bytes spilled, outside the inner loop by the timings: at
// 2 CTAs the k = 25..28 sampler steps are 15-18 % and the k = 29, 30 steps
// 12 % slower); 36 to 44 columns 2 CTAs.
template <int KB>
struct MinorsMinBlocks {
    static constexpr int G = BS_MINORS_FP32_GROUP_KB(KB);
    static constexpr int NP = KB / (2 * G);
    static constexpr int value = G == 4 ? (NP <= 3 ? 5 : 1) : (KB <= 20 ? 4 : (KB <= 32 ? 3 : 2));
};

template <int KB>
__global__ void __launch_bounds__(kMinorsBlock, MinorsMinBlocks<KB>::value) walk_fp32_minors_kernel(WalkArgs a) {
    extern __shared__ float4 smem_fp32[];
    const int lane = threadIdx.x & 31;
    const int stride = blockDim.x;
    float4* sm_ff = smem_fp32 + threadIdx.x;
    const bs_job* __restrict__ jobs = a.jobs;
    const unsigned long long total = task_total(a);
    const int njobs = job_count(a);
    const unsigned long long deadline = warp_deadline(a.deadline_rel_ns);
    for (;;) {
        unsigned long long t = next_task(a.counter, total, a.status, deadline, lane);
        if (t >= total) break;
        const bs_job jb = jobs[find_job(jobs, a.job_list, njobs, t)];
        if (((jb.K + 3) >> 2) != KB / 4 || jb.kind != BS_KIND_MINORS) {
            if (lane == 0) atomicExch(a.status, BS_STATUS_BADJOB);
            continue;
        }
        walk_task_minors_fp32<KB>(jb, a.data, a.meta + BS_META_RADIX(jb), a.partials, (uint32_t)(t - jb.task_begin) + jb.task_offset,
                                  lane, sm_ff, stride);
    }
}

template <typename Kern>
static int persistent_grid(Kern k, int block, size_t smem, const WalkArgs& a) {
    int dev = 0;
    cudaGetDevice(&dev);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)per_sm * sm_count(dev);
    if (!a.total_dev) {
        long long need = ((long long)a.total_tasks * 32 + block - 1) / block;
        if (need < grid) grid = need;
    }
    if (a.grid_cap > 0 && grid > a.grid_cap) grid = a.grid_cap;
    if (grid < 1) grid = 1;
    return (int)grid;
}

template <int KB>
static cudaError_t run_perm(const WalkArgs& a, cudaStream_t s) {
    int grid = persistent_grid(walk_fp32_perm_kernel<KB>, kPermBlock, 0, a);
    walk_fp32_perm_kernel<KB><<<grid, kPermBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KB>
static cudaError_t run_minors(const WalkArgs& a, cudaStream_t s) {
    size_t smem = (size_t)kMinorsBlock * (KB / BS_MINORS_FP32_GROUP_KB(KB)) * sizeof(float4);
    cudaError_t e =
        cudaFuncSetAttribute(walk_fp32_minors_kernel<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = persistent_grid(walk_fp32_minors_kernel<KB>, kMinorsBlock, smem, a);
    walk_fp32_minors_kernel<KB><<<grid, kMinorsBlock, smem, s>>>(a);
    return cudaGetLastError();
}

#define BS_B48(X) X(1, 4) X(2, 8) X(3, 12) X(4, 16) X(5, 20) X(6, 24) X(7, 28) X(8, 32) X(9, 36) X(10, 40) X(11, 44) X(12, 48)

cudaError_t launch_walk_fp32_perm(const WalkArgs& a, cudaStream_t s) {
    if (a.total_tasks == 0 && !a.total_dev) return cudaSuccess;
    switch ((a.max_K + 3) >> 2) {
#define BS_CASE(b, kb) \
    case b: return run_perm<kb>(a, s);
        BS_B48(BS_CASE)
#undef BS_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_walk_fp32_minors(const WalkArgs& a, cudaStream_t s) {
    if (a.total_tasks == 0 && !a.total_dev) return cudaSuccess;
    switch ((a.max_K + 3) >> 2) {
#define BS_CASE(b, kb) \
    case b: return run_minors<kb>(a, s);
        BS_B48(BS_CASE)
#undef BS_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace bs
