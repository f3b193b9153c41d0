// Double-float walk kernels (walk_df.cuh): permanents and fused Laplace
// minors with FP64-class accuracy on the FP32 pipe.  One instantiation per
// 8-column bucket (K in (KB - 8, KB]); persistent grids pull warp tasks from
// an atomic counter, as the FP64 and FP32 kernels do.
#include "kernels.h"
#include "walk_df.cuh"

namespace bs {

constexpr int kDfBlock = 128;

template <int KB>
__global__ void __launch_bounds__(kDfBlock) walk_df_perm_kernel(WalkArgs a) {
    const int lane = threadIdx.x & 31;
    const bs_job* __restrict__ jobs = a.jobs;
    const unsigned long long total = task_total(a);
    const int njobs = job_count(a);
    const unsigned long long deadline = warp_deadline(a.deadline_rel_ns);
    for (;;) {
        unsigned long long t = next_task(a.counter, total, a.status, deadline, lane);
        if (t >= total) break;
        const bs_job jb = jobs[find_job(jobs, a.job_list, njobs, t)];
        if (((jb.K + 7) >> 3) != KB / 8 || jb.kind != BS_KIND_PERM) {
            if (lane == 0) atomicExch(a.status, BS_STATUS_BADJOB);
            continue;
        }
        walk_task_perm_df<KB>(jb, a.data, a.meta + BS_META_RADIX(jb), a.partials,
                              (uint32_t)(t - jb.task_begin) + jb.task_offset, lane);
    }
}

// Resident CTAs per SM the fused-minor kernel is compiled for (register
// cap 65536 / (128 x value)): 3 at widths 24 and 48 (three pairs per lane,
// no spill at 168 registers; width 24 measured 8 % faster than uncapped), 1
// (no cap) elsewhere (widths 16, 32 and 40 spill at 168 registers; width 32
// measured 4 % slower with the cap).  A build may override it for every
// width with -DBS_DF_MINORS_MIN_BLOCKS=n to time the alternatives.
template <int KB>
struct DfMinorsMinBlocks {
#ifdef BS_DF_MINORS_MIN_BLOCKS
    static constexpr int value = BS_DF_MINORS_MIN_BLOCKS;
#else
    static constexpr int value = (KB == 24 || KB == 48) ? 3 : 1;
#endif
};

template <int KB>
__global__ void __launch_bounds__(kDfBlock, DfMinorsMinBlocks<KB>::value) walk_df_minors_kernel(WalkArgs a) {
    extern __shared__ float4 smem_df[];
    const int lane = threadIdx.x & 31;
    const int stride = blockDim.x;
    // [column][thread] double-float sums, then [column][thread] staging
    float4* sm = smem_df + threadIdx.x;
    float4* stage = smem_df + (size_t)(KB / BS_DF_GROUP_KB(KB)) * stride + threadIdx.x;
    const bs_job* __restrict__ jobs = a.jobs;
    const unsigned long long total = task_total(a);
    const int njobs = job_count(a);
    const unsigned long long deadline = warp_deadline(a.deadline_rel_ns);
    for (;;) {
        unsigned long long t = next_task(a.counter, total, a.status, deadline, lane);
        if (t >= total) break;
        const bs_job jb = jobs[find_job(jobs, a.job_list, njobs, t)];
        if (((jb.K + 7) >> 3) != KB / 8 || jb.kind != BS_KIND_MINORS) {
            if (lane == 0) atomicExch(a.status, BS_STATUS_BADJOB);
            continue;
        }
        walk_task_minors_df<KB>(jb, a.data, a.meta + BS_META_RADIX(jb), a.partials,
                                (uint32_t)(t - jb.task_begin) + jb.task_offset, lane, sm, stage, stride);
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
    int grid = persistent_grid(walk_df_perm_kernel<KB>, kDfBlock, 0, a);
    walk_df_perm_kernel<KB><<<grid, kDfBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KB>
static cudaError_t run_minors(const WalkArgs& a, cudaStream_t s) {
    // per owned column and thread: a float4 fold slot and a float4 staging slot
    const size_t smem = (size_t)kDfBlock * (KB / BS_DF_GROUP_KB(KB)) * 2 * sizeof(float4);
    cudaError_t e =
        cudaFuncSetAttribute(walk_df_minors_kernel<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = persistent_grid(walk_df_minors_kernel<KB>, kDfBlock, smem, a);
    walk_df_minors_kernel<KB><<<grid, kDfBlock, smem, s>>>(a);
    return cudaGetLastError();
}

#define BS_DF_B48(X) X(1, 8) X(2, 16) X(3, 24) X(4, 32) X(5, 40) X(6, 48)

// a.max_K selects the 8-column bucket: every job of the launch must share it.
cudaError_t launch_walk_df_perm(const WalkArgs& a, cudaStream_t s) {
    if (a.total_tasks == 0 && !a.total_dev) return cudaSuccess;
    switch ((a.max_K + 7) >> 3) {
#define BS_CASE(b, kb) \
    case b: return run_perm<kb>(a, s);
        BS_DF_B48(BS_CASE)
#undef BS_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_walk_df_minors(const WalkArgs& a, cudaStream_t s) {
    if (a.total_tasks == 0 && !a.total_dev) return cudaSuccess;
    switch ((a.max_K + 7) >> 3) {
#define BS_CASE(b, kb) \
    case b: return run_minors<kb>(a, s);
        BS_DF_B48(BS_CASE)
#undef BS_CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace bs
