// FP64 walk kernels: permanents and fused Laplace minors, every step in
// double precision (column sums, products, weights; compensated sums).
// One kernel per column bucket KB (K in (KB-4, KB]); the host groups jobs by
// bucket, so each kernel keeps its own register allocation.  Inside, each
// task runs the walk instance for its job's exact column count (permanents)
// or owned-column count (minors), so no dead bucket column costs FP64 slots.
#include "kernels.h"
#include "walk.cuh"

namespace bs {

constexpr int kPermBlock = 128;
constexpr int kMinorsBlock = 64;

template <int KB>
__global__ void __launch_bounds__(kPermBlock) walk_fp64_perm_kernel(WalkArgs a) {
    const int lane = threadIdx.x & 31;
    const bs_job* __restrict__ jobs = a.jobs;
    const cx<double>* __restrict__ data = static_cast<const cx<double>*>(a.data);
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
        const uint32_t local = (uint32_t)(t - jb.task_begin) + jb.task_offset;
        const int* radix = a.meta + BS_META_RADIX(jb);
        // the instance with the job's exact column count (K in (KB-4, KB])
        switch (jb.K - (KB - 4)) {
            case 1: walk_task_perm_fp64<KB, KB - 3>(jb, data, radix, a.partials, local, lane); break;
            case 2: walk_task_perm_fp64<KB, KB - 2>(jb, data, radix, a.partials, local, lane); break;
            case 3: walk_task_perm_fp64<KB, KB - 1>(jb, data, radix, a.partials, local, lane); break;
            default: walk_task_perm_fp64<KB, KB>(jb, data, radix, a.partials, local, lane); break;
        }
    }
}

// Resident CTAs per SM the fused-minor kernel is compiled for (64 threads
// each).  Two walk instances inlined into one kernel raise the compiler's
// register choice (width 32: 168 -> 216, 6 -> 4 CTAs per SM), so the kernel
// keeps the budgets its one-instance form ran at, with no spills: 168
// registers (6 CTAs) at widths 24 to 32, 128 (8) at 16 and 20, 96 (10) at 8
// and 12, 72 (14) at 4, and the compiler's choice (4 CTAs) above 32.
template <int KB>
struct MinorsMinBlocks {
    static constexpr int value = KB <= 4 ? 14 : KB <= 12 ? 10 : KB <= 20 ? 8 : KB <= 32 ? 6 : 4;
};

template <int KB>
__global__ void __launch_bounds__(kMinorsBlock, MinorsMinBlocks<KB>::value) walk_fp64_minors_kernel(WalkArgs a) {
    extern __shared__ double2 smem_fp64[];
    const int lane = threadIdx.x & 31;
    const int stride = blockDim.x;
    // [col][thread] plain-double runs, then per warp KB double-double totals
    cx<double>* sm_acc = reinterpret_cast<cx<double>*>(smem_fp64) + threadIdx.x;
    double4* wtot = reinterpret_cast<double4*>(smem_fp64 + (size_t)(KB / 2) * stride) + (threadIdx.x >> 5) * KB;
    const bs_job* __restrict__ jobs = a.jobs;
    const cx<double>* __restrict__ data = static_cast<const cx<double>*>(a.data);
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
        const uint32_t local = (uint32_t)(t - jb.task_begin) + jb.task_offset;
        const int* radix = a.meta + BS_META_RADIX(jb);
        // the instance whose lanes own exactly Hr = ceil(K / 2) columns
        if (((jb.K + 1) >> 1) == KB / 2)
            walk_task_minors_fp64<KB, KB / 2>(jb, data, radix, a.partials, local, lane, sm_acc, wtot, stride);
        else
            walk_task_minors_fp64<KB, KB / 2 - 1>(jb, data, radix, a.partials, local, lane, sm_acc, wtot, stride);
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
    int grid = persistent_grid(walk_fp64_perm_kernel<KB>, kPermBlock, 0, a);
    walk_fp64_perm_kernel<KB><<<grid, kPermBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int KB>
static cudaError_t run_minors(const WalkArgs& a, cudaStream_t s) {
    // per thread and owned column a 16-byte run; per warp and column a
    // 32-byte double-double total
    size_t smem = (size_t)kMinorsBlock * (KB / 2) * sizeof(cx<double>) + (size_t)(kMinorsBlock / 32) * KB * sizeof(double4);
    cudaError_t e =
        cudaFuncSetAttribute(walk_fp64_minors_kernel<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = persistent_grid(walk_fp64_minors_kernel<KB>, kMinorsBlock, smem, a);
    walk_fp64_minors_kernel<KB><<<grid, kMinorsBlock, smem, s>>>(a);
    return cudaGetLastError();
}

#define BS_B48(X) X(1, 4) X(2, 8) X(3, 12) X(4, 16) X(5, 20) X(6, 24) X(7, 28) X(8, 32) X(9, 36) X(10, 40) X(11, 44) X(12, 48)

// a.max_K selects the bucket: every job of the launch must share it.
cudaError_t launch_walk_fp64_perm(const WalkArgs& a, cudaStream_t s) {
    if (a.total_tasks == 0 && !a.total_dev) return cudaSuccess;
    switch ((a.max_K + 3) >> 2) {
#define BS_CASE(b, kb) \
    case b: return run_perm<kb>(a, s);
        BS_B48(BS_CASE)
#undef BS_CASE
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_walk_fp64_minors(const WalkArgs& a, cudaStream_t s) {
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
