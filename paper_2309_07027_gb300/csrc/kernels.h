// Launch wrappers for the device code (host side, stream-ordered, no sync).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "bs_job.h"

namespace bs {

struct WalkArgsBase {
    const bs_job* jobs;                    // device, sorted by task_begin
    int njobs;
    const int* job_list;                   // if non-null: job i is jobs[job_list[i]]
    const int* njobs_dev;                  // if non-null: the job count, planned on the device
    const void* data;                      // device: complex double or float arena
    const int* meta;                       // device
    bs_zdd* partials;                      // device
    unsigned long long total_tasks;        // sum of ntasks (host-planned launches)
    const unsigned long long* total_dev;   // if non-null: the total, planned on the device
    unsigned long long* counter;           // device, zeroed before the launch
    int* status;                           // device status word
    unsigned long long deadline_rel_ns;    // per-warp deadline after its start, 0 = none
    int max_K;                             // bucket: every job has (K+3)/4 == (max_K+3)/4
    int grid_cap;                          // upper bound on CTAs (0 = fill the GPU)
};
typedef WalkArgsBase WalkArgs;

cudaError_t launch_walk_fp64_perm(const WalkArgs& a, cudaStream_t s);
cudaError_t launch_walk_fp64_minors(const WalkArgs& a, cudaStream_t s);
cudaError_t launch_walk_fp32_perm(const WalkArgs& a, cudaStream_t s);
cudaError_t launch_walk_fp32_minors(const WalkArgs& a, cudaStream_t s);
// Double-float kernels: 8-column buckets (max_K selects (K + 7) / 8).
cudaError_t launch_walk_df_perm(const WalkArgs& a, cudaStream_t s);
cudaError_t launch_walk_df_minors(const WalkArgs& a, cudaStream_t s);

// Builds c0 / 2a (and column scales) of every job from its source matrix.
// prec (BS_PREC_*) selects the layout: complex doubles (FP64), packed float
// pairs (FP32, the float arena) or double-float pairs (DF, 16-byte units).
cudaError_t launch_pack(const bs_job* jobs, int njobs, const double2* src, int* meta, void* data, int prec,
                        cudaStream_t s);

// Sums each job's task partials in a fixed order and applies 2^(1-n) and the
// column scales; writes out[out_index + col] (and the low parts to out_lo when
// non-null).
cudaError_t launch_reduce(const bs_job* jobs, int njobs, const bs_zdd* partials, const int* meta, double2* out,
                          double2* out_lo, int max_cols, cudaStream_t s);

// Measured issue rates (lane-operations per second) of the FP64 and FP32
// fused multiply-add pipes, from a timed microbenchmark on this device.
cudaError_t measure_fma_rates(int device, double* fp64_per_s, double* fp32_per_s);

int sm_count(int device);

}  // namespace bs
