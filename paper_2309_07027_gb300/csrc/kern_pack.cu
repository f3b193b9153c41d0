// Pack and reduce kernels.
//
// pack:   for every job, reads its source matrix (device) and writes
//           c0[col]   = sum over all rows of M_row * a_row,col  (all delta = +1)
//           2a[j][col] = 2 * a_digit_j,col
//         in the job's working precision.  With normalize set, column col is
//         first scaled by 2^-e, e the smallest integer with
//         sum_rows M_row (|Re a| + |Im a|) <= 2^e, so every column sum of the
//         walk has modulus <= sqrt(2) and FP32 products cannot overflow; the
//         exponents go to colexp[] and are undone exactly by the reduce
//         kernel (Appendix A.5 normalises columns for the same reason; here the
//         factors are powers of two, so the rescaling is exact).
// reduce: sums each job's task partials (Sum2, twice double precision) in a fixed order and
//         applies 2^(1-n) (Eq. bbfgrepeated prefactor) and the column scales.
#include <cuda_runtime.h>
#include "kernels.h"
#include "pack.cuh"
#include "walk.cuh"

namespace bs {

__global__ void pack_kernel(const bs_job* __restrict__ jobs, const double2* __restrict__ src, int* __restrict__ meta,
                            void* __restrict__ data, int prec) {
    const bs_job jb = jobs[blockIdx.x];
    pack_job(jb, src, meta, data, prec, threadIdx.x, blockDim.x);
}

cudaError_t launch_pack(const bs_job* jobs, int njobs, const double2* src, int* meta, void* data, int prec,
                        cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    pack_kernel<<<njobs, 64, 0, s>>>(jobs, src, meta, data, prec);
    return cudaGetLastError();
}

constexpr int kReduceBlock = 256;

// One Sum2 step: (s, c) + (hi, lo) -> (s', c + e + lo) with s' + e = s + hi
// exactly (TwoSum, Knuth).
__device__ __forceinline__ ddv sum2_add(ddv a, double hi, double lo) {
    const double s = __dadd_rn(a.hi, hi);
    const double bb = __dsub_rn(s, a.hi);
    const double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(hi, bb));
    return ddv{s, __dadd_rn(a.lo, __dadd_rn(e, lo))};
}

// (s, c) -> normalised double-double (TwoSum of s and c: c may exceed s when
// the sum cancels).
__device__ __forceinline__ ddv sum2_final(ddv a) {
    const double h = __dadd_rn(a.hi, a.lo);
    const double bb = __dsub_rn(h, a.hi);
    return ddv{h, __dadd_rn(__dsub_rn(a.hi, __dsub_rn(h, bb)), __dsub_rn(a.lo, bb))};
}

__global__ void __launch_bounds__(kReduceBlock) reduce_kernel(const bs_job* __restrict__ jobs,
                                                              const bs_zdd* __restrict__ partials,
                                                              const int* __restrict__ meta, double2* __restrict__ out,
                                                              double2* __restrict__ out_lo) {
    // Sum2 (Ogita, Rump and Oishi 2005): the high parts are added with TwoSum,
    // the TwoSum errors and the low parts go to one plain double c; result
    // (s, c) as accurate as a sum in twice the working precision, at 8 FP64
    // operations per addition instead of about 20 for a double-double add.
    __shared__ ddv sre[kReduceBlock];
    __shared__ ddv sim[kReduceBlock];
    const bs_job jb = jobs[blockIdx.x];
    const int ncols = jb.kind == BS_KIND_PERM ? 1 : jb.K;
    const int col = blockIdx.y;
    if (col >= ncols) return;
    ddv re = {0.0, 0.0}, im = {0.0, 0.0};  // (s, c)
    for (uint32_t t = threadIdx.x; t < jb.ntasks; t += kReduceBlock) {
        bs_zdd p = partials[jb.partial_off + (int64_t)t * ncols + col];
        re = sum2_add(re, p.re_hi, p.re_lo);
        im = sum2_add(im, p.im_hi, p.im_lo);
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int w = kReduceBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const ddv r2 = sre[threadIdx.x + w], i2 = sim[threadIdx.x + w];
            sre[threadIdx.x] = sum2_add(sre[threadIdx.x], r2.hi, r2.lo);
            sim[threadIdx.x] = sum2_add(sim[threadIdx.x], i2.hi, i2.lo);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sre[0] = sum2_final(sre[0]);
        sim[0] = sum2_final(sim[0]);
    }
    if (threadIdx.x == 0) {
        // prefactor: 2^(1-n) times the column scales (Eq. bbfgrepeated), or
        // (-1)^n (Eq. ryser), or (-1)^(n-1) 2 (Nijenhuis-Wilf)
        int e = 0;
        double sgn = 1.0;
        if (jb.formula == BS_JOB_BBFG) {
            const int* colexp = meta + BS_META_COLEXP(jb);
            e = 1 - jb.n;
            for (int c = 0; c < jb.K; ++c) e += colexp[c];
            if (jb.kind == BS_KIND_MINORS) e -= colexp[col];
        } else if (jb.formula == BS_JOB_RYSER) {
            sgn = (jb.n & 1) ? -1.0 : 1.0;
        } else {
            e = 1;
            sgn = ((jb.n - 1) & 1) ? -1.0 : 1.0;
        }
        ddv r = sre[0], i = sim[0];
        out[jb.out_index + col] = make_double2(sgn * ldexp(r.hi, e), sgn * ldexp(i.hi, e));
        if (out_lo) out_lo[jb.out_index + col] = make_double2(sgn * ldexp(r.lo, e), sgn * ldexp(i.lo, e));
    }
}

cudaError_t launch_reduce(const bs_job* jobs, int njobs, const bs_zdd* partials, const int* meta, double2* out,
                          double2* out_lo, int max_cols, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    dim3 grid(njobs, max_cols < 1 ? 1 : max_cols);
    reduce_kernel<<<grid, kReduceBlock, 0, s>>>(jobs, partials, meta, out, out_lo);
    return cudaGetLastError();
}

}  // namespace bs
