// Packing of one job (shared by the batch pack kernel and the sampler's
// device planner): c0[col] = sum over rows of M_row * a_row,col (every
// delta = +1), computed in double-double and rounded, and 2a[j][col] for every
// digit row, in the job's working precision, rows of stride
// KP = BS_ROW_STRIDE(K) with a zero pad column.  With normalize set, column col
// is scaled by 2^-e (e: smallest integer with sum_rows M_row (|Re a| + |Im a|)
// <= 2^e) and e is stored in colexp[col] for the reduce kernel.
#pragma once
#include <cuda_runtime.h>
#include "bs_job.h"
#include "gray.h"
#include "walk.cuh"

namespace bs {

__device__ __forceinline__ double2 src_elem(const double2* __restrict__ src, const bs_job& jb, int r, int c) {
    return jb.src_trans ? src[jb.src_off + (int64_t)c * jb.src_ld + r] : src[jb.src_off + (int64_t)r * jb.src_ld + c];
}

__device__ __forceinline__ void pack_job(const bs_job& jb, const double2* __restrict__ src, int* __restrict__ meta,
                         void* __restrict__ data, int fp32, int tid, int nthreads) {
    const int* radix = meta + BS_META_RADIX(jb);
    const int* dsrc = meta + BS_META_DIGIT_SRC(jb);
    const int* csrc = meta + BS_META_COL_SRC(jb);
    int* colexp = meta + BS_META_COLEXP(jb);
    const int prow = meta[BS_META_PINNED(jb)];
    // binomial table C(M_j, d), digit after digit
    if (tid == 0) {
        uint64_t* binom = reinterpret_cast<uint64_t*>(meta + BS_META_BINOM(jb));
        int at = 0;
        for (int j = 0; j < jb.nrows; ++j)
            for (int d = 0; d < radix[j]; ++d) binom[at++] = bs_binom(radix[j] - 1, d);
    }
    const int KP = BS_ROW_STRIDE(jb.K);
    for (int col = tid; col < KP; col += nthreads) {
        if (col >= jb.K) {  // pad column: zeros
            if (fp32) {
                cx<float>* out = static_cast<cx<float>*>(data) + jb.data_off;
                for (int j = 0; j <= jb.nrows; ++j) out[(size_t)j * KP + col] = cx<float>{0.f, 0.f};
            } else {
                cx<double>* out = static_cast<cx<double>*>(data) + jb.data_off;
                for (int j = 0; j <= jb.nrows; ++j) out[(size_t)j * KP + col] = cx<double>{0.0, 0.0};
            }
            continue;
        }
        const int sc = csrc[col];
        int e = 0;
        if (jb.normalize) {
            double2 a = src_elem(src, jb, prow, sc);
            double b = fabs(a.x) + fabs(a.y);
            for (int j = 0; j < jb.nrows; ++j) {
                double2 d = src_elem(src, jb, dsrc[j], sc);
                b += (double)(radix[j] - 1) * (fabs(d.x) + fabs(d.y));
            }
            if (b > 0.0) (void)frexp(b, &e);  // b = f 2^e, f in [0.5, 1)
        }
        colexp[col] = e;
        // c0 in double-double (each product split exactly with an FMA), rounded
        double2 a = src_elem(src, jb, prow, sc);
        ddv sre = {ldexp(a.x, -e), 0.0}, sim = {ldexp(a.y, -e), 0.0};
        for (int j = 0; j < jb.nrows; ++j) {
            double2 d = src_elem(src, jb, dsrc[j], sc);
            double m = (double)(radix[j] - 1);
            double dre = ldexp(d.x, -e), dim = ldexp(d.y, -e);
            double pre = m * dre, pim = m * dim;
            double ere = __fma_rn(m, dre, -pre), eim = __fma_rn(m, dim, -pim);
            sre = dd_add_d(dd_add_d(sre, pre), ere);
            sim = dd_add_d(dd_add_d(sim, pim), eim);
        }
        if (fp32) {
            cx<float>* out = static_cast<cx<float>*>(data) + jb.data_off;
            out[col] = cx<float>{(float)sre.hi, (float)sim.hi};
            for (int j = 0; j < jb.nrows; ++j) {
                double2 d = src_elem(src, jb, dsrc[j], sc);
                out[(size_t)(1 + j) * KP + col] = cx<float>{(float)ldexp(d.x, 1 - e), (float)ldexp(d.y, 1 - e)};
            }
        } else {
            cx<double>* out = static_cast<cx<double>*>(data) + jb.data_off;
            out[col] = cx<double>{sre.hi, sim.hi};
            for (int j = 0; j < jb.nrows; ++j) {
                double2 d = src_elem(src, jb, dsrc[j], sc);
                out[(size_t)(1 + j) * KP + col] = cx<double>{ldexp(d.x, 1 - e), ldexp(d.y, 1 - e)};
            }
        }
    }
}

}  // namespace bs
