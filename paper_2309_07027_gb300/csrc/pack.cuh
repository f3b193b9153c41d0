// Packing of one job (shared by the batch pack kernel and the sampler's
// device planner): c0[col] = sum over rows of M_row * a_row,col (every
// delta = +1), computed in double-double and rounded, and 2a[j][col] for every
// digit row, in the job's working precision, rows of stride
// KP = BS_ROW_STRIDE(K).  FP64 rows are plain complex doubles; FP32 rows are
// column pairs {re(2p), re(2p+1), im(2p), im(2p+1)} (the packed layout of
// walk_fp32.cuh).  Pad columns: zero rows, c0 = 1 in FP32 jobs (a neutral
// factor) and 0 in FP64 jobs.  With normalize set, column col
// is scaled by 2^-e (e: smallest integer with sum_rows M_row (|Re a| + |Im a|)
// <= 2^e) and e is stored in colexp[col] for the reduce kernel.
// Double-float (DF) jobs: rows of stride BS_ROW_STRIDE_DF(K) (a multiple of
// 8), column col scaled by 2^(2 - e) (colexp = e - 2) so that every column
// sum has |Re|, |Im| <= 4, and every entry quantised to a high part on the
// grid 2^-20 and a low part on the grid 2^-44, both exact floats
// (walk_df.cuh); pair p of a row is {re h, re h, im h, im h} of columns
// (2p, 2p+1), then the same for the low parts; pad columns have c0 = 1.
#pragma once
#include <cuda_runtime.h>
#include "bs_job.h"
#include "gray.h"
#include "walk.cuh"

namespace bs {

__device__ __forceinline__ double2 src_elem(const double2* __restrict__ src, const bs_job& jb, int r, int c) {
    return jb.src_trans ? src[jb.src_off + (int64_t)c * jb.src_ld + r] : src[jb.src_off + (int64_t)r * jb.src_ld + c];
}

// Element (row r, column col) of an FP32 job's packed rows.
__device__ __forceinline__ void put_f32(void* data, const bs_job& jb, int KP, int r, int col, float re, float im) {
    float* q = static_cast<float*>(data) + 2 * (jb.data_off + (int64_t)r * KP) + 4 * (col >> 1) + (col & 1);
    q[0] = re;
    q[2] = im;
}

// The DF split of v (|v| < 16): hi = v rounded to the grid 2^-20, lo = the
// rest rounded to the grid 2^-44; vlo: a low-order double added to v
// (double-double input), 0 otherwise.
__device__ __forceinline__ float2 df_quantise(double v, double vlo) {
    const double hi = rint(v * 0x1p20) * 0x1p-20;
    const double rest = (v - hi) + vlo;  // v - hi is exact
    const double lo = rint(rest * 0x1p44) * 0x1p-44;
    return make_float2((float)hi, (float)lo);
}

// Element (row r, column col) of a DF job's packed rows.
__device__ __forceinline__ void put_df(void* data, const bs_job& jb, int KP, int r, int col, float2 re, float2 im) {
    float* q = static_cast<float*>(data) + 4 * (jb.data_off + (int64_t)r * KP) + 8 * (col >> 1) + (col & 1);
    q[0] = re.x;
    q[2] = im.x;
    q[4] = re.y;
    q[6] = im.y;
}

__device__ __forceinline__ void pack_job(const bs_job& jb, const double2* __restrict__ src, int* __restrict__ meta,
                         void* __restrict__ data, int prec, int tid, int nthreads) {
    const int fp32 = prec == BS_PREC_FP32;
    const int df = prec == BS_PREC_DF;
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
    const int KP = df ? BS_ROW_STRIDE_DF(jb.K) : BS_ROW_STRIDE(jb.K);
    if (jb.formula != BS_JOB_BBFG) {
        // Ryser / Nijenhuis-Wilf (FP64): product column col is matrix row
        // sc; digit j is matrix column dsrc[j], added with +1 when it enters
        // the subset, so the packed row is -a (the walk subtracts rows of
        // digits whose Delta is 1).  Start sums: 0 (Ryser) or
        // x = a_(sc, n-1) - (sum_j a_(sc, j)) / 2 (Nijenhuis-Wilf).
        cx<double>* out = static_cast<cx<double>*>(data) + jb.data_off;
        for (int col = tid; col < KP; col += nthreads) {
            if (col >= jb.K) {
                for (int j = 0; j <= jb.nrows; ++j) out[(size_t)j * KP + col] = cx<double>{0.0, 0.0};
                continue;
            }
            colexp[col] = 0;
            const int sc = csrc[col];
            ddv sre = {0.0, 0.0}, sim = {0.0, 0.0};
            if (jb.formula == BS_JOB_NW) {
                for (int j = 0; j < jb.n; ++j) {
                    const double2 d = src_elem(src, jb, j, sc);
                    sre = dd_add_d(sre, -0.5 * d.x);
                    sim = dd_add_d(sim, -0.5 * d.y);
                }
                const double2 last = src_elem(src, jb, jb.n - 1, sc);
                sre = dd_add_d(sre, last.x);
                sim = dd_add_d(sim, last.y);
            }
            out[col] = cx<double>{sre.hi, sim.hi};
            for (int j = 0; j < jb.nrows; ++j) {
                const double2 d = src_elem(src, jb, dsrc[j], sc);
                out[(size_t)(1 + j) * KP + col] = cx<double>{-d.x, -d.y};
            }
        }
        return;
    }
    for (int col = tid; col < KP; col += nthreads) {
        if (col >= jb.K) {  // pad column
            if (df) {
                put_df(data, jb, KP, 0, col, make_float2(1.f, 0.f), make_float2(0.f, 0.f));
                for (int j = 1; j <= jb.nrows; ++j) put_df(data, jb, KP, j, col, make_float2(0.f, 0.f), make_float2(0.f, 0.f));
            } else if (fp32) {
                put_f32(data, jb, KP, 0, col, 1.f, 0.f);
                for (int j = 1; j <= jb.nrows; ++j) put_f32(data, jb, KP, j, col, 0.f, 0.f);
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
            if (df) e -= 2;                   // DF: column sums up to 4 (walk_df.cuh)
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
        if (df) {
            put_df(data, jb, KP, 0, col, df_quantise(sre.hi, sre.lo), df_quantise(sim.hi, sim.lo));
            for (int j = 0; j < jb.nrows; ++j) {
                double2 d = src_elem(src, jb, dsrc[j], sc);
                put_df(data, jb, KP, 1 + j, col, df_quantise(ldexp(d.x, 1 - e), 0.0),
                       df_quantise(ldexp(d.y, 1 - e), 0.0));
            }
        } else if (fp32) {
            put_f32(data, jb, KP, 0, col, (float)sre.hi, (float)sim.hi);
            for (int j = 0; j < jb.nrows; ++j) {
                double2 d = src_elem(src, jb, dsrc[j], sc);
                put_f32(data, jb, KP, 1 + j, col, (float)ldexp(d.x, 1 - e), (float)ldexp(d.y, 1 - e));
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
