// Gray-walk kernels for the generalized BB/FG sum (Eq. bbfgrepeated) and its
// fused Laplace-minor variant.
//
// Work decomposition (Sec. 2.1: contiguous index ranges walked
// independently, each seeded by decoding its first index):
//   * a job's index range [0, C) is cut into chunks of L = 2^log2L addends;
//   * a warp task is a run of consecutive chunks: one per lane for the
//     permanents, one per lane pair (FP64) or per group of 2 or 4 lanes
//     (FP32) for the Laplace minors, the group's lanes splitting the columns;
//   * persistent warps pull tasks from a global counter (largest jobs are
//     planned first), so uneven jobs share one launch;
//   * every lane decodes its chunk start (re-seeding its column sums from the
//     matrix, which bounds the drift of the incremental updates, Sec. 3.2)
//     and then steps through the chunk one digit move at a time.
// Because chunk starts are multiples of L, all lanes of a warp flip the same
// binary digit at each step except at the rare carries past bit log2L, so the
// row they read is a broadcast load.
//
// Per addend (thread-owns-chunk; all column sums in registers):
//   update   c_col += coef * (2 a_row,col)       K complex FMAs
//   product  P = prod_col c_col                   K-1 complex multiplies, two
//                                                 independent chains
//   weight   acc += (+-W) * P                      (Eq. bbfgrepeated weight)
// Minors additionally form, for every column l, prod_{col != l} c_col from a
// suffix pass and a running prefix (about 2.3x the FP64 work of one
// permanent instead of K x).
//
// Accumulation: each lane sums its addends in plain precision for a short
// run, folds the run into a compensated accumulator (double-double in FP64
// mode, float-float in FP32 mode), and the lanes of a task are combined in a
// fixed shuffle order.  Tasks write one partial per output; the
// reduce kernel sums them in a fixed order, so results do not depend on which
// warp ran which task or on what else was in the launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "bs_job.h"
#include "gray.h"
#include "kernels.h"

namespace bs {

template <typename T>
struct cx {
    T re, im;
};

__device__ __forceinline__ float bfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double bfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    cx<T> r;
    r.re = bfma(a.re, b.re, -(a.im * b.im));
    r.im = bfma(a.re, b.im, a.im * b.re);
    return r;
}

// ---------------------------------------------------------------- compensated sums
struct ddv {
    double hi, lo;
};

// TwoSum (Knuth) then renormalisation; adds a double into a double-double.
__device__ __forceinline__ ddv dd_add_d(ddv a, double b) {
    double s = __dadd_rn(a.hi, b);
    double bb = __dsub_rn(s, a.hi);
    double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    e = __dadd_rn(e, a.lo);
    double h = __dadd_rn(s, e);
    ddv r;
    r.hi = h;
    r.lo = __dsub_rn(e, __dsub_rn(h, s));
    return r;
}

// Double-double addition (two TwoSums, two renormalisations).
__device__ __forceinline__ ddv dd_add(ddv a, ddv b) {
    double s = __dadd_rn(a.hi, b.hi);
    double bb = __dsub_rn(s, a.hi);
    double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b.hi, bb));
    double t = __dadd_rn(a.lo, b.lo);
    double tb = __dsub_rn(t, a.lo);
    double f = __dadd_rn(__dsub_rn(a.lo, __dsub_rn(t, tb)), __dsub_rn(b.lo, tb));
    e = __dadd_rn(e, t);
    double h = __dadd_rn(s, e);
    e = __dsub_rn(e, __dsub_rn(h, s));
    e = __dadd_rn(e, f);
    ddv r;
    r.hi = __dadd_rn(h, e);
    r.lo = __dsub_rn(e, __dsub_rn(r.hi, h));
    return r;
}

// Double-double addition in Sum2 form (Ogita, Rump and Oishi 2005): TwoSum
// of the high parts, its error and both low parts added in double, one
// renormalisation; 11 FP64 operations instead of 20.  Sums of many terms
// formed this way are as accurate as summation in twice double precision,
// which is what the task and cross-lane combinations need (the FP64 pipe is
// 1/64 of the FP32 pipe here, and a small job's latency is its warps' FP64
// instruction count).
__device__ __forceinline__ ddv dd_add_sum2(ddv a, ddv b) {
    const double s = __dadd_rn(a.hi, b.hi);
    const double bb = __dsub_rn(s, a.hi);
    double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b.hi, bb));
    e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
    ddv r;
    r.hi = __dadd_rn(s, e);
    r.lo = __dsub_rn(e, __dsub_rn(r.hi, s));
    return r;
}

// Sum2 accumulation of single doubles: s holds the rounded sum, e the
// running sum of the TwoSum errors.
__device__ __forceinline__ void sum2_acc(double& s, double& e, double x) {
    const double t = __dadd_rn(s, x);
    const double bb = __dsub_rn(t, s);
    e = __dadd_rn(e, __dadd_rn(__dsub_rn(s, __dsub_rn(t, bb)), __dsub_rn(x, bb)));
    s = t;
}

struct ffv {
    float hi, lo;
};

// TwoSum in single precision: adds a float into a float-float.
__device__ __forceinline__ ffv ff_add_f(ffv a, float b) {
    float s = __fadd_rn(a.hi, b);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    e = __fadd_rn(e, a.lo);
    ffv r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ ddv dd_from_ff(ffv a) {
    ddv r;
    r.hi = (double)a.hi;
    r.lo = 0.0;
    return dd_add_d(r, (double)a.lo);
}

// Float-float addition (TwoSum of the high parts, low parts added, one
// renormalisation); used for cross-lane sums in the FP32 kernels so that no
// FP64 instruction runs in their loops.
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    ffv r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ ffv shfl_down_ff(ffv v, int off) {
    ffv r;
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return r;
}

__device__ __forceinline__ ddv shfl_down_dd(ddv v, int off) {
    ddv r;
    r.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    r.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return r;
}

// Fixed-order warp reduction of a double-double complex value; lane 0 ends
// with the sum.
__device__ __forceinline__ void warp_reduce_zdd(ddv& re, ddv& im) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ddv ore = shfl_down_dd(re, off);
        ddv oim = shfl_down_dd(im, off);
        re = dd_add_sum2(re, ore);
        im = dd_add_sum2(im, oim);
    }
}

__device__ __forceinline__ double flip_sign(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ float flip_sign(float x) {
    return __int_as_float(__float_as_int(x) ^ (int)0x80000000u);
}

// +1 or -1 (neg = 1) built from bits, so no int-to-float conversion runs in
// the loop.
__device__ __forceinline__ float unit_sign_f(uint32_t neg) { return __int_as_float(0x3f800000u | (neg << 31)); }
__device__ __forceinline__ double unit_sign_d(uint32_t neg) {
    return __longlong_as_double((long long)(0x3ff0000000000000ull | ((unsigned long long)neg << 63)));
}

// In-chunk stepper.  A chunk starts at a multiple i0 of L = 2^log2L and
// takes fewer than L steps, so the index i0 + s has exactly the trailing
// ones of s: the digit that moves at step s -> s + 1 is t = ctz(s + 1) < 12
// when t < nbin (a binary flip, 32-bit arithmetic only), and otherwise every
// binary digit is saturated and a repeated-row digit moves (general step).
// The stepper itself holds only scalars (kept in registers); the full Gray
// state g, whose repeated-row digit arrays are indexed at run time and so
// live in local memory, is a separate object that only the general step
// touches.
struct ChunkStepper {
    uint64_t i0;
    const uint64_t* binom;
    uint32_t dlo;   // Delta bits of binary digits 0..31
    int parity0;    // parity at the chunk start
    int nbin;

    __device__ __forceinline__ void init(bs_gray& g, uint64_t start, int nb, int nrows, const int* radix,
                                         const uint64_t* tab) {
        binom = tab;
        bs_gray_decode(g, start, nb, nrows, radix, tab);
        i0 = start;
        dlo = (uint32_t)g.dbin;
        parity0 = g.parity;
        nbin = nb;
    }
    // The step to index i0 + u when it moves a binary digit (ctz(u) < nbin,
    // which the caller guarantees): returns the row, *neg as in step().
    __device__ __forceinline__ int step_bin(uint32_t u, uint32_t* neg) {
        const int t = __ffs((int)u) - 1;
        const uint32_t was = (dlo >> t) & 1u;
        dlo ^= 1u << t;
        *neg = was ^ 1u;
        return t;
    }
    // Move from index i0 + s to i0 + s + 1.  Returns the digit row; *neg is 1
    // when the column sums move by -2a_row (Delta rises), 0 for +2a_row;
    // *wch is 1 when the binomial weight changed (then g.w, g.parity are
    // current).
    __device__ __forceinline__ int step(bs_gray& g, uint32_t s, const int* radix, uint32_t* neg, int* wch) {
        const int t = __ffs((int)(s + 1u)) - 1;
        if (t < nbin) {
            const uint32_t was = (dlo >> t) & 1u;
            dlo ^= 1u << t;
            *neg = was ^ 1u;
            *wch = 0;
            return t;
        }
        g.i = i0 + s;
        g.parity = parity0 ^ (int)(s & 1u);
        g.dbin = (g.dbin & ~0xffffffffull) | (uint64_t)dlo;
        int coef;
        const int row = bs_gray_step(g, radix, &coef, wch, binom);
        *neg = coef < 0 ? 1u : 0u;
        return row;
    }
};

// The packed rows of a job with K columns have stride BS_ROW_STRIDE(K), the
// width KB of the bucket kernel that walks it: inside a kernel the stride is
// the compile-time KB.
static_assert(BS_ROW_STRIDE(29) == 32 && BS_ROW_STRIDE(32) == 32 && BS_ROW_STRIDE(1) == 4,
              "row stride must equal the 4-column bucket width");

// Column `col` of a bucket KB is live when col < K; K >= KB - 3 always, so
// only the last three columns of a bucket need a runtime test.  (The FP32
// kernels need none: their pad columns are neutral, see walk_fp32.cuh.)
#define BS_LIVE(col) ((col) < KB - 3 || (col) < K)

// Seed the column sums of the decoded state: c = c0 - sum_j Delta_j * 2a_j
// (rows of the packed matrix have stride KP).
template <typename T, int KB>
__device__ __forceinline__ void seed_columns(cx<T> (&c)[KB], const bs_gray& g, const cx<T>* __restrict__ c0,
                                             const cx<T>* __restrict__ a2, int K, int KP, int nbin, int nrows) {
#pragma unroll
    for (int col = 0; col < KB; ++col)
        if (BS_LIVE(col)) c[col] = c0[col];
    uint64_t bits = g.dbin;
    while (bits) {
        int j = bs_ctz64(bits);
        bits &= bits - 1;
        const cx<T>* row = a2 + (size_t)j * KP;
#pragma unroll
        for (int col = 0; col < KB; ++col)
            if (BS_LIVE(col)) {
                cx<T> a = row[col];
                c[col].re -= a.re;
                c[col].im -= a.im;
            }
    }
    for (int j = nbin; j < nrows; ++j) {
        int d = g.del[j];
        if (d == 0) continue;
        T fd = (T)(-d);
        const cx<T>* row = a2 + (size_t)j * KP;
#pragma unroll
        for (int col = 0; col < KB; ++col)
            if (BS_LIVE(col)) {
                cx<T> a = row[col];
                c[col].re = bfma(fd, a.re, c[col].re);
                c[col].im = bfma(fd, a.im, c[col].im);
            }
    }
}

__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return cx<double>{v.x, v.y};
}

// c_col += cf * row_col for the KX live columns (one 16-byte load per
// column).  KX is the job's exact column count, a template parameter: a
// runtime test on the bucket's last columns becomes predicated instructions
// that occupy FP64 issue slots even where the column is dead.
template <int KB, int KX>
__device__ __forceinline__ void update_columns(cx<double> (&c)[KB], const cx<double>* __restrict__ row, double cf) {
    static_assert(KX >= 1 && KX <= KB, "live columns lie in the bucket");
#pragma unroll
    for (int col = 0; col < KX; ++col) {
        cx<double> a = ldg_cx(row + col);
        c[col].re = bfma(cf, a.re, c[col].re);
        c[col].im = bfma(cf, a.im, c[col].im);
    }
}
// prod_col c_col over the KX live columns with two interleaved chains (even
// / odd columns).
template <typename T, int KB, int KX>
__device__ __forceinline__ cx<T> product_columns(const cx<T> (&c)[KB]) {
    if constexpr (KX == 1) {
        return c[0];
    } else {
        cx<T> pe = c[0];
        cx<T> po = c[1];
#pragma unroll
        for (int col = 2; col < KX; ++col) {
            if (col & 1)
                po = cmul(po, c[col]);
            else
                pe = cmul(pe, c[col]);
        }
        return cmul(pe, po);
    }
}

template <typename T>
__device__ __forceinline__ T signed_weight(uint64_t w, int parity) {
    T x = (T)w;
    return parity ? -x : x;
}

__device__ __forceinline__ void store_partial(bs_zdd* p, ddv re, ddv im) {
    bs_zdd o;
    o.re_hi = re.hi;
    o.re_lo = re.lo;
    o.im_hi = im.hi;
    o.im_lo = im.lo;
    *p = o;
}

// ---------------------------------------------------------------- one task: permanent, FP64
// Each lane: plain double runs of FOLD addends folded into a double-double
// sum; the 32 lanes are combined in double-double in a fixed shuffle order
// and lane 0 writes the task's partial.  KX = K, the job's column count, is
// compile-time (the kernel picks the instance per task), so the per-addend
// update and product run exactly K columns.  (The FP32 permanent runs on
// packed pairs, walk_fp32.cuh.)
template <int KB, int KX>
__device__ void walk_task_perm_fp64(const bs_job& jb, const cx<double>* __restrict__ data,
                                    const int* __restrict__ radix, bs_zdd* __restrict__ partials, uint32_t local,
                                    int lane) {
    constexpr uint32_t FOLD = 64;
    constexpr int K = KX;
    constexpr int KP = KB;  // = BS_ROW_STRIDE(K) for every K of the bucket
    const cx<double>* c0 = data + jb.data_off;
    const cx<double>* a2 = c0 + KP;
    ddv sre = {0.0, 0.0}, sim = {0.0, 0.0};
    const uint64_t i0 = ((uint64_t)local * 32u + (uint64_t)lane) << jb.log2L;
    if (i0 < jb.C) {
        const uint64_t rem = jb.C - i0;
        const uint32_t len = (uint32_t)(rem < (1ull << jb.log2L) ? rem : (1ull << jb.log2L));
        bs_gray g;
        ChunkStepper st;
        st.init(g, i0, jb.nbin, jb.nrows, radix, reinterpret_cast<const uint64_t*>(radix + (BS_META_BINOM(jb) - jb.meta_off)));
        cx<double> c[KB];
        seed_columns<double, KB>(c, g, c0, a2, K, KP, jb.nbin, jb.nrows);
        double ws = signed_weight<double>(g.w, g.parity);
        cx<double> acc = {0.0, 0.0};
        uint32_t run = 0;
        for (uint32_t s = 0;; ++s) {
            const cx<double> p = product_columns<double, KB, KX>(c);
            acc.re = bfma(ws, p.re, acc.re);
            acc.im = bfma(ws, p.im, acc.im);
            if (++run == FOLD) {
                run = 0;
                sre = dd_add_d(sre, acc.re);
                sim = dd_add_d(sim, acc.im);
                acc = cx<double>{0.0, 0.0};
            }
            if (s + 1 == len) break;
            uint32_t neg;
            int wch;
            const int row = st.step(g, s, radix, &neg, &wch);
            ws = wch ? signed_weight<double>(g.w, g.parity) : flip_sign(ws);
            update_columns<KB, KX>(c, a2 + (size_t)row * KP, unit_sign_d(neg));
        }
        sre = dd_add_d(sre, acc.re);
        sim = dd_add_d(sim, acc.im);
    }
    warp_reduce_zdd(sre, sim);
    if (lane == 0) store_partial(partials + jb.partial_off + local, sre, sim);
}

// Fold the plain-double runs of the warp's 16 chunks into the warp's
// double-double column totals and clear the runs: lane 16 h + u takes
// column t = u + 16 r of half h (rounds r), sums the runs of lanes 2p + h
// in Sum2 form and adds them to the total of that column (only it touches
// that total and those runs).  wacc: the warp's runs ([col][thread], thread
// 0 of the warp at column 0); wtot: its K totals {re hi, re lo, im hi, im lo}.
__device__ __forceinline__ void minors_fold_fp64(cx<double>* __restrict__ wacc, double4* __restrict__ wtot,
                                                 int stride, int lane, int K, int Hr, int H) {
    const int hh = lane >> 4;
    const int Kh = hh ? K - Hr : Hr;
    __syncwarp();
#pragma unroll 1
    for (int t = lane & 15; t < Kh && t < H; t += 16) {
        double sr = 0.0, er = 0.0, si = 0.0, ei = 0.0;
#pragma unroll 4
        for (int p = 0; p < 16; ++p) {
            cx<double>* q = wacc + t * stride + 2 * p + hh;
            const cx<double> r = *q;
            *q = cx<double>{0.0, 0.0};
            sum2_acc(sr, er, r.re);
            sum2_acc(si, ei, r.im);
        }
        double4* w = wtot + hh * Hr + t;
        const double4 v = *w;
        const ddv re = dd_add_sum2(ddv{v.x, v.y}, dd_add_d(ddv{sr, 0.0}, er));
        const ddv im = dd_add_sum2(ddv{v.z, v.w}, dd_add_d(ddv{si, 0.0}, ei));
        *w = make_double4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncwarp();
}

// ---------------------------------------------------------------- one task: minors, FP64
// Two lanes share one chunk: lane (2p + h) owns the columns
// [h Hr, h Hr + KH), Hr = ceil(K / 2), KH = Hr (h = 0) or K - Hr (h = 1), so
// both lanes run the same number of columns except one for odd K.  Per
// addend each lane
//   1. forms suffix products over its own columns (in registers), the last
//      one being Q_own, the product of its columns,
//   2. swaps Q_own with its partner (one shuffle of a complex double),
//   3. runs the prefix pass from X = (+-W) Q_partner:
//          acc[l] += X * prefix_l * suffix_l,
// with the per-column accumulators in shared memory, [col][thread]: plain
// double runs of FOLD addends, which the warp folds, column by column and
// transposed across lanes, into one double-double total per column of the
// warp (minors_fold_fp64).  Each lane holds half the column sums and
// suffixes of the one-lane form, so more warps fit on an SM and the
// dependent product chains are half as long, for the same FP64 work plus
// one real-by-complex product per lane and addend; with the totals per warp
// rather than per thread, shared memory (16 bytes per owned column and
// thread) no longer limits the CTAs per SM before registers do.  All lanes
// run the warp's longest chunk length (a finished or absent chunk continues
// with weight 0), so the shuffle has the full warp.  A warp task covers 16
// chunks; its last fold leaves the task's sums in the warp's totals, which
// lanes 16 h + u write as the task's double-double partials.
//
// HX = Hr, the most columns a lane owns, is compile-time (the kernel picks
// the instance per task: KB / 2 or KB / 2 - 1), so the per-addend loops run
// exactly Hr columns; only lane h = 1 of an odd K has one predicated column.
template <int KB, int HX>
__device__ void walk_task_minors_fp64(const bs_job& jb, const cx<double>* __restrict__ data,
                                      const int* __restrict__ radix, bs_zdd* __restrict__ partials, uint32_t local,
                                      int lane, cx<double>* __restrict__ sm_acc, double4* __restrict__ wtot,
                                      int stride) {
    // fold interval: each lane spends about 7 FP64 operations per column and
    // addend, a fold about 16 per column, so folds every 256 addends cost
    // about 1 % (every 64: 4.8 %, measured on the 29 x 30 minors)
    constexpr uint32_t FOLD = 256;
    constexpr int H = HX;  // most columns a lane owns: Hr
    static_assert(HX >= 1 && 2 * HX <= KB, "owned columns lie in the bucket");
    const int K = jb.K;
    constexpr int KP = KB;  // = BS_ROW_STRIDE(K) for every K of the bucket
    const int half = lane & 1;
    const int Hr = (K + 1) >> 1;
    const int cbase = half * Hr;
    const int KH = half ? K - Hr : Hr;  // own columns, >= 1 for K >= 2
    const cx<double>* c0 = data + jb.data_off;
    const cx<double>* a2 = c0 + KP;
    cx<double>* wacc = sm_acc - lane;  // this warp's thread 0
#define BS_OWN(t) ((t) < H - 1 || (t) < KH)
#pragma unroll
    for (int t = 0; t < H; ++t)
        if (BS_OWN(t)) sm_acc[t * stride] = cx<double>{0.0, 0.0};
    for (int t = lane; t < K; t += 32) wtot[t] = make_double4(0.0, 0.0, 0.0, 0.0);
    const uint64_t i0_own = ((uint64_t)local * 16u + (uint64_t)(lane >> 1)) << jb.log2L;
    const bool has = i0_own < jb.C;
    const uint64_t i0 = has ? i0_own : 0ull;
    uint32_t len = 0;
    if (has) {
        const uint64_t rem = jb.C - i0;
        len = (uint32_t)(rem < (1ull << jb.log2L) ? rem : (1ull << jb.log2L));
    }
    const uint32_t steps = __reduce_max_sync(0xffffffffu, len);
    bs_gray g;
    ChunkStepper st;
    st.init(g, i0, jb.nbin, jb.nrows, radix, reinterpret_cast<const uint64_t*>(radix + (BS_META_BINOM(jb) - jb.meta_off)));
    cx<double> c[H];
    {
        // seed own columns: c = c0 - sum_j Delta_j 2a_j
#pragma unroll
        for (int t = 0; t < H; ++t)
            if (BS_OWN(t)) c[t] = c0[cbase + t];
        uint64_t bits = g.dbin;
        while (bits) {
            const int j = bs_ctz64(bits);
            bits &= bits - 1;
            const cx<double>* row = a2 + (size_t)j * KP + cbase;
#pragma unroll
            for (int t = 0; t < H; ++t)
                if (BS_OWN(t)) {
                    c[t].re -= row[t].re;
                    c[t].im -= row[t].im;
                }
        }
        for (int j = jb.nbin; j < jb.nrows; ++j) {
            const int d = g.del[j];
            if (d == 0) continue;
            const double fd = (double)(-d);
            const cx<double>* row = a2 + (size_t)j * KP + cbase;
#pragma unroll
            for (int t = 0; t < H; ++t)
                if (BS_OWN(t)) {
                    c[t].re = bfma(fd, row[t].re, c[t].re);
                    c[t].im = bfma(fd, row[t].im, c[t].im);
                }
        }
    }
    double ws = has ? signed_weight<double>(g.w, g.parity) : 0.0;
    for (uint32_t s = 0; s < steps; ++s) {
        // 1. suffix products over own columns (suf[t] = prod_{own u > t} c_u)
        cx<double> suf[H];
        cx<double> sfx = {1.0, 0.0};
        bool first = true;
#pragma unroll
        for (int t = H - 1; t >= 0; --t)
            if (BS_OWN(t)) {
                suf[t] = sfx;
                sfx = first ? c[t] : cmul(sfx, c[t]);
                first = false;
            }
        // 2. swap Q_own with the partner lane
        cx<double> q;
        q.re = __shfl_xor_sync(0xffffffffu, sfx.re, 1);
        q.im = __shfl_xor_sync(0xffffffffu, sfx.im, 1);
        // 3. prefix pass from X = ws Q_partner
        cx<double> pre = {ws * q.re, ws * q.im};
#pragma unroll
        for (int t = 0; t < H; ++t)
            if (BS_OWN(t)) {
                cx<double> a = sm_acc[t * stride];
                a.re = bfma(pre.re, suf[t].re, a.re);
                a.re = bfma(-pre.im, suf[t].im, a.re);
                a.im = bfma(pre.re, suf[t].im, a.im);
                a.im = bfma(pre.im, suf[t].re, a.im);
                sm_acc[t * stride] = a;
                if (BS_OWN(t + 1)) pre = cmul(pre, c[t]);
            }
        if (((s + 1u) & (FOLD - 1u)) == 0) minors_fold_fp64(wacc, wtot, stride, lane, K, Hr, H);
        if (s + 1 >= len) {  // this lane's chunk is done: weight 0 from here on
            ws = 0.0;
            continue;
        }
        uint32_t neg;
        int wch;
        const int row = st.step(g, s, radix, &neg, &wch);
        ws = wch ? signed_weight<double>(g.w, g.parity) : flip_sign(ws);
        const cx<double>* rp = a2 + (size_t)row * KP + cbase;
        const double cf = unit_sign_d(neg);
#pragma unroll
        for (int t = 0; t < H; ++t)
            if (BS_OWN(t)) {
                const cx<double> v = ldg_cx(rp + t);
                c[t].re = bfma(cf, v.re, c[t].re);
                c[t].im = bfma(cf, v.im, c[t].im);
            }
    }
    // the last runs into the totals, then the task's partials (the reduce
    // kernel sums the partials of all tasks in Sum2 form)
    minors_fold_fp64(wacc, wtot, stride, lane, K, Hr, H);
    for (int t = lane; t < K; t += 32) {
        const double4 v = wtot[t];
        store_partial(partials + jb.partial_off + (int64_t)local * K + t, ddv{v.x, v.y}, ddv{v.z, v.w});
    }
    __syncwarp();  // the next task's initialisation overwrites the totals
#undef BS_OWN
}

#undef BS_LIVE

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Job owning global task t: the last job (in list order) whose task_begin
// <= t.  Jobs are jobs[i], or jobs[list[i]] when a device-built list is
// given.
__device__ __forceinline__ int find_job(const bs_job* __restrict__ jobs, const int* __restrict__ list, int njobs,
                                        unsigned long long t) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        const int jm = list ? list[mid] : mid;
        if (jobs[jm].task_begin <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return list ? list[lo] : lo;
}

// Pull the next warp task (lane 0 takes it, all lanes learn it).  A task
// index >= total means stop: either the work is done or the deadline passed
// (then the status word says so and the host reports a timeout).
// deadline_ns is absolute (%globaltimer), 0 = none.
__device__ __forceinline__ unsigned long long next_task(unsigned long long* counter, unsigned long long total,
                                                        int* status, unsigned long long deadline_ns, int lane) {
    unsigned long long t = 0;
    if (lane == 0) {
        if (deadline_ns != 0ull && global_ns() > deadline_ns) {
            atomicExch(status, BS_STATUS_TIMEOUT);
            t = total;
        } else {
            t = atomicAdd(counter, 1ull);
        }
    }
    return __shfl_sync(0xffffffffu, t, 0);
}

// Per-warp absolute deadline from a relative one (0 = none).
__device__ __forceinline__ unsigned long long warp_deadline(unsigned long long rel_ns) {
    return rel_ns == 0ull ? 0ull : global_ns() + rel_ns;
}

// Task total and job count: from device memory when planned on the device.
__device__ __forceinline__ unsigned long long task_total(const WalkArgsBase& a) {
    return a.total_dev ? *a.total_dev : a.total_tasks;
}
__device__ __forceinline__ int job_count(const WalkArgsBase& a) { return a.njobs_dev ? *a.njobs_dev : a.njobs; }

}  // namespace bs
