// Double-float ("DF") Gray-walk tasks: FP64-class accuracy on the FP32 pipe.
//
// FP64 runs at 1/64 of the FP32 rate on this part, so the DF kernels carry
// every quantity as an unevaluated pair of floats (about 48 significant bits)
// and do all arithmetic with single-precision FMAs, packed two columns per
// instruction (fma / add / sub / mul .rn.f32x2: even column in the low half,
// odd column in the high half, as in walk_fp32.cuh).
//
// Column sums: exact fixed point.  The pack kernel scales column j by
// 2^(2 - e_j), 2^e_j >= sum_rows M (|Re a| + |Im a|), so every column sum
// has |Re|, |Im| <= 4 for every Delta, and quantises c0 and every 2a to a
// high part on the grid 2^-20 and a low part on the grid 2^-44 (input error
// <= 2^-45 per entry).  The walk keeps each column sum as such a pair
// (h, l): h + A_h and l + A_l are exact float additions (|h| < 16, |l| <=
// 2^-20 fit 24 bits on their grids), and a carry moves the part of l that
// is a multiple of 2^-20 into h after every step: t = (l + 12) - 12 rounds l
// to that grid (ulp of 12 is 2^-20), h += t, l -= t, all exact.  The column
// sums therefore never drift, whatever the chunk length: every addend sees
// exactly c0 - sum_j Delta_j 2a_j of the quantised matrix (a fixed backward
// perturbation of at most 2^-45 per entry).  Before a product the pair is
// normalised by FastTwoSum (exact: |h| >= 2^-20 > |l| or h = 0).
//
// Products: double-float complex multiplication with FMA-based TwoProd:
// for x = (xh + xl), y = (yh + yl) componentwise, each real part of x y is
// formed from exact products xh yh (product and FMA error), one exact TwoSum
// of the two main products, and the cross terms xh yl + xl yh in single
// precision; the dropped xl yl term and the roundings are about 2^-46 of
// |x| |y|.  Outputs are not renormalised (their low parts stay within a few
// ulps of |x| |y|), which the next product tolerates.  A negated addend of
// an FMA would cost a separate instruction on this part, so one multiplicand
// carries the negations of its high parts ("neg" fields) and products are
// formed as -round(a b) = a (-b), with subtractions (sub.rn.f32x2) instead
// of negations.
//
// Sums: each column accumulates Sum2-style (TwoSum on the high parts, the
// errors and low parts in one float) for FOLD addends, then folds into a
// double-float accumulator in shared memory (accurate double-float
// addition); chunk totals are combined across lanes in double-float and
// written as double-double partials, which the reduce kernel sums in twice
// double precision and scales by 2^(1-n) and the column exponents.
#pragma once
#include "sample.h"
#include "walk.cuh"

namespace bs {

// ---------------------------------------------------------------- packed primitives
__device__ __forceinline__ unsigned long long df_bits(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 df_f2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(df_bits(a)), "l"(df_bits(b)));
    return df_f2(d);
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_splat(float x) { return make_float2(x, x); }

// Packed double-float complex pair (two columns).
struct dfc {
    float2 rh, rl, ih, il;
};
// The same with the negated high parts (a multiplicand).
struct dfy {
    float2 rh, rl, ih, il, nrh, nih;
};
// Fixed-point column-sum state of a pair of columns.
struct dfst {
    float2 rh, rl, ih, il;
};

__device__ __forceinline__ dfc df_one() {
    return dfc{make_float2(1.f, 1.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
}
__device__ __forceinline__ dfc df_drop(const dfy& y) { return dfc{y.rh, y.rl, y.ih, y.il}; }

// c += sg * A (A: packed high / low parts of one row pair), exact, then the
// carry of the low part into the high part.
__device__ __forceinline__ void df_update(dfst& c, float4 ah, float4 al, float2 sg) {
    const float2 C = p_splat(12.0f);
    c.rh = p_fma(sg, make_float2(ah.x, ah.y), c.rh);
    c.ih = p_fma(sg, make_float2(ah.z, ah.w), c.ih);
    c.rl = p_fma(sg, make_float2(al.x, al.y), c.rl);
    c.il = p_fma(sg, make_float2(al.z, al.w), c.il);
    const float2 tr = p_sub(p_add(c.rl, C), C);
    const float2 ti = p_sub(p_add(c.il, C), C);
    c.rh = p_add(c.rh, tr);
    c.ih = p_add(c.ih, ti);
    c.rl = p_sub(c.rl, tr);
    c.il = p_sub(c.il, ti);
}

// Normalised double-float value of the state (FastTwoSum, exact).
__device__ __forceinline__ dfc df_norm(const dfst& c) {
    dfc r;
    r.rh = p_add(c.rh, c.rl);
    r.rl = p_sub(c.rl, p_sub(r.rh, c.rh));
    r.ih = p_add(c.ih, c.il);
    r.il = p_sub(c.il, p_sub(r.ih, c.ih));
    return r;
}
__device__ __forceinline__ dfy df_norm_neg(const dfst& c) {
    const dfc v = df_norm(c);
    const float2 z = make_float2(0.f, 0.f);
    return dfy{v.rh, v.rl, v.ih, v.il, p_sub(z, v.rh), p_sub(z, v.ih)};
}

// The real and imaginary parts of x y before the final rounding of the
// imaginary high part: re = (re_h, re_l); im = -(im_nh) + im_l.
struct dfraw {
    float2 re_h, re_l, im_nh, im_l;
};
__device__ __forceinline__ dfraw df_cmul_raw(const dfc& x, const dfy& y) {
    dfraw o;
    // re = xr yr - xi yi
    const float2 np1 = p_mul(x.rh, y.nrh);   // -round(xr yr)
    const float2 e1 = p_fma(x.rh, y.rh, np1);  // xr yr - round(xr yr)
    const float2 np2 = p_mul(x.ih, y.nih);   // -round(xi yi)
    const float2 e2 = p_fma(x.ih, y.ih, np2);
    const float2 s = p_sub(np2, np1);         // round(xr yr) - round(xi yi), rounded
    const float2 bb = p_add(s, np1);
    const float2 t = p_sub(p_sub(np2, bb), p_add(np1, p_sub(s, bb)));  // its TwoSum error
    float2 c = p_fma(x.rh, y.rl, e1);
    c = p_fma(x.rl, y.rh, c);
    float2 d = p_fma(x.ih, y.il, e2);
    d = p_fma(x.il, y.ih, d);
    o.re_h = s;
    o.re_l = p_add(p_sub(c, d), t);
    // im = xr yi + xi yr = -(np3 + np4) + errors
    const float2 np3 = p_mul(x.rh, y.nih);
    const float2 e3 = p_fma(x.rh, y.ih, np3);
    const float2 np4 = p_mul(x.ih, y.nrh);
    const float2 e4 = p_fma(x.ih, y.rh, np4);
    const float2 sn = p_add(np3, np4);
    const float2 bb2 = p_sub(sn, np3);
    const float2 t2 = p_add(p_sub(np3, p_sub(sn, bb2)), p_sub(np4, bb2));  // sn + t2 = np3 + np4
    float2 c2 = p_fma(x.rh, y.il, e3);
    c2 = p_fma(x.rl, y.ih, c2);
    c2 = p_fma(x.ih, y.rl, c2);
    c2 = p_fma(x.il, y.rh, c2);
    o.im_nh = sn;
    o.im_l = p_sub(p_add(c2, e4), t2);
    return o;
}

// x y as a double-float complex pair.
__device__ __forceinline__ dfc df_cmul(const dfc& x, const dfy& y) {
    const dfraw o = df_cmul_raw(x, y);
    return dfc{o.re_h, o.re_l, p_sub(make_float2(0.f, 0.f), o.im_nh), o.im_l};
}
// x y with the negated high parts (to serve as the next multiplicand).
__device__ __forceinline__ dfy df_cmul_neg(const dfc& x, const dfy& y) {
    const dfraw o = df_cmul_raw(x, y);
    const float2 z = make_float2(0.f, 0.f);
    return dfy{o.re_h, o.re_l, p_sub(z, o.im_nh), o.im_l, p_sub(z, o.re_h), o.im_nh};
}

// Sum2 accumulator of a pair of columns: h by TwoSum, errors and low parts in l.
struct dfacc {
    float2 rh, rl, ih, il;
};
// acc += x y.
__device__ __forceinline__ void df_cmul_acc(dfacc& a, const dfc& x, const dfy& y) {
    const dfraw o = df_cmul_raw(x, y);
    // re: TwoSum(a.rh, re_h)
    const float2 s = p_add(a.rh, o.re_h);
    const float2 bb = p_sub(s, a.rh);
    const float2 er = p_add(p_sub(a.rh, p_sub(s, bb)), p_sub(o.re_h, bb));
    a.rh = s;
    a.rl = p_add(a.rl, p_add(er, o.re_l));
    // im: TwoSum(a.ih, -im_nh) as a difference
    const float2 s2 = p_sub(a.ih, o.im_nh);
    const float2 bb2 = p_sub(s2, a.ih);
    const float2 ei = p_sub(p_sub(a.ih, p_sub(s2, bb2)), p_add(o.im_nh, bb2));
    a.ih = s2;
    a.il = p_add(a.il, p_add(ei, o.im_l));
}

// ---------------------------------------------------------------- scalar double-float
struct dfs {
    float h, l;
};
struct dfsc {
    dfs re, im;
};

__device__ __forceinline__ dfs s_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return dfs{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfs s_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfs{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// Accurate double-float addition (two TwoSums, two renormalisations).
__device__ __forceinline__ dfs s_add(dfs a, dfs b) {
    dfs s = s_two_sum(a.h, b.h);
    const dfs t = s_two_sum(a.l, b.l);
    s.l = __fadd_rn(s.l, t.h);
    s = s_fast_two_sum(s.h, s.l);
    s.l = __fadd_rn(s.l, t.l);
    return s_fast_two_sum(s.h, s.l);
}
// x y for scalar double-float complex numbers (the compiler folds the
// negations of scalar operands into the FMAs).
__device__ __forceinline__ dfsc s_cmul(const dfsc& x, const dfsc& y) {
    dfsc o;
    {
        const float p1 = __fmul_rn(x.re.h, y.re.h), e1 = __fmaf_rn(x.re.h, y.re.h, -p1);
        const float p2 = __fmul_rn(x.im.h, y.im.h), e2 = __fmaf_rn(x.im.h, y.im.h, -p2);
        const dfs s = s_two_sum(p1, -p2);
        float c = __fmaf_rn(x.re.h, y.re.l, e1);
        c = __fmaf_rn(x.re.l, y.re.h, c);
        c = __fmaf_rn(-x.im.h, y.im.l, c);
        c = __fmaf_rn(-x.im.l, y.im.h, c);
        o.re = dfs{s.h, __fadd_rn(__fsub_rn(c, e2), s.l)};
    }
    {
        const float p3 = __fmul_rn(x.re.h, y.im.h), e3 = __fmaf_rn(x.re.h, y.im.h, -p3);
        const float p4 = __fmul_rn(x.im.h, y.re.h), e4 = __fmaf_rn(x.im.h, y.re.h, -p4);
        const dfs s = s_two_sum(p3, p4);
        float c = __fmaf_rn(x.re.h, y.im.l, e3);
        c = __fmaf_rn(x.re.l, y.im.h, c);
        c = __fmaf_rn(x.im.h, y.re.l, c);
        c = __fmaf_rn(x.im.l, y.re.h, c);
        o.im = dfs{s.h, __fadd_rn(__fadd_rn(c, e4), s.l)};
    }
    return o;
}
// w x for a double-float real w.
__device__ __forceinline__ dfsc s_rmul(dfs w, const dfsc& x) {
    dfsc o;
    const float p = __fmul_rn(w.h, x.re.h), e = __fmaf_rn(w.h, x.re.h, -p);
    o.re = dfs{p, __fmaf_rn(w.h, x.re.l, __fmaf_rn(w.l, x.re.h, e))};
    const float q = __fmul_rn(w.h, x.im.h), f = __fmaf_rn(w.h, x.im.h, -q);
    o.im = dfs{q, __fmaf_rn(w.h, x.im.l, __fmaf_rn(w.l, x.im.h, f))};
    return o;
}
__device__ __forceinline__ dfsc shfl_xor_dfsc(const dfsc& v, int m) {
    return dfsc{dfs{__shfl_xor_sync(0xffffffffu, v.re.h, m), __shfl_xor_sync(0xffffffffu, v.re.l, m)},
                dfs{__shfl_xor_sync(0xffffffffu, v.im.h, m), __shfl_xor_sync(0xffffffffu, v.im.l, m)}};
}
__device__ __forceinline__ dfs shfl_down_dfs(dfs v, int off) {
    return dfs{__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off)};
}
// Low / high half of a packed pair as a scalar complex.
__device__ __forceinline__ dfsc df_half(const dfc& v, int hi) {
    return hi ? dfsc{dfs{v.rh.y, v.rl.y}, dfs{v.ih.y, v.il.y}} : dfsc{dfs{v.rh.x, v.rl.x}, dfs{v.ih.x, v.il.x}};
}

// The signed binomial weight (-1)^parity W as an exact double-float
// (W < 2^48: its high and low 24 bits are exact floats).
__device__ __forceinline__ dfs df_weight(uint64_t w, int parity) {
    const float hi = (float)(w & ~0xFFFFFFull), lo = (float)(w & 0xFFFFFFull);
    const dfs r = s_fast_two_sum(hi, lo);
    return parity ? dfs{-r.h, -r.l} : r;
}

// Exact double-double of a double-float (the sum of two floats fits a double).
__device__ __forceinline__ ddv dd_from_dfs(dfs a) { return ddv{(double)a.h + (double)a.l, 0.0}; }

// Packed DF rows: pair p of a row is two float4, {re h (2p), re h (2p+1),
// im h (2p), im h (2p+1)} then the low parts; a row of the bucket width KB
// takes KB float4 (16 bytes per column, as one complex double).
__device__ __forceinline__ void df_load_pair(const float4* __restrict__ row, int p, float4& h, float4& l) {
    h = __ldg(row + 2 * p);
    l = __ldg(row + 2 * p + 1);
}

// Seed the fixed-point state of NP pairs (from pair p0) at the decoded Gray
// state: c = c0 - sum_j Delta_j 2a_j by exact additions (a repeated digit's
// row is added Delta_j times).
template <int NP>
__device__ __forceinline__ void df_seed(dfst (&c)[NP], const bs_gray& g, const float4* __restrict__ c0,
                                        const float4* __restrict__ a2, int KB4, int p0, int nbin, int nrows) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float4 h, l;
        df_load_pair(c0, p0 + p, h, l);
        c[p] = dfst{make_float2(h.x, h.y), make_float2(l.x, l.y), make_float2(h.z, h.w), make_float2(l.z, l.w)};
    }
    const float2 m1 = p_splat(-1.0f);
    uint64_t bits = g.dbin;
    while (bits) {
        const int j = bs_ctz64(bits);
        bits &= bits - 1;
        const float4* row = a2 + (size_t)j * KB4;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float4 h, l;
            df_load_pair(row, p0 + p, h, l);
            df_update(c[p], h, l, m1);
        }
    }
    for (int j = nbin; j < nrows; ++j) {
        const float4* row = a2 + (size_t)j * KB4;
        for (int d = 0; d < g.del[j]; ++d) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float4 h, l;
                df_load_pair(row, p0 + p, h, l);
                df_update(c[p], h, l, m1);
            }
        }
    }
}

// Fold the Sum2 accumulators into the double-float sums in shared memory
// ([column][thread] float4 {re h, re l, im h, im l}) and clear them.  The
// accumulators are first staged to a second [column][thread] array; the
// additions then run in a rolled loop, so their temporaries stay out of the
// walk's registers.
template <int NP>
__device__ __forceinline__ void df_fold(float4* __restrict__ sm, float4* __restrict__ stage, int stride,
                                        dfacc (&a)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        stage[(2 * p) * stride] = make_float4(a[p].rh.x, a[p].rl.x, a[p].ih.x, a[p].il.x);
        stage[(2 * p + 1) * stride] = make_float4(a[p].rh.y, a[p].rl.y, a[p].ih.y, a[p].il.y);
        a[p] = dfacc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    }
#pragma unroll 1
    for (int t = 0; t < 2 * NP; ++t) {
        const float4 f = sm[t * stride], g = stage[t * stride];
        const dfs re = s_add(dfs{f.x, f.y}, s_two_sum(g.x, g.y));
        const dfs im = s_add(dfs{f.z, f.w}, s_two_sum(g.z, g.w));
        sm[t * stride] = make_float4(re.h, re.l, im.h, im.l);
    }
}

// ---------------------------------------------------------------- one task: minors
// G lanes share one chunk; lane (G c + q) owns the NP = KB / (2G) column
// pairs [q NP, q NP + NP).  Per addend each lane
//   1. forms the suffix products of its own pairs from 1 (two chains, even
//      and odd columns, in the packed halves); the last is {Q_even, Q_odd};
//   2. learns the product Q' of the other lanes' Q = Q_even Q_odd by G - 1
//      butterfly rounds;
//   3. runs the prefix pass from X = (+-W) Q' times the other half of its
//      own columns, {X Q_odd, X Q_even}:  acc[l] += suffix_l * prefix_l.
// All lanes run the warp's longest chunk; a lane past its chunk keeps its
// column sums and continues with weight 0, so the shuffles have the full
// warp.
template <int KB>
__device__ void walk_task_minors_df(const bs_job& jb, const void* __restrict__ data_v,
                                    const int* __restrict__ radix, bs_zdd* __restrict__ partials, uint32_t local,
                                    int lane, float4* __restrict__ sm, float4* __restrict__ stage, int stride) {
    constexpr uint32_t FOLD = 64;
    constexpr int G = BS_DF_GROUP_KB(KB);
    constexpr int NP = KB / (2 * G);
    constexpr int CPT = 32 / G;
    static_assert(KB % (2 * G) == 0, "bucket must split into G groups of column pairs");
    const int K = jb.K;
    const int q = lane & (G - 1);
    const int p0 = q * NP;
    const int cbase = 2 * p0;
    const float4* c0 = static_cast<const float4*>(data_v) + jb.data_off;  // 16-byte units
    const float4* a2 = c0 + KB;
#pragma unroll
    for (int t = 0; t < 2 * NP; ++t) sm[t * stride] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint64_t i0_own = ((uint64_t)local * CPT + (uint64_t)(lane / G)) << jb.log2L;
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
    dfst c[NP];
    df_seed<NP>(c, g, c0, a2, KB, p0, jb.nbin, jb.nrows);
    dfs ws = has ? df_weight(g.w, g.parity) : dfs{0.f, 0.f};
    dfacc acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
        acc[p] = dfacc{make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    for (uint32_t s = 0; s < steps; ++s) {
        // 1. suffix products over own pairs
        dfc suf[NP];
        suf[NP - 1] = df_one();
        dfc sfx = df_norm(c[NP - 1]);
#pragma unroll
        for (int p = NP - 2; p >= 0; --p) {
            suf[p] = sfx;
            sfx = df_cmul(sfx, df_norm_neg(c[p]));
        }
        const dfsc qe = df_half(sfx, 0), qo = df_half(sfx, 1);
        // 2. the other lanes' product Q'
        dfsc qx = dfsc{dfs{1.f, 0.f}, dfs{0.f, 0.f}};
        if constexpr (G > 1) {
            const dfsc qown = s_cmul(qe, qo);
            qx = shfl_xor_dfsc(qown, 1);
            if constexpr (G >= 4) {
                const dfsc pair = s_cmul(qown, qx);
                qx = s_cmul(qx, shfl_xor_dfsc(pair, 2));
                if constexpr (G >= 8) {
                    const dfsc quad = s_cmul(pair, shfl_xor_dfsc(pair, 2));
                    qx = s_cmul(qx, shfl_xor_dfsc(quad, 4));
                }
            }
        }
        // 3. prefix pass from {X Q_odd, X Q_even}, X = (+-W) Q'
        const dfsc X = s_rmul(ws, qx);
        const dfc xs = {p_splat(X.re.h), p_splat(X.re.l), p_splat(X.im.h), p_splat(X.im.l)};
        const float2 z = make_float2(0.f, 0.f);
        const dfy qsw = {make_float2(qo.re.h, qe.re.h), make_float2(qo.re.l, qe.re.l),
                         make_float2(qo.im.h, qe.im.h), make_float2(qo.im.l, qe.im.l),
                         p_sub(z, make_float2(qo.re.h, qe.re.h)), p_sub(z, make_float2(qo.im.h, qe.im.h))};
        dfy pre = df_cmul_neg(xs, qsw);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            df_cmul_acc(acc[p], suf[p], pre);
            if (p + 1 < NP) pre = df_cmul_neg(df_norm(c[p]), pre);
        }
        if (((s + 1u) & (FOLD - 1u)) == 0) df_fold<NP>(sm, stage, stride, acc);
        if (s + 1u >= steps) break;
        if (s + 1u >= len) {  // this lane's chunk is done: weight 0 from here on
            ws = dfs{0.f, 0.f};
            continue;
        }
        uint32_t neg;
        int wch;
        const int row = st.step(g, s, radix, &neg, &wch);
        ws = wch ? df_weight(g.w, g.parity) : dfs{-ws.h, -ws.l};
        const float2 sg = p_splat(neg ? -1.0f : 1.0f);
        const float4* rp = a2 + (size_t)row * KB;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float4 h, l;
            df_load_pair(rp, p0 + p, h, l);
            df_update(c[p], h, l, sg);
        }
    }
    df_fold<NP>(sm, stage, stride, acc);
    // combine the chunks of the task (lanes of equal q) in double-float;
    // lane q < G ends with the sums of its columns
    const int KH = min(2 * NP, max(K - cbase, 0));
    for (int t = 0; t < 2 * NP; ++t) {
        const float4 f = sm[t * stride];
        dfs re = {f.x, f.y}, im = {f.z, f.w};
#pragma unroll
        for (int off = 16; off >= G; off >>= 1) {
            re = s_add(re, shfl_down_dfs(re, off));
            im = s_add(im, shfl_down_dfs(im, off));
        }
        if (lane < G && t < KH)
            store_partial(partials + jb.partial_off + (int64_t)local * K + cbase + t, dd_from_dfs(re),
                          dd_from_dfs(im));
    }
}

// ---------------------------------------------------------------- one task: permanent
// G lanes share one chunk, each owning NP column pairs; per addend a lane
// forms the product of its pairs (two packed chains), Q = Q_even Q_odd, and
// the G lanes multiply their Q in a butterfly; lane q = 0 of each group adds
// (+-W) prod Q to its Sum2 accumulator, folded into a double-float total
// every FOLD addends.
template <int KB>
__device__ void walk_task_perm_df(const bs_job& jb, const void* __restrict__ data_v, const int* __restrict__ radix,
                                  bs_zdd* __restrict__ partials, uint32_t local, int lane) {
    constexpr uint32_t FOLD = 64;
    constexpr int G = BS_DF_GROUP_KB(KB);
    constexpr int NP = KB / (2 * G);
    constexpr int CPT = 32 / G;
    static_assert(KB % (2 * G) == 0, "bucket must split into G groups of column pairs");
    const int q = lane & (G - 1);
    const int p0 = q * NP;
    const float4* c0 = static_cast<const float4*>(data_v) + jb.data_off;
    const float4* a2 = c0 + KB;
    const uint64_t i0_own = ((uint64_t)local * CPT + (uint64_t)(lane / G)) << jb.log2L;
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
    dfst c[NP];
    df_seed<NP>(c, g, c0, a2, KB, p0, jb.nbin, jb.nrows);
    dfs ws = has ? df_weight(g.w, g.parity) : dfs{0.f, 0.f};
    dfs are = {0.f, 0.f}, aim = {0.f, 0.f};   // Sum2 state
    dfs tre = {0.f, 0.f}, tim = {0.f, 0.f};   // folded totals
    for (uint32_t s = 0; s < steps; ++s) {
        dfc pr = df_norm(c[NP - 1]);
#pragma unroll
        for (int p = NP - 2; p >= 0; --p) pr = df_cmul(pr, df_norm_neg(c[p]));
        dfsc Q = s_cmul(df_half(pr, 0), df_half(pr, 1));
        if constexpr (G > 1) {
            Q = s_cmul(Q, shfl_xor_dfsc(Q, 1));
            if constexpr (G >= 4) Q = s_cmul(Q, shfl_xor_dfsc(Q, 2));
            if constexpr (G >= 8) Q = s_cmul(Q, shfl_xor_dfsc(Q, 4));
        }
        const dfsc a = s_rmul(ws, Q);
        // Sum2: TwoSum of the high parts, errors and low parts in l
        const dfs sr = s_two_sum(are.h, a.re.h);
        are = dfs{sr.h, __fadd_rn(are.l, __fadd_rn(sr.l, a.re.l))};
        const dfs si = s_two_sum(aim.h, a.im.h);
        aim = dfs{si.h, __fadd_rn(aim.l, __fadd_rn(si.l, a.im.l))};
        if (((s + 1u) & (FOLD - 1u)) == 0) {
            tre = s_add(tre, s_two_sum(are.h, are.l));
            tim = s_add(tim, s_two_sum(aim.h, aim.l));
            are = aim = dfs{0.f, 0.f};
        }
        if (s + 1u >= steps) break;
        if (s + 1u >= len) {
            ws = dfs{0.f, 0.f};
            continue;
        }
        uint32_t neg;
        int wch;
        const int row = st.step(g, s, radix, &neg, &wch);
        ws = wch ? df_weight(g.w, g.parity) : dfs{-ws.h, -ws.l};
        const float2 sg = p_splat(neg ? -1.0f : 1.0f);
        const float4* rp = a2 + (size_t)row * KB;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float4 h, l;
            df_load_pair(rp, p0 + p, h, l);
            df_update(c[p], h, l, sg);
        }
    }
    tre = s_add(tre, s_two_sum(are.h, are.l));
    tim = s_add(tim, s_two_sum(aim.h, aim.l));
    // lanes q = 0 hold the chunk totals; combine them over the task
    if (q != 0) tre = tim = dfs{0.f, 0.f};
    ddv re = dd_from_dfs(tre), im = dd_from_dfs(tim);
    warp_reduce_zdd(re, im);
    if (lane == 0) store_partial(partials + jb.partial_off + local, re, im);
}

}  // namespace bs
