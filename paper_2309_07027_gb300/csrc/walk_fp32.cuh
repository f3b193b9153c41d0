// FP32 ("mixed") Gray-walk tasks on packed single-precision pairs.
//
// Data layout (written by pack_job for FP32 jobs): every row of the packed
// matrix (c0, then 2a per digit row) stores its columns in pairs,
//     pair p = { re(2p), re(2p+1), im(2p), im(2p+1) }    (16 bytes),
// so one 16-byte load fills the two packed registers {re even, re odd} and
// {im even, im odd}.  Each thread keeps its column sums as such pairs and
// runs the even and the odd columns as two independent chains in the two
// halves of `fma.rn.f32x2` / `mul.rn.f32x2` instructions: one issue slot
// does the work of two scalar FP32 instructions, and the two chains give the
// scheduler independent work.
//
// The one minus sign of a complex product, re(a b) = re a re b - im a im b,
// is a negation of the packed product im a im b before the packed FMA.
// (Carrying nim = -im beside every column sum instead costs one packed FMA
// per pair and step on the FMA pipe, which bounds these kernels: without it
// the permanent runs 7 % and the sampler's fused minors 1.4 % faster.)
//
// Rounding: every product, update and accumulation rounds exactly as the
// scalar single-precision form of the same expression order (packed
// instructions round each half as the scalar instruction does), so the
// error model of the MIXED precision rule applies unchanged.
#pragma once
#include "sample.h"
#include "walk.cuh"

namespace bs {

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2splat(float x) { return make_float2(x, x); }

// Two complex numbers (even column, odd column) as packed halves.
struct cx2 {
    float2 re, im;
};

__device__ __forceinline__ float2 f2neg(float2 x) { return make_float2(-x.x, -x.y); }

// A pair of column sums.
struct colsum {
    float2 re, im;
};

// a * c for both halves.
__device__ __forceinline__ cx2 cmul2(cx2 a, const colsum& c) {
    cx2 r;
    r.re = f2fma(a.re, c.re, f2neg(f2mul(a.im, c.im)));
    r.im = f2fma(a.re, c.im, f2mul(a.im, c.re));
    return r;
}

__device__ __forceinline__ cx2 as_cx2(const colsum& c) { return cx2{c.re, c.im}; }

// Scalar complex product of the two halves (even * odd).
__device__ __forceinline__ cx<float> halves_product(cx2 a) {
    return cmul(cx<float>{a.re.x, a.im.x}, cx<float>{a.re.y, a.im.y});
}

// One packed row pair: 16 bytes at pair index p of a row.
__device__ __forceinline__ void load_pair(const float4* __restrict__ row, int p, float2& re, float2& im) {
    const float4 v = __ldg(row + p);
    re = make_float2(v.x, v.y);
    im = make_float2(v.z, v.w);
}

// c[p] += cf * row pair p for the NP pairs starting at pair p0.
template <int NP>
__device__ __forceinline__ void update_pairs(colsum (&c)[NP], const float4* __restrict__ row, int p0, float cf) {
    const float2 f = f2splat(cf);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 re, im;
        load_pair(row, p0 + p, re, im);
        c[p].re = f2fma(f, re, c[p].re);
        c[p].im = f2fma(f, im, c[p].im);
    }
}

// Seed NP column pairs (from pair p0) of the decoded state:
// c = c0 - sum_j Delta_j 2a_j; rows have KP / 2 pairs.
template <int NP>
__device__ __forceinline__ void seed_pairs(colsum (&c)[NP], const bs_gray& g, const float4* __restrict__ c0,
                                           const float4* __restrict__ a2, int KP2, int p0, int nbin, int nrows) {
#pragma unroll
    for (int p = 0; p < NP; ++p) load_pair(c0, p0 + p, c[p].re, c[p].im);
    uint64_t bits = g.dbin;
    while (bits) {
        const int j = bs_ctz64(bits);
        bits &= bits - 1;
        const float4* row = a2 + (size_t)j * KP2;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 re, im;
            load_pair(row, p0 + p, re, im);
            c[p].re = make_float2(c[p].re.x - re.x, c[p].re.y - re.y);
            c[p].im = make_float2(c[p].im.x - im.x, c[p].im.y - im.y);
        }
    }
    for (int j = nbin; j < nrows; ++j) {
        const int d = g.del[j];
        if (d == 0) continue;
        const float2 fd = f2splat((float)(-d));
        const float4* row = a2 + (size_t)j * KP2;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 re, im;
            load_pair(row, p0 + p, re, im);
            c[p].re = f2fma(fd, re, c[p].re);
            c[p].im = f2fma(fd, im, c[p].im);
        }
    }
}

// Re-seeding inside a chunk (jobs with reseed_log2 > 0, set by the MIXED
// rule): at the steps s + 1 that are multiples of 2^reseed_log2 the column
// sums are computed afresh from the matrix for the current Gray state
// instead of updated, so the incremental FP32 sums drift no further than in
// a chunk of that length.  The stepper's binary Delta bits are written back
// to the Gray state first (between general steps it holds them alone).
__device__ __forceinline__ bool reseed_due(const bs_job& jb, uint32_t s1) {
    return jb.reseed_log2 > 0 && (s1 & ((1u << jb.reseed_log2) - 1u)) == 0;
}

// ---------------------------------------------------------------- one task: permanent
// One lane = one chunk; all KB columns as KB/2 packed pairs (pad columns are
// neutral).  Per addend: the packed update, one packed product chain (even
// and odd columns), the product of its two halves, and the weighted sum in a
// short single-precision run folded into float-float every 32 addends.
template <int KB>
__device__ void walk_task_perm_fp32(const bs_job& jb, const void* __restrict__ data_v, const int* __restrict__ radix,
                                    bs_zdd* __restrict__ partials, uint32_t local, int lane) {
    constexpr uint32_t FOLD = 32;
    constexpr int NP = KB / 2;
    const int K = jb.K;
    constexpr int KP2 = KB / 2;  // pairs per row: BS_ROW_STRIDE(K) = KB in the bucket
    const float4* c0 = static_cast<const float4*>(data_v) + jb.data_off / 2;
    const float4* a2 = c0 + KP2;
    ffv fre = {0.f, 0.f}, fim = {0.f, 0.f};
    const uint64_t i0 = ((uint64_t)local * 32u + (uint64_t)lane) << jb.log2L;
    if (i0 < jb.C) {
        const uint64_t rem = jb.C - i0;
        const uint32_t len = (uint32_t)(rem < (1ull << jb.log2L) ? rem : (1ull << jb.log2L));
        bs_gray g;
        ChunkStepper st;
        st.init(g, i0, jb.nbin, jb.nrows, radix, reinterpret_cast<const uint64_t*>(radix + (BS_META_BINOM(jb) - jb.meta_off)));
        colsum c[NP];
        float ws = signed_weight<float>(g.w, g.parity);
        cx<float> acc = {0.f, 0.f};
        uint32_t run = 0;
        // segments of 2^reseed_log2 steps (the whole chunk without
        // re-seeding), each starting from column sums seeded afresh
        const uint32_t seg_mask = jb.reseed_log2 > 0 ? (1u << jb.reseed_log2) - 1u : 0xffffffffu;
        for (uint32_t s = 0;; ++s) {
            seed_pairs<NP>(c, g, c0, a2, KP2, 0, jb.nbin, jb.nrows);
            const uint32_t s_last = min(len - 1u, s | seg_mask);
            for (;; ++s) {
                cx2 pr = as_cx2(c[0]);
#pragma unroll
                for (int p = 1; p < NP; ++p) pr = cmul2(pr, c[p]);
                const cx<float> prod = halves_product(pr);
                acc.re = bfma(ws, prod.re, acc.re);
                acc.im = bfma(ws, prod.im, acc.im);
                if (++run == FOLD) {
                    run = 0;
                    fre = ff_add_f(fre, acc.re);
                    fim = ff_add_f(fim, acc.im);
                    acc = cx<float>{0.f, 0.f};
                }
                if (s == s_last) break;
                uint32_t neg;
                int wch;
                const int row = st.step(g, s, radix, &neg, &wch);
                ws = wch ? signed_weight<float>(g.w, g.parity) : flip_sign(ws);
                update_pairs<NP>(c, a2 + (size_t)row * KP2, 0, unit_sign_f(neg));
            }
            if (s + 1u == len) break;
            // into the next segment: its column sums are seeded at the top
            uint32_t neg;
            int wch;
            (void)st.step(g, s, radix, &neg, &wch);
            ws = wch ? signed_weight<float>(g.w, g.parity) : flip_sign(ws);
            g.dbin = (g.dbin & ~0xffffffffull) | (uint64_t)st.dlo;
        }
        fre = ff_add_f(fre, acc.re);
        fim = ff_add_f(fim, acc.im);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        fre = ff_add(fre, shfl_down_ff(fre, off));
        fim = ff_add(fim, shfl_down_ff(fim, off));
    }
    if (lane == 0) store_partial(partials + jb.partial_off + local, dd_from_ff(fre), dd_from_ff(fim));
}

// ---------------------------------------------------------------- one task: minors
// G lanes share one chunk (bs_minors_fp32_group): lane (G c + q) owns the
// NP = KB / (2G) column pairs [q NP, q NP + NP), i.e. columns
// [2 q NP, 2 q NP + 2 NP).  Per addend each lane
//   1. forms packed suffix products over its own pairs, starting from 1;
//      the last one is {Q_even, Q_odd}, the products of its even and of its
//      odd columns, and Q = Q_even Q_odd;
//   2. learns the product Q' of the other lanes' Q by butterfly shuffles:
//      Q' = Q_(q^1) (G = 2), or Q_(q^1) (Q_(q^2) Q_(q^3)) (G = 4);
//   3. runs the packed prefix pass from X = (+-W) Q' times the other half of
//      its own columns, {X Q_odd, X Q_even}:
//          acc[l] += X_half * prefix_l * suffix_l.
// The lanes run the same instructions; a warp task covers 32 / G chunks.  Pad
// columns are neutral (sum 1), so every lane runs all its pairs without
// tests.  All lanes run the warp's longest chunk length: a lane whose chunk is
// shorter (the job's last chunk) or absent continues with weight 0, so the
// shuffles always have the full warp.  Float-float fold targets live in
// shared memory, [col][thread]; the cross-lane sums stay in float-float.
//
// Schedule.  Chunk starts are multiples of L, so at step s every lane moves
// the same digit: a binary digit (row ctz(s + 1)) unless s + 1 is a multiple
// of 2^nbin.  The walk therefore runs in blocks that end at every such step
// and at every fold point (s + 1 a multiple of FOLD); inside a block the loop
// body is branch-free and software-pipelined: the prefix pass of addend s
// (which reads the column sums of s) and the step plus steps 1-2 of addend
// s + 1 are independent, so the scheduler can overlap the shuffles and the
// dependent product chains of one addend with the arithmetic of the other.
// A lane past the end of its chunk keeps stepping binary digits inside a
// block (any row < nbin is a valid row; its weight is 0) and stops stepping
// at block ends, where the mixed-radix step is taken.

// Steps 1-2 for the current column sums: suffix products, {Q_even, Q_odd} and
// the other lanes' product Q'.
template <int NP, int G>
__device__ __forceinline__ void minors_suffix(const colsum (&c)[NP], cx2 (&suf)[NP], cx<float>& qe,
                                              cx<float>& qo, cx<float>& qx) {
    suf[NP - 1] = cx2{make_float2(1.f, 1.f), make_float2(0.f, 0.f)};
    cx2 sfx = as_cx2(c[NP - 1]);
#pragma unroll
    for (int p = NP - 2; p >= 0; --p) {
        suf[p] = sfx;
        sfx = cmul2(sfx, c[p]);
    }
    qe = cx<float>{sfx.re.x, sfx.im.x};
    qo = cx<float>{sfx.re.y, sfx.im.y};
    const cx<float> qown = cmul(qe, qo);
    qx.re = __shfl_xor_sync(0xffffffffu, qown.re, 1);
    qx.im = __shfl_xor_sync(0xffffffffu, qown.im, 1);
    if constexpr (G == 4) {
        const cx<float> pair = cmul(qown, qx);
        cx<float> q2;
        q2.re = __shfl_xor_sync(0xffffffffu, pair.re, 2);
        q2.im = __shfl_xor_sync(0xffffffffu, pair.im, 2);
        qx = cmul(qx, q2);
    }
}

// Step 3: the packed prefix pass from {X Q_odd, X Q_even}, X = ws Q'.
template <int NP>
__device__ __forceinline__ void minors_prefix(const colsum (&c)[NP], const cx2 (&suf)[NP], cx<float> qe,
                                              cx<float> qo, cx<float> qx, float ws, float2 (&are)[NP],
                                              float2 (&aim)[NP]) {
    const cx<float> x = {ws * qx.re, ws * qx.im};
    const cx<float> xe = cmul(x, qo), xo = cmul(x, qe);
    cx2 pre = {make_float2(xe.re, xo.re), make_float2(xe.im, xo.im)};
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        are[p] = f2fma(pre.re, suf[p].re, are[p]);
        are[p] = f2fma(f2neg(pre.im), suf[p].im, are[p]);
        aim[p] = f2fma(pre.re, suf[p].im, aim[p]);
        aim[p] = f2fma(pre.im, suf[p].re, aim[p]);
        if (p + 1 < NP) pre = cmul2(pre, c[p]);
    }
}

// Fold the plain-float runs into the float-float sums in shared memory.
template <int NP>
__device__ __forceinline__ void minors_fold(float4* __restrict__ sm_ff, int stride, float2 (&are)[NP],
                                            float2 (&aim)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4* slot = sm_ff + (2 * p + h) * stride;
            float4 f = *slot;
            ffv re = {f.x, f.y}, im = {f.z, f.w};
            re = ff_add_f(re, h ? are[p].y : are[p].x);
            im = ff_add_f(im, h ? aim[p].y : aim[p].x);
            *slot = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
        are[p] = aim[p] = make_float2(0.f, 0.f);
    }
}

template <int KB>
__device__ void walk_task_minors_fp32(const bs_job& jb, const void* __restrict__ data_v,
                                      const int* __restrict__ radix, bs_zdd* __restrict__ partials, uint32_t local,
                                      int lane, float4* __restrict__ sm_ff, int stride) {
    constexpr uint32_t FOLD = 128;
    constexpr int LOG2_FOLD = 7;
    constexpr int G = BS_MINORS_FP32_GROUP_KB(KB);
    constexpr int NP = KB / (2 * G);
    constexpr int CPT = 32 / G;
    static_assert(KB % (2 * G) == 0, "bucket must split into G groups of column pairs");
    static_assert(FOLD == 1u << LOG2_FOLD, "fold length is a power of two");
    static_assert(BS_FP32_RESEED_LOG2 >= LOG2_FOLD, "re-seed points must be block ends");
    const int K = jb.K;
    constexpr int KP2 = KB / 2;  // pairs per row: BS_ROW_STRIDE(K) = KB in the bucket
    const int q = lane & (G - 1);
    const int p0 = q * NP;         // first own pair
    const int cbase = 2 * p0;      // first own column
    const float4* c0 = static_cast<const float4*>(data_v) + jb.data_off / 2;
    const float4* a2 = c0 + KP2;
#pragma unroll
    for (int t = 0; t < 2 * NP; ++t) sm_ff[t * stride] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint64_t i0_own = ((uint64_t)local * CPT + (uint64_t)(lane / G)) << jb.log2L;
    const bool has = i0_own < jb.C;
    const uint64_t i0 = has ? i0_own : 0ull;
    uint32_t len = 0;
    if (has) {
        const uint64_t rem = jb.C - i0;
        len = (uint32_t)(rem < (1ull << jb.log2L) ? rem : (1ull << jb.log2L));
    }
    const uint32_t steps = __reduce_max_sync(0xffffffffu, len);  // >= 1: a task's first chunk exists
    bs_gray g;
    ChunkStepper st;
    st.init(g, i0, jb.nbin, jb.nrows, radix, reinterpret_cast<const uint64_t*>(radix + (BS_META_BINOM(jb) - jb.meta_off)));
    colsum c[NP];
    seed_pairs<NP>(c, g, c0, a2, KP2, p0, jb.nbin, jb.nrows);
    float ws = has ? signed_weight<float>(g.w, g.parity) : 0.f;
    float2 are[NP], aim[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) are[p] = aim[p] = make_float2(0.f, 0.f);
    cx2 suf[NP];
    cx<float> qe, qo, qx;
    minors_suffix<NP, G>(c, suf, qe, qo, qx);
    // blocks end where s + 1 is a multiple of min(FOLD, 2^nbin)
    const uint32_t block_mask = (1u << min(jb.nbin, LOG2_FOLD)) - 1u;
    uint32_t s = 0;
    for (;;) {
        const uint32_t e = min(steps - 1u, s | block_mask);
        for (; s < e; ++s) {
            minors_prefix<NP>(c, suf, qe, qo, qx, ws, are, aim);
            uint32_t neg;
            const int row = st.step_bin(s + 1u, &neg);
            ws = s + 1u < len ? flip_sign(ws) : 0.f;
            update_pairs<NP>(c, a2 + (size_t)row * KP2, p0, unit_sign_f(neg));
            minors_suffix<NP, G>(c, suf, qe, qo, qx);
        }
        minors_prefix<NP>(c, suf, qe, qo, qx, ws, are, aim);
        if (((s + 1u) & (FOLD - 1u)) == 0) minors_fold<NP>(sm_ff, stride, are, aim);
        if (s + 1u >= steps) break;
        if (s + 1u < len) {
            uint32_t neg;
            int wch;
            const int row = st.step(g, s, radix, &neg, &wch);
            ws = wch ? signed_weight<float>(g.w, g.parity) : flip_sign(ws);
            // re-seed points (multiples of 2^reseed_log2 >= 2^8) are block ends
            if (reseed_due(jb, s + 1u)) {
                g.dbin = (g.dbin & ~0xffffffffull) | (uint64_t)st.dlo;
                seed_pairs<NP>(c, g, c0, a2, KP2, p0, jb.nbin, jb.nrows);
            } else {
                update_pairs<NP>(c, a2 + (size_t)row * KP2, p0, unit_sign_f(neg));
            }
        } else {
            ws = 0.f;
        }
        minors_suffix<NP, G>(c, suf, qe, qo, qx);
        ++s;
    }
    minors_fold<NP>(sm_ff, stride, are, aim);
    // reduce over the chunks of the task in float-float (lanes of equal q);
    // lane q < G ends with the sums of its columns
    const int KH = min(2 * NP, max(K - cbase, 0));
    for (int t = 0; t < 2 * NP; ++t) {
        const float4 f = sm_ff[t * stride];
        ffv re = {f.x, f.y}, im = {f.z, f.w};
#pragma unroll
        for (int off = 16; off >= G; off >>= 1) {
            re = ff_add(re, shfl_down_ff(re, off));
            im = ff_add(im, shfl_down_ff(im, off));
        }
        if (lane < G && t < KH)
            store_partial(partials + jb.partial_off + (int64_t)local * K + cbase + t, dd_from_ff(re), dd_from_ff(im));
    }
}

}  // namespace bs
