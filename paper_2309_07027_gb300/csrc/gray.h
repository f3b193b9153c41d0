// Reflected n-ary (Guan) Gray counter over the digit rows of a job
// (Sec. 2.2, Eq. bbfgrepeated; the binary special case is Sec. 2.1).
//
// Index i in [0, C) is a mixed-radix number with digit j of radix R_j
// (digit 0 least significant), counter digits a_j.  Its Gray code is
//     Delta_j = a_j                 if floor(i / (R_0...R_j)) is even
//     Delta_j = R_j - 1 - a_j       otherwise.
// Going from i to i+1 exactly one digit changes by +-1: the lowest j with
// a_j != R_j - 1; it moves up when floor(i / (R_0...R_j)) is even, down
// otherwise, and every lower digit (all at their end) reverses direction.
// Any index can be decoded in O(#digits), so index ranges can be walked
// independently (Sec. 2.1: contiguous subsets processed concurrently).
//
// The first nbin digits have radix 2 (rows of multiplicity 1).  Their Delta
// bits are kept as a mask: for those digits the code is the binary reflected
// code of the low bits, lo ^ (lo >> 1), whose top bit is reflected once more
// by the parity of the higher part; a step inside the binary part flips the
// bit at the lowest zero bit of lo (Sec. 2.1: the changed bit is the lowest
// set bit of the next index).
//
// Weights: W = prod_j C(M_j, Delta_j) over multi digits (binary digits have
// weight 1) kept as an exact 64-bit integer.  The kernels read C(M_j, d)
// from a per-job table and recompute the product after a multi-digit move
// (no integer division on the device).  Without a table the update is the
// ratio form of Appendix A.3 (Eq. simplified_binomial, with the +-1 cases as
// derived here): on a +1 move C(M, D+1) = C(M, D) (M - D) / (D + 1), on a -1
// move C(M, D-1) = C(M, D) D / (M - D + 1), both exact integer quotients.
#pragma once
#include <stdint.h>
#include "bs_job.h"

#if defined(__CUDACC__)
#define BS_HD __host__ __device__ __forceinline__
#else
#define BS_HD inline
#endif

BS_HD int bs_ctz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}

BS_HD int bs_popc64(uint64_t x) {
#if defined(__CUDA_ARCH__)
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}

// Exact C(m, d) for 0 <= d <= m <= 60 (each partial product is an integer).
BS_HD uint64_t bs_binom(int m, int d) {
    if (d < 0 || d > m) return 0;
    if (d > m - d) d = m - d;
    uint64_t v = 1;
    for (int t = 1; t <= d; ++t) v = v * (uint64_t)(m - d + t) / (uint64_t)t;
    return v;
}

struct bs_gray {
    uint64_t i;        // current addend index
    uint64_t binmask;  // (1 << nbin) - 1
    uint64_t dbin;     // Delta bits of the binary digits
    uint64_t w;        // prod of binomials over multi digits (exact)
    int parity;        // (sum Delta) mod 2 -> sign of the addend
    int nbin, nrows;
    int8_t cnt[BS_MAX_DIGITS];  // mixed-radix counter digits (multi digits)
    int8_t dir[BS_MAX_DIGITS];  // +1 / -1 move direction (multi digits)
    int8_t del[BS_MAX_DIGITS];  // Delta (multi digits)
};

// Decode index i (constant time per digit).  binom (nullable): the job's
// table of C(M_j, d), digit after digit (binary digits first, 2 entries
// each); without it the weights are computed directly.
BS_HD void bs_gray_decode(bs_gray& g, uint64_t i, int nbin, int nrows, const int* radix,
                          const uint64_t* binom = nullptr) {
    g.i = i;
    g.nbin = nbin;
    g.nrows = nrows;
    g.binmask = nbin >= 64 ? ~0ull : ((1ull << nbin) - 1ull);
    uint64_t lo = i & g.binmask;
    uint64_t q = nbin >= 64 ? 0 : (i >> nbin);
    uint64_t code = lo ^ (lo >> 1);
    if (nbin > 0 && (q & 1ull)) code ^= 1ull << (nbin - 1);
    g.dbin = code;
    int par = bs_popc64(code) & 1;
    uint64_t w = 1;
    int toff = 2 * nbin;
    for (int j = nbin; j < nrows; ++j) {
        const int R = radix[j];
        int a;
        if (q <= 0xffffffffull) {  // 32-bit division (64-bit division is slow)
            const uint32_t q32 = (uint32_t)q;
            a = (int)(q32 % (uint32_t)R);
            q = (uint64_t)(q32 / (uint32_t)R);
        } else {
            a = (int)(q % (uint64_t)R);
            q = q / (uint64_t)R;
        }
        const int odd = (int)(q & 1ull);
        const int d = odd ? R - 1 - a : a;
        g.cnt[j] = (int8_t)a;
        g.dir[j] = (int8_t)(odd ? -1 : 1);
        g.del[j] = (int8_t)d;
        par ^= d & 1;
        w *= binom ? binom[toff + d] : bs_binom(R - 1, d);
        toff += R;
    }
    g.parity = par;
    g.w = w;
}

// Advance from i to i+1 (requires i + 1 < C).  Returns the digit row that
// changed; *coef is the change of its coefficient (M - 2 Delta) divided by 2,
// i.e. the column sums move by coef * (2 a_row).  Sets *wchanged when the
// binomial weight changed (only on multi-digit moves); the new weight is
// the product of table entries (binom non-null) or the exact ratio update.
BS_HD int bs_gray_step(bs_gray& g, const int* radix, int* coef, int* wchanged, const uint64_t* binom = nullptr) {
    uint64_t lo = g.i & g.binmask;
    int row;
    g.parity ^= 1;
    g.i += 1;
    if (lo != g.binmask) {
        int t = bs_ctz64(~lo);
        int was = (int)((g.dbin >> t) & 1ull);
        g.dbin ^= 1ull << t;
        *coef = was ? 1 : -1;
        *wchanged = 0;
        return t;
    }
    int j = g.nbin;
    while ((int)g.cnt[j] == radix[j] - 1) {
        g.cnt[j] = 0;
        g.dir[j] = (int8_t)(-g.dir[j]);
        ++j;
    }
    row = j;
    g.cnt[j] = (int8_t)(g.cnt[j] + 1);
    const int M = radix[j] - 1;
    const int d0 = g.del[j];
    const int d1 = d0 + g.dir[j];
    g.del[j] = (int8_t)d1;
    *coef = g.dir[j] > 0 ? -1 : 1;
    *wchanged = 1;
    if (binom) {
        uint64_t w = 1;
        int toff = 2 * g.nbin;
        for (int k = g.nbin; k < g.nrows; ++k) {
            w *= binom[toff + g.del[k]];
            toff += radix[k];
        }
        g.w = w;
    } else if (d1 > d0) {
        g.w = g.w * (uint64_t)(M - d0) / (uint64_t)(d0 + 1);
    } else {
        g.w = g.w * (uint64_t)d0 / (uint64_t)(M - d0 + 1);
    }
    return row;
}

// Delta of digit j in the current state (binary or multi).
BS_HD int bs_gray_delta(const bs_gray& g, int j) {
    if (j < g.nbin) return (int)((g.dbin >> j) & 1ull);
    return (int)g.del[j];
}
