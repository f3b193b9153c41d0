/*
 * oracle.c -- plain, slow CPU oracle for the generalized BB/FG permanent,
 * its Laplace minors and the Clifford & Clifford sampler.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA path (its own
 * double-double arithmetic, its own Philox generator, its own Gray walk).
 *
 * Arithmetic is complex double-double (about 106 significand bits) built from
 * published error-free transforms:
 *   TwoSum            Knuth, TAOCP vol. 2, Sec. 4.2.2 (Moller's algorithm)
 *   FastTwoSum        Dekker 1971 (requires |a| >= |b|)
 *   TwoProd           via fused multiply-add (Ogita, Rump, Oishi 2005)
 *   dd add / mul      Hida, Li, Bailey, "QD" library paper (2001)
 * Compile with -ffp-contract=off so the compiler never fuses the transforms.
 *
 * Entry points (all return 0 on success, a negative number on bad input):
 *   orc_perm_bruteforce   Eq. (perm_def): sum over all permutations, n <= 10
 *   orc_bbfg_gray         Eq. (bbfg) with delta_1 = +1 walked in binary
 *                         reflected Gray order (Sec. 2.1, Table "gray");
 *                         accepts rectangular r x c input (Appendix A.1)
 *   orc_gray_sequence     the Gray codes that walk visits, in order
 *   orc_bbfg_direct       Eq. (bbfg) with every column sum recomputed from
 *                         scratch (the O(n^2 2^n) form, Sec. 3.2)
 *   orc_ryser_gray        Eq. (ryser), subsets walked in Gray order
 *   orc_ryser_exact_gauss Eq. (ryser) in exact 128-bit integers for
 *                         Gaussian-integer matrices
 *   orc_nw_gray           the Nijenhuis-Wilf form of Eq. (ryser) (Sec. 2:
 *                         x_i = a_in - sum_j a_ij / 2, subsets of the first
 *                         n-1 columns), walked in Gray order
 *   orc_nw_exact_gauss    the same in exact 128-bit integers
 *   orc_formula_abs       modulus-sum of the addends of Eq. (ryser) or of
 *                         the Nijenhuis-Wilf form (times their prefactor)
 *   orc_perm_mult         Eq. (bbfgrepeated) evaluated term by term: every
 *                         Delta vector enumerated in plain odometer order,
 *                         binomials and column sums computed directly
 *   orc_perm_expanded     per(A expanded by row/col multiplicities), via
 *                         orc_bbfg_gray on the expanded matrix
 *   orc_minors            Laplace minors: per(expanded A with one copy of
 *                         distinct column l removed), each by orc_bbfg_gray
 *   orc_perm_mult_abs     modulus-sum of the addends of Eq. (bbfgrepeated)
 *   orc_bbfg_mult_extremes  sums of the positive and the negative real
 *                         addends of Eq. (bbfgrepeated) (Appendix A.5)
 *   orc_philox4x32_10     counter-based generator (Salmon et al., SC'11)
 *   orc_cc_sample         Clifford & Clifford sampler (Sec. 4; algorithm B of
 *                         Clifford & Clifford 2018) with minors by
 *                         orc_perm_expanded
 *
 * Complex matrices are passed as interleaved (re, im) doubles, row-major with
 * a leading dimension `ld` counted in complex elements.  Double-double
 * complex results are written as 4 doubles: re.hi, re.lo, im.hi, im.lo.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* double-double                                                        */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } zdd;

static dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd r = { s, e };
    return r;
}
static dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    dd r = { s, e };
    return r;
}
static dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    dd r = { p, e };
    return r;
}
static dd dd_make(double a) { dd r = { a, 0.0 }; return r; }
static dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd x) { dd r = { -x.hi, -x.lo }; return r; }
static dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }
static dd dd_mul(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p.hi, p.lo);
}
static dd dd_mul_d(dd x, double y) {
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return fast_two_sum(p.hi, p.lo);
}
static dd dd_ldexp(dd x, int e) { dd r = { ldexp(x.hi, e), ldexp(x.lo, e) }; return r; }

static zdd z_zero(void) { zdd r = { { 0, 0 }, { 0, 0 } }; return r; }
static zdd z_one(void) { zdd r = { { 1, 0 }, { 0, 0 } }; return r; }
static zdd z_from(double re, double im) { zdd r = { dd_make(re), dd_make(im) }; return r; }
static zdd z_add(zdd a, zdd b) { zdd r = { dd_add(a.re, b.re), dd_add(a.im, b.im) }; return r; }
static zdd z_sub(zdd a, zdd b) { zdd r = { dd_sub(a.re, b.re), dd_sub(a.im, b.im) }; return r; }
static zdd z_mul(zdd a, zdd b) {
    zdd r;
    r.re = dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
    r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
    return r;
}
/* multiply by a real double (used for exact small integers and +-1, +-2) */
static zdd z_mul_d(zdd a, double s) { zdd r = { dd_mul_d(a.re, s), dd_mul_d(a.im, s) }; return r; }
static zdd z_mul_dd(zdd a, dd s) { zdd r = { dd_mul(a.re, s), dd_mul(a.im, s) }; return r; }
static zdd z_ldexp(zdd a, int e) { zdd r = { dd_ldexp(a.re, e), dd_ldexp(a.im, e) }; return r; }
static void z_store(zdd a, double* out) {
    out[0] = a.re.hi; out[1] = a.re.lo; out[2] = a.im.hi; out[3] = a.im.lo;
}
static zdd z_elem(const double* A, int ld, int i, int j) {
    return z_from(A[2 * ((size_t)i * ld + j)], A[2 * ((size_t)i * ld + j) + 1]);
}

/* ------------------------------------------------------------------ */
/* Eq. (perm_def): brute force over S_n                                 */
/* ------------------------------------------------------------------ */
static void bf_rec(int n, int row, const double* A, int ld, int* used, zdd prod, zdd* acc) {
    if (row == n) { *acc = z_add(*acc, prod); return; }
    for (int j = 0; j < n; ++j) {
        if (used[j]) continue;
        used[j] = 1;
        bf_rec(n, row + 1, A, ld, used, z_mul(prod, z_elem(A, ld, row, j)), acc);
        used[j] = 0;
    }
}

int orc_perm_bruteforce(int n, const double* A, int ld, double* out) {
    if (n < 0 || n > 10) return -1;
    int used[16] = { 0 };
    zdd acc = z_zero();
    bf_rec(n, 0, A, ld, used, z_one(), &acc);
    z_store(acc, out);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. (bbfg): delta_1 = +1, binary reflected Gray walk over rows 2..r  */
/* Column sums c_j = sum_i delta_i a_ij (Sec. 2, column orientation).   */
/* Works for r x c (Appendix A.1): the product runs over the c columns, */
/* the prefactor is 2^(1-r).                                            */
/* ------------------------------------------------------------------ */
int orc_bbfg_gray(int r, int c, const double* A, int ld, double* out) {
    if (r < 0 || c < 0 || r > 40 || c > 64) return -1;
    if (r == 0) {
        /* empty row set: every column sum is 0; the empty product is 1 */
        zdd v = (c == 0) ? z_one() : z_zero();
        z_store(v, out);
        return 0;
    }
    zdd cs[64];
    for (int j = 0; j < c; ++j) {
        cs[j] = z_zero();
        for (int i = 0; i < r; ++i) cs[j] = z_add(cs[j], z_elem(A, ld, i, j));
    }
    zdd acc = z_zero();
    uint64_t count = (uint64_t)1 << (r - 1);
    uint64_t gray_prev = 0;
    int sign = 1;
    for (uint64_t g = 0; g < count; ++g) {
        if (g > 0) {
            /* the changed Gray bit is the lowest set bit of the index g */
            int t = __builtin_ctzll(g);
            int row = t + 1;
            int was_minus = (int)((gray_prev >> t) & 1u);
            /* bit 0 -> delta = +1, bit 1 -> delta = -1 */
            double coef = was_minus ? 2.0 : -2.0;
            for (int j = 0; j < c; ++j)
                cs[j] = z_add(cs[j], z_mul_d(z_elem(A, ld, row, j), coef));
            gray_prev ^= (uint64_t)1 << t;
            sign = -sign;
        }
        zdd p = z_one();
        for (int j = 0; j < c; ++j) p = z_mul(p, cs[j]);
        acc = (sign > 0) ? z_add(acc, p) : z_sub(acc, p);
    }
    z_store(z_ldexp(acc, 1 - r), out);
    return 0;
}

/* The same Gray walk in plain double arithmetic (no compensation, no
 * double-double): the plain-FP64 CPU form of Eq. (bbfg), a timing baseline
 * beside the double-double walk above.  out = {re, im}. */
int orc_bbfg_gray_fp64(int r, int c, const double* A, int ld, double* out) {
    if (r < 0 || c < 0 || r > 40 || c > 64) return -1;
    if (r == 0) {
        out[0] = (c == 0) ? 1.0 : 0.0;
        out[1] = 0.0;
        return 0;
    }
    double sr[64], si[64];
    for (int j = 0; j < c; ++j) {
        sr[j] = 0.0; si[j] = 0.0;
        for (int i = 0; i < r; ++i) { sr[j] += A[2 * ((size_t)i * ld + j)]; si[j] += A[2 * ((size_t)i * ld + j) + 1]; }
    }
    double ar = 0.0, ai = 0.0;
    uint64_t count = (uint64_t)1 << (r - 1);
    uint64_t gray_prev = 0;
    int sign = 1;
    for (uint64_t g = 0; g < count; ++g) {
        if (g > 0) {
            int t = __builtin_ctzll(g);
            int row = t + 1;
            double coef = ((gray_prev >> t) & 1u) ? 2.0 : -2.0;
            for (int j = 0; j < c; ++j) {
                sr[j] += coef * A[2 * ((size_t)row * ld + j)];
                si[j] += coef * A[2 * ((size_t)row * ld + j) + 1];
            }
            gray_prev ^= (uint64_t)1 << t;
            sign = -sign;
        }
        double pr = 1.0, pi = 0.0;
        for (int j = 0; j < c; ++j) {
            const double t = pr * sr[j] - pi * si[j];
            pi = pr * si[j] + pi * sr[j];
            pr = t;
        }
        if (sign > 0) { ar += pr; ai += pi; } else { ar -= pr; ai -= pi; }
    }
    out[0] = ldexp(ar, 1 - r);
    out[1] = ldexp(ai, 1 - r);
    return 0;
}

/* The sequence of Gray codes visited by orc_bbfg_gray's walk over `bits`
 * delta bits (bit t <-> row t+1; 1 means delta = -1), reconstructed from the
 * same flip rule: at index g the bit at the lowest set bit of g changes. */
int orc_gray_sequence(int bits, uint64_t* out) {
    if (bits < 0 || bits > 20) return -1;
    uint64_t count = (uint64_t)1 << bits;
    uint64_t gray = 0;
    for (uint64_t g = 0; g < count; ++g) {
        if (g > 0) gray ^= (uint64_t)1 << __builtin_ctzll(g);
        out[g] = gray;
    }
    return 0;
}

/* Eq. (bbfg) with every column sum recomputed for every delta (no Gray
 * reuse): the O(n^2 2^(n-1)) form discussed in Sec. 3.2. */
int orc_bbfg_direct(int r, int c, const double* A, int ld, double* out) {
    if (r < 1 || c < 0 || r > 30 || c > 64) return -1;
    zdd acc = z_zero();
    uint64_t count = (uint64_t)1 << (r - 1);
    for (uint64_t mask = 0; mask < count; ++mask) {
        /* bit (i-1) of mask set <=> delta_i = -1, for rows i = 1..r-1 */
        int neg = __builtin_popcountll(mask) & 1;
        zdd p = z_one();
        for (int j = 0; j < c; ++j) {
            zdd s = z_elem(A, ld, 0, j);
            for (int i = 1; i < r; ++i) {
                zdd a = z_elem(A, ld, i, j);
                s = ((mask >> (i - 1)) & 1u) ? z_sub(s, a) : z_add(s, a);
            }
            p = z_mul(p, s);
        }
        acc = neg ? z_sub(acc, p) : z_add(acc, p);
    }
    z_store(z_ldexp(acc, 1 - r), out);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. (ryser): perm = (-1)^n sum_S (-1)^|S| prod_i sum_{j in S} a_ij   */
/* subsets S of columns walked in Gray order (Sec. 2, O(n 2^n) form).   */
/* ------------------------------------------------------------------ */
int orc_ryser_gray(int n, const double* A, int ld, double* out) {
    if (n < 0 || n > 30) return -1;
    if (n == 0) { z_store(z_one(), out); return 0; }
    zdd rs[64];
    for (int i = 0; i < n; ++i) rs[i] = z_zero();
    zdd acc = z_zero();
    uint64_t count = (uint64_t)1 << n;
    uint64_t gray_prev = 0;
    int card = 0;
    for (uint64_t g = 1; g < count; ++g) {
        int t = __builtin_ctzll(g);
        int in_set = (int)((gray_prev >> t) & 1u);
        for (int i = 0; i < n; ++i) {
            zdd a = z_elem(A, ld, i, t);
            rs[i] = in_set ? z_sub(rs[i], a) : z_add(rs[i], a);
        }
        gray_prev ^= (uint64_t)1 << t;
        card += in_set ? -1 : 1;
        zdd p = z_one();
        for (int i = 0; i < n; ++i) p = z_mul(p, rs[i]);
        acc = (card & 1) ? z_sub(acc, p) : z_add(acc, p);
    }
    if (n & 1) acc = z_mul_d(acc, -1.0);
    z_store(acc, out);
    return 0;
}

/* Eq. (ryser) in exact arithmetic for Gaussian-integer matrices.  Entries
 * are passed as int64 pairs; the result as two __int128 values split into
 * (hi, lo) 64-bit halves: out[0..1] = re, out[2..3] = im. */
typedef __int128 i128;
int orc_ryser_exact_gauss(int n, const int64_t* A, int64_t* out) {
    if (n < 0 || n > 14) return -1;
    i128 are = 0, aim = 0;
    if (n == 0) { are = 1; }
    uint64_t count = (uint64_t)1 << n;
    for (uint64_t S = 1; S < count && n > 0; ++S) {
        i128 pre = 1, pim = 0;
        for (int i = 0; i < n; ++i) {
            i128 sre = 0, sim = 0;
            for (int j = 0; j < n; ++j)
                if ((S >> j) & 1u) { sre += A[2 * (i * n + j)]; sim += A[2 * (i * n + j) + 1]; }
            i128 tre = pre * sre - pim * sim;
            i128 tim = pre * sim + pim * sre;
            pre = tre; pim = tim;
        }
        int card = __builtin_popcountll(S);
        if (card & 1) { are -= pre; aim -= pim; } else { are += pre; aim += pim; }
    }
    if (n & 1) { are = -are; aim = -aim; }
    out[0] = (int64_t)(are >> 64); out[1] = (int64_t)(uint64_t)are;
    out[2] = (int64_t)(aim >> 64); out[3] = (int64_t)(uint64_t)aim;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Nijenhuis-Wilf form of Eq. (ryser) (Sec. 2):                         */
/*   perm = (-1)^(n-1) 2 sum_{S in {1..n-1}} (-1)^|S|                   */
/*          prod_i (x_i + sum_{j in S} a_ij),                           */
/*   x_i = a_in - (a_i1 + ... + a_in) / 2.                              */
/* Subsets of the first n-1 columns walked in Gray order.               */
/* ------------------------------------------------------------------ */
int orc_nw_gray(int n, const double* A, int ld, double* out) {
    if (n < 0 || n > 30) return -1;
    if (n == 0) { z_store(z_one(), out); return 0; }
    zdd rs[64];
    for (int i = 0; i < n; ++i) {
        zdd row = z_zero();
        for (int j = 0; j < n; ++j) row = z_add(row, z_elem(A, ld, i, j));
        rs[i] = z_sub(z_elem(A, ld, i, n - 1), z_ldexp(row, -1));
    }
    zdd acc = z_zero();
    uint64_t count = (uint64_t)1 << (n - 1);
    uint64_t gray_prev = 0;
    int card = 0;
    for (uint64_t g = 0; g < count; ++g) {
        if (g > 0) {
            int t = __builtin_ctzll(g);
            int in_set = (int)((gray_prev >> t) & 1u);
            for (int i = 0; i < n; ++i) {
                zdd a = z_elem(A, ld, i, t);
                rs[i] = in_set ? z_sub(rs[i], a) : z_add(rs[i], a);
            }
            gray_prev ^= (uint64_t)1 << t;
            card += in_set ? -1 : 1;
        }
        zdd p = z_one();
        for (int i = 0; i < n; ++i) p = z_mul(p, rs[i]);
        acc = (card & 1) ? z_sub(acc, p) : z_add(acc, p);
    }
    acc = z_ldexp(acc, 1);
    if ((n - 1) & 1) acc = z_mul_d(acc, -1.0);
    z_store(acc, out);
    return 0;
}

/* The Nijenhuis-Wilf form in exact integers for Gaussian-integer matrices.
 * With y_i = 2 x_i + 2 sum_{j in S} a_ij (an integer),
 *   perm = (-1)^(n-1) 2^(1-n) sum_S (-1)^|S| prod_i y_i;
 * the sum must be divisible by 2^(n-1) (else -2 is returned).  Output as in
 * orc_ryser_exact_gauss. */
int orc_nw_exact_gauss(int n, const int64_t* A, int64_t* out) {
    if (n < 0 || n > 14) return -1;
    i128 are = 0, aim = 0;
    if (n == 0) are = 1;
    if (n > 0) {
        i128 x2re[64], x2im[64];
        for (int i = 0; i < n; ++i) {
            i128 sre = 0, sim = 0;
            for (int j = 0; j < n; ++j) { sre += A[2 * (i * n + j)]; sim += A[2 * (i * n + j) + 1]; }
            x2re[i] = 2 * (i128)A[2 * (i * n + n - 1)] - sre;
            x2im[i] = 2 * (i128)A[2 * (i * n + n - 1) + 1] - sim;
        }
        uint64_t count = (uint64_t)1 << (n - 1);
        for (uint64_t S = 0; S < count; ++S) {
            i128 pre = 1, pim = 0;
            for (int i = 0; i < n; ++i) {
                i128 yre = x2re[i], yim = x2im[i];
                for (int j = 0; j < n - 1; ++j)
                    if ((S >> j) & 1u) { yre += 2 * (i128)A[2 * (i * n + j)]; yim += 2 * (i128)A[2 * (i * n + j) + 1]; }
                i128 tre = pre * yre - pim * yim;
                i128 tim = pre * yim + pim * yre;
                pre = tre; pim = tim;
            }
            if (__builtin_popcountll(S) & 1) { are -= pre; aim -= pim; } else { are += pre; aim += pim; }
        }
        const i128 div = (i128)1 << (n - 1);
        if (are % div != 0 || aim % div != 0) return -2;
        are /= div; aim /= div;
        if ((n - 1) & 1) { are = -are; aim = -aim; }
    }
    out[0] = (int64_t)(are >> 64); out[1] = (int64_t)(uint64_t)are;
    out[2] = (int64_t)(aim >> 64); out[3] = (int64_t)(uint64_t)aim;
    return 0;
}

/* Modulus-sum of the addends of Eq. (ryser) (which = 1) or of the
 * Nijenhuis-Wilf form (which = 2), each addend |prod_i inner sum| times the
 * modulus of the prefactor (1, or 2); every subset evaluated directly in
 * plain double.  The scale of the rounding error of those formulas. */
int orc_formula_abs(int which, int n, const double* A, int ld, double* out) {
    if (n < 0 || n > 24 || (which != 1 && which != 2)) return -1;
    if (n == 0) { out[0] = 1.0; return 0; }
    double xre[64], xim[64];
    for (int i = 0; i < n; ++i) {
        xre[i] = 0.0; xim[i] = 0.0;
        if (which == 2) {
            double sre = 0.0, sim = 0.0;
            for (int j = 0; j < n; ++j) { sre += A[2 * (i * ld + j)]; sim += A[2 * (i * ld + j) + 1]; }
            xre[i] = A[2 * (i * ld + n - 1)] - 0.5 * sre;
            xim[i] = A[2 * (i * ld + n - 1) + 1] - 0.5 * sim;
        }
    }
    const int cols = which == 1 ? n : n - 1;
    const uint64_t count = (uint64_t)1 << cols;
    double acc = 0.0;
    for (uint64_t S = 0; S < count; ++S) {
        double mag = 1.0;
        for (int i = 0; i < n; ++i) {
            double re = xre[i], im = xim[i];
            for (int j = 0; j < cols; ++j)
                if ((S >> j) & 1u) { re += A[2 * (i * ld + j)]; im += A[2 * (i * ld + j) + 1]; }
            mag *= hypot(re, im);
        }
        acc += mag;
    }
    out[0] = which == 2 ? 2.0 * acc : acc;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. (bbfgrepeated), evaluated term by term.                          */
/*                                                                      */
/* A is R x K (distinct rows x distinct columns), row multiplicities    */
/* M_k, column multiplicities N_j, n = sum M = sum N.  Row 0 is the     */
/* first row of Eq. (bbfgrepeated) and carries delta = +1 with          */
/* multiplicity 1 (Sec. 2.2); when M_0 > 1 its remaining M_0 - 1 copies */
/* form an extra repeated row.  Every Delta vector is visited in plain  */
/* odometer order; the weight prod (-1)^Delta_k C(M_k, Delta_k) and the */
/* column sums sum_k (M_k - 2 Delta_k) a_kj are computed from scratch.  */
/* ------------------------------------------------------------------ */
static double binom_exact(int m, int d) {
    /* exact for m <= 60 (values < 2^63 computed in 64-bit integers) */
    if (d < 0 || d > m) return 0.0;
    uint64_t v = 1;
    for (int t = 1; t <= d; ++t) v = v * (uint64_t)(m - d + t) / (uint64_t)t;
    return (double)v;
}

typedef struct {
    int R, K, n;
    int rows[64];      /* source row of each formula row (after the split) */
    int M[64];         /* multiplicity of each formula row */
    int N[64];         /* column multiplicities (zero ones dropped) */
    int cols[64];      /* source column index */
} mult_problem;

static int mult_setup(int R, int K, const int* M, const int* N, mult_problem* p) {
    if (R < 0 || K < 0 || R > 60 || K > 64) return -1;
    int sm = 0, sn = 0;
    p->R = 0; p->K = 0;
    int first = -1;
    for (int k = 0; k < R; ++k) { if (M[k] < 0) return -1; sm += M[k]; if (M[k] > 0 && first < 0) first = k; }
    for (int j = 0; j < K; ++j) { if (N[j] < 0) return -1; sn += N[j]; }
    if (sm != sn || sm > 60) return -2;
    p->n = sm;
    for (int j = 0; j < K; ++j) if (N[j] > 0) { p->cols[p->K] = j; p->N[p->K] = N[j]; p->K++; }
    if (first < 0) return 0;
    /* row 0 of the formula: one copy of the first occupied row, delta = +1 */
    p->rows[0] = first; p->M[0] = 1; p->R = 1;
    if (M[first] > 1) { p->rows[p->R] = first; p->M[p->R] = M[first] - 1; p->R++; }
    for (int k = first + 1; k < R; ++k)
        if (M[k] > 0) { p->rows[p->R] = k; p->M[p->R] = M[k]; p->R++; }
    return 0;
}

int orc_perm_mult(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    mult_problem p;
    int rc = mult_setup(R, K, M, N, &p);
    if (rc) return rc;
    if (p.n == 0) { z_store(z_one(), out); return 0; }
    int D[64];
    memset(D, 0, sizeof(D));
    zdd acc = z_zero();
    for (;;) {
        /* weight prod_k (-1)^Delta_k C(M_k, Delta_k) over rows k >= 1 */
        dd w = dd_make(1.0);
        int parity = 0;
        for (int k = 1; k < p.R; ++k) { w = dd_mul_d(w, binom_exact(p.M[k], D[k])); parity ^= (D[k] & 1); }
        zdd prod = z_one();
        for (int j = 0; j < p.K; ++j) {
            zdd s = z_zero();
            for (int k = 0; k < p.R; ++k)
                s = z_add(s, z_mul_d(z_elem(A, ld, p.rows[k], p.cols[j]), (double)(p.M[k] - 2 * D[k])));
            for (int e = 0; e < p.N[j]; ++e) prod = z_mul(prod, s);
        }
        zdd term = z_mul_dd(prod, w);
        acc = parity ? z_sub(acc, term) : z_add(acc, term);
        /* odometer over Delta_k in [0, M_k], k = 1..R-1 */
        int k = 1;
        while (k < p.R && D[k] == p.M[k]) { D[k] = 0; ++k; }
        if (k >= p.R) break;
        D[k]++;
    }
    z_store(z_ldexp(acc, 1 - p.n), out);
    return 0;
}

/* The same term-by-term evaluation of Eq. (bbfgrepeated) in plain double
 * arithmetic (no compensation): the plain-FP64 CPU form of the method, a
 * timing baseline beside the double-double oracle above.  out = {re, im}. */
int orc_perm_mult_fp64(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    mult_problem p;
    int rc = mult_setup(R, K, M, N, &p);
    if (rc) return rc;
    if (p.n == 0) { out[0] = 1.0; out[1] = 0.0; return 0; }
    int D[64];
    memset(D, 0, sizeof(D));
    double acc_re = 0.0, acc_im = 0.0;
    for (;;) {
        double w = 1.0;
        int parity = 0;
        for (int k = 1; k < p.R; ++k) { w *= binom_exact(p.M[k], D[k]); parity ^= (D[k] & 1); }
        double pr = 1.0, pi = 0.0;
        for (int j = 0; j < p.K; ++j) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < p.R; ++k) {
                const double c = (double)(p.M[k] - 2 * D[k]);
                sr += c * A[2 * (p.rows[k] * ld + p.cols[j])];
                si += c * A[2 * (p.rows[k] * ld + p.cols[j]) + 1];
            }
            for (int e = 0; e < p.N[j]; ++e) {
                const double t = pr * sr - pi * si;
                pi = pr * si + pi * sr;
                pr = t;
            }
        }
        if (parity) { acc_re -= w * pr; acc_im -= w * pi; }
        else { acc_re += w * pr; acc_im += w * pi; }
        int k = 1;
        while (k < p.R && D[k] == p.M[k]) { D[k] = 0; ++k; }
        if (k >= p.R) break;
        D[k]++;
    }
    out[0] = ldexp(acc_re, 1 - p.n);
    out[1] = ldexp(acc_im, 1 - p.n);
    return 0;
}

/* S_abs = 2^(1-n) sum over Delta of prod_k C(M_k, Delta_k) |prod_j c_j^N_j|,
 * the modulus-sum of the addends of Eq. (bbfgrepeated): the scale of the
 * rounding error of any evaluation of the sum (each addend carries a
 * relative error, so |error| <= rel * S_abs).  out[0] = S_abs. */
int orc_perm_mult_abs(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    mult_problem p;
    int rc = mult_setup(R, K, M, N, &p);
    if (rc) return rc;
    if (p.n == 0) { out[0] = 1.0; return 0; }
    int D[64];
    memset(D, 0, sizeof(D));
    dd acc = dd_make(0.0);
    for (;;) {
        dd w = dd_make(1.0);
        for (int k = 1; k < p.R; ++k) w = dd_mul_d(w, binom_exact(p.M[k], D[k]));
        double mag = 1.0;
        for (int j = 0; j < p.K; ++j) {
            zdd s = z_zero();
            for (int k = 0; k < p.R; ++k)
                s = z_add(s, z_mul_d(z_elem(A, ld, p.rows[k], p.cols[j]), (double)(p.M[k] - 2 * D[k])));
            double m = hypot(s.re.hi + s.re.lo, s.im.hi + s.im.lo);
            for (int e = 0; e < p.N[j]; ++e) mag *= m;
        }
        acc = dd_add(acc, dd_mul_d(w, mag));
        int k = 1;
        while (k < p.R && D[k] == p.M[k]) { D[k] = 0; ++k; }
        if (k >= p.R) break;
        D[k]++;
    }
    out[0] = ldexp(acc.hi + acc.lo, 1 - p.n);
    return 0;
}

/* Sums of the positive and of the negative real parts of the addends of
 * Eq. (bbfgrepeated) (each addend weighted by its binomial count), without
 * the 2^(1-n) prefactor; out[0] = positive sum, out[1] = negative sum.
 * Appendix A.5 bounds these partial sums for the normalized all-ones
 * matrix. */
int orc_bbfg_mult_extremes(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    mult_problem p;
    int rc = mult_setup(R, K, M, N, &p);
    if (rc) return rc;
    int D[64];
    memset(D, 0, sizeof(D));
    dd pos = dd_make(0.0), neg = dd_make(0.0);
    if (p.n == 0) { out[0] = 1.0; out[1] = 0.0; return 0; }
    for (;;) {
        dd w = dd_make(1.0);
        int parity = 0;
        for (int k = 1; k < p.R; ++k) { w = dd_mul_d(w, binom_exact(p.M[k], D[k])); parity ^= (D[k] & 1); }
        zdd prod = z_one();
        for (int j = 0; j < p.K; ++j) {
            zdd s = z_zero();
            for (int k = 0; k < p.R; ++k)
                s = z_add(s, z_mul_d(z_elem(A, ld, p.rows[k], p.cols[j]), (double)(p.M[k] - 2 * D[k])));
            for (int e = 0; e < p.N[j]; ++e) prod = z_mul(prod, s);
        }
        dd v = dd_mul(prod.re, w);
        if (parity) v = dd_neg(v);
        if (v.hi >= 0) pos = dd_add(pos, v); else neg = dd_add(neg, v);
        int k = 1;
        while (k < p.R && D[k] == p.M[k]) { D[k] = 0; ++k; }
        if (k >= p.R) break;
        D[k]++;
    }
    out[0] = pos.hi + pos.lo;
    out[1] = neg.hi + neg.lo;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Expanded matrix: repeat row k M_k times and column j N_j times       */
/* (Sec. 4: U_ST), then Eq. (bbfg) on the square result.                */
/* ------------------------------------------------------------------ */
static int expand(int R, int K, const double* A, int ld, const int* M, const int* N,
                  int skip_col, double* E, int* n_out) {
    int rr[64], cc[64];
    int nr = 0, nc = 0;
    for (int k = 0; k < R; ++k) for (int t = 0; t < M[k]; ++t) { if (nr >= 60) return -1; rr[nr++] = k; }
    for (int j = 0; j < K; ++j) {
        int cnt = N[j] - (j == skip_col ? 1 : 0);
        for (int t = 0; t < cnt; ++t) { if (nc >= 60) return -1; cc[nc++] = j; }
    }
    if (nr != nc) return -2;
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nc; ++j) {
            E[2 * (i * nr + j)] = A[2 * ((size_t)rr[i] * ld + cc[j])];
            E[2 * (i * nr + j) + 1] = A[2 * ((size_t)rr[i] * ld + cc[j]) + 1];
        }
    *n_out = nr;
    return 0;
}

int orc_perm_expanded(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    for (int k = 0; k < R; ++k) if (M[k] < 0) return -1;
    for (int j = 0; j < K; ++j) if (N[j] < 0) return -1;
    double* E = (double*)malloc(sizeof(double) * 2 * 60 * 60);
    if (!E) return -3;
    int n = 0;
    int rc = expand(R, K, A, ld, M, N, -1, E, &n);
    if (rc == 0) rc = orc_bbfg_gray(n, n, E, n, out);
    free(E);
    return rc;
}

/* Laplace minors: for each distinct column l with N_l >= 1, the permanent of
 * the expanded matrix with one copy of column l removed; requires
 * sum M = sum N - 1.  out holds 4 doubles per column (zeros for N_l = 0).
 * Expanding per(A') of the square matrix A' = [A; row a] along its last row
 * gives per(A') = sum_l N_l a_l minor_l. */
int orc_minors(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    int sm = 0, sn = 0;
    for (int k = 0; k < R; ++k) { if (M[k] < 0) return -1; sm += M[k]; }
    for (int j = 0; j < K; ++j) { if (N[j] < 0) return -1; sn += N[j]; }
    if (sm != sn - 1) return -2;
    double* E = (double*)malloc(sizeof(double) * 2 * 60 * 60);
    if (!E) return -3;
    int rc = 0;
    for (int l = 0; l < K && rc == 0; ++l) {
        if (N[l] == 0) { memset(out + 4 * l, 0, 4 * sizeof(double)); continue; }
        int n = 0;
        rc = expand(R, K, A, ld, M, N, l, E, &n);
        if (rc == 0) rc = orc_bbfg_gray(n, n, E, n, out + 4 * l);
    }
    free(E);
    return rc;
}

/* Laplace minors as orc_minors, each by the plain-double walk
 * orc_bbfg_gray_fp64 (timing baseline).  out: K x {re, im}. */
int orc_minors_fp64(int R, int K, const double* A, int ld, const int* M, const int* N, double* out) {
    int sm = 0, sn = 0;
    for (int k = 0; k < R; ++k) { if (M[k] < 0) return -1; sm += M[k]; }
    for (int j = 0; j < K; ++j) { if (N[j] < 0) return -1; sn += N[j]; }
    if (sm != sn - 1) return -2;
    double* E = (double*)malloc(sizeof(double) * 2 * 60 * 60);
    if (!E) return -3;
    int rc = 0;
    for (int l = 0; l < K && rc == 0; ++l) {
        if (N[l] == 0) { out[2 * l] = 0.0; out[2 * l + 1] = 0.0; continue; }
        int n = 0;
        rc = expand(R, K, A, ld, M, N, l, E, &n);
        if (rc == 0) rc = orc_bbfg_gray_fp64(n, n, E, n, out + 2 * l);
    }
    free(E);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC 2011): 10 rounds of the 4x32 Philox S-box,   */
/* multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments             */
/* 0x9E3779B9 / 0xBB67AE85.                                             */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw for (seed, sample, purpose, index): the 4 Philox words of counter
 * (sample_lo, sample_hi, purpose, index) under key (seed_lo, seed_hi). */
static void draw(uint64_t seed, uint64_t sample, uint32_t purpose, uint32_t index, uint32_t w[4]) {
    uint32_t ctr[4] = { (uint32_t)sample, (uint32_t)(sample >> 32), purpose, index };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------------ */
/* Clifford & Clifford sampler (Sec. 4, algorithm B of Clifford &       */
/* Clifford, SODA 2018), single-threaded, minors by orc_perm_expanded.  */
/*                                                                      */
/* Random numbers (shared definition with the GPU sampler):             */
/*   column shuffle: Fisher-Yates for j = n-1 .. 1, swap positions j and */
/*     floor(w0 * (j+1) / 2^32), w = draw(seed, s, 0, j);               */
/*   step k (1-based): u = (((uint64)w0 << 32 | w1) >> 11) * 2^-53,     */
/*     w = draw(seed, s, 1, k);                                          */
/*   r_k = smallest row i with cdf_i > u * total, where cdf is the       */
/*     running FP64 sum of the weights in row order.                     */
/* U is m x m' (row-major, ld = m'); the first m_det rows are counted in */
/* the output (all m when m_det <= 0).                                    */
/* out: n_samples x m_det occupation counts; margin (nullable): per       */
/* sample, the smallest |u*total - cdf boundary| / total over its steps.  */
/* rows_out (nullable): n_samples x max_steps drawn rows r_1, r_2, ...,   */
/* in draw order; step_margin (nullable, same shape): that smallest       */
/* distance for each step alone.                                        */
/* ------------------------------------------------------------------ */
int orc_cc_sample(int m, int mcols, const double* U, int ld, const int* occ, int n_samples,
                  uint64_t seed, int m_det, int max_steps, int* out, double* margin,
                  double* addend_ops, int* rows_out, double* step_margin) {
    if (m <= 0 || mcols <= 0 || n_samples < 0) return -1;
    if (m_det <= 0 || m_det > m) m_det = m;
    int n = 0;
    int cols0[64];
    for (int i = 0; i < mcols; ++i) {
        if (occ[i] < 0) return -1;
        for (int t = 0; t < occ[i]; ++t) { if (n >= 48) return -1; cols0[n++] = i; }
    }
    if (max_steps <= 0 || max_steps > n) max_steps = n;
    double* w = (double*)malloc(sizeof(double) * (size_t)m);
    double* A = (double*)malloc(sizeof(double) * 2 * 64 * 64);
    double* minors = (double*)malloc(sizeof(double) * 4 * 64);
    if (!w || !A || !minors) { free(w); free(A); free(minors); return -3; }
    double ops = 0.0;
    for (int s = 0; s < n_samples; ++s) {
        int cols[64];
        memcpy(cols, cols0, sizeof(int) * (size_t)n);
        for (int j = n - 1; j >= 1; --j) {
            uint32_t wd[4];
            draw(seed, (uint64_t)s, 0u, (uint32_t)j, wd);
            int t = (int)(((uint64_t)wd[0] * (uint64_t)(j + 1)) >> 32);
            int tmp = cols[j]; cols[j] = cols[t]; cols[t] = tmp;
        }
        int rows[64];
        double min_margin = INFINITY;
        for (int k = 1; k <= max_steps; ++k) {
            /* minors of the (k-1) x k matrix U[rows[0..k-2], cols[0..k-1]] */
            for (int i = 0; i < k - 1; ++i)
                for (int l = 0; l < k; ++l) {
                    A[2 * (i * 64 + l)] = U[2 * ((size_t)rows[i] * ld + cols[l])];
                    A[2 * (i * 64 + l) + 1] = U[2 * ((size_t)rows[i] * ld + cols[l]) + 1];
                }
            int ones_r[64], ones_c[64];
            for (int t = 0; t < 64; ++t) { ones_r[t] = 1; ones_c[t] = 1; }
            if (k == 1) {
                minors[0] = 1.0; minors[1] = 0.0; minors[2] = 0.0; minors[3] = 0.0;
            } else {
                int rc = orc_minors(k - 1, k, A, 64, ones_r, ones_c, minors);
                if (rc) { free(w); free(A); free(minors); return rc; }
                ops += (double)k * (double)(k - 1) * ldexp(1.0, k - 2);
            }
            /* w_i = |sum_l U[i, cols[l]] * minor_l|^2 */
            for (int i = 0; i < m; ++i) {
                zdd acc = z_zero();
                for (int l = 0; l < k; ++l) {
                    zdd mnr = { { minors[4 * l], minors[4 * l + 1] }, { minors[4 * l + 2], minors[4 * l + 3] } };
                    acc = z_add(acc, z_mul(z_elem(U, ld, i, cols[l]), mnr));
                }
                dd p2 = dd_add(dd_mul(acc.re, acc.re), dd_mul(acc.im, acc.im));
                w[i] = p2.hi + p2.lo;
            }
            double total = 0.0;
            for (int i = 0; i < m; ++i) total += w[i];
            uint32_t wd[4];
            draw(seed, (uint64_t)s, 1u, (uint32_t)k, wd);
            double u = (double)((((uint64_t)wd[0] << 32) | wd[1]) >> 11) * 0x1.0p-53;
            double target = u * total;
            double cdf = 0.0;
            double step_min = INFINITY;
            int pick = -1;
            for (int i = 0; i < m; ++i) {
                cdf += w[i];
                double d = fabs(cdf - target) / total;
                if (d < step_min) step_min = d;
                if (pick < 0 && cdf > target) pick = i;
            }
            if (step_min < min_margin) min_margin = step_min;
            if (step_margin) step_margin[(size_t)s * max_steps + (k - 1)] = step_min;
            if (pick < 0) { for (int i = m - 1; i >= 0; --i) if (w[i] > 0) { pick = i; break; } }
            if (pick < 0) pick = 0;
            rows[k - 1] = pick;
            if (rows_out) rows_out[(size_t)s * max_steps + (k - 1)] = pick;
        }
        int* o = out + (size_t)s * m_det;
        for (int i = 0; i < m_det; ++i) o[i] = 0;
        for (int k = 0; k < max_steps; ++k) if (rows[k] < m_det) o[rows[k]]++;
        if (margin) margin[s] = min_margin;
    }
    if (addend_ops) *addend_ops = ops;
    free(w); free(A); free(minors);
    return 0;
}
