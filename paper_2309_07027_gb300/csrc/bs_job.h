// Job descriptor shared by the host planner and the walk kernels.
//
// A job is one generalized BB/FG sum (Eq. bbfgrepeated) in canonical form:
//   * K product columns, each with multiplicity 1 (repeated columns are
//     expanded by the planner, so the product length equals K);
//   * one pinned row (delta = +1, Sec. 2.2) folded into the base column sums;
//   * nrows digit rows; digit j has radix R_j = M_j + 1 and counts the -1
//     entries Delta_j among the M_j copies of that row (Eq. Deltak).  The
//     first nbin digits are binary (M_j = 1) and vary fastest.
// The addend index i in [0, C), C = prod_j R_j, is read as a mixed-radix
// number (digit 0 least significant) and mapped to the reflected n-ary Gray
// code of Sec. 2.2; each addend is
//     (-1)^{sum Delta} prod_j C(M_j, Delta_j) * prod_col c_col
// with c_col = c0_col - sum_j Delta_j * (2 a_j,col).
//
// kind == BS_KIND_PERM   : one output, sum * 2^{scale_exp}
// kind == BS_KIND_MINORS : K outputs, output l = sum over addends of
//                          (-1)^.. C(..) prod_{col != l} c_col, scaled by
//                          2^{colexp[l]} (Laplace minors, one column removed).
#pragma once
#include <stdint.h>

#define BS_KIND_PERM 0
#define BS_KIND_MINORS 1

#define BS_MAX_COLS 48     // product columns per job
#define BS_MAX_DIGITS 48   // digit rows per job
#define BS_MAX_PHOTONS 48  // n = sum of multiplicities

struct bs_job {
    uint64_t C;            // number of addends = prod of radices
    uint64_t task_begin;   // first global warp-task index of this job
    uint32_t ntasks;       // warp tasks in this launch: 32 (or 16) chunks of 2^log2L addends each
    uint32_t task_offset;  // job-local number of this launch's first task (a launch may walk a slice)
    int32_t K;             // product columns
    int32_t nrows;         // digit rows
    int32_t nbin;          // leading binary digits
    int32_t kind;          // BS_KIND_PERM or BS_KIND_MINORS
    int32_t log2L;         // chunk length exponent (one chunk per lane per task)
    int32_t out_index;     // perm: output slot; minors: first of K output slots
    int32_t n;             // photons of the formula (prefactor 2^(1-n))
    int32_t normalize;     // 1: scale each column by a power of two (FP32 range)
    int32_t prec;          // BS_PREC_*: which kernels walk the job
    int64_t data_off;      // complex elements: c0[KP] then 2a[nrows][KP], KP = BS_ROW_STRIDE(K)
    int64_t meta_off;      // ints, see BS_META_* below
    int64_t partial_off;   // double-double complex slots: ntasks * (perm ? 1 : K)
    int64_t src_off;       // source matrix: element offset of entry (0, 0)
    int32_t src_ld;        // source leading dimension (complex elements)
    int32_t src_trans;     // 1: formula row r / column c read source (c, r)
    int32_t formula;       // BS_JOB_BBFG (0), BS_JOB_RYSER or BS_JOB_NW (plain permanents, FP64)
    int32_t reseed_log2;   // FP32 jobs: > 0 re-seeds the column sums from the matrix every 2^reseed_log2
                           // steps inside a chunk as well (0: at chunk starts only)
};

// Formula of a job (see bs_perm_formula).  Ryser and Nijenhuis-Wilf jobs
// walk the columns of the matrix as binary digits with the rows as product
// columns; the walk kernels are the same, only packing and prefactor differ.
#define BS_JOB_BBFG 0
#define BS_JOB_RYSER 1
#define BS_JOB_NW 2

// Integer metadata of a job, at meta_off (int32 units; meta_off even):
//   radix[nrows]        digit radices R_j = M_j + 1 (binary digits first)
//   digit_src[nrows]    source row of each digit
//   col_src[K]          source column of each product column
//   colexp[K]           power-of-two column scale chosen by the pack kernel
//   pinned_src          source row of the pinned (delta = +1) row
//   (one int of padding to an 8-byte boundary)
//   binom[]             uint64 table written by the pack kernel: for each
//                       digit j in order, C(M_j, d) for d = 0..M_j
//                       (nrows + n - 1 entries in all)
#define BS_META_RADIX(jb) ((jb).meta_off)
#define BS_META_DIGIT_SRC(jb) ((jb).meta_off + (jb).nrows)
#define BS_META_COL_SRC(jb) ((jb).meta_off + 2 * (jb).nrows)
#define BS_META_COLEXP(jb) ((jb).meta_off + 2 * (jb).nrows + (jb).K)
#define BS_META_PINNED(jb) ((jb).meta_off + 2 * (jb).nrows + 2 * (jb).K)
#define BS_META_BINOM(jb) ((jb).meta_off + 2 * (jb).nrows + 2 * (jb).K + 2)
#define BS_META_SIZE(nrows, K, n) (2 * (nrows) + 2 * (K) + 2 + 2 * ((nrows) + (n)))

// Row stride of the packed matrix c0 / 2a: K rounded up to a multiple of 4,
// the width KB of the bucket kernel that walks the job (inside a kernel the
// stride is the compile-time KB), so FP32 rows are whole 16-byte column pairs
// and every bucket column has a slot.  Pad columns are neutral: rows hold
// zeros, and in FP32 jobs c0 holds 1, so a pad column sum stays exactly 1 and
// leaves every product unchanged (FP64 jobs keep c0 = 0 there and test
// columns against K instead).
#define BS_ROW_STRIDE(K) ((((K) + 3) / 4) * 4)
// Double-float jobs: K rounded up to a multiple of 8 (the DF bucket width).
#define BS_ROW_STRIDE_DF(K) ((((K) + 7) / 8) * 8)
#define BS_ROW_STRIDE_P(K, prec) ((prec) == BS_PREC_DF ? BS_ROW_STRIDE_DF(K) : BS_ROW_STRIDE(K))

// Precision of a job: the kernel family that walks it.
//   FP64: double column sums, products and runs (data in complex doubles);
//   FP32: single-precision packed pairs (data in complex floats);
//   DF:   double-float (float pairs, exact fixed-point column sums; data in
//         16-byte units like FP64).
#define BS_PREC_FP64 0
#define BS_PREC_FP32 1
#define BS_PREC_DF 2
#define BS_NPREC 3

// Double-double complex partial: re = (re_hi, re_lo), im = (im_hi, im_lo).
struct bs_zdd {
    double re_hi, re_lo, im_hi, im_lo;
};

// Device status word values (written by kernels, read by the host).
#define BS_STATUS_OK 0
#define BS_STATUS_TIMEOUT 1
#define BS_STATUS_BADJOB 2
