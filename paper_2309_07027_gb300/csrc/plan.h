// Host planner shared by the library entry points (no allocation).
#pragma once
#include <stdint.h>

#include "bs.h"
#include "bs_job.h"

namespace bs {

// Formats the calling thread's error text (fixed buffer) and returns code.
int fail(int code, const char* fmt, ...);
const char* last_error();

// Canonical form of a permanent (kind BS_KIND_PERM) or minors
// (BS_KIND_MINORS) problem: orientation, pinned row, digit order (binary
// digits first), product columns (repeated columns expanded).
struct IntPlan {
    int kind = BS_KIND_PERM;
    int formula = BS_JOB_BBFG;
    bool trivial = false;  // result known without a walk
    int n = 0;             // photons of the formula
    int K = 0, nrows = 0, nbin = 0;
    uint64_t C = 1;
    bool trans = false;
    int pinned_src = 0;
    int pinned_m = 1;      // multiplicity of the pinned row
    int radix[BS_MAX_DIGITS];
    int digit_src[BS_MAX_DIGITS];
    int col_src[BS_MAX_COLS];
};

// Addends of an orientation whose row multiplicities are m[0..cnt).
uint64_t pin_cost(const int* m, int cnt);

// Plans rows x cols with multiplicities M, N; BS_OK or BS_EINVAL (text via
// last_error()).
int plan_job(int rows, int cols, const int* M, const int* N, int kind, IntPlan& p);

// Plans the permanent of an n x n matrix by Ryser's formula or its
// Nijenhuis-Wilf form (formula BS_JOB_RYSER / BS_JOB_NW): the matrix columns
// are the binary digits (all n, or the first n - 1), the matrix rows the
// product columns (read transposed).  BS_OK or BS_EINVAL.
int plan_formula(int n, int formula, IntPlan& p);

// Product column of the first copy of source column c in a minors plan; -1
// when N[c] == 0.
int first_product_col(const int* N, int c);

}  // namespace bs
