// Host planner (canonicalisation of a permanent / minors problem, Sec. 2.2,
// Eq. bbfgrepeated) and per-thread error text.  Neither allocates memory.
#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "plan.h"

namespace bs {

namespace {
thread_local char g_err[512] = "no error";
}

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

const char* last_error() { return g_err; }


// Addends of the orientation whose row multiplicities are m[0..cnt): the
// smallest one is pinned (its other copies form a digit of radix m_p).
uint64_t pin_cost(const int* m, int cnt) {
    if (cnt <= 0) return 1;
    int p = 0;
    for (int i = 1; i < cnt; ++i)
        if (m[i] < m[p]) p = i;
    uint64_t c = (uint64_t)m[p];
    for (int i = 0; i < cnt; ++i)
        if (i != p) c *= (uint64_t)(m[i] + 1);
    return c;
}

int plan_formula(int n, int formula, IntPlan& p) {
    if (n < 0 || n > BS_MAX_N) return fail(BS_EINVAL, "matrix size %d outside [0, %d]", n, BS_MAX_N);
    if (formula != BS_JOB_RYSER && formula != BS_JOB_NW) return fail(BS_EINVAL, "unknown formula %d", formula);
    p = IntPlan();
    p.kind = BS_KIND_PERM;
    p.formula = formula;
    p.n = n;
    if (n == 0) {
        p.trivial = true;
        return BS_OK;
    }
    p.K = n;
    p.nrows = formula == BS_JOB_RYSER ? n : n - 1;
    p.nbin = p.nrows;
    p.C = 1ull << p.nrows;
    p.trans = true;
    p.pinned_src = 0;  // unused: the start sums do not come from a pinned row
    for (int j = 0; j < p.nrows; ++j) {
        p.radix[j] = 2;
        p.digit_src[j] = j;
    }
    for (int i = 0; i < n; ++i) p.col_src[i] = i;
    return BS_OK;
}

// Canonicalisation without heap allocation (fixed capacities: at most
// BS_MAX_N photons, so at most BS_MAX_N occupied rows or columns).
int plan_job(int rows, int cols, const int* M, const int* N, int kind, IntPlan& p) {
    if (rows < 0 || cols < 0) return fail(BS_EINVAL, "negative matrix size %d x %d", rows, cols);
    if ((rows > 0 && !M) || (cols > 0 && !N)) return fail(BS_EINVAL, "multiplicity array is NULL");
    long sm = 0, sn = 0;
    for (int r = 0; r < rows; ++r) {
        if (M[r] < 0) return fail(BS_EINVAL, "row multiplicity %d of row %d is negative", M[r], r);
        sm += M[r];
    }
    for (int j = 0; j < cols; ++j) {
        if (N[j] < 0) return fail(BS_EINVAL, "column multiplicity %d of column %d is negative", N[j], j);
        sn += N[j];
    }
    p = IntPlan();
    p.kind = kind;
    if (kind == BS_KIND_PERM) {
        if (sm != sn) return fail(BS_EINVAL, "sum of row multiplicities %ld != sum of column multiplicities %ld", sm, sn);
        if (sm > BS_MAX_N) return fail(BS_EINVAL, "n = %ld photons exceeds the limit %d", sm, BS_MAX_N);
    } else {
        if (sm != sn - 1)
            return fail(BS_EINVAL, "minors need sum(row_mult) = sum(col_mult) - 1, got %ld and %ld", sm, sn);
        if (sn > BS_MAX_N) return fail(BS_EINVAL, "n + 1 = %ld columns exceeds the limit %d", sn, BS_MAX_N);
    }
    p.n = (int)sm;
    if (p.n == 0) {
        p.trivial = true;  // per(0 x 0) = 1 (minors: the single column with N = 1)
        return BS_OK;
    }
    int rsrc[BS_MAX_N], rmul[BS_MAX_N], csrc[BS_MAX_N + 1], cmul[BS_MAX_N + 1];
    int nr = 0, nc = 0;
    for (int r = 0; r < rows; ++r)
        if (M[r] > 0) {
            rsrc[nr] = r;
            rmul[nr++] = M[r];
        }
    for (int j = 0; j < cols; ++j)
        if (N[j] > 0) {
            csrc[nc] = j;
            cmul[nc++] = N[j];
        }
    const int* Rs = rsrc;
    const int* Rm = rmul;
    const int* Cs = csrc;
    const int* Cm = cmul;
    int nR = nr, nC = nc;
    if (kind == BS_KIND_PERM && pin_cost(cmul, nc) < pin_cost(rmul, nr)) {
        p.trans = true;
        Rs = csrc;
        Rm = cmul;
        nR = nc;
        Cs = rsrc;
        Cm = rmul;
        nC = nr;
    }
    int pin = 0;
    for (int i = 1; i < nR; ++i)
        if (Rm[i] < Rm[pin]) pin = i;
    p.pinned_src = Rs[pin];
    p.pinned_m = Rm[pin];
    // digits: binary first (order of appearance, then a split pinned row of
    // multiplicity 2), then repeated rows by increasing multiplicity
    int dm[BS_MAX_DIGITS], ds[BS_MAX_DIGITS], nd = 0;
    for (int i = 0; i < nR; ++i)
        if (i != pin && Rm[i] == 1) {
            dm[nd] = 1;
            ds[nd++] = Rs[i];
        }
    if (Rm[pin] == 2) {
        dm[nd] = 1;
        ds[nd++] = Rs[pin];
    }
    p.nbin = nd;
    for (int i = 0; i <= nR; ++i) {
        int m, s;
        if (i < nR) {
            if (i == pin || Rm[i] == 1) continue;
            m = Rm[i];
            s = Rs[i];
        } else {
            if (Rm[pin] <= 2) continue;
            m = Rm[pin] - 1;
            s = Rs[pin];
        }
        int pos = nd;
        while (pos > p.nbin && dm[pos - 1] > m) {  // stable insertion sort
            dm[pos] = dm[pos - 1];
            ds[pos] = ds[pos - 1];
            --pos;
        }
        dm[pos] = m;
        ds[pos] = s;
        ++nd;
    }
    p.nrows = nd;
    p.C = 1;
    for (int d = 0; d < nd; ++d) {
        p.radix[d] = dm[d] + 1;
        p.digit_src[d] = ds[d];
        p.C *= (uint64_t)(dm[d] + 1);
    }
    p.K = 0;
    for (int j = 0; j < nC; ++j)
        for (int t = 0; t < Cm[j]; ++t) p.col_src[p.K++] = Cs[j];
    return BS_OK;
}

// Product column of the first copy of source column c in a minors plan
// (columns expanded in source order); -1 when col_mult[c] == 0.
int first_product_col(const int* N, int c) {
    if (N[c] <= 0) return -1;
    int at = 0;
    for (int j = 0; j < c; ++j) at += N[j] > 0 ? N[j] : 0;
    return at;
}

}  // namespace bs
