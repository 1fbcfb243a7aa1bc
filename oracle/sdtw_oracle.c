/*
 * sdtw_oracle.c -- plain, slow, obviously-correct CPU subsequence DTW.
 *
 * TEST INFRASTRUCTURE ONLY.  The parity tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this file's shared object; the CUDA
 * library never links, includes or calls it, and it shares no code with the
 * CUDA sources.
 *
 * What it computes (paper Section 2):
 *   Eq. 1    D(i,j) = d(x_i, y_j) + min{ D(i-1,j), D(i,j-1), D(i-1,j-1) }
 *   cost d   the paper only calls d "a measure of distance"; it is read here
 *            as the squared difference d(x,y) = (x - y)^2, with no square root.
 *   subsequence form (Section 2): the query x (length n, one row per sample)
 *            may start and end anywhere in the reference y (length m, one
 *            column per sample).  The start is free: row 0 holds only the local
 *            cost, D(0,j) = d(x_0, y_j), which is Eq. 1 with a virtual row -1 of
 *            zeros.  Column 0 has no left neighbours: D(i,0) = D(i-1,0) + d.
 *            The end is free: cost = min_j D(n-1, j), and end = the smallest j
 *            attaining that minimum.
 *   walk-back (Section 2): after the matrix is filled, the warp path is traced
 *            from (n-1, end) back to row 0, each step moving to the neighbour
 *            with the smallest accumulated cost among (i-1,j-1), (i,j-1),
 *            (i-1,j) -- the three cells of Eq. 1.  Exact ties go to the first
 *            of that list.  In column 0 the only neighbour is (i-1,0); the path
 *            stops on reaching row 0.
 *
 *   z-normalisation (Section 5.1, Eq. 2): the standardisation the paper
 *            applies to the reference and every query before the fill.
 *
 * Floating point is double throughout, except the binary16 variant (the
 * paper's own precision, each operation rounded to binary16); the integer
 * variant uses int64 and is exact.  Everything is a straightforward
 * row-by-row scalar loop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* ------------------------------------------------------------------ f64 -- */

static double local_cost_f64(double a, double b)
{
    double d = a - b;
    return d * d;
}

/* min over the last row, smallest index on exact ties */
static void last_row_min_f64(const double* row, int64_t m, double* cost, int64_t* end)
{
    double best = row[0];
    int64_t arg = 0;
    for (int64_t j = 1; j < m; ++j) {
        if (row[j] < best) {
            best = row[j];
            arg = j;
        }
    }
    *cost = best;
    *end = arg;
}

/*
 * Forward sDTW of one query x[0..n) against y[0..m) in double precision.
 * Writes the minimum cost and its (smallest) end column; if last_row is not
 * NULL it receives D(n-1, j) for every j.  Returns 0, or a negative code.
 */
int sdtw_oracle_forward_f64(const double* x, int64_t n, const double* y, int64_t m,
                            double* cost, int64_t* end, double* last_row)
{
    if (!x || !y || !cost || !end || n < 1 || m < 1) return ORACLE_EINVAL;
    double* prev = (double*)malloc((size_t)m * sizeof(double));
    double* cur = (double*)malloc((size_t)m * sizeof(double));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return ORACLE_ENOMEM;
    }
    /* row 0: free start */
    for (int64_t j = 0; j < m; ++j) prev[j] = local_cost_f64(x[0], y[j]);
    for (int64_t i = 1; i < n; ++i) {
        /* column 0: only the cell above */
        cur[0] = prev[0] + local_cost_f64(x[i], y[0]);
        for (int64_t j = 1; j < m; ++j) {
            double best = prev[j - 1];            /* (i-1, j-1) */
            if (cur[j - 1] < best) best = cur[j - 1]; /* (i, j-1) */
            if (prev[j] < best) best = prev[j];   /* (i-1, j) */
            cur[j] = best + local_cost_f64(x[i], y[j]);
        }
        double* t = prev;
        prev = cur;
        cur = t;
    }
    last_row_min_f64(prev, m, cost, end);
    if (last_row) memcpy(last_row, prev, (size_t)m * sizeof(double));
    free(prev);
    free(cur);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ i64 -- */

static int64_t local_cost_i64(int64_t a, int64_t b)
{
    int64_t d = a - b;
    return d * d;
}

/* Same algorithm as sdtw_oracle_forward_f64, in exact int64 arithmetic. */
int sdtw_oracle_forward_i64(const int64_t* x, int64_t n, const int64_t* y, int64_t m,
                            int64_t* cost, int64_t* end, int64_t* last_row)
{
    if (!x || !y || !cost || !end || n < 1 || m < 1) return ORACLE_EINVAL;
    int64_t* prev = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    int64_t* cur = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return ORACLE_ENOMEM;
    }
    for (int64_t j = 0; j < m; ++j) prev[j] = local_cost_i64(x[0], y[j]);
    for (int64_t i = 1; i < n; ++i) {
        cur[0] = prev[0] + local_cost_i64(x[i], y[0]);
        for (int64_t j = 1; j < m; ++j) {
            int64_t best = prev[j - 1];
            if (cur[j - 1] < best) best = cur[j - 1];
            if (prev[j] < best) best = prev[j];
            cur[j] = best + local_cost_i64(x[i], y[j]);
        }
        int64_t* t = prev;
        prev = cur;
        cur = t;
    }
    int64_t best = prev[0], arg = 0;
    for (int64_t j = 1; j < m; ++j) {
        if (prev[j] < best) {
            best = prev[j];
            arg = j;
        }
    }
    *cost = best;
    *end = arg;
    if (last_row) memcpy(last_row, prev, (size_t)m * sizeof(int64_t));
    free(prev);
    free(cur);
    return ORACLE_OK;
}

/* ----------------------------------------------------------------- f16 -- */

/*
 * The paper's own precision (Section 5.2 runs its fill in float16, packed as
 * __half2): Eq. 1 evaluated with every operation rounded to IEEE 754
 * binary16, round to nearest with ties to even,
 *     d = fl16(x_i - y_j),   D(i,j) = fl16(d * d + min{ D(i-1,j), D(i,j-1), D(i-1,j-1) }),
 * the product and the sum rounded once (a fused multiply-add); the minimum is
 * exact.  Boundaries and the free start and end as in the double version
 * (row 0: D(0,j) = fl16(d * d + 0)).  Values are carried in doubles, each
 * one a binary16 value; a sum at or beyond 65520 rounds to +inf.
 */

/* The binary16 value nearest to v (ties to the even significand).  Normal
 * binary16 numbers have 11 significant bits, so in [2^(e-1), 2^e) the spacing
 * is 2^(e-11); below 2^-14 the spacing is that of the subnormals, 2^-24. */
static double round_f16(double v)
{
    if (v == 0.0 || isnan(v) || isinf(v)) return v;
    const double a = fabs(v);
    int e;
    frexp(a, &e);
    const double ulp = ldexp(1.0, e - 11 < -24 ? -24 : e - 11);
    const double q = a / ulp;              /* exact: a power-of-two scaling */
    double r = floor(q);
    const double f = q - r;                /* exact */
    if (f > 0.5 || (f == 0.5 && fmod(r, 2.0) != 0.0)) r += 1.0;
    double res = r * ulp;
    if (res > 65504.0) res = INFINITY;     /* 65520 and above: beyond the largest finite value */
    return copysign(res, v);
}

/* fl16(a * b + c) for binary16 a, b, c, rounded once.  a * b is exact in
 * double (two 11-bit significands); the sum s = fl64(a * b + c) plus its
 * exact error t (TwoSum) give the exact value s + t.  Rounding s alone is
 * right unless s lies exactly halfway between two binary16 values and t != 0,
 * in which case the exact value lies on t's side of that midpoint. */
static double fma_f16(double a, double b, double c)
{
    const double p = a * b;
    const double s = p + c;
    if (isinf(s) || isnan(s)) return s;
    const double bb = s - p;
    const double t = (p - (s - bb)) + (c - bb);
    const double r = round_f16(s);
    if (t == 0.0 || r == s) return r;
    /* is s a midpoint?  then the nearer neighbour on t's side wins */
    const double a_s = fabs(s);
    int e;
    frexp(a_s, &e);
    const double ulp = ldexp(1.0, e - 11 < -24 ? -24 : e - 11);
    const double q = a_s / ulp;
    if (q - floor(q) != 0.5) return r;
    const double lo = copysign(floor(q) * ulp, s), hi = copysign((floor(q) + 1.0) * ulp, s);
    const double below = s > 0 ? lo : hi, above = s > 0 ? hi : lo;   /* as signed values */
    const double pick = t > 0 ? above : below;
    return fabs(pick) > 65504.0 ? copysign(INFINITY, pick) : pick;
}

/* Test hooks for the two rounding routines (pinned against numpy's float16
 * conversion and against exact rational arithmetic). */
int sdtw_oracle_round_f16(const double* in, int64_t n, double* out)
{
    if (!in || !out || n < 0) return ORACLE_EINVAL;
    for (int64_t k = 0; k < n; ++k) out[k] = round_f16(in[k]);
    return ORACLE_OK;
}

int sdtw_oracle_fma_f16(const double* a, const double* b, const double* c, int64_t n, double* out)
{
    if (!a || !b || !c || !out || n < 0) return ORACLE_EINVAL;
    for (int64_t k = 0; k < n; ++k) out[k] = fma_f16(a[k], b[k], c[k]);
    return ORACLE_OK;
}

/* Eq. 1 in binary16 arithmetic; x and y must hold binary16 values. */
int sdtw_oracle_forward_f16(const double* x, int64_t n, const double* y, int64_t m,
                            double* cost, int64_t* end, double* last_row)
{
    if (!x || !y || !cost || !end || n < 1 || m < 1) return ORACLE_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (!(round_f16(x[i]) == x[i]) || isinf(x[i])) return ORACLE_EINVAL;
    for (int64_t j = 0; j < m; ++j)
        if (!(round_f16(y[j]) == y[j]) || isinf(y[j])) return ORACLE_EINVAL;
    double* prev = (double*)malloc((size_t)m * sizeof(double));
    double* cur = (double*)malloc((size_t)m * sizeof(double));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return ORACLE_ENOMEM;
    }
    for (int64_t j = 0; j < m; ++j) {
        const double d = round_f16(x[0] - y[j]);   /* x - y is exact in double */
        prev[j] = fma_f16(d, d, 0.0);
    }
    for (int64_t i = 1; i < n; ++i) {
        const double d0 = round_f16(x[i] - y[0]);
        cur[0] = fma_f16(d0, d0, prev[0]);
        for (int64_t j = 1; j < m; ++j) {
            double best = prev[j - 1];
            if (cur[j - 1] < best) best = cur[j - 1];
            if (prev[j] < best) best = prev[j];
            const double d = round_f16(x[i] - y[j]);
            cur[j] = fma_f16(d, d, best);
        }
        double* t = prev;
        prev = cur;
        cur = t;
    }
    double best = prev[0];
    int64_t arg = 0;
    for (int64_t j = 1; j < m; ++j) {
        if (prev[j] < best) {
            best = prev[j];
            arg = j;
        }
    }
    *cost = best;
    *end = arg;
    if (last_row) memcpy(last_row, prev, (size_t)m * sizeof(double));
    free(prev);
    free(cur);
    return ORACLE_OK;
}

/* -------------------------------------------------- early-INF pruning -- */

/*
 * Section 8 of the paper (future work) proposes pruning: when the two samples
 * of a cell are "far" apart, the cell is taken not to lie on the path and its
 * cost is infinite instead of being computed.  Read here for the integer
 * modes: a cell with |x_i - y_j| > gap costs +inf, and +inf absorbs every
 * sum.  Eq. 1 is otherwise unchanged (free start, free end); the cost is +inf
 * when every cell of the last row is, and then no column ends a path (end -1).
 * gap >= 0.  PRUNED_INF stands for +inf: above every finite sum of at most
 * n * 2^17 int8 or uint8 local costs.
 */
#define PRUNED_INF ((int64_t)1 << 62)

static int64_t pruned_cost_i64(int64_t a, int64_t b, int64_t gap)
{
    const int64_t d = a - b;
    return (d > gap || -d > gap) ? PRUNED_INF : d * d;
}

static int64_t sat_add(int64_t a, int64_t b)
{
    return (a >= PRUNED_INF || b >= PRUNED_INF) ? PRUNED_INF : a + b;
}

int sdtw_oracle_forward_pruned_i64(const int64_t* x, int64_t n, const int64_t* y, int64_t m, int64_t gap,
                                   int64_t* cost, int64_t* end)
{
    if (!x || !y || !cost || !end || n < 1 || m < 1 || gap < 0) return ORACLE_EINVAL;
    int64_t* prev = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    int64_t* cur = (int64_t*)malloc((size_t)m * sizeof(int64_t));
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return ORACLE_ENOMEM;
    }
    for (int64_t j = 0; j < m; ++j) prev[j] = pruned_cost_i64(x[0], y[j], gap);
    for (int64_t i = 1; i < n; ++i) {
        cur[0] = sat_add(prev[0], pruned_cost_i64(x[i], y[0], gap));
        for (int64_t j = 1; j < m; ++j) {
            int64_t best = prev[j - 1];
            if (cur[j - 1] < best) best = cur[j - 1];
            if (prev[j] < best) best = prev[j];
            cur[j] = sat_add(best, pruned_cost_i64(x[i], y[j], gap));
        }
        int64_t* t = prev;
        prev = cur;
        cur = t;
    }
    int64_t best = prev[0], arg = 0;
    for (int64_t j = 1; j < m; ++j) {
        if (prev[j] < best) {
            best = prev[j];
            arg = j;
        }
    }
    *cost = best;
    *end = best >= PRUNED_INF ? -1 : arg;
    free(prev);
    free(cur);
    return ORACLE_OK;
}

/* ------------------------------------------------------------- walk-back -- */

/*
 * Fill the whole n x m matrix D (double), then walk back from (n-1, end).
 *
 * Outputs, for a path of L cells listed from the end cell back to row 0:
 *   path_i[k], path_j[k]  the k-th cell (capacity n + m - 1 each)
 *   *path_len             L
 *   margin[k]             for a cell with three neighbours, the gap between
 *                         the second-smallest and the smallest neighbour D
 *                         (0 on an exact tie); -1 where the step had a single
 *                         choice (column 0) or none (row 0).  May be NULL.
 * end must lie in [0, m).  The matrix needs n*m doubles; the caller bounds n*m.
 */
int sdtw_oracle_walkback_f64(const double* x, int64_t n, const double* y, int64_t m,
                             int64_t end, int64_t* path_i, int64_t* path_j,
                             int64_t* path_len, double* margin)
{
    if (!x || !y || !path_i || !path_j || !path_len || n < 1 || m < 1) return ORACLE_EINVAL;
    if (end < 0 || end >= m) return ORACLE_EINVAL;
    double* D = (double*)malloc((size_t)n * (size_t)m * sizeof(double));
    if (!D) return ORACLE_ENOMEM;
#define AT(i, j) D[(size_t)(i) * (size_t)m + (size_t)(j)]
    for (int64_t j = 0; j < m; ++j) AT(0, j) = local_cost_f64(x[0], y[j]);
    for (int64_t i = 1; i < n; ++i) {
        AT(i, 0) = AT(i - 1, 0) + local_cost_f64(x[i], y[0]);
        for (int64_t j = 1; j < m; ++j) {
            double best = AT(i - 1, j - 1);
            if (AT(i, j - 1) < best) best = AT(i, j - 1);
            if (AT(i - 1, j) < best) best = AT(i - 1, j);
            AT(i, j) = best + local_cost_f64(x[i], y[j]);
        }
    }
    int64_t i = n - 1, j = end, L = 0;
    for (;;) {
        path_i[L] = i;
        path_j[L] = j;
        if (i == 0) {
            if (margin) margin[L] = -1.0;
            ++L;
            break;
        }
        if (j == 0) {
            if (margin) margin[L] = -1.0;
            ++L;
            i -= 1;
            continue;
        }
        /* neighbours in tie order: (i-1,j-1), (i,j-1), (i-1,j) */
        double v[3] = {AT(i - 1, j - 1), AT(i, j - 1), AT(i - 1, j)};
        int k = 0;
        for (int c = 1; c < 3; ++c)
            if (v[c] < v[k]) k = c;
        if (margin) {
            double second = -1.0;
            for (int c = 0; c < 3; ++c) {
                if (c == k) continue;
                double g = v[c] - v[k];
                if (second < 0.0 || g < second) second = g;
            }
            margin[L] = second;
        }
        ++L;
        if (k == 0) {
            i -= 1;
            j -= 1;
        } else if (k == 1) {
            j -= 1;
        } else {
            i -= 1;
        }
    }
#undef AT
    *path_len = L;
    free(D);
    return ORACLE_OK;
}

/* ------------------------------------------------------------ z-norm -- */

/*
 * Eq. 2 (paper Section 5.1): z = (x - mean) / S, with the series' own mean
 * and standard deviation.  The paper's text says "sample" statistics but its
 * code divides by n; the population form (divide by n) is taken.  Two passes
 * in double: the mean, then the centred second moment.  A series with S == 0
 * (constant, or of length 1) is only centred.  out may equal x.
 */
int sdtw_oracle_znorm_f64(const double* x, int64_t n, double* out)
{
    if (n < 0 || (n > 0 && (!x || !out))) return ORACLE_EINVAL;
    if (n == 0) return ORACLE_OK;
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) sum += x[i];
    const double mean = sum / (double)n;
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double c = x[i] - mean;
        ss += c * c;
    }
    double s = sqrt(ss / (double)n);
    if (!(s > 0.0)) s = 1.0;
    for (int64_t i = 0; i < n; ++i) out[i] = (x[i] - mean) / s;
    return ORACLE_OK;
}
