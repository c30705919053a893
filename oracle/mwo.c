/*
 * mwo.c -- CPU oracle for multiword (DD/TD/QD) LU with partial pivoting,
 * forward/back substitution, the exact long residual and mixed-precision
 * iterative refinement.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * It is deliberately plain and slow: every operation is written out in the
 * order the algorithm states it, with no blocking, fusion or reordering.
 * Build flags: -O2 -ffp-contract=off -fno-fast-math (a contracted a*b+c would
 * change the bits; aarch64 GCC contracts by default).
 *
 * Method (Kouya, "Accelerated Multiple Precision Direct Method and Mixed
 * Precision Iterative Refinement on Python Programming Environment"):
 *   - DD/TD/QD arithmetic made of 2/3/4 binary64 words (Section 1, Section 2);
 *     the paper names the QD library of Bailey et al. but does not print the
 *     algorithms, so the published ones below are used (readings listed in
 *     the design notes);
 *   - LU decomposition with partial pivoting and forward/back substitution
 *     in DD/TD/QD (Section 2, Listing 1: TDLUdecompPM, SolveTDLSPM);
 *   - mixed precision iterative refinement (Section 2, Listing 1) with the
 *     stopping test of Eq. (2); the long precision is 424 bits = 8 words.
 *
 * Data layout: a matrix of w-word values is w planes of lda*n doubles,
 * column-major; word c of A(i,j) is A[c*lda*n + j*lda + i].  A vector of
 * w-word values is w planes of n doubles: word c of v(i) is v[c*n + i].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MWO_MAXW 8

/* ------------------------------------------------------------------------ */
/* Error-free transformations                                                */
/* ------------------------------------------------------------------------ */

/* Knuth's TwoSum: s = fl(a+b), e = (a+b) - s exactly, for any a, b. */
static void two_sum(double a, double b, double *s, double *e)
{
    double ss = a + b;
    double ap = ss - b;
    double bp = ss - ap;
    double da = a - ap;
    double db = b - bp;
    *s = ss;
    *e = da + db;
}

/* Dekker's FastTwoSum: exact when exponent(a) >= exponent(b). */
static void fast_two_sum(double a, double b, double *s, double *e)
{
    double ss = a + b;
    double z = ss - a;
    *s = ss;
    *e = b - z;
}

/* TwoProd with a fused multiply-add: p = fl(a*b), e = a*b - p exactly
 * (barring underflow). */
static void two_prod(double a, double b, double *p, double *e)
{
    double pp = a * b;
    *p = pp;
    *e = fma(a, b, -pp);
}

/* ------------------------------------------------------------------------ */
/* Double-double: Joldes, Muller, Popescu, "Tight and rigorous error bounds  */
/* for basic building blocks of double-word arithmetic", ACM TOMS 44(2),     */
/* 2017: AccurateDWPlusDW (Alg. 6), DWTimesDW3 (Alg. 12), and the division   */
/* DWDivDW2 shape (Alg. 17) with the FMA form of the DW-times-FP product.    */
/* ------------------------------------------------------------------------ */

static void dd_add(const double *x, const double *y, double *z)
{
    double sh, sl, th, tl, c, vh, vl, w;
    two_sum(x[0], y[0], &sh, &sl);
    two_sum(x[1], y[1], &th, &tl);
    c = sl + th;
    fast_two_sum(sh, c, &vh, &vl);
    w = tl + vl;
    fast_two_sum(vh, w, &z[0], &z[1]);
}

static void dd_mul(const double *x, const double *y, double *z)
{
    double ch, cl1, tl0, tl1, cl2, cl3;
    two_prod(x[0], y[0], &ch, &cl1);
    tl0 = x[1] * y[1];
    tl1 = fma(x[0], y[1], tl0);
    cl2 = fma(x[1], y[0], tl1);
    cl3 = cl1 + cl2;
    fast_two_sum(ch, cl3, &z[0], &z[1]);
}

static void dd_div(const double *x, const double *y, double *z)
{
    double q0, ph, pl, rh, rl, dh, dl, d, q1;
    q0 = x[0] / y[0];
    two_prod(y[0], q0, &ph, &pl);     /* y*q0 as a double-word ...        */
    pl = fma(y[1], q0, pl);           /* ... including the low word of y  */
    fast_two_sum(ph, pl, &rh, &rl);
    dh = x[0] - rh;
    dl = x[1] - rl;
    d = dh + dl;
    q1 = d / y[0];
    fast_two_sum(q0, q1, &z[0], &z[1]);
}

/* ------------------------------------------------------------------------ */
/* Triple- and quad-word arithmetic (w = 3, 4).  The shape follows Hida, Li  */
/* and Bailey, "Algorithms for quad-double precision floating point          */
/* arithmetic" (ARITH 2001): exact partial results are gathered and then     */
/* renormalised.  The renormalisation is a bottom-up TwoSum cascade (the     */
/* VecSum of Ogita, Rump and Oishi, 2005), a top-down extraction that skips */
/* zero errors and folds everything past word w-1 into the last word, and a  */
/* top-down FastTwoSum sweep over the w result words.                        */
/* ------------------------------------------------------------------------ */

/* Renormalise the m terms t[0..m-1] (roughly ordered by decreasing
 * magnitude; t is overwritten) into w words z[0..w-1]. */
static void renorm(int w, int m, double *t, double *z)
{
    double s, hi, lo;
    int i, k;
    /* pass 1: exact bottom-up cascade */
    s = t[m - 1];
    for (i = m - 2; i >= 0; --i) {
        two_sum(t[i], s, &hi, &lo);
        s = hi;
        t[i + 1] = lo;
    }
    t[0] = s;
    /* pass 2: top-down extraction of w words */
    k = 0;
    s = t[0];
    for (i = 1; i < m; ++i) {
        if (k < w - 1) {
            two_sum(s, t[i], &hi, &lo);
            if (lo != 0.0) {
                z[k] = hi;
                k = k + 1;
                s = lo;
            } else {
                s = hi;
            }
        } else {
            s = s + t[i];
        }
    }
    z[k] = s;
    for (k = k + 1; k < w; ++k)
        z[k] = 0.0;
    /* pass 3: top-down FastTwoSum sweep, so that no word exceeds one ulp
     * of the word above it */
    for (i = 0; i < w - 1; ++i) {
        fast_two_sum(z[i], z[i + 1], &hi, &lo);
        z[i] = hi;
        z[i + 1] = lo;
    }
}

static void mw_add_gen(int w, const double *x, const double *y, double *z)
{
    double s[4] = {0, 0, 0, 0}, e[4] = {0, 0, 0, 0}, t[8];
    int i, m = 0;
    for (i = 0; i < w; ++i)
        two_sum(x[i], y[i], &s[i], &e[i]);
    /* order: s0, s1, e0, s2, e1, ..., s_{w-1}, e_{w-2}; e_{w-1} is dropped */
    t[m++] = s[0];
    for (i = 1; i < w; ++i) {
        t[m++] = s[i];
        t[m++] = e[i - 1];
    }
    renorm(w, m, t, z);
}

static void mw_mul_gen(int w, const double *x, const double *y, double *z)
{
    double t[10];
    double p00, q00, p01, q01, p10, q10, c;
    two_prod(x[0], y[0], &p00, &q00);
    two_prod(x[0], y[1], &p01, &q01);
    two_prod(x[1], y[0], &p10, &q10);
    if (w == 3) {
        c = x[1] * y[1];
        c = fma(x[0], y[2], c);
        c = fma(x[2], y[0], c);
        c = c + q01;
        c = c + q10;
        t[0] = p00; t[1] = q00; t[2] = p01; t[3] = p10; t[4] = c;
        renorm(3, 5, t, z);
    } else {
        double p02, q02, p11, q11, p20, q20;
        two_prod(x[0], y[2], &p02, &q02);
        two_prod(x[1], y[1], &p11, &q11);
        two_prod(x[2], y[0], &p20, &q20);
        c = x[1] * y[2];
        c = fma(x[2], y[1], c);
        c = fma(x[0], y[3], c);
        c = fma(x[3], y[0], c);
        c = c + q02;
        c = c + q11;
        c = c + q20;
        t[0] = p00; t[1] = q00; t[2] = p01; t[3] = p10; t[4] = q01;
        t[5] = q10; t[6] = p02; t[7] = p11; t[8] = p20; t[9] = c;
        renorm(4, 10, t, z);
    }
}

/* w-word value times a double */
static void mw_mul_d_gen(int w, const double *x, double d, double *z)
{
    double p[4], q[4], t[8];
    int i, m = 0;
    for (i = 0; i < w - 1; ++i)
        two_prod(x[i], d, &p[i], &q[i]);
    p[w - 1] = x[w - 1] * d;
    t[m++] = p[0];
    for (i = 1; i < w; ++i) {
        t[m++] = p[i];
        t[m++] = q[i - 1];
    }
    renorm(w, m, t, z);
}

/* long division: w+1 quotient digits, then renormalise */
static void mw_div_gen(int w, const double *x, const double *y, double *z)
{
    double q[5], r[4], p[4], nr[4], t[5];
    int i, c;
    q[0] = x[0] / y[0];
    for (c = 0; c < w; ++c)
        r[c] = x[c];
    for (i = 1; i <= w; ++i) {
        mw_mul_d_gen(w, y, q[i - 1], p);
        for (c = 0; c < w; ++c)
            p[c] = -p[c];
        mw_add_gen(w, r, p, nr);
        for (c = 0; c < w; ++c)
            r[c] = nr[c];
        q[i] = r[0] / y[0];
    }
    for (i = 0; i <= w; ++i)
        t[i] = q[i];
    renorm(w, w + 1, t, z);
}

/* ------------------------------------------------------------------------ */
/* Precision dispatch                                                       */
/* ------------------------------------------------------------------------ */

static void mw_add(int w, const double *x, const double *y, double *z)
{
    if (w == 2) dd_add(x, y, z); else mw_add_gen(w, x, y, z);
}

static void mw_sub(int w, const double *x, const double *y, double *z)
{
    double ny[4];
    int c;
    for (c = 0; c < w; ++c)
        ny[c] = -y[c];
    mw_add(w, x, ny, z);
}

static void mw_mul(int w, const double *x, const double *y, double *z)
{
    if (w == 2) dd_mul(x, y, z); else mw_mul_gen(w, x, y, z);
}

static void mw_div(int w, const double *x, const double *y, double *z)
{
    if (w == 2) dd_div(x, y, z); else mw_div_gen(w, x, y, z);
}

/* Compare |x| with |y| lexicographically on the sign-adjusted words
 * (|x0|, s*x1, s*x2, ...), s = sign of x0.  Returns -1, 0, +1. */
static int mw_cmpabs(int w, const double *x, const double *y)
{
    int c;
    double sx = (x[0] < 0.0) ? -1.0 : 1.0;
    double sy = (y[0] < 0.0) ? -1.0 : 1.0;
    for (c = 0; c < w; ++c) {
        double a = sx * x[c], b = sy * y[c];
        if (a > b) return 1;
        if (a < b) return -1;
    }
    return 0;
}

static int mw_iszero(int w, const double *x)
{
    int c;
    for (c = 0; c < w; ++c)
        if (x[c] != 0.0) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Element access helpers for the planar layout                             */
/* ------------------------------------------------------------------------ */

static void ld_m(int w, const double *A, int64_t plane, int64_t idx, double *v)
{
    int c;
    for (c = 0; c < w; ++c) v[c] = A[c * plane + idx];
}

static void st_m(int w, double *A, int64_t plane, int64_t idx, const double *v)
{
    int c;
    for (c = 0; c < w; ++c) A[c * plane + idx] = v[c];
}

/* ------------------------------------------------------------------------ */
/* Exported: element-wise arithmetic for the tests                          */
/* ------------------------------------------------------------------------ */

/* op: 0 TwoSum, 1 FastTwoSum, 2 TwoProd.  Outputs s[i], e[i]. */
int mwo_eft(int op, int64_t cnt, const double *a, const double *b, double *s, double *e)
{
    int64_t i;
    for (i = 0; i < cnt; ++i) {
        if (op == 0) two_sum(a[i], b[i], &s[i], &e[i]);
        else if (op == 1) fast_two_sum(a[i], b[i], &s[i], &e[i]);
        else if (op == 2) two_prod(a[i], b[i], &s[i], &e[i]);
        else return -1;
    }
    return 0;
}

/* op: 0 add, 1 sub, 2 mul, 3 div, 4 cmpabs (z plane 0 gets -1/0/+1),
 *     5 times-a-double (y is a plain array of cnt doubles),
 *     6 renorm of the 2w words of x followed by y, read as terms
 *       x0,y0,x1,y1,... (w output words).
 * x, y, z: w planes of cnt doubles. */
int mwo_arith(int op, int w, int64_t cnt, const double *x, const double *y, double *z)
{
    int64_t i;
    if (w < 2 || w > 4) return -2;
    for (i = 0; i < cnt; ++i) {
        double a[4], b[4], r[4], t[8];
        int c;
        ld_m(w, x, cnt, i, a);
        if (op == 5) b[0] = y[i]; else ld_m(w, y, cnt, i, b);
        switch (op) {
        case 0: mw_add(w, a, b, r); break;
        case 1: mw_sub(w, a, b, r); break;
        case 2: mw_mul(w, a, b, r); break;
        case 3: mw_div(w, a, b, r); break;
        case 4:
            r[0] = (double)mw_cmpabs(w, a, b);
            for (c = 1; c < w; ++c) r[c] = 0.0;
            break;
        case 5:
            if (w == 2) {
                /* DD times double: the FMA form used inside dd_div */
                double ph, pl;
                two_prod(a[0], b[0], &ph, &pl);
                pl = fma(a[1], b[0], pl);
                fast_two_sum(ph, pl, &r[0], &r[1]);
            } else {
                mw_mul_d_gen(w, a, b[0], r);
            }
            break;
        case 6:
            for (c = 0; c < w; ++c) { t[2 * c] = a[c]; t[2 * c + 1] = b[c]; }
            renorm(w, 2 * w, t, r);
            break;
        default:
            return -1;
        }
        st_m(w, z, cnt, i, r);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LU decomposition with partial pivoting (Section 2, Listing 1:            */
/* TDLUdecompPM).  Unblocked right-looking k-j-i order, LAPACK getf2        */
/* semantics:                                                               */
/*   for k: p = argmax_{i>=k} |a_ik| (first index on ties); swap rows k, p  */
/*   over all columns; piv[k] = p; if a_kk == 0 record info = k+1 (first)   */
/*   and skip the scaling, else l_ik = a_ik / a_kk (a division per entry);  */
/*   then a_ij = a_ij - l_ik * a_kj for i, j > k (a rounded multiply then a */
/*   rounded subtraction).                                                  */
/* In place: A <- L\U, unit lower L implicit.  piv is 0-based.              */
/* ------------------------------------------------------------------------ */

/* The first `ksteps` elimination steps only (ksteps >= n: the whole
 * factorisation).  Used to time a bounded sample of a large factorisation. */
int mwo_lu_steps(int w, int64_t n, double *A, int64_t lda, int64_t *piv, int64_t *info,
                 int64_t ksteps)
{
    int64_t plane, k, kend;
    if (w < 2 || w > 4) return -1;
    if (n < 0) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    plane = lda * n;
    *info = 0;
    kend = ksteps < n ? ksteps : n;
    for (k = 0; k < kend; ++k) {
        double best[4], v[4], akk[4];
        int64_t p = k, i, j;
        ld_m(w, A, plane, k * lda + k, best);
        for (i = k + 1; i < n; ++i) {
            ld_m(w, A, plane, k * lda + i, v);
            if (mw_cmpabs(w, v, best) > 0) {
                p = i;
                memcpy(best, v, sizeof(v));
            }
        }
        piv[k] = p;
        if (p != k) {
            for (j = 0; j < n; ++j) {
                int c;
                for (c = 0; c < w; ++c) {
                    double tmp = A[c * plane + j * lda + k];
                    A[c * plane + j * lda + k] = A[c * plane + j * lda + p];
                    A[c * plane + j * lda + p] = tmp;
                }
            }
        }
        ld_m(w, A, plane, k * lda + k, akk);
        if (mw_iszero(w, akk)) {
            if (*info == 0) *info = k + 1;
        } else {
            for (i = k + 1; i < n; ++i) {
                double l[4];
                ld_m(w, A, plane, k * lda + i, v);
                mw_div(w, v, akk, l);
                st_m(w, A, plane, k * lda + i, l);
            }
        }
        /* trailing update; columns are independent, so the loop over j can
         * run in parallel without changing any element's operation order */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (j = k + 1; j < n; ++j) {
            double u[4], l[4], a[4], prod[4], res[4];
            int64_t ii;
            ld_m(w, A, plane, j * lda + k, u);
            for (ii = k + 1; ii < n; ++ii) {
                ld_m(w, A, plane, k * lda + ii, l);
                ld_m(w, A, plane, j * lda + ii, a);
                mw_mul(w, l, u, prod);
                mw_sub(w, a, prod, res);
                st_m(w, A, plane, j * lda + ii, res);
            }
        }
    }
    return 0;
}

int mwo_lu(int w, int64_t n, double *A, int64_t lda, int64_t *piv, int64_t *info)
{
    return mwo_lu_steps(w, n, A, lda, piv, info, n);
}

/* ------------------------------------------------------------------------ */
/* Forward/back substitution (Section 2, Listing 1: SolveTDLSPM).           */
/*   y = P b (swaps in order k = 0..n-1);                                   */
/*   y_i = y_i - l_ij * y_j   for j ascending (unit lower L);               */
/*   d_j = 1 / u_jj (a multiword division, for every j first), then        */
/*   x_j = y_j * d_j and y_i = y_i - u_ij * x_j for j descending.           */
/* b and x are w planes of n; b may alias x.                                */
/* ------------------------------------------------------------------------ */

int mwo_solve(int w, int64_t n, const double *LU, int64_t lda, const int64_t *piv,
              const double *b, double *x)
{
    int64_t plane, i, j, k;
    double *y, *d;
    if (w < 2 || w > 4) return -1;
    if (n == 0) return 0;
    plane = lda * n;
    y = (double *)malloc(sizeof(double) * (size_t)(w * n));
    d = (double *)malloc(sizeof(double) * (size_t)(w * n));
    if (!y || !d) { free(y); free(d); return -100; }
    memcpy(y, b, sizeof(double) * (size_t)(w * n));
    for (k = 0; k < n; ++k) {
        int64_t p = piv[k];
        if (p != k) {
            int c;
            for (c = 0; c < w; ++c) {
                double tmp = y[c * n + k];
                y[c * n + k] = y[c * n + p];
                y[c * n + p] = tmp;
            }
        }
    }
    for (j = 0; j < n; ++j) {
        double yj[4];
        ld_m(w, y, n, j, yj);
        for (i = j + 1; i < n; ++i) {
            double l[4], yi[4], prod[4], res[4];
            ld_m(w, LU, plane, j * lda + i, l);
            ld_m(w, y, n, i, yi);
            mw_mul(w, l, yj, prod);
            mw_sub(w, yi, prod, res);
            st_m(w, y, n, i, res);
        }
    }
    for (j = 0; j < n; ++j) {
        double one[4] = {1.0, 0.0, 0.0, 0.0}, ujj[4], dj[4];
        ld_m(w, LU, plane, j * lda + j, ujj);
        mw_div(w, one, ujj, dj);
        st_m(w, d, n, j, dj);
    }
    for (j = n - 1; j >= 0; --j) {
        double yj[4], dj[4], xj[4];
        ld_m(w, y, n, j, yj);
        ld_m(w, d, n, j, dj);
        mw_mul(w, yj, dj, xj);
        st_m(w, y, n, j, xj);
        for (i = 0; i < j; ++i) {
            double u[4], yi[4], prod[4], res[4];
            ld_m(w, LU, plane, j * lda + i, u);
            ld_m(w, y, n, i, yi);
            mw_mul(w, u, xj, prod);
            mw_sub(w, yi, prod, res);
            st_m(w, y, n, i, res);
        }
    }
    memcpy(x, y, sizeof(double) * (size_t)(w * n));
    free(y);
    free(d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact accumulation (the long-precision residual of Listing 1, computed   */
/* exactly and then rounded once).  A fixed-point integer of NLIMB 32-bit   */
/* digits held in int64 slots; digit k weighs 2^(LOWBIT + 32 k).  Every     */
/* product of two finite doubles lies on this grid (its lowest bit is at    */
/* least 2^-2148), so deposits are exact.                                   */
/* ------------------------------------------------------------------------ */

#define NLIMB 140
#define LOWBIT (-2176)

typedef struct { int64_t d[NLIMB]; } acc_t;

/* odd integer mantissa and exponent: v = m * 2^e, m odd (v != 0) */
static void decompose(double v, uint64_t *m, int *e)
{
    int ex;
    double f = frexp(fabs(v), &ex);      /* |v| = f * 2^ex, f in [0.5, 1) */
    uint64_t mm = (uint64_t)ldexp(f, 53); /* exact: f has <= 53 bits */
    int ee = ex - 53;
    while ((mm & 1u) == 0) { mm >>= 1; ee += 1; }
    *m = mm;
    *e = ee;
}

/* add sign * mag * 2^e, mag < 2^128 */
static void acc_add_u128(acc_t *a, int neg, unsigned __int128 mag, int e)
{
    int off = e - LOWBIT, k, sh, q;
    if (mag == 0) return;
    k = off / 32;
    sh = off % 32;
    for (q = 0; q < 4; ++q) {
        uint64_t chunk = (uint64_t)((mag >> (32 * q)) & 0xffffffffu);
        uint64_t v;
        if (chunk == 0) continue;
        v = chunk << sh;
        if (neg) {
            a->d[k + q] -= (int64_t)(v & 0xffffffffu);
            a->d[k + q + 1] -= (int64_t)(v >> 32);
        } else {
            a->d[k + q] += (int64_t)(v & 0xffffffffu);
            a->d[k + q + 1] += (int64_t)(v >> 32);
        }
    }
}

static void acc_add_double(acc_t *a, double v, int extra_exp)
{
    uint64_t m;
    int e;
    if (v == 0.0) return;
    decompose(v, &m, &e);
    acc_add_u128(a, v < 0.0, (unsigned __int128)m, e + extra_exp);
}

/* add (sign) * x * y * 2^extra_exp exactly */
static void acc_add_prod(acc_t *a, double x, double y, int negate, int extra_exp)
{
    uint64_t mx, my;
    int ex, ey, neg;
    if (x == 0.0 || y == 0.0) return;
    decompose(x, &mx, &ex);
    decompose(y, &my, &ey);
    neg = ((x < 0.0) != (y < 0.0));
    if (negate) neg = !neg;
    acc_add_u128(a, neg, (unsigned __int128)mx * my, ex + ey + extra_exp);
}

/* carry-propagate: digits 0..NLIMB-2 in [0, 2^32), top digit signed */
static void acc_norm(acc_t *a)
{
    int k;
    for (k = 0; k < NLIMB - 1; ++k) {
        int64_t c = a->d[k] >> 32;  /* arithmetic shift = floor division */
        a->d[k] -= c * ((int64_t)1 << 32);
        a->d[k + 1] += c;
    }
}

static int acc_bit(const acc_t *a, int pos) /* pos: absolute bit exponent */
{
    int r = pos - LOWBIT;
    if (r < 0) return 0;
    return (int)((a->d[r / 32] >> (r % 32)) & 1);
}

static int acc_any_below(const acc_t *a, int pos) /* any bit at exponent < pos */
{
    int r = pos - LOWBIT, k;
    if (r <= 0) return 0;
    for (k = 0; k < r / 32; ++k)
        if (a->d[k] != 0) return 1;
    if (r % 32) {
        uint64_t mask = ((uint64_t)1 << (r % 32)) - 1;
        if (((uint64_t)a->d[r / 32] & mask) != 0) return 1;
    }
    return 0;
}

/* Round the accumulated value to nearest (ties to even, IEEE binary64
 * including subnormals and overflow) and remove the rounded value from the
 * accumulator.  Returns the rounded double. */
static double acc_take_rn(acc_t *a)
{
    int neg = 0, k, top = -1, hb, H, lsb, b;
    uint64_t q = 0;
    double res;
    acc_norm(a);
    if (a->d[NLIMB - 1] < 0) {
        neg = 1;
        for (k = 0; k < NLIMB; ++k) a->d[k] = -a->d[k];
        acc_norm(a);
    }
    for (k = NLIMB - 1; k >= 0; --k)
        if (a->d[k] != 0) { top = k; break; }
    if (top < 0) {
        if (neg) { for (k = 0; k < NLIMB; ++k) a->d[k] = -a->d[k]; acc_norm(a); }
        return 0.0;
    }
    hb = 63;
    while (((a->d[top] >> hb) & 1) == 0) --hb;
    H = LOWBIT + 32 * top + hb;           /* exponent of the leading bit */
    lsb = H - 52;
    if (lsb < -1074) lsb = -1074;
    for (b = H; b >= lsb; --b)
        q = (q << 1) | (uint64_t)acc_bit(a, b);
    if (acc_bit(a, lsb - 1) && (acc_any_below(a, lsb - 1) || (q & 1u)))
        q += 1;
    if (lsb > 1023 - 52 || (lsb == 1023 - 52 + 1 && q != 0) ||
        ldexp((double)q, lsb) == INFINITY)
        res = INFINITY;
    else
        res = ldexp((double)q, lsb);
    /* remove the rounded value (still in magnitude form) */
    if (res != INFINITY)
        acc_add_u128(a, 1, (unsigned __int128)q, lsb);
    if (neg) {
        for (k = 0; k < NLIMB; ++k) a->d[k] = -a->d[k];
        res = -res;
    }
    acc_norm(a);
    return res;
}

/* greedy round-to-nearest into nw words: c_i = RN(S - sum_{j<i} c_j) */
static void acc_round_words(acc_t *a, int nw, double *out, int64_t stride)
{
    int c;
    for (c = 0; c < nw; ++c)
        out[c * stride] = acc_take_rn(a);
}

/* Exported for the tests: out = greedy RN words of sum(terms[0..cnt-1]). */
int mwo_exact_sum(int64_t cnt, const double *terms, int nw, double *out)
{
    acc_t *a = (acc_t *)calloc(1, sizeof(acc_t));
    int64_t i;
    if (!a) return -100;
    for (i = 0; i < cnt; ++i) acc_add_double(a, terms[i], 0);
    acc_round_words(a, nw, out, 1);
    free(a);
    return 0;
}

/* Exported for the tests: out = greedy RN words of sum_i x[i]*y[i]. */
int mwo_exact_dot(int64_t cnt, const double *x, const double *y, int nw, double *out)
{
    acc_t *a = (acc_t *)calloc(1, sizeof(acc_t));
    int64_t i;
    if (!a) return -100;
    for (i = 0; i < cnt; ++i) acc_add_prod(a, x[i], y[i], 0, 0);
    acc_round_words(a, nw, out, 1);
    free(a);
    return 0;
}

/* r = b - A x, computed exactly and rounded greedily to wr words.
 * A: wa planes (lda, n); b: wb planes of n; x: wx planes of n;
 * r: wr planes of n. */
int mwo_residual(int64_t n, const double *A, int64_t lda, int wa,
                 const double *b, int wb, const double *x, int wx,
                 double *r, int wr)
{
    int64_t plane = lda * n, i;
    int fail = 0;
    if (wa < 1 || wa > MWO_MAXW || wb < 1 || wb > MWO_MAXW || wx < 1 || wx > MWO_MAXW ||
        wr < 1 || wr > MWO_MAXW) return -1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (i = 0; i < n; ++i) {
        acc_t *a = (acc_t *)calloc(1, sizeof(acc_t));
        int64_t j;
        int c, d;
        if (!a) { fail = 1; continue; }
        for (c = 0; c < wb; ++c) acc_add_double(a, b[c * n + i], 0);
        for (j = 0; j < n; ++j)
            for (c = 0; c < wa; ++c) {
                double aij = A[c * plane + j * lda + i];
                if (aij == 0.0) continue;
                for (d = 0; d < wx; ++d)
                    acc_add_prod(a, aij, x[d * n + j], 1, 0);
            }
        acc_round_words(a, wr, r + i, n);
        free(a);
    }
    return fail ? -100 : 0;
}

/* RN of sum_i (v_i * 2^-e)^2 over the leading words v_i, exactly. */
static double exact_sumsq_scaled(int64_t cnt, const double *v, int64_t stride, int e)
{
    acc_t *a = (acc_t *)calloc(1, sizeof(acc_t));
    int64_t i;
    double res;
    if (!a) return NAN;
    for (i = 0; i < cnt; ++i) acc_add_prod(a, v[i * stride], v[i * stride], 0, -2 * e);
    res = acc_take_rn(a);
    free(a);
    return res;
}

/* 2-norm from leading words: ldexp(sqrt(RN(sum (v*2^-e)^2)), e),
 * e = ilogb(max |v|).  Returns 0 for a zero vector. */
static double norm2_lead(int64_t cnt, const double *v, int64_t stride)
{
    double mx = 0.0;
    int64_t i;
    int e;
    for (i = 0; i < cnt; ++i) {
        double t = fabs(v[i * stride]);
        if (t > mx) mx = t;
    }
    if (mx == 0.0) return 0.0;
    e = ilogb(mx);
    return ldexp(sqrt(exact_sumsq_scaled(cnt, v, stride, e)), e);
}

/* ------------------------------------------------------------------------ */
/* Mixed precision iterative refinement (Section 2, Listing 1).             */
/*   LU in w_in words of A; x0 = solve(b rounded to w_in) promoted to wx     */
/*   words; repeat: r = b - A x exactly, rounded to wx words; stopping test; */
/*   r_hat = first w_in words of 2^-e r, e = ilogb(max|r_0|) (power-of-two   */
/*   normalisation); z = solve(r_hat); x = RN_wx(x + 2^e z) exactly.         */
/* stop_mode 0: Eq. (2), ||r||_2 <= sqrt(n) rtol ||A||_F ||x||_2 + atol,     */
/*   norms taken from the leading words.                                    */
/* stop_mode 1: converged when the applied correction satisfies             */
/*   max|2^e z_0| <= 2^(-target_bits-2) max|x_0|; stops as not converged    */
/*   when a correction exceeds half the previous one (from the second on).  */
/* Returns 0 converged, 1 singular LU (info in stats[2]), 2 not converged.  */
/* stats: [0] corrections applied, [1] residuals evaluated, [2] LU info.    */
/* ------------------------------------------------------------------------ */

int mwo_refine(int64_t n, const double *A, int64_t lda, int wa,
               const double *b, int wb, int w_in, int max_iter, int stop_mode,
               double rtol, double atol, int target_bits,
               double *x, int wx, int64_t *stats)
{
    int64_t plane = lda * n, i, j, info = 0;
    int c, status = 2, corrections = 0, residuals = 0;
    double *LU = NULL, *bin = NULL, *xin = NULL, *r = NULL, *rh = NULL, *z = NULL;
    int64_t *piv = NULL;
    double nA = 0.0, prev = INFINITY;
    if (w_in < 2 || w_in > 4 || wx < w_in || wx > MWO_MAXW || wa < 1 || wa > MWO_MAXW ||
        wb < 1 || wb > MWO_MAXW) return -1;
    LU = (double *)calloc((size_t)(w_in * plane), sizeof(double));
    piv = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    bin = (double *)calloc((size_t)(w_in * n + 1), sizeof(double));
    xin = (double *)calloc((size_t)(w_in * n + 1), sizeof(double));
    r = (double *)calloc((size_t)(wx * n + 1), sizeof(double));
    rh = (double *)calloc((size_t)(w_in * n + 1), sizeof(double));
    z = (double *)calloc((size_t)(w_in * n + 1), sizeof(double));
    if (!LU || !piv || !bin || !xin || !r || !rh || !z) { status = -100; goto done; }
    for (c = 0; c < w_in && c < wa; ++c)
        memcpy(LU + c * plane, A + c * plane, sizeof(double) * (size_t)plane);
    mwo_lu(w_in, n, LU, lda, piv, &info);
    stats[2] = info;
    if (info != 0) { status = 1; goto done; }
    for (c = 0; c < w_in && c < wb; ++c)
        memcpy(bin + c * n, b + c * n, sizeof(double) * (size_t)n);
    mwo_solve(w_in, n, LU, lda, piv, bin, xin);
    memset(x, 0, sizeof(double) * (size_t)(wx * n));
    memcpy(x, xin, sizeof(double) * (size_t)(w_in * n));
    if (stop_mode == 0) {
        /* ||A||_F from the leading words, over the n x n entries */
        double mx = 0.0;
        acc_t *a;
        for (j = 0; j < n; ++j)
            for (i = 0; i < n; ++i) {
                double t = fabs(A[j * lda + i]);
                if (t > mx) mx = t;
            }
        if (mx > 0.0) {
            int e = ilogb(mx);
            a = (acc_t *)calloc(1, sizeof(acc_t));
            if (!a) { status = -100; goto done; }
            for (j = 0; j < n; ++j)
                for (i = 0; i < n; ++i)
                    acc_add_prod(a, A[j * lda + i], A[j * lda + i], 0, -2 * e);
            nA = ldexp(sqrt(acc_take_rn(a)), e);
            free(a);
        }
    }
    for (;;) {
        double rmax = 0.0;
        int er;
        mwo_residual(n, A, lda, wa, b, wb, x, wx, r, wx);
        residuals++;
        for (i = 0; i < n; ++i) {
            double t = fabs(r[i]);
            if (t > rmax) rmax = t;
        }
        if (rmax == 0.0) { status = 0; break; }
        er = ilogb(rmax);
        if (stop_mode == 0) {
            double nr = norm2_lead(n, r, 1);
            double nx = norm2_lead(n, x, 1);
            double rhs = sqrt((double)n) * rtol;
            rhs = rhs * nA;
            rhs = rhs * nx;
            rhs = rhs + atol;
            if (nr <= rhs) { status = 0; break; }
        }
        if (corrections >= max_iter) { status = 2; break; }
        for (c = 0; c < w_in; ++c)
            for (i = 0; i < n; ++i)
                rh[c * n + i] = ldexp(r[c * n + i], -er);
        mwo_solve(w_in, n, LU, lda, piv, rh, z);
        /* x = RN_wx(x + 2^er z), exactly */
        for (i = 0; i < n; ++i) {
            acc_t a;
            memset(&a, 0, sizeof(a));
            for (c = 0; c < wx; ++c) acc_add_double(&a, x[c * n + i], 0);
            for (c = 0; c < w_in; ++c) acc_add_double(&a, z[c * n + i], er);
            acc_round_words(&a, wx, x + i, n);
        }
        corrections++;
        if (stop_mode == 1) {
            double zmax = 0.0, xmax = 0.0, corr;
            for (i = 0; i < n; ++i) {
                double t = fabs(z[i]);
                if (t > zmax) zmax = t;
                t = fabs(x[i]);
                if (t > xmax) xmax = t;
            }
            corr = ldexp(zmax, er);
            if (corr <= ldexp(xmax, -target_bits - 2)) { status = 0; break; }
            if (corrections >= 2 && corr > 0.5 * prev) { status = 2; break; }
            prev = corr;
        }
    }
done:
    stats[0] = corrections;
    stats[1] = residuals;
    free(LU); free(piv); free(bin); free(xin); free(r); free(rh); free(z);
    return status;
}

int mwo_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}
