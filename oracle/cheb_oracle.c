/*
 * Plain FP64 CPU oracle of the tensorial Chebyshev method for the
 * transboundary pollution game (de Castro, Gaton, Gomez, arXiv 2307.04688).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * reference that the CUDA path is checked against. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never calls it, includes it or shares a header, helper or table with it.
 *
 * Conventions. Arrays are row-major with the last mode fastest. Node k of a
 * mode sits at alpha^k = cos(pi k / N), N = n - 1, so k = 0 is x = +1 and the
 * nodes descend (Section 3.1). Everything is IEEE double; the library is
 * compiled without contraction of a*b+c into fused multiply-adds.
 *
 * Every function states the passage of the paper it follows. Where the paper
 * is garbled the reading taken is stated beside the code.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

void orc_set_threads(int t)
{
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : 1);
#else
    (void)t;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Section 3.1: Chebyshev polynomials, nodes, one-dimensional interpolant */
/* ------------------------------------------------------------------ */

/* Chebyshev-Lobatto nodes alpha^k = cos(pi k / N), k = 0..N (Section 3.1). */
void orc_nodes(int n, double *alpha)
{
    int N = n - 1;
    for (int k = 0; k < n; ++k) alpha[k] = cos(M_PI * (double)k / (double)N);
}

/* Affine map [a,b] -> [-1,1], the inverse of the change of variable of
 * Section 3.1 (x~ = (b-a)/2 x + (b+a)/2). */
double orc_to_ref(double a, double b, double xt)
{
    return (2.0 * xt - (a + b)) / (b - a);
}

/* T_0(x)..T_{n-1}(x) by the three-term recurrence T_{k+1} = 2x T_k - T_{k-1}.
 * On [-1,1] this equals T_k(x) = cos(k arccos x) (Section 3.1); off [-1,1]
 * it is the same polynomial continued, which the game needs because next
 * states can leave the state box. */
void orc_cheb_T(int n, double x, double *T)
{
    if (n <= 0) return;
    T[0] = 1.0;
    if (n == 1) return;
    T[1] = x;
    for (int k = 2; k < n; ++k) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
}

/* T_l(alpha^k) = cos(l * arccos(cos(pi k/N))) = cos(pi l k / N). The integer
 * product l*k is reduced modulo 2N before the cosine, which is exact. */
static double T_at_node(int l, int k, int N)
{
    long t = ((long)l * (long)k) % (2L * N);
    return cos(M_PI * (double)t / (double)N);
}

/* One-dimensional interpolation coefficients by eq. (forcoef)
 * (Definition 3.1): p_l = (c_l / N) sum''_k F_k T_l(alpha^k), with c_l = 1
 * for l in {0, N} and 2 otherwise, and the double prime halving the k = 0
 * and k = N terms. F and p are read/written with the given strides. */
static void fit_1d_strided(int n, const double *F, ptrdiff_t fs, double *p, ptrdiff_t ps,
                           const double *Tn /* n*n table T_l(alpha^k), [l*n+k] */)
{
    int N = n - 1;
    for (int l = 0; l <= N; ++l) {
        double s = 0.0;
        for (int k = 0; k <= N; ++k) {
            double w = (k == 0 || k == N) ? 0.5 : 1.0;
            s += w * F[(ptrdiff_t)k * fs] * Tn[l * n + k];
        }
        double cl = (l == 0 || l == N) ? 1.0 : 2.0;
        p[(ptrdiff_t)l * ps] = cl / (double)N * s;
    }
}

static double *node_table(int n)
{
    int N = n - 1;
    double *Tn = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int l = 0; l < n; ++l)
        for (int k = 0; k < n; ++k) Tn[l * n + k] = T_at_node(l, k, N);
    return Tn;
}

void orc_fit_1d(int n, const double *F, double *p)
{
    double *Tn = node_table(n);
    fit_1d_strided(n, F, 1, p, 1, Tn);
    free(Tn);
}

/* Algorithm C1v (Section 3.1) with a plain O(n^2) discrete Fourier transform
 * standing in for the FFT:
 *   1. z = [F_0, F_1, ..., F_N, F_{N-1}, ..., F_1]  (length 2N),
 *   2. y = real(DFT(z)) / (2N), DFT(z)_q = sum_t z_t exp(-2 pi i q t / 2N),
 *   3. p_0 = y_0, p_l = y_l + y_{2N-l} (0 < l < N), p_N = y_N.
 * The paper prints p_N = y(N) (1-based), which would be y_{N-1}; the value
 * consistent with eq. (forcoef) is y(N+1), i.e. y_N, and that is used. */
void orc_c1v(int n, const double *F, double *p)
{
    int N = n - 1, L = 2 * N;
    double *z = (double *)malloc(sizeof(double) * (size_t)L);
    double *y = (double *)malloc(sizeof(double) * (size_t)L);
    for (int k = 0; k <= N; ++k) z[k] = F[k];
    for (int k = N + 1; k < L; ++k) z[k] = F[L - k];
    for (int q = 0; q < L; ++q) {
        double s = 0.0;
        for (int t = 0; t < L; ++t) {
            long qt = ((long)q * (long)t) % L;
            s += z[t] * cos(2.0 * M_PI * (double)qt / (double)L);
        }
        y[q] = s / (double)L;
    }
    p[0] = y[0];
    for (int l = 1; l < N; ++l) p[l] = y[l] + y[L - l];
    p[N] = y[N];
    free(z);
    free(y);
}

/* Derivative of a Chebyshev series (Proposition 3.1, Section 3.1):
 * (sum_{l=0}^N p_l T_l)' = sum_{l=0}^{N-1} q_l T_l with
 * q_l = (2 / c_l) sum_{j = l+1, j + l odd}^{N} j p_j, c_0 = 2, c_l = 1 (l>0).
 * The printed formula reads "2/c_l +"; the product (2/c_l) * sum is the
 * standard identity and is used. The factor 2/(b-a) of the change of
 * variable is left to the caller. q has n entries and q[N] = 0. */
void orc_deriv_coeffs(int n, const double *p, double *q)
{
    int N = n - 1;
    for (int l = 0; l < N; ++l) {
        double s = 0.0;
        for (int j = l + 1; j <= N; ++j)
            if ((j + l) % 2 == 1) s += (double)j * p[j];
        q[l] = (l == 0 ? 1.0 : 2.0) * s;
    }
    if (N >= 0) q[N] = 0.0;
}

/* Sum_{l} p_l T_l(x), by forming T_l with the recurrence. */
double orc_series(int n, const double *p, double x)
{
    double *T = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    orc_cheb_T(n, x, T);
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += p[l] * T[l];
    free(T);
    return s;
}

/* ------------------------------------------------------------------ */
/* Section 3.1-3.2: n-dimensional interpolant, fit and evaluation        */
/* ------------------------------------------------------------------ */

static size_t prod_i(int d, const int *v)
{
    size_t p = 1;
    for (int s = 0; s < d; ++s) p *= (size_t)v[s];
    return p;
}

/* out = in x_s B: the mode-s product of a row-major tensor of the given
 * shape with an (m x shape[s]) matrix B, out[.., j, ..] = sum_k B[j,k] in[.., k, ..]. */
static void mode_apply(int d, const int *shape, int s, int m, const double *B,
                       const double *in, double *out)
{
    size_t pre = 1, post = 1;
    for (int t = 0; t < s; ++t) pre *= (size_t)shape[t];
    for (int t = s + 1; t < d; ++t) post *= (size_t)shape[t];
    int n = shape[s];
    long long total = (long long)pre * (long long)m;
#pragma omp parallel for schedule(static)
    for (long long pj = 0; pj < total; ++pj) {
        size_t a = (size_t)(pj / m);
        int j = (int)(pj % m);
        double *o = out + (a * (size_t)m + (size_t)j) * post;
        const double *ib = in + a * (size_t)n * post;
        for (size_t c = 0; c < post; ++c) o[c] = 0.0;
        for (int k = 0; k < n; ++k) {
            double bjk = B[(size_t)j * n + k];
            const double *ik = ib + (size_t)k * post;
            for (size_t c = 0; c < post; ++c) o[c] += bjk * ik[c];
        }
    }
}

/* n-dimensional coefficients (Definition 3.2): eq. (forcoef) applied along
 * every mode, p_l = prod_s (c_{l_s}/N_s) sum''_k F(alpha^k) prod_s T_{l_s}(alpha^{k_s}).
 * The sum over the multi-index k factorises mode by mode. */
void orc_fit_nd(int d, const int *n, const double *Gamma, double *coef)
{
    size_t total = prod_i(d, n);
    double *cur = (double *)malloc(sizeof(double) * total);
    double *nxt = (double *)malloc(sizeof(double) * total);
    memcpy(cur, Gamma, sizeof(double) * total);
    for (int s = 0; s < d; ++s) {
        int ns = n[s], N = ns - 1;
        /* matrix form of eq. (forcoef) for this mode: Mf[l,k] */
        double *Mf = (double *)malloc(sizeof(double) * (size_t)ns * (size_t)ns);
        for (int l = 0; l < ns; ++l)
            for (int k = 0; k < ns; ++k) {
                double w = (k == 0 || k == N) ? 0.5 : 1.0;
                double cl = (l == 0 || l == N) ? 1.0 : 2.0;
                Mf[l * ns + k] = cl / (double)N * w * T_at_node(l, k, N);
            }
        mode_apply(d, n, s, ns, Mf, cur, nxt);
        free(Mf);
        double *t = cur; cur = nxt; nxt = t;
    }
    memcpy(coef, cur, sizeof(double) * total);
    free(cur);
    free(nxt);
}

/* Algorithm Cnv as printed (Section 3.1): apply C1v to every fibre of the
 * leading mode, then rotate the modes, d times. The paper's arrays are
 * column-major (first mode contiguous) and rotate with permute([2:n 1]); in
 * this row-major layout the contiguous mode is the last one, so each pass
 * applies C1v along the last mode and rotates it to the front. After d
 * passes the modes are back in their original order. */
void orc_cnv(int d, const int *n, const double *Gamma, double *coef)
{
    size_t total = prod_i(d, n);
    double *A = (double *)malloc(sizeof(double) * total);
    double *B = (double *)malloc(sizeof(double) * total);
    int shape[16];
    for (int s = 0; s < d; ++s) shape[s] = n[s];
    memcpy(A, Gamma, sizeof(double) * total);
    for (int pass = 0; pass < d; ++pass) {
        int nl = shape[d - 1];
        size_t rows = total / (size_t)nl;
        double *fib = (double *)malloc(sizeof(double) * (size_t)nl);
        double *res = (double *)malloc(sizeof(double) * (size_t)nl);
        /* B(rows, nl) = C1v along the last mode; then rotate: B -> A(nl, rows) */
        for (size_t r = 0; r < rows; ++r) {
            for (int k = 0; k < nl; ++k) fib[k] = A[r * (size_t)nl + (size_t)k];
            orc_c1v(nl, fib, res);
            for (int l = 0; l < nl; ++l) B[(size_t)l * rows + r] = res[l];
        }
        free(fib);
        free(res);
        for (int s = d - 1; s > 0; --s) shape[s] = shape[s - 1];
        shape[0] = nl;
        double *t = A; A = B; B = t;
    }
    memcpy(coef, A, sizeof(double) * total);
    free(A);
    free(B);
}

/* Tensor-grid evaluation D(j_1..j_d) = I_N F(b^1_{j_1}, ..., b^d_{j_d})
 * (Section 3.2): successive mode products with B_s(j, l) = T_l(x_{s,j}).
 * Points are given on [a_s, b_s] and mapped to [-1,1]. */
void orc_eval_grid(int d, const int *n, const double *coef, const double *a, const double *b,
                   const int *m, const double *const *x, double *out)
{
    int shape[16];
    for (int s = 0; s < d; ++s) shape[s] = n[s];
    size_t cap = 1;
    {
        /* the largest intermediate: modes 0..s evaluated, s+1..d-1 still coefficients */
        for (int s = 0; s <= d; ++s) {
            size_t sz = 1;
            for (int t = 0; t < d; ++t) sz *= (size_t)(t < s ? m[t] : n[t]);
            if (sz > cap) cap = sz;
        }
    }
    double *cur = (double *)malloc(sizeof(double) * cap);
    double *nxt = (double *)malloc(sizeof(double) * cap);
    memcpy(cur, coef, sizeof(double) * prod_i(d, n));
    for (int s = 0; s < d; ++s) {
        double *Bm = (double *)malloc(sizeof(double) * (size_t)m[s] * (size_t)n[s]);
        for (int j = 0; j < m[s]; ++j)
            orc_cheb_T(n[s], orc_to_ref(a[s], b[s], x[s][j]), Bm + (size_t)j * n[s]);
        mode_apply(d, shape, s, m[s], Bm, cur, nxt);
        free(Bm);
        shape[s] = m[s];
        double *t = cur; cur = nxt; nxt = t;
    }
    memcpy(out, cur, sizeof(double) * prod_i(d, m));
    free(cur);
    free(nxt);
}

/* Direct summation of the n-dimensional interpolant at one point of
 * [-1,1]^d (Definition 3.2): sum_l p_l prod_s T_{l_s}(x_s). */
double orc_eval_direct(int d, const int *n, const double *coef, const double *xref)
{
    int nmax = 1;
    for (int s = 0; s < d; ++s) if (n[s] > nmax) nmax = n[s];
    double *T = (double *)malloc(sizeof(double) * (size_t)d * (size_t)nmax);
    for (int s = 0; s < d; ++s) orc_cheb_T(n[s], xref[s], T + (size_t)s * nmax);
    size_t total = prod_i(d, n);
    double sum = 0.0;
    int idx[16] = {0};
    for (size_t f = 0; f < total; ++f) {
        double t = coef[f];
        for (int s = 0; s < d; ++s) t *= T[(size_t)s * nmax + idx[s]];
        sum += t;
        for (int s = d - 1; s >= 0; --s) {
            if (++idx[s] < n[s]) break;
            idx[s] = 0;
        }
    }
    free(T);
    return sum;
}

/* Point evaluation f(x_j) = sum_l p_l prod_s T_{l_s}(x_{j,s}) at P points
 * given row-major (P x d) on the box prod [a_s, b_s] (Section 3.3 asks for
 * the values of the interpolant at a different point per evaluation). */
void orc_eval_points(int d, const int *n, const double *coef, const double *a, const double *b,
                     long P, const double *x, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (long j = 0; j < P; ++j) {
        double xr[16];
        for (int s = 0; s < d; ++s) xr[s] = orc_to_ref(a[s], b[s], x[(size_t)j * d + s]);
        out[j] = orc_eval_direct(d, n, coef, xr);
    }
}

/* Nested contraction at one point: contract the last mode first, mode by
 * mode. Identical to orc_eval_direct up to rounding order; O(n^d) instead
 * of O(d n^d). The game oracle uses it for speed. */
double orc_eval_nested(int d, const int *n, const double *coef, const double *xref, double *work)
{
    /* work must hold prod(n) / n[d-1] + prod(n) / (n[d-1] n[d-2]) + ... doubles */
    size_t len = prod_i(d, n);
    const double *src = coef;
    double *dst = work;
    double T[128];
    for (int s = d - 1; s >= 0; --s) {
        int ns = n[s];
        orc_cheb_T(ns, xref[s], T);
        size_t rows = len / (size_t)ns;
        for (size_t r = 0; r < rows; ++r) {
            double acc = 0.0;
            const double *row = src + r * (size_t)ns;
            for (int k = 0; k < ns; ++k) acc += row[k] * T[k];
            dst[r] = acc;
        }
        src = dst;
        dst = dst + rows;
        len = rows;
    }
    return src[0];
}
