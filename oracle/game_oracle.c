/*
 * Plain FP64 CPU oracle of the Chebyshev collocation method for the
 * J-player pollution game (arXiv 2307.04688, Section 2.1 Steps 0-4 and
 * Section 3.4), plus the closed-form linear-quadratic recursion that pins it.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the library.
 *
 * Model (Section 2, linear-quadratic specification, all m_i equal to m):
 *   g_i(p, u) = (1/m) sum_{j != i} k_ij (p_j - p_i) - c_i p_i + beta_i u_i
 *               + u_i sum_{l != i} gamma_il u_l,
 * where the last term (an emission-interaction coupling, zero in the paper's
 * examples) makes g non-separable in the controls: Section 2.1 Step 0 then
 * interpolates g at every state node as a function of all controls on
 * [0, U_M]^J (the "g-interpolants"), and Steps 1-2 evaluate those
 * interpolants at the controls (Section 3.3); with gamma = 0 the same code
 * evaluates g directly, which the interpolant reproduces exactly.
 *   G_i(p, u_i) = u_i (A_i - u_i / 2) - (phi_i / 2) p_i^2,
 *   delta_h = 1 - rho h, next state p + h g(p, u)           (eq. ecgtimedisc),
 *   V_i(p) = max_{u_i >= 0} { h G_i + delta_h V_i(p + h g(p, [u_i, u*_{-i}])) }.
 * Readings of garbled or unstated passages:
 *   - the printed coupling term is k_ij (p_i - p_j) with k_ij >= 0, which is
 *     anti-diffusive; the neighbour matrices the paper prints have rows
 *     summing to zero, so the term is read as k_ij (p_j - p_i), i.e.
 *     (1/m) (K p)_i with the printed K;
 *   - Step 2 as printed leaves out h G_i; the Bellman form above is used;
 *   - the tolerance test is the maximum over players and state nodes of
 *     |V^[r+1] - V^[r]| at the nodes;
 *   - players update simultaneously from the previous iterate (Step 1 fixes
 *     the other players' controls at u^[r]).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* from cheb_oracle.c */
void orc_nodes(int n, double *alpha);
void orc_cheb_T(int n, double x, double *T);
void orc_c1v(int n, const double *F, double *p);
void orc_deriv_coeffs(int n, const double *p, double *q);
double orc_series(int n, const double *p, double x);
void orc_fit_nd(int d, const int *n, const double *Gamma, double *coef);
double orc_eval_nested(int d, const int *n, const double *coef, const double *xref, double *work);
double orc_eval_direct(int d, const int *n, const double *coef, const double *xref);

typedef struct {
    int J;
    double K[16];      /* J x J row-major neighbour matrix, rows summing to zero */
    double m;          /* common region measure m_i */
    double A[4], beta[4], phi[4], c[4];
    double rho;
    double gamma[16];  /* J x J emission-interaction coupling (diagonal unused) */
} orc_game_params;

typedef struct {
    double h, P_M, U_M, tol;
    int n;             /* state nodes per player (N^p + 1) */
    int n_u;           /* control nodes (N^u + 1) */
    long max_iter;
    int g_interp;      /* 1: Steps 1-2 evaluate g through the Step 0 interpolants */
} orc_game_opts;

static long ipow(int b, int e)
{
    long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* g(p, u) of Section 2.1 under the reading stated in the header. */
void orc_game_dynamics(const orc_game_params *P, const double *p, const double *u, double *g)
{
    int J = P->J;
    for (int i = 0; i < J; ++i) {
        double coup = 0.0;
        for (int j = 0; j < J; ++j)
            if (j != i) coup += P->K[i * J + j] * (p[j] - p[i]);
        double inter = 0.0;
        for (int l = 0; l < J; ++l)
            if (l != i) inter += P->gamma[i * J + l] * u[l];
        g[i] = coup / P->m - P->c[i] * p[i] + P->beta[i] * u[i] + u[i] * inter;
    }
}

/* Step 0 (Section 2.1): the interpolants of g_l(pbar, .) at one state node in
 * all J controls, on the tensor grid of n_u Chebyshev-Lobatto control nodes
 * per player, u~_k = (U_M/2)(cos(pi k/N_u) + 1) on [0, U_M]. gc receives J
 * coefficient tensors of n_u^J entries (component l first), fitted by
 * eq. (forcoef) mode by mode. */
void orc_game_g_interp(const orc_game_params *P, const orc_game_opts *O, const double *pbar, double *gc)
{
    int J = P->J, nu = O->n_u, Nu = nu - 1;
    long NU = ipow(nu, J);
    int nd[4];
    for (int s = 0; s < J; ++s) nd[s] = nu;
    double *vals = (double *)malloc(sizeof(double) * (size_t)NU * (size_t)J);
    for (long t = 0; t < NU; ++t) {
        double uu[4], g[4];
        long rem = t;
        for (int s = J - 1; s >= 0; --s) {
            int k = (int)(rem % nu);
            rem /= nu;
            uu[s] = 0.5 * O->U_M * (cos(M_PI * (double)k / (double)Nu) + 1.0);
        }
        orc_game_dynamics(P, pbar, uu, g);
        for (int l = 0; l < J; ++l) vals[(size_t)l * NU + t] = g[l];
    }
    for (int l = 0; l < J; ++l) orc_fit_nd(J, nd, vals + (size_t)l * NU, gc + (size_t)l * NU);
    free(vals);
}

/* g(pbar, u) through the Step 0 interpolants gc (Section 3.3: the node's own
 * interpolant evaluated at its controls). */
void orc_game_g_eval(const orc_game_params *P, const orc_game_opts *O, const double *gc, const double *u,
                     double *g)
{
    int J = P->J, nu = O->n_u;
    long NU = ipow(nu, J);
    int nd[4];
    double xr[4];
    for (int s = 0; s < J; ++s) {
        nd[s] = nu;
        xr[s] = 2.0 * u[s] / O->U_M - 1.0;
    }
    double *work = (double *)malloc(sizeof(double) * (size_t)NU);
    for (int l = 0; l < J; ++l) g[l] = orc_eval_nested(J, nd, gc + (size_t)l * NU, xr, work);
    free(work);
}

/* State node j (row-major multi-index, last player fastest) on [0, P_M]^J:
 * p~_k = (P_M/2)(cos(pi k/N) + 1) (Section 3.4, Step 0). */
void orc_game_node(const orc_game_opts *O, int J, long j, double *pbar, double *xref)
{
    int N = O->n - 1;
    long rem = j;
    for (int s = J - 1; s >= 0; --s) {
        int k = (int)(rem % O->n);
        rem /= O->n;
        double a = cos(M_PI * (double)k / (double)N);
        if (xref) xref[s] = a;
        pbar[s] = 0.5 * O->P_M * (a + 1.0);
    }
}

/* Maximiser of sum_m a_m T_m(y) over y in [-1, 1]: sample 8 n_u + 1
 * Chebyshev-spaced points (endpoints included), then polish the best sample
 * with Newton on the derivative series (Proposition 3.1 applied twice),
 * safeguarded by bisection on a sign-changing bracket. Candidates are the
 * two endpoints, the best sample and the polished point; the largest value
 * wins, ties going to the smaller y (smaller control). Returns y*, writes
 * the value; *concave is set to 0 if the second derivative at an interior
 * optimum is not negative. */
static double argmax_series(int nu, const double *a, double *val, int *concave)
{
    double q1[128], q2[128];
    orc_deriv_coeffs(nu, a, q1);
    orc_deriv_coeffs(nu, q1, q2);
    int S = 8 * nu;
    int best = 0;
    double bestv = -INFINITY;
    for (int t = S; t >= 0; --t) {           /* ascending y: t = S is y = -1 */
        double y = cos(M_PI * (double)t / (double)S);
        double v = orc_series(nu, a, y);
        if (v > bestv) { bestv = v; best = t; }
    }
    double ybest = cos(M_PI * (double)best / (double)S);
    double ylo = cos(M_PI * (double)(best < S ? best + 1 : S) / (double)S);
    double yhi = cos(M_PI * (double)(best > 0 ? best - 1 : 0) / (double)S);
    double cand[4];
    int nc = 0;
    cand[nc++] = -1.0;
    cand[nc++] = 1.0;
    cand[nc++] = ybest;
    double dlo = orc_series(nu, q1, ylo), dhi = orc_series(nu, q1, yhi);
    if (dlo > 0.0 && dhi < 0.0) {
        double y = ybest, lo = ylo, hi = yhi;
        for (int it = 0; it < 60; ++it) {
            double d1 = orc_series(nu, q1, y), d2 = orc_series(nu, q2, y);
            if (d1 > 0.0) lo = y; else hi = y;
            double yn = (d2 < 0.0) ? y - d1 / d2 : 0.5 * (lo + hi);
            if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
            double step = fabs(yn - y);
            y = yn;
            if (step < 1e-15 || hi - lo < 1e-15) break;
        }
        cand[nc++] = y;
    }
    double ys = cand[0], vs = orc_series(nu, a, cand[0]);
    for (int c = 1; c < nc; ++c) {
        double v = orc_series(nu, a, cand[c]);
        if (v > vs || (v == vs && cand[c] < ys)) { vs = v; ys = cand[c]; }
    }
    if (concave) *concave = (ys <= -1.0 || ys >= 1.0) ? 1 : (orc_series(nu, q2, ys) < 0.0);
    *val = vs;
    return ys;
}

/* Steps 1-3 (Sections 2.1 and 3.4) for player i at one state node:
 * for every control node u~_k on [0, U_M] evaluate
 *   W_k = h G_i(pbar, u~_k) + delta_h V_i(pbar + h g(pbar, [u~_k, u_{-i}])),
 * interpolate W in u with C1v, and maximise the interpolant on [0, U_M].
 * u_old holds u^[r](pbar) for all players. Returns 1 if the optimum was
 * strictly inside (0, U_M) and 0 if a bound was active. */
int orc_game_node_update(const orc_game_params *P, const orc_game_opts *O, int i,
                         const double *pbar, const double *u_old, const double *Vcoef_i,
                         double *u_star, double *V_star, int *concave)
{
    int J = P->J, nu = O->n_u, Nu = nu - 1;
    double delta = 1.0 - P->rho * O->h;
    int nd[4];
    for (int s = 0; s < J; ++s) nd[s] = O->n;
    long NP = ipow(O->n, J);
    double *work = (double *)malloc(sizeof(double) * (size_t)NP);
    double *gc = NULL;
    if (O->g_interp) {
        gc = (double *)malloc(sizeof(double) * (size_t)J * (size_t)ipow(nu, J));
        orc_game_g_interp(P, O, pbar, gc);
    }
    double W[128], a[128];
    for (int k = 0; k <= Nu; ++k) {
        double uk = 0.5 * O->U_M * (cos(M_PI * (double)k / (double)Nu) + 1.0);
        double uu[4], g[4], xr[4];
        for (int s = 0; s < J; ++s) uu[s] = u_old[s];
        uu[i] = uk;
        if (gc)
            orc_game_g_eval(P, O, gc, uu, g);
        else
            orc_game_dynamics(P, pbar, uu, g);
        for (int s = 0; s < J; ++s) xr[s] = 2.0 * (pbar[s] + O->h * g[s]) / O->P_M - 1.0;
        double Vq = orc_eval_nested(J, nd, Vcoef_i, xr, work);
        double G = uk * (P->A[i] - 0.5 * uk) - 0.5 * P->phi[i] * pbar[i] * pbar[i];
        W[k] = O->h * G + delta * Vq;
    }
    free(work);
    free(gc);
    orc_c1v(nu, W, a);
    double val;
    double y = argmax_series(nu, a, &val, concave);
    *u_star = 0.5 * O->U_M * (y + 1.0);
    *V_star = val;
    return (y > -1.0 && y < 1.0);
}

/* One pass r -> r+1 of Steps 1-4 for all players (Jacobi). Inputs are the
 * coefficient tensors Vcoef (J x N_P), the nodal values Vnod (J x N_P) and the
 * nodal controls u (J x N_P, u[s*N_P + j] = u_s(pbar_j)). Writes the new
 * nodal values, controls and refitted coefficients and returns the residual
 * max_{i,j} |V^[r+1]_i(pbar_j) - V^[r]_i(pbar_j)|. *interior counts the
 * node updates whose optimum was strictly inside (0, U_M); *nonconcave the
 * interior optima whose second derivative was not negative. */
double orc_game_iterate(const orc_game_params *P, const orc_game_opts *O, const double *Vcoef,
                        const double *Vnod, const double *u, double *Vcoef_new, double *Vnod_new,
                        double *u_new, long *interior, long *nonconcave)
{
    int J = P->J;
    long NP = ipow(O->n, J);
    long n_in = 0, n_nc = 0;
    double res = 0.0;
    for (int i = 0; i < J; ++i) {
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : n_in, n_nc) reduction(max : res)
        for (long j = 0; j < NP; ++j) {
            double pbar[4], uo[4];
            orc_game_node(O, J, j, pbar, NULL);
            for (int s = 0; s < J; ++s) uo[s] = u[(size_t)s * NP + j];
            double us, vs;
            int cc = 1;
            n_in += orc_game_node_update(P, O, i, pbar, uo, Vcoef + (size_t)i * NP, &us, &vs, &cc);
            n_nc += (cc == 0);
            u_new[(size_t)i * NP + j] = us;
            Vnod_new[(size_t)i * NP + j] = vs;
            double dv = fabs(vs - Vnod[(size_t)i * NP + j]);
            if (dv > res) res = dv;
        }
    }
    int nd[4];
    for (int s = 0; s < J; ++s) nd[s] = O->n;
    for (int i = 0; i < J; ++i)
        orc_fit_nd(J, nd, Vnod_new + (size_t)i * NP, Vcoef_new + (size_t)i * NP);
    if (interior) *interior = n_in;
    if (nonconcave) *nonconcave = n_nc;
    return res;
}

/* The whole method: Step 0 (initial nodal values V0 and controls u0, zero
 * when NULL; fit), then Steps 1-4 until the residual is below tol or
 * max_iter passes were made. Returns 0 on convergence and 1 otherwise;
 * *iters counts the passes made, res_hist (if given, max_iter entries)
 * receives every residual. */
int orc_game_solve(const orc_game_params *P, const orc_game_opts *O, const double *V0,
                   const double *u0, double *Vcoef, double *Vnod, double *u, long *iters,
                   double *residual, double *res_hist)
{
    int J = P->J;
    long NP = ipow(O->n, J);
    size_t sz = (size_t)J * (size_t)NP;
    double *Vc2 = (double *)malloc(sizeof(double) * sz);
    double *Vn2 = (double *)malloc(sizeof(double) * sz);
    double *u2 = (double *)malloc(sizeof(double) * sz);
    int nd[4];
    for (int s = 0; s < J; ++s) nd[s] = O->n;
    for (size_t t = 0; t < sz; ++t) {
        Vnod[t] = V0 ? V0[t] : 0.0;
        u[t] = u0 ? u0[t] : 0.0;
    }
    for (int i = 0; i < J; ++i) orc_fit_nd(J, nd, Vnod + (size_t)i * NP, Vcoef + (size_t)i * NP);
    long r = 0;
    double res = INFINITY;
    int status = 1;
    while (r < O->max_iter) {
        res = orc_game_iterate(P, O, Vcoef, Vnod, u, Vc2, Vn2, u2, NULL, NULL);
        memcpy(Vcoef, Vc2, sizeof(double) * sz);
        memcpy(Vnod, Vn2, sizeof(double) * sz);
        memcpy(u, u2, sizeof(double) * sz);
        if (res_hist) res_hist[r] = res;
        ++r;
        if (res < O->tol) { status = 0; break; }
    }
    free(Vc2);
    free(Vn2);
    free(u2);
    *iters = r;
    *residual = res;
    return status;
}

/* ------------------------------------------------------------------ */
/* Closed-form pin: the linear-quadratic recursion                      */
/* ------------------------------------------------------------------ */
/* While the bound u >= 0 (and u <= U_M) is inactive at every node, the
 * iteration above keeps V_i quadratic, V_i(p) = 1/2 p'Q_i p + b_i'p + a_i,
 * and the controls affine, u_i(p) = F_i p + f_i, because a quadratic is
 * reproduced exactly by the interpolant (n >= 3), the next state is affine
 * in p and u, and the objective is quadratic in u. Substituting into the
 * Bellman step of Section 2.1 gives, for each player i with
 *   S_i = I + h (K/m - diag c) + h sum_{l != i} beta_l e_l F_l,
 *   s_i = h sum_{l != i} beta_l f_l e_l,
 *   D = 1 - delta h beta_i^2 Q_i[i,i],
 *   F = delta beta_i e_i' Q_i S_i / D,  f = (A_i + delta beta_i e_i'(Q_i s_i + b_i)) / D,
 *   S' = S_i + h beta_i e_i F,  s' = s_i + h beta_i f e_i,
 * the update
 *   Q_i <- h(-F'F - phi_i e_i e_i') + delta S'' Q_i S',
 *   b_i <- h (A_i - f) F' + delta S''(Q_i s' + b_i),
 *   a_i <- h (A_i f - f^2/2) + delta (1/2 s''Q_i s' + b_i's' + a_i),
 *   (F_i, f_i) <- (F, f),
 * all players at once from the previous iterate. Starting from V = 0, u = 0,
 * R passes are written out: Q (R x J x J x J), b (R x J x J), a (R x J),
 * F (R x J x J), f (R x J). */
void orc_game_lq(const orc_game_params *P, double h, int R, double *Qo, double *bo, double *ao,
                 double *Fo, double *fo)
{
    int J = P->J;
    double delta = 1.0 - P->rho * h;
    double Q[4][16], b[4][4], a[4], F[4][4], f[4];
    double Qn[4][16], bn[4][4], an[4], Fn[4][4], fn[4];
    memset(Q, 0, sizeof Q); memset(b, 0, sizeof b); memset(a, 0, sizeof a);
    memset(F, 0, sizeof F); memset(f, 0, sizeof f);
    for (int r = 0; r < R; ++r) {
        for (int i = 0; i < J; ++i) {
            double S[16], s[4], Sp[16], sp[4], Fi[4], fi;
            for (int x = 0; x < J; ++x)
                for (int y = 0; y < J; ++y)
                    S[x * J + y] = (x == y ? 1.0 : 0.0) + h * (P->K[x * J + y] / P->m - (x == y ? P->c[x] : 0.0));
            for (int x = 0; x < J; ++x) s[x] = 0.0;
            for (int l = 0; l < J; ++l) {
                if (l == i) continue;
                for (int y = 0; y < J; ++y) S[l * J + y] += h * P->beta[l] * F[l][y];
                s[l] += h * P->beta[l] * f[l];
            }
            double Qii = Q[i][i * J + i];
            double D = 1.0 - delta * h * P->beta[i] * P->beta[i] * Qii;
            for (int y = 0; y < J; ++y) {       /* e_i' Q_i S_i */
                double t = 0.0;
                for (int x = 0; x < J; ++x) t += Q[i][i * J + x] * S[x * J + y];
                Fi[y] = delta * P->beta[i] * t / D;
            }
            {
                double t = b[i][i];
                for (int x = 0; x < J; ++x) t += Q[i][i * J + x] * s[x];
                fi = (P->A[i] + delta * P->beta[i] * t) / D;
            }
            memcpy(Sp, S, sizeof(double) * J * J);
            memcpy(sp, s, sizeof(double) * J);
            for (int y = 0; y < J; ++y) Sp[i * J + y] += h * P->beta[i] * Fi[y];
            sp[i] += h * P->beta[i] * fi;
            /* Q' = h(-F'F - phi e_i e_i') + delta Sp' Q Sp */
            double QS[16];
            for (int x = 0; x < J; ++x)
                for (int y = 0; y < J; ++y) {
                    double t = 0.0;
                    for (int z = 0; z < J; ++z) t += Q[i][x * J + z] * Sp[z * J + y];
                    QS[x * J + y] = t;
                }
            for (int x = 0; x < J; ++x)
                for (int y = 0; y < J; ++y) {
                    double t = 0.0;
                    for (int z = 0; z < J; ++z) t += Sp[z * J + x] * QS[z * J + y];
                    double q = h * (-Fi[x] * Fi[y] - (x == i && y == i ? P->phi[i] : 0.0)) + delta * t;
                    Qn[i][x * J + y] = q;
                }
            double Qs_b[4];
            for (int x = 0; x < J; ++x) {
                double t = b[i][x];
                for (int z = 0; z < J; ++z) t += Q[i][x * J + z] * sp[z];
                Qs_b[x] = t;
            }
            for (int y = 0; y < J; ++y) {
                double t = 0.0;
                for (int z = 0; z < J; ++z) t += Sp[z * J + y] * Qs_b[z];
                bn[i][y] = h * (P->A[i] - fi) * Fi[y] + delta * t;
            }
            {
                double sQs = 0.0, bs = 0.0;
                for (int x = 0; x < J; ++x) {
                    double t = 0.0;
                    for (int z = 0; z < J; ++z) t += Q[i][x * J + z] * sp[z];
                    sQs += sp[x] * t;
                    bs += b[i][x] * sp[x];
                }
                an[i] = h * (P->A[i] * fi - 0.5 * fi * fi) + delta * (0.5 * sQs + bs + a[i]);
            }
            for (int y = 0; y < J; ++y) Fn[i][y] = Fi[y];
            fn[i] = fi;
        }
        memcpy(Q, Qn, sizeof Q); memcpy(b, bn, sizeof b); memcpy(a, an, sizeof a);
        memcpy(F, Fn, sizeof F); memcpy(f, fn, sizeof f);
        for (int i = 0; i < J; ++i) {
            for (int t = 0; t < J * J; ++t) Qo[((size_t)r * J + i) * J * J + t] = Q[i][t];
            for (int t = 0; t < J; ++t) bo[((size_t)r * J + i) * J + t] = b[i][t];
            ao[(size_t)r * J + i] = a[i];
            for (int t = 0; t < J; ++t) Fo[((size_t)r * J + i) * J + t] = F[i][t];
            fo[(size_t)r * J + i] = f[i];
        }
    }
}

/* Equilibrium time paths (Section 4: the emission and pollution-stock paths
 * along the equilibrium strategy). The feedback policy of player i is the
 * Chebyshev interpolant of its nodal controls on [0, P_M]^J (Definition 3.2,
 * fitted by eq. (forcoef)), clamped to [0, U_M]; from each initial stock, T
 * explicit steps of the dynamics with the discretisation's time step h:
 *     p_{t+1} = p_t + h g(p_t, u(p_t)).
 * u_nodal: J x n^J nodal controls (row-major, last player fastest); p0: K x J;
 * p_path: K x (T + 1) x J (p_path[k][0] = p0[k]); u_path: K x T x J or NULL. */
void orc_game_paths(const orc_game_params *P, const orc_game_opts *O, const double *u_nodal, long K,
                    const double *p0, long T, double *p_path, double *u_path)
{
    const int J = P->J;
    const long NP = ipow(O->n, J);
    int nd[4];
    for (int s = 0; s < J; ++s) nd[s] = O->n;
    double *coef = (double *)malloc(sizeof(double) * (size_t)J * (size_t)NP);
    for (int i = 0; i < J; ++i) orc_fit_nd(J, nd, u_nodal + (size_t)i * NP, coef + (size_t)i * NP);
#pragma omp parallel for schedule(dynamic, 1)
    for (long k = 0; k < K; ++k) {
        double p[4], u[4], g[4], xref[4];
        for (int s = 0; s < J; ++s) {
            p[s] = p0[(size_t)k * J + s];
            p_path[((size_t)k * (T + 1)) * J + s] = p[s];
        }
        for (long t = 0; t < T; ++t) {
            for (int s = 0; s < J; ++s) xref[s] = 2.0 * p[s] / O->P_M - 1.0;
            for (int i = 0; i < J; ++i) {
                const double v = orc_eval_direct(J, nd, coef + (size_t)i * NP, xref);
                u[i] = fmin(fmax(v, 0.0), O->U_M);
            }
            orc_game_dynamics(P, p, u, g);
            for (int s = 0; s < J; ++s) {
                p[s] += O->h * g[s];
                p_path[((size_t)k * (T + 1) + (size_t)t + 1) * J + s] = p[s];
                if (u_path) u_path[((size_t)k * T + (size_t)t) * J + s] = u[s];
            }
        }
    }
    free(coef);
}
