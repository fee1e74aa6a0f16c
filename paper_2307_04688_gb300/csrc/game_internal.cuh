// Shared declarations of the game solver (game.cu, game_tc.cu).
#pragma once

#include <cstdint>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {
namespace game {

constexpr int kGameNMax = 33;     // nodes per player

// One instance, device-resident (read-only during the iteration).
struct GameDev {
    int J, n, NP;                 // players, nodes per player, n^J
    double K[16], minv;           // neighbour matrix, 1/m
    double A[4], beta[4], phi[4], c[4];
    double h, delta, P_M, U_M, tol;
    // per player, formed on the host: dx_i/du_i = 2 h beta_i / P_M, h A_i and
    // -h phi_i / 2 (the FP64 pipe is slow; no division per node)
    double slope[4], hA[4], hphi2[4];
    long long max_iter;
    int polish, stall_window;
    double *C;                    // J x NP coefficient tensors of the current iterate
    double *u, *Vn;               // nodal controls / values of the current iterate
    double *u_new, *Vn_new;       // of the next iterate
    double *X;                    // J x NP next-state reference coordinates
    const double *nodes;          // cos(pi k / N), k < n
    const double *V0, *u0;        // optional initial nodal values / controls
    // split-precision path (game_tc.cu)
    void *bsplit;                 // pre-split coefficient operands, J x chunks
    // double-float path (game_df.cu)
    float *Cdf;                   // J x NP coefficient pairs (hi, lo)
    float *Vdf;                   // J x NP pairs (hi, lo) of Vn_new: the double-float refit's input
    double two_over_PM;           // 2 / P_M (next-state coordinates without a division)
    int polish_mode;              // mode a stalled split iteration continues in (0 FP64, 2 double-float)
    // general method (game_general.cu): dynamics coupled through gamma
    int general, n_u;             // general method on; control nodes per player
    double gamma[16];             // J x J emission-interaction coupling
    double *Gc;                   // NP x J x n_u^J coefficients of the g-interpolants
    const double *Mu;             // n_u x n_u DCT-I matrix of the control interpolant
    const double *unodes;         // cos(pi k / (n_u - 1)), k < n_u
};

// One instance's progress, written by the commit kernel.
struct GameStat {
    int done;
    int mode;                     // 0: FP64 evaluation, 1: split precision, 2: double-float
    int mode_initial;             // the mode a (re)start begins in
    int status;                   // cheb_status once done
    int since_best;
    int warm;                     // started from given V0 / u0 (a divergence restarts cold)
    int restart;                  // 1: reset to the cold start at the next iteration
    int restarts;                 // cold restarts performed
    long long iters, iters_split;
    unsigned long long res_bits;  // running max |dV| of this iteration (bits of a double >= 0)
    double last_res, best_res;
};

// Node j: multi-index (j_0..j_{J-1}), last fastest; reference coordinate
// cos(pi j_s / N), physical pbar_s = (P_M / 2)(x_s + 1) (Section 3.4, Step 0).
__device__ __forceinline__ void node_coords(const GameDev &g, int j, double *xr, double *pb)
{
    int rem = j;
    for (int s = g.J - 1; s >= 0; --s) {
        const int k = rem % g.n;
        rem /= g.n;
        xr[s] = g.nodes[k];
        pb[s] = 0.5 * g.P_M * (xr[s] + 1.0);
    }
}

// W(u) = h (u (A - u/2) - phi pbar_i^2 / 2) + delta sum_m w_m T_m(xc + slope u)
// (the Bellman objective of Section 2.1 along the next states, which are
// affine in the player's own control) and its first two derivatives; T, T'
// and T'' by differentiating the three-term recurrence, valid for any x.
__device__ __forceinline__ void objective(const double *w, int n, double xc, double slope, double hA,
                                          double hG0, double h, double delta, double u, double *W,
                                          double *W1, double *W2)
{
    const double x = xc + slope * u;
    double t0 = 1.0, t1 = x, d0 = 0.0, d1 = 1.0, e0 = 0.0, e1 = 0.0;
    double s = w[0], s1 = 0.0, s2 = 0.0;
    if (n > 1) {
        s += w[1] * x;
        s1 += w[1];
    }
    for (int m = 2; m < n; ++m) {
        const double t2 = 2.0 * x * t1 - t0;
        const double d2 = 2.0 * t1 + 2.0 * x * d1 - d0;
        const double e2 = 4.0 * d1 + 2.0 * x * e1 - e0;
        s += w[m] * t2;
        s1 += w[m] * d2;
        s2 += w[m] * e2;
        t0 = t1; t1 = t2;
        d0 = d1; d1 = d2;
        e0 = e1; e1 = e2;
    }
    *W = hA * u - 0.5 * h * u * u + hG0 + delta * s;
    *W1 = hA - h * u + delta * slope * s1;
    *W2 = -h + delta * slope * slope * s2;
}

// Step 3: the maximiser of W over [0, U_M]. Projected Newton from u0 (the
// previous control; Section 3.4 recommends Newton), then the two bounds and
// the Newton point compete: the largest W wins, ties to the smaller control.
__device__ __forceinline__ double argmax_control(const double *w, int n, double xc, double slope, double hA,
                                                 double hG0, double h, double delta, double U_M, double u0,
                                                 double *Vbest)
{
    double u = fmin(fmax(u0, 0.0), U_M);
    double W, W1, W2;
    for (int it = 0; it < 30; ++it) {
        objective(w, n, xc, slope, hA, hG0, h, delta, u, &W, &W1, &W2);
        double un;
        if (W2 < 0.0)
            un = u - W1 / W2;
        else
            un = W1 > 0.0 ? 0.5 * (u + U_M) : 0.5 * u;   // not concave here: move towards ascent
        un = fmin(fmax(un, 0.0), U_M);
        const double step = fabs(un - u);
        u = un;
        if (step <= 1e-15 * U_M) break;
    }
    double best_u = 0.0, best_W;
    objective(w, n, xc, slope, hA, hG0, h, delta, 0.0, &best_W, &W1, &W2);
    objective(w, n, xc, slope, hA, hG0, h, delta, u, &W, &W1, &W2);
    if (W > best_W) { best_W = W; best_u = u; }
    objective(w, n, xc, slope, hA, hG0, h, delta, U_M, &W, &W1, &W2);
    if (W > best_W) { best_W = W; best_u = U_M; }
    *Vbest = best_W;
    return best_u;
}

// Vn_new[idx] = V and, for groups that refit in double-float, its split
// (hi = V rounded to FP32, lo = the rest rounded), the refit's input: formed
// here once per value instead of by every refit CTA that reads it (the FP64
// conversions run on GB300's slow FP64 pipe).
__device__ __forceinline__ void store_vn_new(const GameDev &g, int idx, double V)
{
    g.Vn_new[idx] = V;
    if (g.Vdf) {
        const float hi = (float)V;
        g.Vdf[2 * idx] = hi;
        g.Vdf[2 * idx + 1] = (float)(V - (double)hi);
    }
}

// Given the series w (player i's coordinate, node j), maximise, store the
// new control and value, and fold |V_new - V_old| into the residual.
__device__ __forceinline__ void player_finish(const GameDev &g, GameStat *st, int i, int j, const double *w)
{
    double xr[4], pb[4];
    node_coords(g, j, xr, pb);
    const int NP = g.NP;
    const double ui = g.u[i * NP + j];
    const double slope = g.slope[i];                               // dx_i / du_i
    const double xc = g.X[i * NP + j] - slope * ui;
    const double hA = g.hA[i];
    const double hG0 = g.hphi2[i] * pb[i] * pb[i];
    double V;
    const double us = argmax_control(w, g.n, xc, slope, hA, hG0, g.h, g.delta, g.U_M, ui, &V);
    g.u_new[i * NP + j] = us;
    store_vn_new(g, i * NP + j, V);
    const double d = fabs(V - g.Vn[i * NP + j]);
    atomicMax(&st->res_bits, (unsigned long long)__double_as_longlong(d));
}

cheb_status solve_group(cheb_ctx *ctx, int J, int n, int NP, int prec, int general, int n_u,
                        const std::vector<int> &members, const cheb_game_params *params,
                        const cheb_game_opts *opts, cheb_game_result *res, cudaStream_t st);

// ---- general method (game_general.cu): Step 0 g-interpolants of every instance
// into Gc (tmp0, tmp1: workspaces of the same size, B NP J n_u^J doubles), and the
// Steps 1-3 update of every player at every node (instances in FP64 mode) ----
cheb_status game_general_prepare(cheb_ctx *ctx, const GameDev *d_inst, int B, int J, int NP, int n_u, double *Gc,
                                 double *tmp0, double *tmp1, cudaStream_t st);
cheb_status game_general_player(const GameDev *d_inst, GameStat *d_stat, int B, int J, int NP, cudaStream_t st);

// ---- double-float player update (game_df.cu): coefficient split + update ----
cheb_status game_df_player(const GameDev *d_inst, GameStat *d_stat, int B, int J, int NP, cudaStream_t st);

// ---- double-float refit of G = B J slabs (game_df.cu), for split-precision
// solves: C = V with eq. (forcoef) applied along each of the J modes, from
// the (hi, lo) pairs Vdf of the nodal values; slabs of finished instances
// skipped when `stats` is given. game_refit_df: one launch per mode, n in
// {5, 9, 17, 33}; game_refit_df_chain: all modes in one launch for small
// groups (bit-identical coefficients; CHEB_EUNSUPPORTED, nothing launched,
// when n^(J-1) > 4913 or G > 65535).
bool game_refit_df_supported(int n);
cheb_status game_refit_df(const float *Vdf, const double *M, double *C, double *tmp0, double *tmp1, int G, int J,
                          int n, int NP, const GameStat *stats, cudaStream_t st);
cheb_status game_refit_df_chain(const float *Vdf, const double *M, double *C, int G, int J, int n,
                                const GameStat *stats, cudaStream_t st);

// ---- split-precision player update (game_tc.cu) ----
bool tc_shape_supported(int J, int n);    // (J, n) with a split player update
size_t game_tc_workspace_bytes(int J, int n, int NP, int B, int prec);
void game_tc_bind(GameDev *hinst, int B, int J, int n, int NP, int prec, uint8_t *ws);
cheb_status game_tc_player(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, const GameDev *hinst, int B,
                           int J, int n, int NP, int prec, uint8_t *ws, cudaStream_t st);
// Tile-shape tuner: before the first iteration of a group (X of that iteration
// already computed), time every tile configuration of the split player update
// on the group itself and keep the fastest for (form, n, batch class) in the
// context. The runs are the first iteration's own work (deterministic; the
// real iteration rewrites the same values), so they change no result.
cheb_status game_tc_tune(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int J, int n, int prec,
                         cudaStream_t st);

}  // namespace game
}  // namespace cheb
