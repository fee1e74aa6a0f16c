// The general method of Section 2.1 for dynamics that are not separable in
// the controls (the game with the emission-interaction coupling gamma):
//
//  Step 0  g-interpolants: at every state node pbar_j, each component g_l of
//          the dynamics is interpolated in all J controls on the tensor grid of
//          n_u Chebyshev-Lobatto control nodes per player on [0, U_M]
//          (eq. (forcoef) along every control mode; computed once per solve);
//  Step 1-2 for player i at node j with the other players' controls fixed at
//          u^[r]_{-i}(pbar_j): the interpolants restricted to player i's
//          control line are one-variable series (a contraction with the
//          Chebyshev rows of the other players' controls: the row-wise form of
//          the paper's location indexes, Section 3.3); at every control node
//          u~_k they give the next state pbar_j + h g(pbar_j, [u~_k, u^[r]_{-i}]),
//          where V_i^[r] is evaluated (its coefficient tensor contracted with
//          the Chebyshev rows of the next state);
//  Step 2-3 the values W_k = h G_i + delta_h V_i are interpolated in the
//          control (C1v as the n_u x n_u DCT-I matrix) and the interpolant is
//          maximised on [0, U_M]: 8 n_u + 1 Chebyshev-spaced samples, Newton
//          on the derivative series (Proposition 3.1) from the best sample,
//          safeguarded by bisection; the bounds, the best sample and the
//          Newton point compete, ties to the smaller control.
// FP64 on the CUDA cores, one thread per (instance, player, node). The refit,
// residual and loop are the ones of game.cu.
#include <algorithm>
#include <cmath>

#include "game_internal.cuh"

namespace cheb {
namespace game {
namespace {

constexpr int kMaxNu = kGameNMax;     // control nodes per player
constexpr int kRowLen = kGameNMax;    // longest Chebyshev row (state or control)

// sum over the multi-index k of C[k] prod_{s in modes, s != skip} T[s][k_s], with
// k_skip fixed at idx (skip < 0: no mode fixed); C row-major with n entries per mode
__device__ double contract(const double *__restrict__ C, int J, int n, int skip, int idx,
                           const double (&T)[4][kRowLen])
{
    int stride[4];
    stride[J - 1] = 1;
    for (int s = J - 2; s >= 0; --s) stride[s] = stride[s + 1] * n;
    int o[4], no = 0;
    for (int s = 0; s < J; ++s)
        if (s != skip) o[no++] = s;
    const double *B = C + (skip >= 0 ? (int64_t)idx * stride[skip] : 0);
    if (no == 0) return B[0];
    if (no == 1) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) acc = fma(B[a * stride[o[0]]], T[o[0]][a], acc);
        return acc;
    }
    if (no == 2) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) {
            double t = 0.0;
            const double *Ba = B + a * stride[o[0]];
            for (int b = 0; b < n; ++b) t = fma(Ba[b * stride[o[1]]], T[o[1]][b], t);
            acc = fma(t, T[o[0]][a], acc);
        }
        return acc;
    }
    if (no == 3) {
        double acc = 0.0;
        for (int a = 0; a < n; ++a) {
            double ta = 0.0;
            for (int b = 0; b < n; ++b) {
                double t = 0.0;
                const double *Bab = B + a * stride[o[0]] + b * stride[o[1]];
                for (int c = 0; c < n; ++c) t = fma(Bab[c * stride[o[2]]], T[o[2]][c], t);
                ta = fma(t, T[o[1]][b], ta);
            }
            acc = fma(ta, T[o[0]][a], acc);
        }
        return acc;
    }
    double acc = 0.0;
    for (int a = 0; a < n; ++a) {
        double ta = 0.0;
        for (int b = 0; b < n; ++b) {
            double tb = 0.0;
            for (int c = 0; c < n; ++c) {
                double t = 0.0;
                const double *Babc = B + a * stride[o[0]] + b * stride[o[1]] + c * stride[o[2]];
                for (int d = 0; d < n; ++d) t = fma(Babc[d * stride[o[3]]], T[o[3]][d], t);
                tb = fma(t, T[o[2]][c], tb);
            }
            ta = fma(tb, T[o[1]][b], ta);
        }
        acc = fma(ta, T[o[0]][a], acc);
    }
    return acc;
}

// T_0..T_{n-1}(x) by the three-term recurrence (valid off [-1, 1] too)
__device__ __forceinline__ void cheb_row(double x, int n, double *T)
{
    T[0] = 1.0;
    if (n > 1) T[1] = x;
    for (int k = 2; k < n; ++k) T[k] = 2.0 * x * T[k - 1] - T[k - 2];
}

// sum_m a_m T_m(y) by Clenshaw's recurrence
__device__ __forceinline__ double series(const double *a, int n, double y)
{
    double b1 = 0.0, b2 = 0.0;
    for (int m = n - 1; m >= 1; --m) {
        const double b0 = fma(2.0 * y, b1, a[m] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(y, b1, a[0] - b2);
}

// coefficients of the derivative of sum_m a_m T_m on [-1, 1] (Proposition 3.1
// with b - a = 2): q_{N-1} = 2 N a_N, q_l = q_{l+2} + 2 (l + 1) a_{l+1}, q_0 halved
__device__ __forceinline__ void deriv(const double *a, int n, double *q)
{
    for (int l = 0; l < n; ++l) q[l] = 0.0;
    if (n < 2) return;
    double q2 = 0.0, q1 = 0.0;      // q_{l+2}, q_{l+1}
    for (int l = n - 2; l >= 0; --l) {
        const double ql = q2 + 2.0 * (double)(l + 1) * a[l + 1];
        q[l] = ql;
        q2 = q1;
        q1 = ql;
    }
    q[0] *= 0.5;
}

// Step 0, values: vals[((q NP + j) J + l) NU + t] = g_l(pbar_j, u_t), t the
// row-major multi-index of the control nodes (last player fastest); one thread
// per (instance, node, control multi-index).
__global__ void g_values_kernel(const GameDev *__restrict__ insts, int B, int NP, int NU, double *__restrict__ vals)
{
    const int64_t total = (int64_t)B * NP * NU;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(e % NU);
        const int64_t qj = e / NU;
        const int j = (int)(qj % NP), q = (int)(qj / NP);
        const GameDev &g = insts[q];
        const int J = g.J, nu = g.n_u;
        double pb[4] = {0.0, 0.0, 0.0, 0.0}, uu[4] = {0.0, 0.0, 0.0, 0.0};
        int rj = j, rt = t;
        for (int s = J - 1; s >= 0; --s) {
            const int kj = rj % g.n, kt = rt % nu;
            rj /= g.n;
            rt /= nu;
            pb[s] = 0.5 * g.P_M * (g.nodes[kj] + 1.0);
            uu[s] = 0.5 * g.U_M * (g.unodes[kt] + 1.0);
        }
        for (int l = 0; l < J; ++l) {
            double coup = 0.0, inter = 0.0;
            for (int s = 0; s < J; ++s) {
                if (s == l) continue;
                coup += g.K[l * J + s] * (pb[s] - pb[l]);
                inter += g.gamma[l * J + s] * uu[s];
            }
            const double gl = coup * g.minv - g.c[l] * pb[l] + g.beta[l] * uu[l] + uu[l] * inter;
            vals[(qj * J + l) * NU + t] = gl;
        }
    }
}

// Steps 1-3 for player blockIdx.y at the nodes of instance blockIdx.z.
__global__ void __launch_bounds__(64)
general_player_kernel(const GameDev *__restrict__ insts, GameStat *__restrict__ stats)
{
    const int q = blockIdx.z, i = blockIdx.y;
    const GameDev &g = insts[q];
    GameStat *st = &stats[q];
    if (st->done || st->mode != 0) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = g.J, n = g.n, NP = g.NP, nu = g.n_u;
    if (j >= NP) return;
    int NU = 1;
    for (int s = 0; s < J; ++s) NU *= nu;
    double pb[4] = {0.0, 0.0, 0.0, 0.0}, uo[4] = {0.0, 0.0, 0.0, 0.0};
    {
        int rj = j;
        for (int s = J - 1; s >= 0; --s) {
            const int k = rj % n;
            rj /= n;
            pb[s] = 0.5 * g.P_M * (g.nodes[k] + 1.0);
            uo[s] = g.u[s * NP + j];
        }
    }
    // Step 1: the g-interpolants of this node on player i's control line
    double T[4][kRowLen];
    for (int s = 0; s < J; ++s)
        if (s != i) cheb_row(2.0 * uo[s] / g.U_M - 1.0, nu, T[s]);
    double a[4][kMaxNu];
    const double *Gc = g.Gc + (int64_t)j * J * NU;
    for (int l = 0; l < J; ++l)
        for (int m = 0; m < nu; ++m) a[l][m] = contract(Gc + (int64_t)l * NU, J, nu, i, m, T);
    // Step 2: V_i^[r] at the next states of the control nodes
    const double *Ci = g.C + (int64_t)i * NP;
    double W[kMaxNu];
    for (int k = 0; k < nu; ++k) {
        const double y = g.unodes[k];
        const double uk = 0.5 * g.U_M * (y + 1.0);
        double x[4];
        for (int l = 0; l < J; ++l) {
            const double gl = series(a[l], nu, y);
            x[l] = 2.0 * (pb[l] + g.h * gl) / g.P_M - 1.0;
        }
        for (int s = 0; s < J; ++s) cheb_row(x[s], n, T[s]);
        const double V = contract(Ci, J, n, -1, 0, T);
        const double G = uk * (g.A[i] - 0.5 * uk) - 0.5 * g.phi[i] * pb[i] * pb[i];
        W[k] = g.h * G + g.delta * V;
    }
    // C1v: coefficients of the control interpolant, w = M_u W
    double w[kMaxNu], d1[kMaxNu], d2[kMaxNu];
    for (int l = 0; l < nu; ++l) {
        double s = 0.0;
        for (int k = 0; k < nu; ++k) s = fma(g.Mu[l * nu + k], W[k], s);
        w[l] = s;
    }
    deriv(w, nu, d1);
    deriv(d1, nu, d2);
    // Step 3: maximise over y in [-1, 1] (u = U_M (y + 1) / 2)
    const int S = 8 * nu;
    int best = S;
    double bestv = -INFINITY;
    for (int t = S; t >= 0; --t) {          // ascending y
        const double v = series(w, nu, cospi((double)t / (double)S));
        if (v > bestv) {
            bestv = v;
            best = t;
        }
    }
    const double yb = cospi((double)best / (double)S);
    const double ylo = cospi((double)(best < S ? best + 1 : S) / (double)S);
    const double yhi = cospi((double)(best > 0 ? best - 1 : 0) / (double)S);
    double cand[4] = {-1.0, 1.0, yb, yb};
    int nc = 3;
    if (series(d1, nu, ylo) > 0.0 && series(d1, nu, yhi) < 0.0) {
        double y = yb, lo = ylo, hi = yhi;
        for (int it = 0; it < 60; ++it) {
            const double f1 = series(d1, nu, y), f2 = series(d2, nu, y);
            if (f1 > 0.0)
                lo = y;
            else
                hi = y;
            double yn = (f2 < 0.0) ? y - f1 / f2 : 0.5 * (lo + hi);
            if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
            const double step = fabs(yn - y);
            y = yn;
            if (step < 1e-15 || hi - lo < 1e-15) break;
        }
        cand[nc++] = y;
    }
    double ys = cand[0], vs = series(w, nu, cand[0]);
    for (int c = 1; c < nc; ++c) {
        const double v = series(w, nu, cand[c]);
        if (v > vs || (v == vs && cand[c] < ys)) {
            vs = v;
            ys = cand[c];
        }
    }
    g.u_new[i * NP + j] = 0.5 * g.U_M * (ys + 1.0);
    store_vn_new(g, i * NP + j, vs);
    const double dv = fabs(vs - g.Vn[i * NP + j]);
    atomicMax(&st->res_bits, (unsigned long long)__double_as_longlong(dv));
}

}  // namespace

cheb_status game_general_prepare(cheb_ctx *ctx, const GameDev *d_inst, int B, int J, int NP, int n_u, double *Gc,
                                 double *tmp0, double *tmp1, cudaStream_t st)
{
    int64_t NU = 1;
    for (int s = 0; s < J; ++s) NU *= n_u;
    const int64_t total = (int64_t)B * NP * NU;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 65535);
    {
        ProfScope prof("game_g_values", st);
        g_values_kernel<<<blocks, 256, 0, st>>>(d_inst, B, NP, (int)NU, tmp0);
    }
    CHEB_CUDA_TRY(cudaGetLastError());
    const double *M = nullptr;
    cheb_status r = dct_matrix(ctx, n_u, &M);
    if (r) return r;
    // eq. (forcoef) along each control mode of every (instance, node, component) slab
    const double *src = tmp0;
    double *bufs[2] = {tmp1, tmp0};
    for (int t = 0; t < J; ++t) {
        double *dst = (t == J - 1) ? Gc : bufs[t & 1];
        if ((r = modeprod_f64_slabs(src, M, dst, (int64_t)B * NP * J, NU / n_u, n_u, n_u, SlabSkip{}, st))) return r;
        src = dst;
    }
    return CHEB_OK;
}

cheb_status game_general_player(const GameDev *d_inst, GameStat *d_stat, int B, int J, int NP, cudaStream_t st)
{
    ProfScope prof("game_player_general", st);
    general_player_kernel<<<dim3((unsigned)((NP + 63) / 64), J, B), 64, 0, st>>>(d_inst, d_stat);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

}  // namespace game
}  // namespace cheb
