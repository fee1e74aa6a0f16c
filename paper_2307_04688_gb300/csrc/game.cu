// The Chebyshev collocation iteration for the J-player pollution game
// (Section 2.1 Steps 0-4, Section 3.4), batched over independent instances.
//
// State per instance (device): coefficient tensors C (J x n^J, the caller's
// V buffer), nodal controls u (the caller's u buffer) and nodal values Vn of
// the current iterate, their successors u_new / Vn_new, and the next-state
// reference coordinates X (J x n^J). One iteration is
//   next_state  : X_l(j) = 2 (pbar_l + h g_l(pbar_j, u^[r](pbar_j))) / P_M - 1
//   player      : for every player i and node j, V_i^[r] along the next states
//                 is a Chebyshev series in the player's own coordinate (the
//                 others are fixed at u^[r]); Newton on it gives u^[r+1]_i(j)
//                 and V^[r+1]_i(j); |V^[r+1] - V^[r]| feeds the residual
//   refit       : C = fit(Vn_new) in FP64 (eq. (forcoef) along every mode)
//   commit      : u, Vn <- u_new, Vn_new; residual test, stall test, counters
// with every kernel skipping instances that are done. Iterations are
// enqueued in chunks captured once into a CUDA graph; the host only reads the
// per-instance status between chunks.
//
// Three evaluation kernels exist: FP64 on the CUDA cores (player_f64_kernel),
// double-float on the FP32 pipe (game_df.cu) and the split-precision
// tensor-core kernel (game_tc.cu). A device-side mode flag per instance
// selects one of them each iteration, so the switch from split to
// FP64-accurate iterations (polish) needs no host round trip.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "cheb_internal.cuh"
#include "game_internal.cuh"

namespace cheb {
namespace game {

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------


// The next states of every node (grid: node blocks x instances):
// p_l + h g_l(p, u) with g_l(p, u) = (1/m) sum_{l' != l} K[l][l'] (p_l' - p_l)
// - c_l p_l + beta_l u_l (Section 2.1), mapped to the reference coordinate.
// The loops run over the fixed maximum of 4 players with guards, so that the
// node's coordinates stay in registers (a by-value copy of the descriptor with
// runtime-indexed arrays put ~560 bytes per thread in local memory); pbar as
// in node_coords.
__global__ void next_state_kernel(const GameDev *__restrict__ insts, const GameStat *__restrict__ stats)
{
    const GameDev &g = insts[blockIdx.y];
    if (stats[blockIdx.y].done) return;
    const int J = g.J, n = g.n, NP = g.NP;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NP) return;
    const double P_M = g.P_M;
    double pb[4] = {0.0, 0.0, 0.0, 0.0};
    int rem = j;
#pragma unroll
    for (int s = 3; s >= 0; --s) {
        if (s < J) {
            const int k = rem % n;
            rem /= n;
            pb[s] = 0.5 * P_M * (g.nodes[k] + 1.0);
        }
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l < J) {
            double coup = 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (t < J && t != l) coup += g.K[l * J + t] * (pb[t] - pb[l]);
            const double dyn = coup * g.minv - g.c[l] * pb[l] + g.beta[l] * g.u[l * NP + j];
            const double q = pb[l] + g.h * dyn;
            g.X[l * NP + j] = g.two_over_PM * q - 1.0;
        }
    }
}

// FP64 player update. A block of 128 threads covers 32 nodes of one player
// and splits the n coefficients k of each node's series over four k groups:
// thread (node q = tid % 32, group kg = tid / 32) contracts
// w[k] = sum over the other modes of C_i[..k..] prod_s T_{k_s}(x_s(j)) by
// nested contraction (last mode first) for its share of k, four k at a time
// (independent FMA chains, each w[k] summed in the same order as one k at a
// time), so a single game gives four times as many warps to hide the FP64
// latency. The Chebyshev rows of the 32 nodes sit in shared memory, w goes
// through shared memory, and the first warp maximises over the controls.
constexpr int kF64Nodes = 32;
__global__ void __launch_bounds__(128)
player_f64_kernel(const GameDev *__restrict__ insts, GameStat *__restrict__ stats)
{
    extern __shared__ double f64_s[];   // T rows [J - 1][n][32], then w [n][32]
    const int inst = blockIdx.z, i = blockIdx.y;
    const GameDev &g = insts[inst];
    GameStat *st = &stats[inst];
    if (st->done || st->mode != 0) return;
    const int J = g.J, n = g.n, NP = g.NP;
    // the J - 1 row blocks and w fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK((size_t)J * n * kF64Nodes * sizeof(double) <= dyn_smem_bytes())) return;
    const int q = threadIdx.x % kF64Nodes, kg = threadIdx.x / kF64Nodes;
    const int j = blockIdx.x * kF64Nodes + q;
    const bool valid = j < NP;
    double *T_s = f64_s;
    double *w_s = f64_s + (size_t)(J - 1) * n * kF64Nodes;
    auto T = [&](int slot, int k) -> double & { return T_s[(slot * n + k) * kF64Nodes + q]; };
    // other mode of slot t (the modes other than i in increasing order)
    auto other = [&](int t) { return t < i ? t : t + 1; };
    auto stride = [&](int s) {
        int v = 1;
        for (int r = s + 1; r < J; ++r) v *= n;
        return v;
    };
    // the rows of the node's other coordinates: group kg takes slots kg, kg + 4, ...
    for (int t = kg; t < J - 1; t += 4) {
        const double x = valid ? g.X[other(t) * NP + j] : 0.0;
        double t0 = 1.0, t1 = x;
        T(t, 0) = 1.0;
        if (n > 1) T(t, 1) = x;
        for (int k = 2; k < n; ++k) {
            const double t2 = 2.0 * x * t1 - t0;
            T(t, k) = t2;
            t0 = t1;
            t1 = t2;
        }
    }
    __syncthreads();
    const int no = J - 1;
    const double *C = g.C + (size_t)i * NP;
    const int si = stride(i);
    const int kq = (n + 3) / 4;
    const int klo = kg * kq, khi = klo + kq < n ? klo + kq : n;
    for (int k0 = klo; valid && k0 < khi; k0 += 4) {
        const int kb = khi - k0 < 4 ? khi - k0 : 4;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        if (no == 0) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < kb) acc[r] = C[(size_t)(k0 + r) * si];
        } else if (no == 1) {
            const int s0 = stride(other(0));
            for (int a = 0; a < n; ++a) {
                const double ta = T(0, a);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < kb) acc[r] = fma(C[(size_t)(k0 + r) * si + a * s0], ta, acc[r]);
            }
        } else if (no == 2) {
            const int s0 = stride(other(0)), s1 = stride(other(1));
            for (int a = 0; a < n; ++a) {
                double t[4] = {0.0, 0.0, 0.0, 0.0};
                const double *Ca = C + (size_t)k0 * si + a * s0;
                for (int b = 0; b < n; ++b) {
                    const double tb = T(1, b);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < kb) t[r] = fma(Ca[(size_t)r * si + b * s1], tb, t[r]);
                }
                const double ta = T(0, a);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < kb) acc[r] = fma(t[r], ta, acc[r]);
            }
        } else {
            const int s0 = stride(other(0)), s1 = stride(other(1)), s2 = stride(other(2));
            for (int a = 0; a < n; ++a) {
                double ta[4] = {0.0, 0.0, 0.0, 0.0};
                for (int b = 0; b < n; ++b) {
                    double t[4] = {0.0, 0.0, 0.0, 0.0};
                    const double *Cab = C + (size_t)k0 * si + a * s0 + b * s1;
                    for (int c = 0; c < n; ++c) {
                        const double tc = T(2, c);
#pragma unroll
                        for (int r = 0; r < 4; ++r)
                            if (r < kb) t[r] = fma(Cab[(size_t)r * si + c * s2], tc, t[r]);
                    }
                    const double tb = T(1, b);
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < kb) ta[r] = fma(t[r], tb, ta[r]);
                }
                const double tA = T(0, a);
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < kb) acc[r] = fma(ta[r], tA, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < kb) w_s[(k0 + r) * kF64Nodes + q] = acc[r];
    }
    __syncthreads();
    if (kg == 0 && valid) {
        double w[kGameNMax];
        for (int k = 0; k < n; ++k) w[k] = w_s[k * kF64Nodes + q];
        player_finish(g, st, i, j, w);
    }
}

// u, Vn <- u_new, Vn_new for instances still running (grid: node blocks x instances).
__global__ void commit_copy_kernel(const GameDev *__restrict__ insts, const GameStat *__restrict__ stats)
{
    if (stats[blockIdx.y].done) return;
    const GameDev g = insts[blockIdx.y];
    const int total = g.J * g.NP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        g.u[t] = g.u_new[t];
        g.Vn[t] = g.Vn_new[t];
    }
}

// Cold restart of instances whose warm start diverged: V = 0, u = 0 (the
// coefficients of V = 0 are 0), as at a cold Step 0.
__global__ void restart_kernel(const GameDev *__restrict__ insts, const GameStat *__restrict__ stats)
{
    if (stats[blockIdx.y].restart != 1) return;
    const GameDev g = insts[blockIdx.y];
    const int total = g.J * g.NP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        g.u[t] = 0.0;
        g.Vn[t] = 0.0;
        store_vn_new(g, t, 0.0);
        g.C[t] = 0.0;
    }
}

// Residual test of Step 4 and the counters (one thread per instance).
__global__ void commit_stat_kernel(const GameDev *__restrict__ insts, GameStat *__restrict__ stats, int B)
{
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= B) return;
    GameStat &s = stats[inst];
    if (s.done) return;
    const GameDev &g = insts[inst];
    const double res = __longlong_as_double((long long)s.res_bits);
    s.res_bits = 0ull;
    if (s.restart == 1) s.restart = 0;          // this iteration ran from the cold state
    s.iters += 1;
    if (s.mode == 1) s.iters_split += 1;
    s.last_res = res;
    if (res < s.best_res * 0.999) {
        s.best_res = res;
        s.since_best = 0;
    } else {
        s.since_best += 1;
    }
    // a warm start that diverges (non-finite residual, or a residual a thousand
    // times above its best after 20 iterations) falls back to the cold start
    if (s.warm && (!isfinite(res) || (s.iters > 20 && res > 1e3 * s.best_res))) {
        s.warm = 0;
        s.restart = 1;
        s.restarts += 1;
        s.best_res = INFINITY;
        s.since_best = 0;
        s.mode = s.mode_initial;
        return;
    }
    if (res < g.tol) {
        s.done = 1;
        s.status = CHEB_OK;
    } else if (s.iters >= g.max_iter) {
        s.done = 1;
        s.status = CHEB_ENOCONV;
    } else if (s.since_best > g.stall_window) {
        if (s.mode == 1 && g.polish) {
            s.mode = g.polish_mode;     // continue with FP64 accuracy (double-float or FP64)
            s.since_best = 0;
            s.best_res = res;
        } else {
            s.done = 1;
            s.status = CHEB_ESTALL;
        }
    }
}

__global__ void init_state_kernel(const GameDev *__restrict__ insts, int has_v0, int has_u0)
{
    const GameDev g = insts[blockIdx.y];
    const int total = g.J * g.NP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const double v = (has_v0 && g.V0) ? g.V0[t] : 0.0;
        store_vn_new(g, t, v);
        g.Vn[t] = v;
        g.u[t] = (has_u0 && g.u0) ? fmin(fmax(g.u0[t], 0.0), g.U_M) : 0.0;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// FP64 refit of every instance's Vn_new into C: the instances of a group are
// contiguous, so the J nodal tensors of all B instances are G = B J slabs of
// n^J values; J mode products per slab (eq. (forcoef) along each player's
// mode), each moving the new mode to the slab's front, leave every slab in
// its original mode order, the last one written straight into C. With
// `stats`, slabs of finished instances are skipped: their coefficients stay as
// last fitted, which is what a refit of their unchanged Vn_new would give.
// Split-precision groups (`Vdf`, the (hi, lo) pairs of Vn_new) refit in
// double-float on the FP32 pipe instead (relative error about 2^-47; the FP64
// pipe runs at ~1.25 TFLOP/s): small groups in one launch (game_refit_df_chain),
// larger ones one launch per mode (game_refit_df).
static_assert(offsetof(GameStat, done) == 0 && sizeof(GameStat) % sizeof(int) == 0, "GameStat layout");
static cheb_status refit_group(cheb_ctx *ctx, int G, int J, int n, int NP, const double *Vn_new_all,
                               const float *Vdf_all, double *C_all, double *tmp0, double *tmp1,
                               const GameStat *stats, cudaStream_t st)
{
    const double *M = nullptr;
    cheb_status r = dct_matrix(ctx, n, &M);
    if (r) return r;
    const bool small = G * n <= 8 * ctx->num_sms;
    if (Vdf_all) {
        if (small) {
            r = game_refit_df_chain(Vdf_all, M, C_all, G, J, n, stats, st);
            if (r != CHEB_EUNSUPPORTED) return r;
        }
        if (game_refit_df_supported(n))
            return game_refit_df(Vdf_all, M, C_all, tmp0, tmp1, G, J, n, NP, stats, st);
    }
    SlabSkip sk;
    if (stats) {
        sk.flags = &stats->done;
        sk.stride = (int64_t)(sizeof(GameStat) / sizeof(int));
        sk.per_flag = J;
    }
    // small groups: all J products in one launch with the intermediates in shared memory
    if (small) {
        r = modeprod_f64_chain(Vn_new_all, M, C_all, G, J, n, sk, st);
        if (r != CHEB_EUNSUPPORTED) return r;
    }
    const double *src = Vn_new_all;
    double *bufs[2] = {tmp0, tmp1};
    for (int t = 0; t < J; ++t) {
        double *dst = (t == J - 1) ? C_all : bufs[t & 1];
        if ((r = modeprod_f64_slabs(src, M, dst, G, NP / n, n, n, sk, st))) return r;
        src = dst;
    }
    return CHEB_OK;
}

cheb_status solve_group(cheb_ctx *ctx, int J, int n, int NP, int prec, int general, int n_u,
                        const std::vector<int> &members, const cheb_game_params *params,
                        const cheb_game_opts *opts, cheb_game_result *res, cudaStream_t st)
{
    const int B = (int)members.size();
    const size_t per = (size_t)J * NP;       // doubles per instance per array
    // All arrays are contiguous across the group (instance-major) so that the
    // refit sees one (B J, n, .., n) tensor.
    const size_t arr = sizeof(double) * per * B;
    const size_t tc_bytes = game_tc_workspace_bytes(J, n, NP, B, prec);
    size_t bytes = 0;
    auto rnd = [](size_t x) { return (x + 255) & ~size_t(255); };
    const bool any_df = prec == CHEB_DF64 || (prec != CHEB_FP64 && opts[members[0]].polish_fp64 == 1);
    // split-precision groups refit in double-float from (hi, lo) pairs of Vn_new
    const bool df_refit = prec != CHEB_FP64 && prec != CHEB_DF64;
    bytes += 9 * rnd(arr) + (any_df ? rnd(arr) : 0) + (df_refit ? rnd(arr) : 0) + rnd(sizeof(double) * 128) +
             rnd(sizeof(GameDev) * B) + rnd(sizeof(GameStat) * B) + rnd(tc_bytes);
    cheb_status r = ctx->game.reserve(bytes);
    if (r) return r;
    uint8_t *base = static_cast<uint8_t *>(ctx->game.ptr);
    size_t off = 0;
    auto take = [&](size_t nbytes) {
        uint8_t *p = base + off;
        off += rnd(nbytes);
        return p;
    };
    double *C_all = reinterpret_cast<double *>(take(arr));
    double *u_all = reinterpret_cast<double *>(take(arr));
    double *Vn_all = reinterpret_cast<double *>(take(arr));
    double *u_new_all = reinterpret_cast<double *>(take(arr));
    double *Vn_new_all = reinterpret_cast<double *>(take(arr));
    double *X_all = reinterpret_cast<double *>(take(arr));
    double *fit0 = reinterpret_cast<double *>(take(arr));
    double *fit1 = reinterpret_cast<double *>(take(arr));
    double *init = reinterpret_cast<double *>(take(arr));
    double *nodes = reinterpret_cast<double *>(take(sizeof(double) * 128));
    GameDev *d_inst = reinterpret_cast<GameDev *>(take(sizeof(GameDev) * B));
    GameStat *d_stat = reinterpret_cast<GameStat *>(take(sizeof(GameStat) * B));
    uint8_t *tc_ws = take(tc_bytes);
    float *Cdf_all = any_df ? reinterpret_cast<float *>(take(arr)) : nullptr;   // (hi, lo) per coefficient
    float *Vdf_all = df_refit ? reinterpret_cast<float *>(take(arr)) : nullptr;  // (hi, lo) per nodal value
    (void)init;

    // nodes cos(pi k / N) (the integer argument is exact); for the general
    // method the control nodes follow them in the same buffer
    std::vector<double> hn(n + (general ? n_u : 0));
    for (int k = 0; k < n; ++k) hn[k] = std::cos(M_PI * (double)k / (double)(n - 1));
    for (int k = 0; general && k < n_u; ++k) hn[n + k] = std::cos(M_PI * (double)k / (double)(n_u - 1));
    CHEB_CUDA_TRY(cudaMemcpyAsync(nodes, hn.data(), sizeof(double) * hn.size(), cudaMemcpyHostToDevice, st));
    // general method: the g-interpolants and two workspaces for their fit
    double *Gc_all = nullptr, *gtmp0 = nullptr, *gtmp1 = nullptr;
    const double *Mu = nullptr;
    size_t gc_per = 0;
    if (general) {
        int64_t NU = 1;
        for (int s = 0; s < J; ++s) NU *= n_u;
        gc_per = (size_t)NP * J * NU;
        const size_t gbytes = sizeof(double) * gc_per * B;
        if ((double)gbytes * 3.0 > 48e9)
            return fail(CHEB_EUNSUPPORTED, "game_solve: the g-interpolants of this batch need more than 48 GB");
        if ((r = ctx->game_aux.reserve(3 * ((gbytes + 255) & ~size_t(255))))) return r;
        uint8_t *gb = static_cast<uint8_t *>(ctx->game_aux.ptr);
        Gc_all = reinterpret_cast<double *>(gb);
        gtmp0 = reinterpret_cast<double *>(gb + ((gbytes + 255) & ~size_t(255)));
        gtmp1 = reinterpret_cast<double *>(gb + 2 * ((gbytes + 255) & ~size_t(255)));
        if ((r = dct_matrix(ctx, n_u, &Mu))) return r;
    }

    std::vector<GameDev> hinst(B);
    std::vector<GameStat> hstat(B);
    bool any_v0 = false, any_u0 = false;
    int64_t max_iter = 0;
    for (int q = 0; q < B; ++q) {
        const int b = members[q];
        const cheb_game_params &p = params[b];
        const cheb_game_opts &o = opts[b];
        GameDev &g = hinst[q];
        std::memset(&g, 0, sizeof(g));
        g.J = J;
        g.n = n;
        g.NP = NP;
        for (int t = 0; t < J * J; ++t) g.K[t] = p.K[t];
        g.minv = 1.0 / p.m;
        for (int t = 0; t < J; ++t) {
            g.A[t] = p.A[t];
            g.beta[t] = p.beta[t];
            g.phi[t] = p.phi[t];
            g.c[t] = p.c[t];
        }
        g.h = o.h;
        g.delta = 1.0 - p.rho * o.h;
        g.P_M = o.P_M;
        g.two_over_PM = 2.0 / o.P_M;
        for (int t = 0; t < J; ++t) {
            g.slope[t] = 2.0 * o.h * p.beta[t] / o.P_M;
            g.hA[t] = o.h * p.A[t];
            g.hphi2[t] = -0.5 * o.h * p.phi[t];
        }
        g.U_M = o.U_M;
        g.tol = o.tol;
        g.max_iter = o.max_iter;
        g.polish = o.polish_fp64 != 0;
        g.polish_mode = o.polish_fp64 == 2 ? 0 : 2;
        g.Cdf = Cdf_all ? Cdf_all + 2 * per * q : nullptr;
        g.Vdf = Vdf_all ? Vdf_all + 2 * per * q : nullptr;
        g.stall_window = 200;
        g.C = C_all + per * q;
        g.u = u_all + per * q;
        g.Vn = Vn_all + per * q;
        g.u_new = u_new_all + per * q;
        g.Vn_new = Vn_new_all + per * q;
        g.X = X_all + per * q;
        g.nodes = nodes;
        g.general = general;
        g.n_u = general ? n_u : 0;
        for (int t = 0; t < J * J; ++t) g.gamma[t] = (t % (J + 1) == 0) ? 0.0 : p.gamma[t];
        g.Gc = general ? Gc_all + gc_per * q : nullptr;
        g.Mu = Mu;
        g.unodes = general ? nodes + n : nullptr;
        g.V0 = res[b].V0;
        g.u0 = res[b].u0;
        any_v0 |= res[b].V0 != nullptr;
        any_u0 |= res[b].u0 != nullptr;
        max_iter = std::max<int64_t>(max_iter, o.max_iter);
        GameStat &s = hstat[q];
        std::memset(&s, 0, sizeof(s));
        s.best_res = INFINITY;
        s.last_res = INFINITY;
        s.mode = prec == CHEB_FP64 ? 0 : prec == CHEB_DF64 ? 2 : 1;
        s.mode_initial = s.mode;
        s.warm = (res[b].V0 != nullptr || res[b].u0 != nullptr) ? 1 : 0;
        s.status = CHEB_ENOCONV;
    }
    game_tc_bind(hinst.data(), B, J, n, NP, prec, tc_ws);
    CHEB_CUDA_TRY(cudaMemcpyAsync(d_inst, hinst.data(), sizeof(GameDev) * B, cudaMemcpyHostToDevice, st));
    CHEB_CUDA_TRY(cudaMemcpyAsync(d_stat, hstat.data(), sizeof(GameStat) * B, cudaMemcpyHostToDevice, st));

    // ---- Step 0: initial nodal values and controls, fit ----
    const unsigned copy_blocks = (unsigned)std::min<int64_t>(((int64_t)per + 255) / 256, 256);
    init_state_kernel<<<dim3(copy_blocks, B), 256, 0, st>>>(d_inst, any_v0, any_u0);
    CHEB_CUDA_TRY(cudaGetLastError());
    if ((r = refit_group(ctx, B * J, J, n, NP, Vn_new_all, Vdf_all, C_all, fit0, fit1, nullptr, st))) return r;
    if (general && (r = game_general_prepare(ctx, d_inst, B, J, NP, n_u, Gc_all, gtmp0, gtmp1, st))) return r;

    // ---- one iteration ----
    // next states: 32-thread blocks for small groups, so that their FP64 work
    // spreads over the SMs
    const int ns_threads = (int64_t)NP * B <= 32768 ? 32 : 128;
    const unsigned node_blocks = (unsigned)((NP + ns_threads - 1) / ns_threads);
    // the FP64 player update: 32 nodes per block, their J - 1 Chebyshev rows and
    // w in shared memory
    const unsigned f64_blocks = (unsigned)((NP + kF64Nodes - 1) / kF64Nodes);
    const size_t f64_smem = sizeof(double) * (size_t)J * (size_t)n * kF64Nodes;
    {
        static PerDevice attr;
        cheb_status ra = per_device_once(attr, [](int *) -> cheb_status {
            CHEB_CUDA_TRY(cudaFuncSetAttribute(player_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(double) * 4 * kGameNMax * kF64Nodes)));
            return CHEB_OK;
        }, nullptr);
        if (ra) return ra;
    }
    auto enqueue_iteration = [&](cudaStream_t s) -> cheb_status {
        cheb_status e;
        if (any_v0 || any_u0) {
            restart_kernel<<<dim3(copy_blocks, B), 256, 0, s>>>(d_inst, d_stat);
            CHEB_CUDA_TRY(cudaGetLastError());
        }
        if (general) {
            // Steps 1-3 of the general method (FP64), then the common refit and commit
            if ((e = game_general_player(d_inst, d_stat, B, J, NP, s))) return e;
        } else {
            ProfScope prof("game_next_state", s);
            next_state_kernel<<<dim3(node_blocks, B), ns_threads, 0, s>>>(d_inst, d_stat);
        }
        CHEB_CUDA_TRY(cudaGetLastError());
        const bool split = prec != CHEB_FP64 && prec != CHEB_DF64;
        if (split) {
            if ((e = game_tc_player(ctx, d_inst, d_stat, hinst.data(), B, J, n, NP, prec, tc_ws, s))) return e;
        }
        if (prec == CHEB_DF64 || (split && hinst[0].polish && hinst[0].polish_mode == 2)) {
            if ((e = game_df_player(d_inst, d_stat, B, J, NP, s))) return e;
        }
        if (!general && (prec == CHEB_FP64 || (split && hinst[0].polish && hinst[0].polish_mode == 0))) {
            ProfScope prof("game_player_f64", s);
            player_f64_kernel<<<dim3(f64_blocks, J, B), 128, f64_smem, s>>>(d_inst, d_stat);
        }
        CHEB_CUDA_TRY(cudaGetLastError());
        if ((e = refit_group(ctx, B * J, J, n, NP, Vn_new_all, Vdf_all, C_all, fit0, fit1, d_stat, s))) return e;
        {
            ProfScope prof("game_commit_copy", s);
            commit_copy_kernel<<<dim3(copy_blocks, B), 256, 0, s>>>(d_inst, d_stat);
        }
        {
            ProfScope prof("game_commit_stat", s);
            commit_stat_kernel<<<(B + 127) / 128, 128, 0, s>>>(d_inst, d_stat, B);
        }
        CHEB_CUDA_TRY(cudaGetLastError());
        return CHEB_OK;
    };

    // ---- tile shapes of the split player update, timed on this group ----
    if (prec != CHEB_FP64 && prec != CHEB_DF64) {
        next_state_kernel<<<dim3(node_blocks, B), ns_threads, 0, st>>>(d_inst, d_stat);
        CHEB_CUDA_TRY(cudaGetLastError());
        if ((r = game_tc_tune(ctx, d_inst, d_stat, B, J, n, prec, st))) return r;
    }

    // ---- chunks of iterations, captured once into a CUDA graph; with kernel
    // timing on, the timing events become event-record nodes of the graph, so
    // the kernels are timed where the graph runs them (the last chunk's launches)
    const int chunk = (int)std::min<int64_t>(max_iter, 32);
    cudaGraphExec_t exec = nullptr;
    {
        cudaStream_t cs = nullptr;
        CHEB_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) {
            cudaStreamDestroy(cs);
            return cuda_fail(ce, "cudaStreamBeginCapture");
        }
        for (int t = 0; t < chunk && r == CHEB_OK; ++t) r = enqueue_iteration(cs);
        ce = cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    }
    GameStat *hs = nullptr;
    CHEB_CUDA_TRY(cudaMallocHost(&hs, sizeof(GameStat) * B * 2));
    cudaEvent_t ev[2];
    cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
    auto launch_chunk = [&](int slot) -> cheb_status {
        CHEB_CUDA_TRY(cudaGraphLaunch(exec, st));
        CHEB_CUDA_TRY(cudaMemcpyAsync(hs + slot * B, d_stat, sizeof(GameStat) * B, cudaMemcpyDeviceToHost, st));
        CHEB_CUDA_TRY(cudaEventRecord(ev[slot], st));
        return CHEB_OK;
    };
    // one chunk stays queued ahead of the one whose status is being read; every
    // instance is marked done at max_iter, so at most max_iter / chunk + 2 chunks run
    const int64_t max_chunks = max_iter / chunk + 2;
    int64_t launched = 0;
    int slot = 0;
    r = launch_chunk(0);
    ++launched;
    while (r == CHEB_OK) {
        bool queued_next = false;
        if (launched < max_chunks) {
            r = launch_chunk(slot ^ 1);
            ++launched;
            queued_next = true;
            if (r) break;
        }
        cudaError_t ce = cudaEventSynchronize(ev[slot]);
        if (ce != cudaSuccess) {
            r = cuda_fail(ce, "game iteration");
            break;
        }
        bool all_done = true;
        for (int q = 0; q < B; ++q) all_done &= hs[slot * B + q].done != 0;
        if (all_done || !queued_next) {
            if (!all_done) {
                r = fail(CHEB_ENOCONV, "game_solve: iteration budget exhausted");
            }
            break;
        }
        slot ^= 1;
    }
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess && r == CHEB_OK) r = cuda_fail(ce, "game iteration");
    if (exec) cudaGraphExecDestroy(exec);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (r == CHEB_OK || r == CHEB_ENOCONV) {
        // the status after the last chunk that ran (later chunks only skip)
        CHEB_CUDA_TRY(cudaMemcpy(hs, d_stat, sizeof(GameStat) * B, cudaMemcpyDeviceToHost));
        int err = 0;
        CHEB_CUDA_TRY(cudaMemcpy(&err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
        for (int q = 0; q < B; ++q) {
            const int b = members[q];
            const GameStat &s = hs[q];
            res[b].iters = s.iters;
            res[b].iters_split = s.iters_split;
            res[b].residual = s.last_res;
            res[b].restarts = s.restarts;
            res[b].status = s.done ? s.status : CHEB_ENOCONV;
            if (err) res[b].status = err;
            CHEB_CUDA_TRY(cudaMemcpyAsync(res[b].V, hinst[q].C, sizeof(double) * per, cudaMemcpyDeviceToDevice, st));
            CHEB_CUDA_TRY(cudaMemcpyAsync(res[b].u, hinst[q].u, sizeof(double) * per, cudaMemcpyDeviceToDevice, st));
            if (res[b].Vn)
                CHEB_CUDA_TRY(cudaMemcpyAsync(res[b].Vn, hinst[q].Vn, sizeof(double) * per, cudaMemcpyDeviceToDevice, st));
        }
        CHEB_CUDA_TRY(cudaStreamSynchronize(st));
        r = CHEB_OK;
    }
    cudaFreeHost(hs);
    return r;
}

}  // namespace game
}  // namespace cheb

using namespace cheb;
using namespace cheb::game;

extern "C" CHEB_API cheb_status game_solve(cheb_ctx *ctx, int32_t batch, const cheb_game_params *params,
                                           const cheb_game_opts *opts, cheb_game_result *res, void *stream)
{
    NvtxRange nvtx_range("game_solve");
    tl_ctx = ctx;
    if (!ctx) return fail(CHEB_EINVAL, "null context");
    if (batch < 1 || !params || !opts || !res) return fail(CHEB_EINVAL, "game_solve: bad batch or null arrays");
    CHEB_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct Key {
        int J, n, prec, general, n_u;
        std::vector<int> members;
    };
    std::vector<Key> groups;
    for (int b = 0; b < batch; ++b) {
        const cheb_game_params &p = params[b];
        const cheb_game_opts &o = opts[b];
        if (p.J < 1 || p.J > 4) return fail(CHEB_EINVAL, "game_solve: J must be in [1, 4]");
        if (o.n < 3 || o.n > kGameNMax) return fail(CHEB_EINVAL, "game_solve: n must be in [3, 33]");
        bool coupled = false;
        for (int x = 0; x < p.J; ++x)
            for (int y = 0; y < p.J; ++y)
                if (x != y && p.gamma[x * p.J + y] != 0.0) coupled = true;
        for (int t = 0; t < p.J * p.J; ++t)
            if (!std::isfinite(p.gamma[t])) return fail(CHEB_EINVAL, "game_solve: gamma not finite");
        if (o.g_interp < 0 || o.g_interp > 1) return fail(CHEB_EINVAL, "game_solve: g_interp must be 0 or 1");
        const int general = (coupled || o.g_interp) ? 1 : 0;
        const int n_u = general ? (o.n_u == 0 ? o.n : o.n_u) : 0;
        if (general) {
            if (n_u < 2 || n_u > kGameNMax)
                return fail(CHEB_EINVAL, "game_solve: the general method needs 2 <= n_u <= 33");
            if (o.prec != CHEB_FP64)
                return fail(CHEB_EUNSUPPORTED, "game_solve: coupled dynamics (the general method) run in CHEB_FP64 only");
        } else if (o.n_u != 0 && o.n_u < o.n) {
            return fail(CHEB_EUNSUPPORTED, "game_solve: n_u must be 0 or >= n (exact control interpolant)");
        }
        if (!(o.h > 0) || !(p.rho > 0) || !(p.rho * o.h < 1) || !(o.P_M > 0) || !(o.U_M > 0) || !(p.m > 0) ||
            !(o.tol >= 0) || o.max_iter < 1)
            return fail(CHEB_EINVAL,
                        "game_solve: need h, rho, P_M, U_M, m > 0, rho h < 1, tol >= 0, max_iter >= 1");
        if (o.prec < CHEB_FP64 || o.prec > CHEB_DF64) return fail(CHEB_EINVAL, "game_solve: bad precision");
        if (o.polish_fp64 < 0 || o.polish_fp64 > 2) return fail(CHEB_EINVAL, "game_solve: polish_fp64 must be 0, 1 or 2");
        if (o.prec != CHEB_FP64 && o.prec != CHEB_DF64 && !tc_shape_supported(p.J, o.n))
            return fail(CHEB_EUNSUPPORTED,
                        "game_solve: the split forms need J in {2, 3} with n in {5, 9, 17, 33}, or J = 4 with n in {5, 9}");
        for (int t = 0; t < p.J * p.J; ++t)
            if (!std::isfinite(p.K[t])) return fail(CHEB_EINVAL, "game_solve: K not finite");
        for (int t = 0; t < p.J; ++t)
            if (!std::isfinite(p.A[t]) || !std::isfinite(p.beta[t]) || !std::isfinite(p.phi[t]) ||
                !std::isfinite(p.c[t]) || !(p.phi[t] >= 0))
                return fail(CHEB_EINVAL, "game_solve: parameters must be finite, phi >= 0");
        if (!res[b].V || !res[b].u || res[b].V == res[b].u)
            return fail(CHEB_EINVAL, "game_solve: V and u must be distinct device buffers");
        res[b].status = CHEB_ENOCONV;
        res[b].iters = 0;
        res[b].iters_split = 0;
        bool found = false;
        for (auto &g : groups)
            if (g.J == p.J && g.n == o.n && g.prec == o.prec && g.general == general && g.n_u == n_u) {
                g.members.push_back(b);
                found = true;
                break;
            }
        if (!found) groups.push_back({p.J, o.n, o.prec, general, n_u, {b}});
    }
    for (auto &g : groups) {
        int NP = 1;
        for (int t = 0; t < g.J; ++t) NP *= g.n;
        const std::string label = "game_solve group J=" + std::to_string(g.J) + " n=" + std::to_string(g.n) +
                                  " prec=" + std::to_string(g.prec) + " batch=" + std::to_string(g.members.size());
        NvtxRange group_range(label.c_str());
        cheb_status r = solve_group(ctx, g.J, g.n, NP, g.prec, g.general, g.n_u, g.members, params, opts, res, st);
        if (r) return r;
    }
    cheb_status first = CHEB_OK;
    for (int b = 0; b < batch; ++b)
        if (res[b].status != CHEB_OK && first == CHEB_OK) first = (cheb_status)res[b].status;
    if (first != CHEB_OK) fail(first, "game_solve: an instance did not converge (see res[].status)");
    return first;
}
