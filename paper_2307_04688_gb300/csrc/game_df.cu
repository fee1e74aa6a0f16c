// Double-float player update of the game iteration (Section 3.4, Steps 1-3):
// the FP64 player update carried out on GB300's FP32 pipe.
//
// GB300 runs FP64 at about 1.25 TFLOP/s, two orders of magnitude below its
// FP32 rate, and the FP64 player update is its slowest stage (n^J FMAs per
// node and player for the series, and a Newton search per node). Here every
// value is a pair of FP32 numbers hi + lo (about 48 significant bits):
// products are error-free (hi*hi exact by fma, plus the cross terms), sums
// compensated (two-sum), so the series w_j[k] and the value at the maximiser
// carry relative errors of a few 1e-14 while using FP32 instructions only.
//  - coefficients: split once per iteration into (hi, lo) pairs by
//    game_coef_df_kernel (the refit of an FP64 or double-float solve stays
//    FP64; split-precision solves refit in double-float, refit_df_kernel);
//  - T_k of the next states by the three-term recurrence in double-float;
//  - the contraction as in the FP64 kernel (last mode innermost), each inner
//    dot product accumulated unnormalised (the rounding errors of the sums
//    and products collected in the low word), renormalised once per dot;
//  - Step 3: projected Newton in FP32 from the previous control, then two
//    double-float Newton steps at a concave interior point (the control must
//    be accurate to about 1e-13: it moves the other players' next states);
//    as in the FP64 update the Newton point and the two bounds compete, their
//    values in double-float. The residual is FP64.
#include <algorithm>
#include <cmath>
#include <string>

#include "game_internal.cuh"

namespace cheb {
namespace game {
namespace {

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl df_of(double x)
{
    dfl r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double df_val(dfl a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dfl df_norm(float s, float e)
{
    dfl r;
    r.hi = s + e;
    r.lo = e - (r.hi - s);
    return r;
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const float s = a.hi + b.hi, bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    return df_norm(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm(p, e);
}

__device__ __forceinline__ dfl df_scale(dfl a, float s) { return {a.hi * s, a.lo * s}; }   // s a power of two

// Running sum of products: hi is the plain FP32 sum, lo collects the rounding
// error of every sum and product (renormalised by the caller).
struct dacc {
    float hi = 0.0f, lo = 0.0f;
};

__device__ __forceinline__ void df_mac(dacc &acc, dfl a, dfl b)
{
    const float p = a.hi * b.hi;
    float pe = fmaf(a.hi, b.hi, -p);
    pe = fmaf(a.hi, b.lo, pe);
    pe = fmaf(a.lo, b.hi, pe);
    const float s = acc.hi + p, bb = s - acc.hi;
    acc.lo += ((acc.hi - (s - bb)) + (p - bb)) + pe;
    acc.hi = s;
}

__device__ __forceinline__ dfl df_done(const dacc &a) { return df_norm(a.hi, a.lo); }

// The Bellman objective along the next states as a function of the player's
// own control, W(u) = h (u (A - u/2) - phi pbar^2 / 2) + delta sum_m w_m T_m(x),
// x = xc + slope u, in FP32 with its first two derivatives (the Newton search).
__device__ __forceinline__ void objective_f32(const float *w, int n, float xc, float slope, float hA, float h,
                                              float delta, float u, float &W, float &W1, float &W2)
{
    const float x = xc + slope * u;
    float t0 = 1.0f, t1 = x, d0 = 0.0f, d1 = 1.0f, e0 = 0.0f, e1 = 0.0f;
    float s = w[0] + (n > 1 ? w[1] * x : 0.0f), s1 = n > 1 ? w[1] : 0.0f, s2 = 0.0f;
    for (int m = 2; m < n; ++m) {
        const float t2 = 2.0f * x * t1 - t0;
        const float d2 = 2.0f * t1 + 2.0f * x * d1 - d0;
        const float e2 = 4.0f * d1 + 2.0f * x * e1 - e0;
        s = fmaf(w[m], t2, s);
        s1 = fmaf(w[m], d2, s1);
        s2 = fmaf(w[m], e2, s2);
        t0 = t1; t1 = t2;
        d0 = d1; d1 = d2;
        e0 = e1; e1 = e2;
    }
    W = hA * u - 0.5f * h * u * u + delta * s;
    W1 = hA - h * u + delta * slope * s1;
    W2 = -h + delta * slope * slope * s2;
}

// sum_m w_m T_m(x) and sum_m w_m T'_m(x) in double-float (T' by differentiating
// the recurrence: T'_m = 2 T_{m-1} + 2 x T'_{m-1} - T'_{m-2})
__device__ __forceinline__ void series_df(const dfl *w, int n, dfl x, dfl &S, dfl &S1)
{
    dfl t0 = {1.0f, 0.0f}, t1 = x, d0 = {0.0f, 0.0f}, d1 = {1.0f, 0.0f};
    dacc s, s1;
    df_mac(s, w[0], t0);
    if (n > 1) {
        df_mac(s, w[1], t1);
        df_mac(s1, w[1], d1);
    }
    for (int m = 2; m < n; ++m) {
        const dfl t2 = df_add(df_scale(df_mul(x, t1), 2.0f), df_neg(t0));
        const dfl d2 = df_add(df_add(df_scale(t1, 2.0f), df_scale(df_mul(x, d1), 2.0f)), df_neg(d0));
        df_mac(s, w[m], t2);
        df_mac(s1, w[m], d2);
        t0 = t1; t1 = t2;
        d0 = d1; d1 = d2;
    }
    S = df_done(s);
    S1 = df_done(s1);
}

__global__ void game_coef_df_kernel(const GameDev *__restrict__ insts, const GameStat *__restrict__ stats)
{
    if (stats[blockIdx.y].done || stats[blockIdx.y].mode != 2) return;
    const GameDev g = insts[blockIdx.y];
    const int total = g.J * g.NP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const dfl c = df_of(g.C[t]);
        g.Cdf[2 * t] = c.hi;
        g.Cdf[2 * t + 1] = c.lo;
    }
}

// Eight threads per (node, player): thread g of a node forms w[k] for
// k = g, g + 8, ..., the node's threads meet in shared memory and the first
// one runs Step 3 (the serial dot products need many warps to hide their
// latency; one thread per node leaves a few warps per SM).
constexpr int kDfGroup = 8;
constexpr int kDfNodes = 16;          // nodes per block of 128 threads

__global__ void __launch_bounds__(kDfGroup * kDfNodes)
game_player_df_kernel(const GameDev *__restrict__ insts, GameStat *__restrict__ stats)
{
    __shared__ float2 w_sm[kDfNodes][kGameNMax];     // w[k] of each node (double-float)
    __shared__ float wf_sm[kDfNodes][kGameNMax];     // and rounded to FP32 (the Newton search)
    __shared__ float2 T_sm[kDfNodes][3][kGameNMax];  // T_k of the next state in each other mode
    const int inst = blockIdx.z, i = blockIdx.y;
    GameStat *st = &stats[inst];
    if (st->done || st->mode != 2) return;
    const GameDev &g = insts[inst];
    const int nl = threadIdx.x / kDfGroup, grp = threadIdx.x % kDfGroup;
    const int j = blockIdx.x * kDfNodes + nl;
    const int J = g.J, n = g.n, NP = g.NP;
    // the node's rows fit the static arrays (uniform)
    if (!CHEB_DCHECK(n <= kGameNMax && J >= 2 && J <= 4)) return;
    const bool valid = j < NP;
    const int jc = valid ? j : NP - 1;
    // mode strides of C_i (row-major) and the modes other than i, by arithmetic
    // (no run-time indexed per-thread arrays)
    auto stride = [&](int s) {
        int v = 1;
        for (int r = s + 1; r < J; ++r) v *= n;
        return v;
    };
    auto other = [&](int t) { return t < i ? t : t + 1; };
    const int no = J - 1;
    // the node's T rows, one other mode per thread, shared by its eight threads,
    // by the double-float recurrence straight into shared memory
    if (grp < no) {
        const dfl xf = df_of(g.X[other(grp) * NP + jc]);
        dfl t0 = {1.0f, 0.0f}, t1 = xf;
        T_sm[nl][grp][0] = make_float2(1.0f, 0.0f);
        if (n > 1) T_sm[nl][grp][1] = make_float2(xf.hi, xf.lo);
        for (int k = 2; k < n; ++k) {
            const dfl t2 = df_add(df_scale(df_mul(xf, t1), 2.0f), df_neg(t0));
            T_sm[nl][grp][k] = make_float2(t2.hi, t2.lo);
            t0 = t1;
            t1 = t2;
        }
    }
    __syncthreads();
    auto Tq = [&](int q, int a) {
        const float2 v = T_sm[nl][q][a];
        return dfl{v.x, v.y};
    };
    const float2 *C = reinterpret_cast<const float2 *>(g.Cdf) + (size_t)i * NP;
    auto coef = [&](size_t idx) {
        const float2 v = __ldg(C + idx);
        return dfl{v.x, v.y};
    };
    // thread grp takes k = grp, grp + 8, ...; three of them at a time as three
    // independent chains (each w[k] summed in the same order as one at a time)
    const int si = stride(i);
    const int s0 = no > 0 ? stride(other(0)) : 0, s1 = no > 1 ? stride(other(1)) : 0,
              s2 = no > 2 ? stride(other(2)) : 0;
    for (int m0 = grp; m0 < n; m0 += 3 * kDfGroup) {
        const int left = (n - m0 + kDfGroup - 1) / kDfGroup;
        const int kb = left < 3 ? left : 3;
        size_t ck[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) ck[r] = (size_t)(m0 + r * kDfGroup) * si;
        dfl wk[3];
        if (no == 0) {
#pragma unroll
            for (int r = 0; r < 3; ++r)
                if (r < kb) wk[r] = coef(ck[r]);
        } else if (no == 1) {
            dacc acc[3];
            for (int a = 0; a < n; ++a) {
                const dfl ta = Tq(0, a);
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    if (r < kb) df_mac(acc[r], coef(ck[r] + (size_t)a * s0), ta);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) wk[r] = df_done(acc[r]);
        } else if (no == 2) {
            dacc acc[3];
            for (int a = 0; a < n; ++a) {
                dacc t[3];
                for (int b = 0; b < n; ++b) {
                    const dfl tb = Tq(1, b);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        if (r < kb) df_mac(t[r], coef(ck[r] + (size_t)a * s0 + (size_t)b * s1), tb);
                }
                const dfl ta = Tq(0, a);
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    if (r < kb) df_mac(acc[r], df_done(t[r]), ta);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) wk[r] = df_done(acc[r]);
        } else {
            dacc acc[3];
            for (int a = 0; a < n; ++a) {
                dacc ta[3];
                for (int b = 0; b < n; ++b) {
                    dacc t[3];
                    for (int c = 0; c < n; ++c) {
                        const dfl tc = Tq(2, c);
#pragma unroll
                        for (int r = 0; r < 3; ++r)
                            if (r < kb)
                                df_mac(t[r], coef(ck[r] + (size_t)a * s0 + (size_t)b * s1 + (size_t)c * s2), tc);
                    }
                    const dfl tb = Tq(1, b);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        if (r < kb) df_mac(ta[r], df_done(t[r]), tb);
                }
                const dfl tA = Tq(0, a);
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    if (r < kb) df_mac(acc[r], df_done(ta[r]), tA);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) wk[r] = df_done(acc[r]);
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (r < kb) {
                const int k = m0 + r * kDfGroup;
                w_sm[nl][k] = make_float2(wk[r].hi, wk[r].lo);
                wf_sm[nl][k] = wk[r].hi + wk[r].lo;
            }
    }
    __syncwarp();       // a node's eight threads share a warp
    if (grp != 0 || !valid) return;
    const dfl *w = reinterpret_cast<const dfl *>(w_sm[nl]);
    const float *wf = wf_sm[nl];
    // Step 3
    double xr[4], pb[4];
    node_coords(g, j, xr, pb);
    const double ui = g.u[i * NP + j];
    const double slope = g.slope[i];
    const double xc = g.X[i * NP + j] - slope * ui;
    const double hA = g.hA[i];
    const double hG0 = g.hphi2[i] * pb[i] * pb[i];
    const float U_M = (float)g.U_M;
    float u = fminf(fmaxf((float)ui, 0.0f), U_M);
    float W, W1, W2;
    for (int it = 0; it < 30; ++it) {
        objective_f32(wf, n, (float)xc, (float)slope, (float)hA, (float)g.h, (float)g.delta, u, W, W1, W2);
        float un = (W2 < 0.0f) ? u - W1 / W2 : (W1 > 0.0f ? 0.5f * (u + U_M) : 0.5f * u);
        un = fminf(fmaxf(un, 0.0f), U_M);
        const float step = fabsf(un - u);
        u = un;
        if (step <= 1e-7f * U_M) break;
    }
    objective_f32(wf, n, (float)xc, (float)slope, (float)hA, (float)g.h, (float)g.delta, u, W, W1, W2);
    const dfl xcd = df_of(xc), sld = df_of(slope), hAd = df_of(hA), hd = df_of(g.h), dd = df_of(g.delta);
    // W and W' at a control in double-float
    auto value = [&](dfl uu, dfl *W1o) {
        dfl S, S1;
        series_df(w, n, df_add(xcd, df_mul(sld, uu)), S, S1);
        const dfl hu = df_mul(hd, uu);
        if (W1o) *W1o = df_add(df_add(hAd, df_neg(hu)), df_mul(df_mul(dd, sld), S1));
        // h A u - h u^2 / 2 + delta S (+ hG0, added in FP64)
        return df_add(df_add(df_mul(hAd, uu), df_neg(df_scale(df_mul(hu, uu), 0.5f))), df_mul(dd, S));
    };
    // a concave interior Newton point is refined by two Newton steps in
    // double-float on W' (W'' from FP32 suffices for the step); then, as in
    // the FP64 update, the bounds and the Newton point compete, ties to the
    // smaller control
    dfl ud = df_of((double)u);
    if (u > 0.0f && u < U_M && W2 < 0.0f) {
        for (int it = 0; it < 2; ++it) {
            dfl W1d;
            value(ud, &W1d);
            ud = df_add(ud, df_of(-df_val(W1d) / (double)W2));
        }
    }
    double us = fmin(fmax(df_val(ud), 0.0), g.U_M);
    double bu = 0.0, V = df_val(value(dfl{0.0f, 0.0f}, nullptr)) + hG0;
    {
        const double vn = df_val(value(df_of(us), nullptr)) + hG0;
        if (vn > V) { V = vn; bu = us; }
        const double vm = df_val(value(df_of(g.U_M), nullptr)) + hG0;
        if (vm > V) { V = vm; bu = g.U_M; }
    }
    us = bu;
    us = fmin(fmax(us, 0.0), g.U_M);
    g.u_new[i * NP + j] = us;
    store_vn_new(g, i * NP + j, V);
    const double d = fabs(V - g.Vn[i * NP + j]);
    atomicMax(&st->res_bits, (unsigned long long)__double_as_longlong(d));
}

// ---- double-float refit (split-precision solves) ------------------------------
// One mode of the refit (Section 3.4, Step 4: eq. (forcoef) along one mode)
// on the FP32 pipe, the same slab-wise product as the FP64 refit:
// out[(g n + j) R + r] = sum_k M[j, k] X[g R + r, k] over G slabs (slab g =
// player g % J of instance g / J) of R rows, slabs of finished instances
// skipped (stats null: none). The input is double-float pairs: the players'
// (hi, lo) split of Vn_new for the first mode, then the previous mode's
// output (8 bytes per value, like the FP64 values they replace); the last
// mode writes FP64 coefficients (OUT_D). A block takes 64 rows and all
// 4Q >= n output columns; each thread one row and Q columns, every product
// error-free and every sum compensated, so a coefficient carries a relative
// error of about 2^-47 (the split forms' own is above 2^-24).
constexpr int kRfRows = 64, kRfThreads = 256;

template <int Q, bool OUT_D>
__global__ void __launch_bounds__(kRfThreads, 4)
refit_df_kernel(const dfl *__restrict__ X, const double *__restrict__ M, void *__restrict__ outv, int64_t G,
                int64_t R, int n, const GameStat *__restrict__ stats, int J)
{
    extern __shared__ dfl rsm[];
    const int ns = n | 1;
    dfl *sX = rsm;
    dfl *sM = rsm + kRfRows * ns;
    const int64_t total = G * R;
    const int64_t r0 = (int64_t)blockIdx.x * kRfRows;
    const int rows = (int)((total - r0) < kRfRows ? (total - r0) : kRfRows);
    // the staged rows and columns fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK(sizeof(dfl) * (size_t)(kRfRows * ns + 4 * Q * n) <= dyn_smem_bytes() && r0 < total)) return;
    if (stats) {
        bool any = false;
        for (int64_t g = r0 / R; g <= (r0 + rows - 1) / R; ++g) any = any || !stats[g / J].done;
        if (!any) return;     // uniform across the block
    }
    for (int t = threadIdx.x; t < rows * n; t += blockDim.x) {
        const int rr = t / n, k = t - rr * n;
        sX[rr * ns + k] = X[r0 * n + t];
    }
    for (int t = threadIdx.x; t < (kRfRows - rows) * n; t += blockDim.x) {
        const int rr = rows + t / n, k = t % n;
        sX[rr * ns + k] = {0.0f, 0.0f};
    }
    for (int t = threadIdx.x; t < 4 * Q * n; t += blockDim.x) {
        const int jj = t / n, k = t - jj * n;
        sM[t] = jj < n ? df_of(M[jj * n + k]) : dfl{0.0f, 0.0f};
    }
    __syncthreads();
    const int tr = threadIdx.x & (kRfRows - 1);
    const int tj = threadIdx.x / kRfRows;
    dacc acc[Q];
    for (int k = 0; k < n; ++k) {
        const dfl xv = sX[tr * ns + k];
#pragma unroll
        for (int q = 0; q < Q; ++q) df_mac(acc[q], sM[(tj + 4 * q) * n + k], xv);
    }
    if (tr < rows) {
        const int64_t rg = r0 + tr, g = rg / R, r = rg - g * R;
        if (!stats || !stats[g / J].done) {
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = tj + 4 * q;
                if (j >= n) continue;
                const dfl v = df_done(acc[q]);
                const int64_t o = (g * n + j) * R + r;
                if (OUT_D)
                    static_cast<double *>(outv)[o] = df_val(v);
                else
                    static_cast<dfl *>(outv)[o] = v;
            }
        }
    }
}

template <int Q>
cheb_status refit_df_mode(const dfl *X, const double *M, void *out, bool out_d, int64_t G, int64_t R, int n,
                          const GameStat *stats, int J, cudaStream_t st)
{
    const int64_t tiles = (G * R + kRfRows - 1) / kRfRows;
    if (tiles > 0x7fffffffLL) return fail(CHEB_EUNSUPPORTED, "refit: too many rows");
    const size_t smem = sizeof(dfl) * (size_t)(kRfRows * (n | 1) + 4 * Q * n);
    const unsigned grid = (unsigned)tiles;
    if (out_d)
        refit_df_kernel<Q, true><<<grid, kRfThreads, smem, st>>>(X, M, out, G, R, n, stats, J);
    else
        refit_df_kernel<Q, false><<<grid, kRfThreads, smem, st>>>(X, M, out, G, R, n, stats, J);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

// All J modes of the double-float refit of a slab in one CTA per (slab g,
// last output index k_J), for small groups (a single game refits 3 slabs:
// the J launches above would leave most SMs idle and each pay a launch).
// The first product (the last mode) is taken for this k_J only and the other
// J - 1 run on the resulting n^(J-1) pairs in shared memory, each moving its
// new index to the front as refit_df_kernel does. Every output is the same
// compensated dot product over k in the same order, and every intermediate
// the same renormalised pair, as in the J launches of refit_df_kernel, so the
// coefficients are bit-identical to game_refit_df's.
constexpr int kRfChainMax = 4913;   // largest n^(J-1) held in shared memory
constexpr int kRfChainThreads = 256;

__global__ void __launch_bounds__(kRfChainThreads)
refit_df_chain_kernel(const dfl *__restrict__ V, const double *__restrict__ M, double *__restrict__ C, int J, int n,
                      const GameStat *__restrict__ stats)
{
    extern __shared__ dfl chain_df[];
    const int kJ = blockIdx.x;
    const int64_t g = blockIdx.y;
    if (stats && stats[g / J].done) return;
    int R = 1;
    for (int s = 0; s < J - 1; ++s) R *= n;
    dfl *sM = chain_df;
    dfl *cur = sM + n * n, *nxt = cur + R;
    // M and the two intermediates fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK(sizeof(dfl) * (size_t)(n * n + 2 * R) <= dyn_smem_bytes() && kJ < n)) return;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sM[t] = df_of(M[t]);
    __syncthreads();
    // the last mode: cur[r] = sum_k M[k_J, k] V_g[r, k]
    const dfl *Vg = V + g * (int64_t)R * n;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const dfl *xr = Vg + (int64_t)r * n;
        dacc acc;
        for (int k = 0; k < n; ++k) df_mac(acc, sM[kJ * n + k], xr[k]);
        cur[r] = df_done(acc);
    }
    __syncthreads();
    // the other modes: cur as [R / n rows x n], nxt[j (R / n) + r] = sum_k M[j, k] cur[r n + k]
    const int Rp = R / n;
    for (int step = 1; step < J; ++step) {
        for (int t = threadIdx.x; t < n * Rp; t += blockDim.x) {
            const int j = t / Rp, r = t - j * Rp;
            const dfl *xr = cur + r * n;
            dacc acc;
            for (int k = 0; k < n; ++k) df_mac(acc, sM[j * n + k], xr[k]);
            nxt[t] = df_done(acc);
        }
        __syncthreads();
        dfl *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    // cur = C_g[k_1 .. k_{J-1}, k_J] for this k_J, (k_1 .. k_{J-1}) row-major
    double *og = C + g * (int64_t)R * n;
    for (int t = threadIdx.x; t < R; t += blockDim.x) og[(int64_t)t * n + kJ] = df_val(cur[t]);
}

}  // namespace

bool game_refit_df_supported(int n) { return n == 5 || n == 9 || n == 17 || n == 33; }

cheb_status game_refit_df(const float *Vdf, const double *M, double *C, double *tmp0, double *tmp1, int G, int J,
                          int n, int NP, const GameStat *stats, cudaStream_t st)
{
    if (!game_refit_df_supported(n)) return fail(CHEB_EUNSUPPORTED, "double-float refit: n not in {5, 9, 17, 33}");
    const dfl *src = reinterpret_cast<const dfl *>(Vdf);
    double *bufs[2] = {tmp0, tmp1};
    ProfScope prof("game_refit_df n=" + std::to_string(n), st);
    for (int t = 0; t < J; ++t) {
        const bool last = t == J - 1;
        void *dst = last ? static_cast<void *>(C) : static_cast<void *>(bufs[t & 1]);
        const int64_t R = NP / n;
        cheb_status r;
        switch (n) {
        case 5: r = refit_df_mode<2>(src, M, dst, last, G, R, n, stats, J, st); break;
        case 9: r = refit_df_mode<3>(src, M, dst, last, G, R, n, stats, J, st); break;
        case 17: r = refit_df_mode<5>(src, M, dst, last, G, R, n, stats, J, st); break;
        default: r = refit_df_mode<9>(src, M, dst, last, G, R, n, stats, J, st); break;
        }
        if (r) return r;
        src = static_cast<const dfl *>(dst);
    }
    return CHEB_OK;
}

cheb_status game_refit_df_chain(const float *Vdf, const double *M, double *C, int G, int J, int n,
                                const GameStat *stats, cudaStream_t st)
{
    int64_t R = 1;
    for (int s = 0; s < J - 1; ++s) R *= n;
    if (J < 1 || n < 1 || R > kRfChainMax || G > 65535) return CHEB_EUNSUPPORTED;
    if (G <= 0) return CHEB_OK;
    static PerDevice attr;
    cheb_status r = per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(refit_df_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(dfl) * (kGameNMax * kGameNMax + 2 * kRfChainMax))));
        return CHEB_OK;
    }, nullptr);
    if (r) return r;
    const size_t smem = sizeof(dfl) * ((size_t)n * n + 2 * (size_t)R);
    ProfScope prof("game_refit_df_chain J=" + std::to_string(J) + " n=" + std::to_string(n) + " G=" + std::to_string(G),
                   st);
    refit_df_chain_kernel<<<dim3((unsigned)n, (unsigned)G), kRfChainThreads, smem, st>>>(
        reinterpret_cast<const dfl *>(Vdf), M, C, J, n, stats);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status game_df_player(const GameDev *d_inst, GameStat *d_stat, int B, int J, int NP, cudaStream_t st)
{
    const unsigned copy_blocks = (unsigned)std::min<int64_t>(((int64_t)J * NP + 255) / 256, 256);
    {
        ProfScope prof("game_coef_df", st);
        game_coef_df_kernel<<<dim3(copy_blocks, B), 256, 0, st>>>(d_inst, d_stat);
        CHEB_CUDA_TRY(cudaGetLastError());
    }
    const unsigned node_blocks = (unsigned)((NP + kDfNodes - 1) / kDfNodes);
    ProfScope prof("game_player_df", st);
    game_player_df_kernel<<<dim3(node_blocks, J, B), kDfGroup * kDfNodes, 0, st>>>(d_inst, d_stat);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

}  // namespace game
}  // namespace cheb
