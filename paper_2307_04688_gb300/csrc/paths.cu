// Equilibrium time paths (Section 4: the emission and pollution-stock paths
// along the equilibrium strategy).
//
// The feedback policy of player i is the Chebyshev interpolant of its nodal
// controls on [0, P_M]^J (fitted once by cheb_fit), clamped to [0, U_M]; from
// each initial stock the path takes T explicit steps of the dynamics with the
// discretisation's time step, p_{t+1} = p_t + h g(p_t, u(p_t)).
//
// Design (GB300): the trajectories are independent, one CTA each, and a CTA
// runs all T steps of its trajectory in one launch (no launch per step). A
// step evaluates the J interpolants at the current stock by contracting the
// coefficient tensor mode by mode in FP64 (the last mode against T(x_{J-1}),
// n^{J-1} dot products spread over the threads, then the next mode in shared
// memory), reading the coefficients from L2 (J n^J doubles, shared by all
// CTAs); thread 0 then applies the clamp and the step. FP64 because the path
// is the reference quality output of the solve; the work per step is
// J (n^J + n^{J-1} + ...) FMAs.
#include <algorithm>
#include <string>

#include "cheb_internal.cuh"

namespace cheb {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxN = 64;

struct PathParams {
    const double *coef;       // J x n^J coefficients of the controls (row-major, last player fastest)
    const double *p0;         // K x J initial stocks
    double *p_path;           // K x (T + 1) x J
    double *u_path;           // K x T x J, or null
    int64_t K, T;
    int J, n;
    int64_t len1;             // n^{J-1}
    double Kmat[16], minv, c[4], beta[4];
    double gamma[16];         // emission-interaction coupling (J x J)
    double h, P_M, U_M;
};

__global__ void __launch_bounds__(kThreads) game_paths_kernel(const PathParams P)
{
    extern __shared__ double sm[];
    double *Tr = sm;                                  // [J][kMaxN]: T_k(x_s)
    double *bufA = Tr + 4 * kMaxN;                    // n^{J-1}
    double *bufB = bufA + P.len1;                     // n^{J-2}
    __shared__ double ps[4], us[4];
    const int tid = threadIdx.x, J = P.J, n = P.n;
    const int64_t NP = P.len1 * n, T = P.T;
    // the rows and both contraction buffers fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK(sizeof(double) * (4 * (size_t)kMaxN + (size_t)P.len1 + (size_t)(P.len1 / n > 0 ? P.len1 / n : 1)) <=
                         dyn_smem_bytes() && n <= kMaxN && J <= 4))
        return;
    for (int64_t k = blockIdx.x; k < P.K; k += gridDim.x) {
        if (tid < J) {
            ps[tid] = P.p0[k * J + tid];
            P.p_path[k * (T + 1) * J + tid] = ps[tid];
        }
        __syncthreads();
        for (int64_t t = 0; t < T; ++t) {
            // T_0..T_{n-1} at x_s = 2 p_s / P_M - 1 (three-term recurrence, valid off [-1, 1])
            if (tid < J) {
                const double x = 2.0 * ps[tid] / P.P_M - 1.0;
                double *row = Tr + tid * kMaxN;
                double t0 = 1.0, t1 = x;
                row[0] = 1.0;
                if (n > 1) row[1] = x;
                for (int m = 2; m < n; ++m) {
                    const double t2 = 2.0 * x * t1 - t0;
                    row[m] = t2;
                    t0 = t1;
                    t1 = t2;
                }
            }
            __syncthreads();
            for (int i = 0; i < J; ++i) {
                // the last mode: n^{J-1} dot products with T(x_{J-1})
                const double *ci = P.coef + (int64_t)i * NP;
                const double *tl = Tr + (J - 1) * kMaxN;
                for (int64_t r = tid; r < P.len1; r += kThreads) {
                    const double *cr = ci + r * n;
                    double s = 0.0;
                    for (int q = 0; q < n; ++q) s = fma(__ldg(cr + q), tl[q], s);
                    bufA[r] = s;
                }
                __syncthreads();
                // the other modes, in shared memory
                int64_t len = P.len1;
                double *src = bufA, *dst = bufB;
                for (int mode = J - 2; mode >= 0; --mode) {
                    len /= n;
                    const double *tm = Tr + mode * kMaxN;
                    for (int64_t r = tid; r < len; r += kThreads) {
                        const double *sr = src + r * n;
                        double s = 0.0;
                        for (int q = 0; q < n; ++q) s = fma(sr[q], tm[q], s);
                        dst[r] = s;
                    }
                    __syncthreads();
                    double *tmp = src;
                    src = dst;
                    dst = tmp;
                }
                if (tid == 0) us[i] = fmin(fmax(src[0], 0.0), P.U_M);
                __syncthreads();
            }
            // the explicit step with g of Section 2.1 (neighbour sum over j != i)
            if (tid == 0) {
                double g[4];
                for (int a = 0; a < J; ++a) {
                    double coup = 0.0;
                    for (int b = 0; b < J; ++b)
                        if (b != a) coup += P.Kmat[a * J + b] * (ps[b] - ps[a]);
                    double inter = 0.0;
                    for (int b = 0; b < J; ++b)
                        if (b != a) inter += P.gamma[a * J + b] * us[b];
                    g[a] = coup * P.minv - P.c[a] * ps[a] + P.beta[a] * us[a] + us[a] * inter;
                }
                for (int a = 0; a < J; ++a) {
                    if (P.u_path) P.u_path[(k * T + t) * J + a] = us[a];
                    ps[a] += P.h * g[a];
                    P.p_path[(k * (T + 1) + t + 1) * J + a] = ps[a];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" CHEB_API cheb_status game_paths(cheb_ctx *ctx, const cheb_game_params *params,
                                           const cheb_game_opts *opts, const double *u_nodal, int64_t K,
                                           const double *p0, int64_t T, double *p_path, double *u_path,
                                           void *stream)
{
    NvtxRange nvtx_range("game_paths");
    if (!ctx) return fail(CHEB_EINVAL, "null context");
    tl_ctx = ctx;
    if (!params || !opts) return fail(CHEB_EINVAL, "game_paths: null params or opts");
    const int J = params->J, n = opts->n;
    if (J < 1 || J > 4) return fail(CHEB_EINVAL, "game_paths: J must be in [1, 4]");
    if (n < 2 || n > kMaxN) return fail(CHEB_EINVAL, "game_paths: n must be in [2, 64]");
    if (K < 0 || T < 0) return fail(CHEB_EINVAL, "game_paths: K and T must be >= 0");
    if (!(opts->h > 0.0) || !(opts->P_M > 0.0) || !(opts->U_M >= 0.0) || !(params->m > 0.0))
        return fail(CHEB_EINVAL, "game_paths: need h > 0, P_M > 0, U_M >= 0, m > 0");
    if (K == 0) return CHEB_OK;
    if (!u_nodal || !p0 || !p_path) return fail(CHEB_EINVAL, "game_paths: null array");
    int64_t len1 = 1;
    for (int s = 0; s < J - 1; ++s) len1 *= n;
    const int64_t NP = len1 * n;
    const size_t smem = sizeof(double) * (4 * (size_t)kMaxN + (size_t)len1 + (size_t)(len1 / n > 0 ? len1 / n : 1));
    if (smem > 200 * 1024)
        return fail(CHEB_EUNSUPPORTED, "game_paths: n^(J-1) too large for the per-CTA contraction (J = 4 needs n <= 24)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the controls' coefficients, player by player (Definition 3.2, eq. (forcoef))
    cheb_status r = ctx->paths.reserve(sizeof(double) * (size_t)J * (size_t)NP);
    if (r) return r;
    double *coef = static_cast<double *>(ctx->paths.ptr);
    int32_t nd[4] = {n, n, n, n};
    for (int i = 0; i < J; ++i)
        if ((r = cheb_fit(ctx, J, nd, u_nodal + (size_t)i * NP, coef + (size_t)i * NP, stream))) return r;
    tl_ctx = ctx;
    PathParams P{};
    P.coef = coef;
    P.p0 = p0;
    P.p_path = p_path;
    P.u_path = u_path;
    P.K = K;
    P.T = T;
    P.J = J;
    P.n = n;
    P.len1 = len1;
    for (int t = 0; t < J * J; ++t) {
        P.Kmat[t] = params->K[t];
        P.gamma[t] = params->gamma[t];
    }
    P.minv = 1.0 / params->m;
    for (int t = 0; t < J; ++t) {
        P.c[t] = params->c[t];
        P.beta[t] = params->beta[t];
    }
    P.h = opts->h;
    P.P_M = opts->P_M;
    P.U_M = opts->U_M;
    static PerDevice attr;
    cheb_status ra = per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(game_paths_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        return CHEB_OK;
    }, nullptr);
    if (ra) return ra;
    const int64_t grid = std::min<int64_t>(K, (int64_t)ctx->num_sms * 8);
    ProfScope prof("game_paths J=" + std::to_string(J) + " n=" + std::to_string(n), st);
    game_paths_kernel<<<(unsigned)grid, kThreads, smem, st>>>(P);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}
