// FP64 CUDA-core kernels: the mode product used by the fit and by the FP64
// grid evaluation, the Chebyshev matrices T_l(x_j), and FP64 point
// evaluation. On GB300 the FP64 pipe is the bound for all of them.
#include <algorithm>
#include <string>

#include "cheb_internal.cuh"

namespace cheb {
namespace {

constexpr int kF64Rows = 64;      // rows r of a tile
constexpr int kF64Threads = 256;  // 64 rows x 4 column groups, Q columns each
constexpr int kF64MaxQ = 9;       // a tile has 4 Q <= 36 output columns
constexpr int kMaxN = 64;

// Whether slab g is skipped: the flag of its group g / per_flag is set.
__device__ __forceinline__ bool slab_skipped(const SlabSkip &sk, int64_t g)
{
    return sk.flags && __ldg(sk.flags + (g / sk.per_flag) * sk.stride) != 0;
}

// Mode product on G slabs, each a row-major [R x n] view (Section 3.2, one
// pagemtimes step per slab): out[(g m + j) R + r] = sum_k B[j, k] X[g R + r, k].
// A block owns 64 consecutive rows of the G R and 4 Q output columns (Q = the
// smallest that covers m <= 36 in one column tile, else 8); a block
// whose rows all lie in skipped slabs returns at once, and rows of skipped
// slabs are not written. X rows are staged with an odd stride so that the
// 64-bit shared loads of consecutive rows fall in different banks; B is read
// as a broadcast. Output stores are coalesced along r.
template <int Q>
__global__ void __launch_bounds__(kF64Threads, 4)
modeprod_f64_kernel(const double *__restrict__ X, const double *__restrict__ B,
                    double *__restrict__ out, int64_t G, int64_t R, int n, int m, const SlabSkip sk)
{
    constexpr int kCols = 4 * Q;
    extern __shared__ double smem[];
    const int ns = n | 1;
    double *sX = smem;
    double *sB = smem + kF64Rows * ns;
    const int64_t total = G * R;
    const int64_t r0 = (int64_t)blockIdx.x * kF64Rows;
    const int j0 = blockIdx.y * kCols;
    const int rows = (int)((total - r0) < kF64Rows ? (total - r0) : kF64Rows);
    // the staged rows and columns fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK((size_t)(kF64Rows * ns + kCols * n) * sizeof(double) <= dyn_smem_bytes() && r0 < total)) return;
    if (sk.flags) {
        bool any = false;
        for (int64_t g = r0 / R; g <= (r0 + rows - 1) / R; ++g) any = any || !slab_skipped(sk, g);
        if (!any) return;     // uniform across the block
    }
    const double *Xt = X + r0 * n;
    for (int t = threadIdx.x; t < rows * n; t += blockDim.x) {
        int rr = t / n, k = t - rr * n;
        sX[rr * ns + k] = Xt[t];
    }
    for (int t = threadIdx.x; t < (kF64Rows - rows) * n; t += blockDim.x) {
        int rr = rows + t / n, k = t % n;
        sX[rr * ns + k] = 0.0;
    }
    for (int t = threadIdx.x; t < kCols * n; t += blockDim.x) {
        int jj = t / n, k = t - jj * n;
        sB[t] = (j0 + jj < m) ? B[(int64_t)(j0 + jj) * n + k] : 0.0;
    }
    __syncthreads();
    const int tr = threadIdx.x & (kF64Rows - 1);
    const int tj = threadIdx.x / kF64Rows;
    double acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.0;
    for (int k = 0; k < n; ++k) {
        const double xv = sX[tr * ns + k];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] = fma(sB[(tj + 4 * q) * n + k], xv, acc[q]);
    }
    if (tr < rows) {
        const int64_t rg = r0 + tr, g = rg / R, r = rg - g * R;
        if (!slab_skipped(sk, g)) {
            double *og = out + g * m * R + r;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int j = j0 + tj + 4 * q;
                if (j < m && CHEB_DCHECK(g < G)) og[(int64_t)j * R] = acc[q];
            }
        }
    }
}

// The same product for small G R (few tiles): one thread per output element,
// so that the FP64 work spreads over the SMs instead of occupying a handful
// of them (GB300's FP64 rate per SM is low). Same order of the k sum and the
// same fma as the tiled kernel, hence bit-identical results.
__global__ void modeprod_f64_small_kernel(const double *__restrict__ X, const double *__restrict__ B,
                                          double *__restrict__ out, int64_t G, int64_t R, int n, int m,
                                          const SlabSkip sk)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * R * m) return;
    const int64_t g = t / (R * m), rem = t - g * R * m;
    if (slab_skipped(sk, g)) return;
    const int j = (int)(rem / R);
    const int64_t r = rem - (int64_t)j * R;
    const double *xr = X + (g * R + r) * n, *bj = B + (int64_t)j * n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(__ldg(bj + k), __ldg(xr + k), acc);
    out[t] = acc;
}

// All J mode products of a slab in one CTA per (slab g, last output index
// k_J): the first product (the last mode, read from global memory) is taken
// for this k_J only, and the other J - 1 products run on the resulting
// n^(J-1) tensor in shared memory, each moving its new index to the front as
// modeprod_f64_slabs does. Every output is the same sum in the same order as
// in J successive slab products, so the results are bit-identical; the
// intermediates never leave the SM and the J launches become one.
constexpr int kChainMax = 4913;     // largest n^(J-1) held in shared memory
constexpr int kChainThreads = 256;

__global__ void __launch_bounds__(kChainThreads)
modeprod_f64_chain_kernel(const double *__restrict__ X, const double *__restrict__ B, double *__restrict__ out,
                          int J, int n, const SlabSkip sk)
{
    extern __shared__ double chain_s[];
    const int kJ = blockIdx.x;
    const int64_t g = blockIdx.y;
    if (slab_skipped(sk, g)) return;
    int R = 1;
    for (int s = 0; s < J - 1; ++s) R *= n;
    double *sB = chain_s;
    double *cur = sB + n * n, *nxt = cur + R;
    // B and the two intermediates fit the dynamic shared memory (uniform)
    if (!CHEB_DCHECK((size_t)(n * n + 2 * R) * sizeof(double) <= dyn_smem_bytes() && kJ < n)) return;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sB[t] = B[t];
    __syncthreads();
    // the last mode: cur[r] = sum_k B[k_J, k] X_g[r, k]
    const double *Xg = X + g * (int64_t)R * n;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double *xr = Xg + (int64_t)r * n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc = fma(sB[kJ * n + k], __ldg(xr + k), acc);
        cur[r] = acc;
    }
    __syncthreads();
    // the other modes: view cur as [R / n rows x n], out[j (R / n) + r] = sum_k B[j, k] cur[r n + k]
    const int Rp = R / n;
    for (int step = 1; step < J; ++step) {
        for (int t = threadIdx.x; t < n * Rp; t += blockDim.x) {
            const int j = t / Rp, r = t - j * Rp;
            const double *xr = cur + r * n;
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc = fma(sB[j * n + k], xr[k], acc);
            nxt[t] = acc;
        }
        __syncthreads();
        double *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    // cur = C_g[k_1 .. k_{J-1}, k_J] for this k_J, (k_1 .. k_{J-1}) row-major
    double *og = out + g * (int64_t)R * n;
    for (int t = threadIdx.x; t < R; t += blockDim.x) og[(int64_t)t * n + kJ] = cur[t];
}

// T[j * n + l] = T_l(x~_j) by the three-term recurrence (valid off [-1,1]).
__global__ void cheb_matrix_kernel(const double *__restrict__ x, int64_t stride, int64_t m, int n,
                                   double a, double b, double *__restrict__ T)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double xr = (2.0 * x[j * stride] - (a + b)) / (b - a);
    double *Tj = T + (int64_t)j * n;
    double t0 = 1.0, t1 = xr;
    Tj[0] = 1.0;
    if (n > 1) Tj[1] = xr;
    for (int l = 2; l < n; ++l) {
        const double t2 = 2.0 * xr * t1 - t0;
        Tj[l] = t2;
        t0 = t1;
        t1 = t2;
    }
}

struct ModeMats {
    const double *x[6];
    double *T[6];
    int m[6], n[6];
    double a[6], b[6];
};

// All d Chebyshev matrices of a grid evaluation in one launch: blockIdx.y is
// the mode, T_s[j * n_s + l] = T_l(x~_{s,j}) by the recurrence.
__global__ void cheb_matrices_kernel(ModeMats M)
{
    const int s = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M.m[s]) return;
    const double xr = (2.0 * M.x[s][j] - (M.a[s] + M.b[s])) / (M.b[s] - M.a[s]);
    double *Tj = M.T[s] + (int64_t)j * M.n[s];
    double t0 = 1.0, t1 = xr;
    Tj[0] = 1.0;
    if (M.n[s] > 1) Tj[1] = xr;
    for (int l = 2; l < M.n[s]; ++l) {
        const double t2 = 2.0 * xr * t1 - t0;
        Tj[l] = t2;
        t0 = t1;
        t1 = t2;
    }
}

struct FilterDims {
    int d;
    int n[6];
    double alpha;
    int order;
};

// c[k] *= prod_s exp(-alpha (k_s / N_s)^(2 order)) (exponential spectral filter)
__global__ void filter_kernel(FilterDims D, double *__restrict__ c, int64_t total)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = t;
        double e = 0.0;
        for (int s = D.d - 1; s >= 0; --s) {
            const int k = (int)(rem % D.n[s]);
            rem /= D.n[s];
            const double eta = D.n[s] > 1 ? (double)k / (double)(D.n[s] - 1) : 0.0;
            double p = 1.0;
            for (int q = 0; q < 2 * D.order; ++q) p *= eta;
            e += p;
        }
        c[t] *= exp(-D.alpha * e);
    }
}

struct PointDims {
    int d;
    int n[6];
    double a[6], b[6];
};

// The Chebyshev rows of each thread's point live in shared memory as
// [row][thread] (rows of mode s from sum_{r<s} n_r), conflict-free and with no
// run-time indexed per-thread array. Returns the row offset of mode s.
__device__ __forceinline__ int point_row_offset(const PointDims &D, int s)
{
    int o = 0;
    for (int r = 0; r < s; ++r) o += D.n[r];
    return o;
}

__device__ __forceinline__ void point_rows(const PointDims &D, int modes, const double *__restrict__ x, int64_t j,
                                           double *Ts)
{
    const int nt = blockDim.x, tid = threadIdx.x;
    int o = 0;
    for (int s = 0; s < modes; ++s) {
        const double xr = (2.0 * x[j * D.d + s] - (D.a[s] + D.b[s])) / (D.b[s] - D.a[s]);
        double t0 = 1.0, t1 = xr;
        Ts[o * nt + tid] = 1.0;
        if (D.n[s] > 1) Ts[(o + 1) * nt + tid] = xr;
        for (int l = 2; l < D.n[s]; ++l) {
            const double t2 = 2.0 * xr * t1 - t0;
            Ts[(o + l) * nt + tid] = t2;
            t0 = t1;
            t1 = t2;
        }
        o += D.n[s];
    }
}

// One thread per point: T values per mode, then the nested contraction
// sum_{l_1} T(x_1) ( sum_{l_2} T(x_2) ( ... sum_{l_d} c_l T(x_d) ) ) with the
// innermost mode contiguous in memory. All threads of a warp read the same
// coefficients at the same time (broadcast through L1).
__global__ void eval_points_f64_kernel(PointDims D, const double *__restrict__ c, int64_t P,
                                       const double *__restrict__ x, double *__restrict__ out)
{
    extern __shared__ double Ts[];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const int d = D.d, nt = blockDim.x, tid = threadIdx.x;
    // this thread's Chebyshev rows fit the dynamic shared memory
    if (!CHEB_DCHECK((size_t)point_row_offset(D, d) * nt * sizeof(double) <= dyn_smem_bytes())) return;
    point_rows(D, d, x, j, Ts);
    auto T = [&](int s, int l) { return Ts[(point_row_offset(D, s) + l) * nt + tid]; };
    int64_t outer = 1;
    for (int s = 0; s < d - 1; ++s) outer *= D.n[s];
    const int nl = D.n[d - 1];
    const double *Tl = Ts + (size_t)point_row_offset(D, d - 1) * nt + tid;
    double part[6] = {0, 0, 0, 0, 0, 0};
    int idx[6] = {0, 0, 0, 0, 0, 0};
    double result = 0.0;
    const double *cp = c;
    for (int64_t o = 0; o < outer; ++o) {
        double t = 0.0;
        for (int k = 0; k < nl; ++k) t = fma(cp[k], Tl[(size_t)k * nt], t);
        cp += nl;
        int s = d - 2;
        double v = t;
        while (s >= 0) {
            part[s] = fma(T(s, idx[s]), v, part[s]);
            if (++idx[s] < D.n[s]) break;
            idx[s] = 0;
            v = part[s];
            part[s] = 0.0;
            --s;
        }
        if (s < 0) result = v;
    }
    out[j] = result;
}

// Second half of the split-precision point evaluation: Y holds, for every
// point j, the partial sums over the last mode, Y[q * P + j] with q the flat
// index of (l_1..l_{d-1}). Each thread finishes its point with the nested
// contraction over modes 1..d-1 in FP64.
__global__ void rowwise_contract_kernel(PointDims D, const float *__restrict__ Y, int64_t P,
                                        const double *__restrict__ x, float *__restrict__ out)
{
    extern __shared__ double Ts[];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const int d = D.d, nt = blockDim.x, tid = threadIdx.x;
    const int dm = d - 1;               // modes still to contract
    if (dm == 0) {
        out[j] = Y[j];
        return;
    }
    if (!CHEB_DCHECK((size_t)point_row_offset(D, dm) * nt * sizeof(double) <= dyn_smem_bytes())) return;
    point_rows(D, dm, x, j, Ts);
    auto T = [&](int s, int l) { return Ts[(point_row_offset(D, s) + l) * nt + tid]; };
    int64_t outer = 1;
    for (int s = 0; s < dm - 1; ++s) outer *= D.n[s];
    const int nl = D.n[dm - 1];
    const double *Tl = Ts + (size_t)point_row_offset(D, dm - 1) * nt + tid;
    double part[6] = {0, 0, 0, 0, 0, 0};
    int idx[6] = {0, 0, 0, 0, 0, 0};
    double result = 0.0;
    const float *yp = Y + j;
    for (int64_t o = 0; o < outer; ++o) {
        double t = 0.0;
        for (int k = 0; k < nl; ++k) t = fma((double)yp[(int64_t)k * P], Tl[(size_t)k * nt], t);
        yp += (int64_t)nl * P;
        int s = dm - 2;
        double v = t;
        while (s >= 0) {
            part[s] = fma(T(s, idx[s]), v, part[s]);
            if (++idx[s] < D.n[s]) break;
            idx[s] = 0;
            v = part[s];
            part[s] = 0.0;
            --s;
        }
        if (s < 0) result = v;
    }
    out[j] = (float)result;
}

// Threads per block of the point kernels and their shared memory: the rows of
// `modes` modes for every thread, at most 96 KB (128 threads, fewer for long rows).
inline int point_threads(const PointDims &D, int modes, size_t *smem)
{
    int rows = 0;
    for (int s = 0; s < modes; ++s) rows += D.n[s];
    int threads = 128;
    while (threads > 32 && (size_t)threads * rows * sizeof(double) > 96 * 1024) threads /= 2;
    *smem = (size_t)threads * rows * sizeof(double);
    return threads;
}

cheb_status point_attrs()
{
    static PerDevice attr;
    return per_device_once(attr, [](int *) -> cheb_status {
        const int bytes = 32 * 6 * kMaxN * (int)sizeof(double);
        CHEB_CUDA_TRY(cudaFuncSetAttribute(eval_points_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           bytes));
        CHEB_CUDA_TRY(cudaFuncSetAttribute(rowwise_contract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           bytes));
        return CHEB_OK;
    }, nullptr);
}

template <int Q>
cheb_status launch_f64(dim3 grid, size_t smem, cudaStream_t st, const double *X, const double *B, double *out,
                       int64_t G, int64_t R, int n, int m, const SlabSkip &skip)
{
    static PerDevice attr;
    cheb_status r = per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(modeprod_f64_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * (kF64Rows * 65 + 4 * Q * 64))));
        return CHEB_OK;
    }, nullptr);
    if (r) return r;
    modeprod_f64_kernel<Q><<<grid, kF64Threads, smem, st>>>(X, B, out, G, R, n, m, skip);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

}  // namespace

cheb_status modeprod_f64(const double *X, const double *B, double *out, int64_t R, int n, int m,
                         cudaStream_t st)
{
    return modeprod_f64_slabs(X, B, out, 1, R, n, m, SlabSkip{}, st);
}

cheb_status modeprod_f64_chain(const double *X, const double *B, double *out, int64_t G, int J, int n,
                               const SlabSkip &skip, cudaStream_t st)
{
    int64_t R = 1;
    for (int s = 0; s < J - 1; ++s) R *= n;
    if (J < 1 || n < 1 || R > kChainMax || G > 65535) return CHEB_EUNSUPPORTED;
    if (G <= 0) return CHEB_OK;
    static PerDevice attr;
    cheb_status r = per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(modeprod_f64_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(double) * (kMaxN * kMaxN + 2 * kChainMax))));
        return CHEB_OK;
    }, nullptr);
    if (r) return r;
    const size_t smem = sizeof(double) * ((size_t)n * n + 2 * (size_t)R);
    ProfScope prof("modeprod_f64_chain J=" + std::to_string(J) + " n=" + std::to_string(n) + " G=" + std::to_string(G),
                   st);
    modeprod_f64_chain_kernel<<<dim3((unsigned)n, (unsigned)G), kChainThreads, smem, st>>>(X, B, out, J, n, skip);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status modeprod_f64_slabs(const double *X, const double *B, double *out, int64_t G, int64_t R, int n, int m,
                               const SlabSkip &skip, cudaStream_t st)
{
    if (G <= 0 || R <= 0 || m <= 0) return CHEB_OK;
    if (n < 1 || n > kMaxN) return fail(CHEB_EUNSUPPORTED, "modeprod_f64: n out of range");
    if (skip.flags && skip.per_flag < 1) return fail(CHEB_EINVAL, "modeprod_f64: slabs per skip flag must be >= 1");
    const int Q = m <= 4 * kF64MaxQ ? (m + 3) / 4 : 8;
    const int cols = 4 * Q;
    const int ns = n | 1;
    const size_t smem = sizeof(double) * (size_t)(kF64Rows * ns + cols * n);
    const int64_t total = G * R;
    const int64_t tiles = (total + kF64Rows - 1) / kF64Rows;
    if (tiles > 0x7fffffffLL) return fail(CHEB_EUNSUPPORTED, "modeprod_f64: too many rows");
    if (tiles * ((m + cols - 1) / cols) < 256 && total * m < (int64_t)1 << 26) {
        ProfScope prof("modeprod_f64 R=" + std::to_string(total) + " n=" + std::to_string(n) +
                           " m=" + std::to_string(m) + " (per element)",
                       st);
        modeprod_f64_small_kernel<<<(unsigned)((total * m + 127) / 128), 128, 0, st>>>(X, B, out, G, R, n, m, skip);
        CHEB_CUDA_TRY(cudaGetLastError());
        return CHEB_OK;
    }
    dim3 grid((unsigned)tiles, (unsigned)((m + cols - 1) / cols));
    if (grid.y > 65535) return fail(CHEB_EUNSUPPORTED, "modeprod_f64: too many columns");
    ProfScope prof("modeprod_f64 R=" + std::to_string(total) + " n=" + std::to_string(n) +
                       " m=" + std::to_string(m), st);
    switch (Q) {
    case 1: return launch_f64<1>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 2: return launch_f64<2>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 3: return launch_f64<3>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 4: return launch_f64<4>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 5: return launch_f64<5>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 6: return launch_f64<6>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 7: return launch_f64<7>(grid, smem, st, X, B, out, G, R, n, m, skip);
    case 8: return launch_f64<8>(grid, smem, st, X, B, out, G, R, n, m, skip);
    default: return launch_f64<9>(grid, smem, st, X, B, out, G, R, n, m, skip);
    }
}

cheb_status cheb_matrix(const double *x, int64_t stride, int64_t m, int n, double a, double b,
                        double *T, cudaStream_t st)
{
    if (m <= 0) return CHEB_OK;
    ProfScope prof("cheb_matrix", st);
    cheb_matrix_kernel<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(x, stride, m, n, a, b, T);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status spectral_filter(int d, const int32_t *n, double *coeffs, double alpha, int order, cudaStream_t st)
{
    FilterDims D{};
    D.d = d;
    int64_t total = 1;
    for (int s = 0; s < d; ++s) {
        D.n[s] = n[s];
        total *= n[s];
    }
    D.alpha = alpha;
    D.order = order;
    ProfScope prof("spectral_filter", st);
    filter_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(D, coeffs, total);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status cheb_matrices(int d, const double *const *x, const int32_t *m, const int32_t *n,
                          const double *a, const double *b, double *const *T, cudaStream_t st)
{
    ModeMats M{};
    int mmax = 0;
    for (int s = 0; s < d; ++s) {
        M.x[s] = x[s];
        M.T[s] = T[s];
        M.m[s] = m[s];
        M.n[s] = n[s];
        M.a[s] = a[s];
        M.b[s] = b[s];
        mmax = std::max(mmax, (int)m[s]);
    }
    if (mmax <= 0) return CHEB_OK;
    ProfScope prof("cheb_matrices", st);
    cheb_matrices_kernel<<<dim3((unsigned)((mmax + 127) / 128), (unsigned)d), 128, 0, st>>>(M);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status eval_points_tc(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                           const double *a, const double *b, int64_t P, const double *x, float *out,
                           cheb_precision prec, cudaStream_t st)
{
    int64_t rest = 1;
    for (int s = 0; s < d - 1; ++s) rest *= n[s];
    if (rest > 256)
        return fail(CHEB_EUNSUPPORTED, "split point evaluation needs prod(n[0..d-2]) <= 256");
    const int nl = n[d - 1];
    cheb_status r;
    // T rows of the last mode (P x n_d, FP64) and the partial sums Y (rest x P, FP32)
    if ((r = ctx->ws[0].reserve(sizeof(double) * (size_t)P * nl))) return r;
    if ((r = ctx->ws[1].reserve(sizeof(float) * (size_t)P * rest))) return r;
    double *T = static_cast<double *>(ctx->ws[0].ptr);
    float *Y = static_cast<float *>(ctx->ws[1].ptr);
    if ((r = cheb_matrix(x + (d - 1), d, P, nl, a[d - 1], b[d - 1], T, st))) return r;
    if ((r = modeprod_tc(ctx, T, 1, coeffs, Y, P, nl, (int)rest, prec, st))) return r;
    PointDims D;
    D.d = d;
    for (int s = 0; s < 6; ++s) {
        D.n[s] = s < d ? n[s] : 1;
        D.a[s] = s < d ? a[s] : -1.0;
        D.b[s] = s < d ? b[s] : 1.0;
    }
    if ((r = point_attrs())) return r;
    size_t smem = 0;
    const int threads = point_threads(D, d - 1, &smem);
    ProfScope prof("rowwise_contract", st);
    rowwise_contract_kernel<<<(unsigned)((P + threads - 1) / threads), threads, smem, st>>>(D, Y, P, x, out);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

cheb_status eval_points_f64(int d, const int32_t *n, const double *coeffs, const double *a,
                            const double *b, int64_t P, const double *x, double *out,
                            cudaStream_t st)
{
    if (P <= 0) return CHEB_OK;
    PointDims D;
    D.d = d;
    for (int s = 0; s < 6; ++s) {
        D.n[s] = s < d ? n[s] : 1;
        D.a[s] = s < d ? a[s] : -1.0;
        D.b[s] = s < d ? b[s] : 1.0;
    }
    cheb_status r = point_attrs();
    if (r) return r;
    size_t smem = 0;
    const int threads = point_threads(D, d, &smem);
    const int64_t blocks = (P + threads - 1) / threads;
    ProfScope prof("eval_points_f64", st);
    eval_points_f64_kernel<<<(unsigned)blocks, threads, smem, st>>>(D, coeffs, P, x, out);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

}  // namespace cheb
