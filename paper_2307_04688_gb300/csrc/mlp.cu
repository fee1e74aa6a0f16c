// The learned warm start: a multilayer perceptron in -> width (x depth) -> out,
// GELU between layers, BF16 operands with FP32 accumulation on the tcgen05
// tensor cores, FP32 master weights, Adam, mean-squared error on normalised
// targets. It maps game parameters to the coefficient tensor of one player's
// value function and warm-starts the iteration (the paper starts from "some
// given" V^[0], Section 2.1 Step 0).
//
// One GEMM kernel serves the forward and backward passes:
//     C[m, n] = epi( sum_k A(m, k) B(n, k) ),  A(m,k) = A[m sa_m + k sa_k],
//                                             B(n,k) = B[n sb_n + k sb_k],
// with FP32 operands rounded to BF16 while they are staged into shared
// memory (arbitrary strides, so the transposed products of backpropagation
// need no copies), tcgen05.mma (M = 128, N = 128, K = 16 steps) into TMEM, and
// an epilogue applying bias, GELU or the GELU derivative.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cheb_internal.cuh"
#include "tc_common.cuh"

namespace cheb {
namespace mlp {

using namespace tc;

constexpr int kBM = 128, kBN = 128, kBK = 64, kThreads = 256;

enum Epi { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

struct GemmArgs {
    const float *A;
    int64_t sa_m, sa_k;
    const float *B;
    int64_t sb_n, sb_k;
    float *C;
    int64_t sc_m, sc_n;
    float *Z;              // EPI_BIAS_GELU: pre-activation output (same strides as C)
    const float *bias;     // EPI_BIAS*: bias[n]
    const float *aux;      // EPI_GELU_BWD: pre-activation Z(m, n) (strides of C)
    int M, N, K;
    int epi;
    int *err;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    return Phi + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

// stage rows [r0, r0 + 128) x K chunk [k0, k0 + 64) of an operand into the
// canonical K-major layout: block kc (8 elements of K) at kc * 2048 bytes,
// row r at r * 16 bytes inside it
__device__ __forceinline__ void stage_operand(uint8_t *dst, const float *src, int64_t s_row, int64_t s_k,
                                              int rows_valid, int r0, int k0, int K, int tid)
{
    for (int t = tid; t < kBM * (kBK / 8); t += kThreads) {
        const int r = t & (kBM - 1), kc = t >> 7;
        const int gr = r0 + r;
        uint32_t w[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float a = 0.0f, b = 0.0f;
            const int k = k0 + kc * 8 + 2 * p;
            if (gr < rows_valid) {
                if (k < K) a = src[gr * s_row + (int64_t)k * s_k];
                if (k + 1 < K) b = src[gr * s_row + (int64_t)(k + 1) * s_k];
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            w[p] = *reinterpret_cast<const uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(dst + kc * (kBM * 16) + r * 16) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void __launch_bounds__(kThreads)
gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(1024) uint8_t sA[kBM * kBK * 2];
    __shared__ __align__(1024) uint8_t sB[kBN * kBK * 2];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, kBN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = make_idesc(1, kBM, kBN);
    uint32_t phase = 0;
    bool mma_pending = false;     // MMAs issued and not yet waited for (timeout path)
    const int nk = (g.K + kBK - 1) / kBK;
    for (int kb = 0; kb < nk; ++kb) {
        stage_operand(sA, g.A, g.sa_m, g.sa_k, g.M, m0, kb * kBK, g.K, tid);
        stage_operand(sB, g.B, g.sb_n, g.sb_k, g.N, n0, kb * kBK, g.K, tid);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int ks = 0; ks < kBK / 16; ++ks) {
                const uint64_t ad = make_sdesc(a0 + ks * 2 * (kBM * 16), kBM * 16, 128);
                const uint64_t bd = make_sdesc(b0 + ks * 2 * (kBN * 16), kBN * 16, 128);
                mma_bf16(tmem, ad, bd, idesc, (kb | ks) != 0);
            }
            mma_commit(&bar);
        }
        mma_pending = true;
        if (mbar_wait_bounded(&bar, phase, g.err)) {
            phase ^= 1u;
            mma_pending = false;
        } else {
            abort_flag = 1;
        }
        tc_fence_after();
        __syncthreads();   // the operands may be overwritten by the next chunk
        if (abort_flag) break;
    }
    // epilogue: warp w -> TMEM lanes 32 (w % 4) .. (rows), column half w / 4
    const int quarter = warp & 3, half = warp >> 2;
    const int m = m0 + quarter * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(lane_addr + c0, v);
        tmem_ld_wait();
        if (m < g.M && !abort_flag) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n = n0 + c0 + e;
                if (n >= g.N) break;
                float acc = __uint_as_float(v[e]);
                const int64_t off = (int64_t)m * g.sc_m + (int64_t)n * g.sc_n;
                if (g.epi == EPI_BIAS || g.epi == EPI_BIAS_GELU) acc += g.bias[n];
                if (g.epi == EPI_BIAS_GELU) {
                    g.Z[off] = acc;
                    acc = gelu_f(acc);
                } else if (g.epi == EPI_GELU_BWD) {
                    acc *= gelu_grad_f(g.aux[off]);
                }
                g.C[off] = acc;
            }
        }
    }
    if (mma_pending) mbar_wait_bounded(&bar, phase, g.err);   // full bound before TMEM is freed
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kBN);
}

cheb_status gemm(const GemmArgs &a, cudaStream_t st)
{
    if (a.M <= 0 || a.N <= 0 || a.K <= 0) return CHEB_OK;
    dim3 grid((unsigned)((a.N + kBN - 1) / kBN), (unsigned)((a.M + kBM - 1) / kBM));
    // 24 KB of otherwise unused dynamic shared memory caps residency at four
    // CTAs per SM, so that their TMEM accumulators (128 columns each) fit in 512
    static PerDevice attr;
    cheb_status r = per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 24 * 1024));
        return CHEB_OK;
    }, nullptr);
    if (r) return r;
    ProfScope prof("mlp_gemm_bf16", st);
    gemm_bf16_kernel<<<grid, kThreads, 24 * 1024, st>>>(a);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

// ---- elementwise kernels ----------------------------------------------------------

// rows[b] of X (FP64, row stride sx) -> normalised FP32 (x - mean) / std
__global__ void gather_norm_kernel(const double *__restrict__ X, int64_t sx, const int *__restrict__ rows, int B,
                                   int F, const float *__restrict__ mean, const float *__restrict__ inv_std,
                                   float *__restrict__ out)
{
    const int64_t total = (int64_t)B * F;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / F), f = (int)(t % F);
        const int64_t r = rows ? rows[b] : b;
        out[t] = (float)((X[r * sx + f] - (double)mean[f]) * (double)inv_std[f]);
    }
}

// per-column mean and 1/std of an S x F FP64 matrix (row stride sx); std floored
__global__ void column_stats_kernel(const double *__restrict__ X, int64_t sx, int64_t S, int F, float floor_frac,
                                    float *__restrict__ mean, float *__restrict__ inv_std, float *__restrict__ std_out)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < S; ++r) {
        const double v = X[r * sx + f];
        s += v;
        s2 += v * v;
    }
    const double mu = s / (double)S;
    const double var = fmax(s2 / (double)S - mu * mu, 0.0);
    mean[f] = (float)mu;
    std_out[f] = (float)sqrt(var);
    (void)floor_frac;
    (void)inv_std;
}

__global__ void finish_inv_std_kernel(const float *__restrict__ std_in, int F, float floor_abs, float *__restrict__ inv_std)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    inv_std[f] = 1.0f / fmaxf(std_in[f], floor_abs);
}

// dY = 2 (Y - T) / (B F); loss accumulated into *loss
__global__ void mse_grad_kernel(const float *__restrict__ Y, const float *__restrict__ T, int64_t total, float scale,
                                float *__restrict__ dY, float *__restrict__ loss)
{
    float local = 0.0f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const float d = Y[t] - T[t];
        dY[t] = 2.0f * d * scale;
        local += d * d * scale;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, local);
}

// gb[n] = sum_b dZ[b, n]
__global__ void bias_grad_kernel(const float *__restrict__ dZ, int B, int N, float *__restrict__ gb)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * N + n];
    gb[n] = s;
}

__global__ void adam_kernel(int64_t nparam, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nparam; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// out (FP64, row stride so) = Y / inv_std + mean (the inverse of the target normalisation)
__global__ void denorm_kernel(const float *__restrict__ Y, int64_t P, int F, const float *__restrict__ mean,
                              const float *__restrict__ inv_std, double *__restrict__ out, int64_t so)
{
    const int64_t total = P * F;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / F;
        const int f = (int)(t % F);
        out[p * so + f] = (double)Y[t] / (double)inv_std[f] + (double)mean[f];
    }
}

inline unsigned blocks_for(int64_t n, int threads = 256)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 8192));
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form
inline uint64_t splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace mlp
}  // namespace cheb

using namespace cheb;
using namespace cheb::mlp;

struct cheb_mlp {
    int device = 0;
    std::vector<int> dims;           // L + 1 widths
    int L = 0;
    int64_t nparam = 0;
    std::vector<int64_t> woff, boff; // offsets of W_l and b_l in the flat parameter vector
    float *w = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    int64_t adam_t = 0;
    // normalisation (inputs and targets)
    float *x_mean = nullptr, *x_inv = nullptr, *x_std = nullptr;
    float *y_mean = nullptr, *y_inv = nullptr, *y_std = nullptr;
    bool normalised = false;
    // batch workspace
    int ws_batch = 0;
    float *Z = nullptr, *H = nullptr, *dZ = nullptr, *dH = nullptr, *X = nullptr, *T = nullptr, *loss = nullptr;
    int *rows = nullptr;
};

namespace {

cheb_status net_ws(cheb_mlp *net, int B)
{
    if (B <= net->ws_batch) return CHEB_OK;
    cudaFree(net->Z);
    cudaFree(net->H);
    cudaFree(net->dZ);
    cudaFree(net->dH);
    cudaFree(net->X);
    cudaFree(net->T);
    cudaFree(net->rows);
    int64_t act = 0, maxw = 0;
    for (int l = 1; l <= net->L; ++l) act += (int64_t)B * net->dims[l];
    for (int l = 0; l <= net->L; ++l) maxw = std::max<int64_t>(maxw, net->dims[l]);
    if (cudaMalloc(&net->Z, sizeof(float) * act) || cudaMalloc(&net->H, sizeof(float) * act) ||
        cudaMalloc(&net->dZ, sizeof(float) * B * maxw) || cudaMalloc(&net->dH, sizeof(float) * B * maxw) ||
        cudaMalloc(&net->X, sizeof(float) * B * net->dims[0]) ||
        cudaMalloc(&net->T, sizeof(float) * B * net->dims[net->L]) || cudaMalloc(&net->rows, sizeof(int) * B))
        return fail(CHEB_ENOMEM, "surrogate workspace allocation failed");
    net->ws_batch = B;
    return CHEB_OK;
}

// activations of layer l (l = 1..L) inside Z / H
int64_t act_off(const cheb_mlp *net, int l, int B)
{
    int64_t o = 0;
    for (int t = 1; t < l; ++t) o += (int64_t)B * net->dims[t];
    return o;
}

GemmArgs base_args(cheb_ctx *ctx)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.err = ctx->d_error;
    return g;
}

// forward pass of a batch whose (normalised) inputs are in net->X
cheb_status forward(cheb_ctx *ctx, cheb_mlp *net, int B, cudaStream_t st)
{
    const float *in = net->X;
    for (int l = 0; l < net->L; ++l) {
        const int ni = net->dims[l], no = net->dims[l + 1];
        GemmArgs g = base_args(ctx);
        g.A = in;
        g.sa_m = ni;
        g.sa_k = 1;
        g.B = net->w + net->woff[l];
        g.sb_n = ni;
        g.sb_k = 1;
        float *Zl = net->Z + act_off(net, l + 1, B);
        float *Hl = net->H + act_off(net, l + 1, B);
        const bool last = (l == net->L - 1);
        g.C = last ? Zl : Hl;
        g.Z = Zl;
        g.sc_m = no;
        g.sc_n = 1;
        g.bias = net->w + net->boff[l];
        g.M = B;
        g.N = no;
        g.K = ni;
        g.epi = last ? EPI_BIAS : EPI_BIAS_GELU;
        cheb_status r = gemm(g, st);
        if (r) return r;
        in = last ? Zl : Hl;
    }
    return CHEB_OK;
}

// output of the last layer (FP32, B x out)
float *output(cheb_mlp *net, int B) { return net->Z + act_off(net, net->L, B); }

// backward pass from dY (in net->dZ) to net->grad
cheb_status backward(cheb_ctx *ctx, cheb_mlp *net, int B, cudaStream_t st)
{
    float *dZ = net->dZ, *dH = net->dH;
    for (int l = net->L - 1; l >= 0; --l) {
        const int ni = net->dims[l], no = net->dims[l + 1];
        const float *in = (l == 0) ? net->X : net->H + act_off(net, l, B);
        // dW_l[o, i] = sum_b dZ[b, o] in[b, i]
        GemmArgs g = base_args(ctx);
        g.A = dZ;
        g.sa_m = 1;
        g.sa_k = no;
        g.B = in;
        g.sb_n = 1;
        g.sb_k = ni;
        g.C = net->grad + net->woff[l];
        g.sc_m = ni;
        g.sc_n = 1;
        g.M = no;
        g.N = ni;
        g.K = B;
        g.epi = EPI_NONE;
        cheb_status r = gemm(g, st);
        if (r) return r;
        {
            ProfScope prof("mlp_bias_grad", st);
            bias_grad_kernel<<<blocks_for(no), 256, 0, st>>>(dZ, B, no, net->grad + net->boff[l]);
        }
        CHEB_CUDA_TRY(cudaGetLastError());
        if (l > 0) {
            // dZ_{l-1}[b, i] = (sum_o dZ[b, o] W_l[o, i]) GELU'(Z_{l-1}[b, i])
            GemmArgs h = base_args(ctx);
            h.A = dZ;
            h.sa_m = no;
            h.sa_k = 1;
            h.B = net->w + net->woff[l];
            h.sb_n = 1;
            h.sb_k = ni;
            h.C = dH;
            h.sc_m = ni;
            h.sc_n = 1;
            h.aux = net->Z + act_off(net, l, B);
            h.M = B;
            h.N = ni;
            h.K = no;
            h.epi = EPI_GELU_BWD;
            if ((r = gemm(h, st))) return r;
            std::swap(dZ, dH);
        }
    }
    return CHEB_OK;
}

cheb_status check_net(cheb_ctx *ctx, cheb_mlp *net)
{
    if (!ctx || !net) return fail(CHEB_EINVAL, "null context or network");
    tl_ctx = ctx;
    CHEB_CUDA_TRY(cudaSetDevice(ctx->device));
    return CHEB_OK;
}

}  // namespace

extern "C" {

CHEB_API cheb_status surrogate_create(cheb_ctx *ctx, int32_t n_in, int32_t width, int32_t depth, int32_t n_out,
                                      uint64_t seed, cheb_mlp **out)
{
    if (!ctx || !out) return fail(CHEB_EINVAL, "null argument");
    if (n_in < 1 || width < 1 || depth < 0 || n_out < 1 || depth > 16 || width > 8192 || n_out > 1 << 20 ||
        n_in > 8192)
        return fail(CHEB_EINVAL, "surrogate_create: bad shape");
    tl_ctx = ctx;
    CHEB_CUDA_TRY(cudaSetDevice(ctx->device));
    cheb_mlp *net = new cheb_mlp();
    net->device = ctx->device;
    net->dims.push_back(n_in);
    for (int l = 0; l < depth; ++l) net->dims.push_back(width);
    net->dims.push_back(n_out);
    net->L = (int)net->dims.size() - 1;
    int64_t off = 0;
    for (int l = 0; l < net->L; ++l) {
        net->woff.push_back(off);
        off += (int64_t)net->dims[l + 1] * net->dims[l];
        net->boff.push_back(off);
        off += net->dims[l + 1];
    }
    net->nparam = off;
    // He-uniform weights (|w| < sqrt(6 / fan_in)), zero biases, from SplitMix64(seed)
    std::vector<float> h(off, 0.0f);
    for (int l = 0; l < net->L; ++l) {
        const double a = std::sqrt(6.0 / net->dims[l]);
        for (int64_t t = 0; t < (int64_t)net->dims[l + 1] * net->dims[l]; ++t) {
            const int64_t idx = net->woff[l] + t;
            const double u = (double)(splitmix64(seed, (uint64_t)idx) >> 11) * (1.0 / 9007199254740992.0);
            h[idx] = (float)(a * (2.0 * u - 1.0));
        }
    }
    const int F = n_in, O = n_out;
    if (cudaMalloc(&net->w, sizeof(float) * off) || cudaMalloc(&net->grad, sizeof(float) * off) ||
        cudaMalloc(&net->m, sizeof(float) * off) || cudaMalloc(&net->v, sizeof(float) * off) ||
        cudaMalloc(&net->x_mean, sizeof(float) * F) || cudaMalloc(&net->x_inv, sizeof(float) * F) ||
        cudaMalloc(&net->x_std, sizeof(float) * F) || cudaMalloc(&net->y_mean, sizeof(float) * O) ||
        cudaMalloc(&net->y_inv, sizeof(float) * O) || cudaMalloc(&net->y_std, sizeof(float) * O) ||
        cudaMalloc(&net->loss, sizeof(float) * 4096)) {
        delete net;
        return fail(CHEB_ENOMEM, "surrogate allocation failed");
    }
    cudaMemcpy(net->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice);
    cudaMemset(net->m, 0, sizeof(float) * off);
    cudaMemset(net->v, 0, sizeof(float) * off);
    std::vector<float> zeros(std::max(F, O), 0.0f), ones(std::max(F, O), 1.0f);
    cudaMemcpy(net->x_mean, zeros.data(), sizeof(float) * F, cudaMemcpyHostToDevice);
    cudaMemcpy(net->x_inv, ones.data(), sizeof(float) * F, cudaMemcpyHostToDevice);
    cudaMemcpy(net->x_std, ones.data(), sizeof(float) * F, cudaMemcpyHostToDevice);
    cudaMemcpy(net->y_mean, zeros.data(), sizeof(float) * O, cudaMemcpyHostToDevice);
    cudaMemcpy(net->y_inv, ones.data(), sizeof(float) * O, cudaMemcpyHostToDevice);
    cudaMemcpy(net->y_std, ones.data(), sizeof(float) * O, cudaMemcpyHostToDevice);
    *out = net;
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_destroy(cheb_mlp *net)
{
    if (!net) return CHEB_OK;
    cudaSetDevice(net->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)net->w, (void *)net->grad, (void *)net->m, (void *)net->v, (void *)net->x_mean,
                    (void *)net->x_inv, (void *)net->x_std, (void *)net->y_mean, (void *)net->y_inv,
                    (void *)net->y_std, (void *)net->Z, (void *)net->H, (void *)net->dZ, (void *)net->dH,
                    (void *)net->X, (void *)net->T, (void *)net->loss, (void *)net->rows})
        if (p) cudaFree(p);
    delete net;
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_params(cheb_mlp *net, float *get, const float *set, int64_t *count)
{
    if (!net) return fail(CHEB_EINVAL, "null network");
    if (count) *count = net->nparam;
    CHEB_CUDA_TRY(cudaSetDevice(net->device));
    if (set) {
        CHEB_CUDA_TRY(cudaMemcpy(net->w, set, sizeof(float) * net->nparam, cudaMemcpyHostToDevice));
        cudaMemset(net->m, 0, sizeof(float) * net->nparam);
        cudaMemset(net->v, 0, sizeof(float) * net->nparam);
        net->adam_t = 0;
    }
    if (get) CHEB_CUDA_TRY(cudaMemcpy(get, net->w, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost));
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_loss_grad(cheb_ctx *ctx, cheb_mlp *net, const float *X, const float *T, int32_t B,
                                         float *loss, float *grad, void *stream)
{
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    if (B < 1 || !X || !T) return fail(CHEB_EINVAL, "surrogate_loss_grad: bad batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = net_ws(net, B))) return r;
    const int F = net->dims[0], O = net->dims[net->L];
    CHEB_CUDA_TRY(cudaMemcpyAsync(net->X, X, sizeof(float) * B * F, cudaMemcpyDeviceToDevice, st));
    if ((r = forward(ctx, net, B, st))) return r;
    CHEB_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(float), st));
    mse_grad_kernel<<<blocks_for((int64_t)B * O), 256, 0, st>>>(output(net, B), T, (int64_t)B * O,
                                                              1.0f / ((float)B * O), net->dZ, net->loss);
    CHEB_CUDA_TRY(cudaGetLastError());
    if ((r = backward(ctx, net, B, st))) return r;
    if (grad) CHEB_CUDA_TRY(cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->nparam, cudaMemcpyDeviceToDevice, st));
    if (loss) {
        CHEB_CUDA_TRY(cudaMemcpyAsync(loss, net->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        CHEB_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_adam_step(cheb_ctx *ctx, cheb_mlp *net, const float *grad, float lr, void *stream)
{
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    if (!(lr > 0)) return fail(CHEB_EINVAL, "surrogate_adam_step: lr must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    net->adam_t += 1;
    const float c1 = 1.0f - std::pow(b1, (float)net->adam_t), c2 = 1.0f - std::pow(b2, (float)net->adam_t);
    {
        ProfScope prof("mlp_adam", st);
        adam_kernel<<<blocks_for(net->nparam), 256, 0, st>>>(net->nparam, net->w, grad ? grad : net->grad, net->m,
                                                            net->v, lr, b1, b2, eps, c1, c2);
    }
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_train(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride,
                                     const double *Y, int64_t y_stride, int64_t S, int32_t epochs, int32_t batch,
                                     float lr, uint64_t seed, float *loss_per_epoch, void *stream)
{
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    const int F = net->dims[0], O = net->dims[net->L];
    if (!X || !Y || S < 1 || epochs < 0 || batch < 1 || x_stride < F || y_stride < O || !(lr > 0))
        return fail(CHEB_EINVAL, "surrogate_train: bad arguments");
    if (epochs > 4096) return fail(CHEB_EINVAL, "surrogate_train: at most 4096 epochs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = (int)std::min<int64_t>(batch, S);
    if ((r = net_ws(net, B))) return r;
    // normalisation from the training set: inputs and targets to zero mean, unit std
    column_stats_kernel<<<(F + 127) / 128, 128, 0, st>>>(X, x_stride, S, F, 0.0f, net->x_mean, net->x_inv, net->x_std);
    column_stats_kernel<<<(O + 127) / 128, 128, 0, st>>>(Y, y_stride, S, O, 0.0f, net->y_mean, net->y_inv, net->y_std);
    CHEB_CUDA_TRY(cudaGetLastError());
    {
        std::vector<float> ys(O);
        CHEB_CUDA_TRY(cudaMemcpyAsync(ys.data(), net->y_std, sizeof(float) * O, cudaMemcpyDeviceToHost, st));
        CHEB_CUDA_TRY(cudaStreamSynchronize(st));
        float ymax = 0.0f;
        for (float s : ys) ymax = std::max(ymax, s);
        // coefficients that barely vary are scaled by a floor of 1e-3 of the largest spread
        finish_inv_std_kernel<<<(O + 127) / 128, 128, 0, st>>>(net->y_std, O, std::max(1e-3f * ymax, 1e-30f), net->y_inv);
        finish_inv_std_kernel<<<(F + 127) / 128, 128, 0, st>>>(net->x_std, F, 1e-30f, net->x_inv);
        CHEB_CUDA_TRY(cudaGetLastError());
    }
    net->normalised = true;
    CHEB_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(float) * std::max(epochs, 1), st));
    std::vector<int> perm(S);
    int *d_perm = nullptr;
    CHEB_CUDA_TRY(cudaMalloc(&d_perm, sizeof(int) * S));
    const int64_t steps = S / B;      // full batches per epoch
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < epochs && r == CHEB_OK; ++e) {
        // Fisher-Yates shuffle driven by SplitMix64(seed), counter = (epoch, position)
        for (int64_t i = 0; i < S; ++i) perm[i] = (int)i;
        for (int64_t i = S - 1; i > 0; --i) {
            const uint64_t z = splitmix64(seed, ((uint64_t)e << 32) + (uint64_t)i);
            const int64_t j = (int64_t)(z % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        CHEB_CUDA_TRY(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
        for (int64_t s = 0; s < steps && r == CHEB_OK; ++s) {
            const int *rows = d_perm + s * B;
            gather_norm_kernel<<<blocks_for((int64_t)B * F), 256, 0, st>>>(X, x_stride, rows, B, F, net->x_mean,
                                                                           net->x_inv, net->X);
            gather_norm_kernel<<<blocks_for((int64_t)B * O), 256, 0, st>>>(Y, y_stride, rows, B, O, net->y_mean,
                                                                           net->y_inv, net->T);
            if ((r = forward(ctx, net, B, st))) break;
            mse_grad_kernel<<<blocks_for((int64_t)B * O), 256, 0, st>>>(
                output(net, B), net->T, (int64_t)B * O, 1.0f / ((float)B * O), net->dZ, net->loss + e);
            if ((r = backward(ctx, net, B, st))) break;
            net->adam_t += 1;
            const float c1 = 1.0f - std::pow(b1, (float)net->adam_t), c2 = 1.0f - std::pow(b2, (float)net->adam_t);
            // cosine decay of the learning rate over the run
            const double prog = (double)(e * steps + s) / (double)std::max<int64_t>(1, (int64_t)epochs * steps);
            const float lr_t = (float)(0.5 * lr * (1.0 + std::cos(M_PI * prog)));
            adam_kernel<<<blocks_for(net->nparam), 256, 0, st>>>(net->nparam, net->w, net->grad, net->m, net->v, lr_t,
                                                                b1, b2, eps, c1, c2);
            cudaError_t ce = cudaGetLastError();
            if (ce != cudaSuccess) r = cuda_fail(ce, "surrogate_train");
        }
    }
    if (loss_per_epoch && epochs > 0 && r == CHEB_OK) {
        std::vector<float> l(epochs);
        CHEB_CUDA_TRY(cudaMemcpyAsync(l.data(), net->loss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st));
        CHEB_CUDA_TRY(cudaStreamSynchronize(st));
        for (int e = 0; e < epochs; ++e) loss_per_epoch[e] = l[e] / (float)std::max<int64_t>(steps, 1);
    }
    cudaStreamSynchronize(st);
    cudaFree(d_perm);
    return r;
}

CHEB_API cheb_status surrogate_predict(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride, int64_t P,
                                       double *Y, int64_t y_stride, void *stream)
{
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    const int F = net->dims[0], O = net->dims[net->L];
    if (P < 0 || (P > 0 && (!X || !Y)) || x_stride < F || y_stride < O)
        return fail(CHEB_EINVAL, "surrogate_predict: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = std::max(net->ws_batch, 256);
    if ((r = net_ws(net, B))) return r;
    for (int64_t p0 = 0; p0 < P; p0 += B) {
        const int nb = (int)std::min<int64_t>(B, P - p0);
        gather_norm_kernel<<<blocks_for((int64_t)nb * F), 256, 0, st>>>(X + p0 * x_stride, x_stride, nullptr, nb, F,
                                                                        net->x_mean, net->x_inv, net->X);
        if ((r = forward(ctx, net, nb, st))) return r;
        denorm_kernel<<<blocks_for((int64_t)nb * O), 256, 0, st>>>(output(net, nb), nb, O, net->y_mean, net->y_inv,
                                                                   Y + p0 * y_stride, y_stride);
        CHEB_CUDA_TRY(cudaGetLastError());
    }
    return CHEB_OK;
}

}  // extern "C"
