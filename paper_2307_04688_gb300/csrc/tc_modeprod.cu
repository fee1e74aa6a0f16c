// Split-precision mode product on the tcgen05 tensor cores.
//
// One mode product of the tensorial method (Section 3.2: B . A(:, i_2..i_n)
// for every page, the pagemtimes step) on a row-major [R x n] view:
//     out[j * R + r] = sum_k B[j, k] X[r, k],   j < m, r < R,
// i.e. D = X B^T written transposed, so that applying it once per mode visits
// every mode and leaves the modes in their original order.
//
// Design (GB300):
//  - persistent CTAs of 256 threads (8 warps), up to four per SM (shared
//    memory decides); a CTA owns a 128-row tile at a time;
//  - the X tile is one contiguous block of global memory, copied to shared
//    memory by the TMA engine (cp.async.bulk, completion on an mbarrier) into
//    one staging slot that is refilled with the next tile as soon as the
//    current one is split, so the copy overlaps the MMA and the epilogue;
//  - two threads per row split the row into S_A BF16 (or TF32) parts in FP32
//    arithmetic (FP64 inputs are rounded to FP32 first: GB300's FP64 pipe is
//    far too slow for this) and write them in the no-swizzle K-major
//    canonical layout; B (m x n, FP64) is split once per CTA the same way;
//  - one thread issues the split products as tcgen05.mma (M = 128, N = m
//    rounded up to 16, K = n rounded down to the instruction K when one or two
//    columns remain, as for the Lobatto sizes n = 2^k + 1, else rounded up)
//    accumulating in FP32 in TMEM, and commits to an mbarrier; the remaining
//    columns are a rank-1 (or rank-2) FP32 update in the epilogue;
//  - the eight warps read TMEM with tcgen05.ld (warp w: lanes 32 (w % 4) ..,
//    column chunks of 16 alternating between w < 4 and w >= 4) and store the
//    tile transposed (coalesced along r).
// Every wait is bounded; a timeout records CHEB_ETIMEOUT in the context's
// device error word and the CTA drains its copies, frees TMEM and returns.
#include <algorithm>
#include <string>

#include "cheb_internal.cuh"
#include "tc_common.cuh"

namespace cheb {
namespace {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kThreads = 256;
// X staging slots. One slot, refilled as soon as the tile in it is split (its
// copy then overlaps the tile's MMA and epilogue), keeps shared memory small
// enough for four CTAs per SM at BF16x6 (three with FP64 rows).
constexpr int kStages = 1;
constexpr int kMaxTail = 2;   // K columns beyond the last full instruction K done in FP32
constexpr int kMaxM = 256;

template <int FORM> struct Form;
// BF16x3: x = x0 + x1, products x1*y0 + x0*y1 + x0*y0 (small terms first).
template <> struct Form<CHEB_BF16X3> {
    static constexpr int SA = 2, SB = 2, NPROD = 3, EBYTES = 2, FMT = 1;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};
// BF16x6: x = x0 + x1 + x2, the six products with i + j <= 2.
template <> struct Form<CHEB_BF16X6> {
    static constexpr int SA = 3, SB = 3, NPROD = 6, EBYTES = 2, FMT = 1;
    __device__ static constexpr int pa(int p)
    {
        return p == 0 ? 2 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 1 : p == 4 ? 0 : 0;
    }
    __device__ static constexpr int pb(int p)
    {
        return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 2 : p == 3 ? 0 : p == 4 ? 1 : 0;
    }
};
// TF32x3: x = x0 + x1 in TF32, products x1*y0 + x0*y1 + x0*y0.
template <> struct Form<CHEB_TF32X3> {
    static constexpr int SA = 2, SB = 2, NPROD = 3, EBYTES = 4, FMT = 2;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};

struct Params {
    const void *X;
    const double *B;          // m x n FP64, or null: then B[j][k] = T_k(x~_j) from xpts
    const double *xpts;       // m points on [ta, tb] (used when B is null)
    double xscale, xshift;    // x~ = xscale x + xshift = (2 x - ta - tb) / (tb - ta)
    float *out;
    int64_t R;
    int n, m;
    int Kp;        // K on the tensor cores: n rounded down (or up) to the instruction K
    int tail;      // n - Kp columns (0..kMaxTail) added in FP32 in the epilogue
    int Np;        // N = m padded to 16
    int tmem_cols; // power of two >= max(32, Np)
    int *err;
    long long wait_limit;   // SM cycles a main-loop wait may take (exit-path waits use the default)
};

__host__ __device__ constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Split 16 bytes worth of consecutive K elements (8 BF16 / 4 TF32) of one
// row into S parts (FP32 arithmetic) and store each part's 16-byte chunk.
template <int FORM, int S>
__device__ __forceinline__ void split_store_chunk(const float (&v)[16 / Form<FORM>::EBYTES],
                                                  uint8_t *dst, uint32_t split_stride)
{
    if constexpr (Form<FORM>::EBYTES == 2) {
        uint32_t w[S][4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float a = v[2 * p], b = v[2 * p + 1];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // .x = a (low half)
                w[s][p] = *reinterpret_cast<const uint32_t *>(&h);
                const float2 f = __bfloat1622float2(h);
                a -= f.x;
                b -= f.y;
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
            *reinterpret_cast<uint4 *>(dst + s * split_stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    } else {
        uint32_t w[S][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float r = v[e];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                w[s][e] = tf32_rna(r);
                r -= __uint_as_float(w[s][e]);
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s)
            *reinterpret_cast<uint4 *>(dst + s * split_stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
}

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return (float)x; }

template <int FORM, typename XT>
__global__ void __launch_bounds__(kThreads, 2)
modeprod_tc_kernel(const Params P)
{
    using F = Form<FORM>;
    constexpr int E = 16 / F::EBYTES;       // K elements per 16-byte chunk
    constexpr int SA = F::SA, SB = F::SB;
    const int n = P.n, m = P.m, Kp = P.Kp, Np = P.Np;
    const int KC = Kp / E;                  // 16-byte chunks along K
    const int ksteps = KC / 2;              // one MMA covers 32 bytes of K
    const uint32_t a_split_bytes = (uint32_t)kTileM * Kp * F::EBYTES;
    const uint32_t b_split_bytes = (uint32_t)Np * Kp * F::EBYTES;
    const uint32_t stage_bytes = (uint32_t)round_up(kTileM * n * (int)sizeof(XT), 128);

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;                                   // SA x [128 x Kp]
    uint8_t *sB = sA + SA * a_split_bytes;                // SB x [Np x Kp]
    float *sBt = reinterpret_cast<float *>(sB + SB * b_split_bytes);   // kMaxTail x Np FP32 tail columns of B
    uint8_t *sX = reinterpret_cast<uint8_t *>(sBt + kMaxTail * kMaxM);  // 2 x staged X tile
    uint64_t *bars = reinterpret_cast<uint64_t *>(sX + kStages * stage_bytes);  // [0,1] loads, [2] mma
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (P.R + kTileM - 1) / kTileM;
    // the carve-up above fits the dynamic shared memory (uniform: all or none return)
    if (!CHEB_DCHECK((uint32_t)(reinterpret_cast<uint8_t *>(abort_flag + 1) - smem) <= dyn_smem_bytes())) return;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, (uint32_t)P.tmem_cols);
        tmem_relinquish();
    }

    // B splits, once per CTA: rows j < Np, chunks c < KC. With xpts given,
    // row j is T_0..T_{n-1} at x~_j = (2 x_j - ta - tb) / (tb - ta) by the
    // three-term recurrence in double-float (one row per thread, then split);
    // the points are caller input, written before the chain started, so this
    // overlaps the previous kernel. A given B may come from the previous
    // kernel in the stream (the T-matrix kernel): it is read only after the
    // wait for that kernel's completion and memory.
    if (P.B) {
        griddep_launch_dependents();
        griddep_wait();
        for (int t = tid; t < Np * KC; t += kThreads) {
            const int j = t / KC, c = t - j * KC;
            float v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = c * E + e;
                v[e] = (j < m && k < n) ? (float)P.B[(int64_t)j * n + k] : 0.0f;
            }
            if (CHEB_DCHECK((uint32_t)(c * Np + j) * 16 + 16 <= b_split_bytes))
                split_store_chunk<FORM, SB>(v, sB + (uint32_t)c * Np * 16 + j * 16, b_split_bytes);
        }
        for (int t = tid; t < P.tail * Np; t += kThreads) {
            const int q = t / Np, j = t - q * Np;
            if (CHEB_DCHECK(q * Np + j < kMaxTail * kMaxM && Kp + q < n))
                sBt[q * Np + j] = j < m ? (float)P.B[(int64_t)j * n + Kp + q] : 0.0f;
        }
    } else {
        for (int j = tid; j < Np; j += kThreads) {
            const double xr = j < m ? fma(P.xscale, P.xpts[j], P.xshift) : 0.0;
            const ff xf = ff_from_double(xr);
            const ff x2 = {2.0f * xf.hi, 2.0f * xf.lo};
            ff t0 = {1.0f, 0.0f}, t1 = xf;
            for (int c = 0; c < KC; ++c) {
                float v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = c * E + e;
                    float tk;
                    if (k == 0) {
                        tk = 1.0f;
                    } else if (k == 1) {
                        tk = xf.hi + xf.lo;
                    } else {
                        const ff t2 = ff_cheb_step(x2, t1, t0);
                        t0 = t1;
                        t1 = t2;
                        tk = t2.hi + t2.lo;
                    }
                    v[e] = (j < m && k < n) ? tk : 0.0f;
                }
                if (CHEB_DCHECK((uint32_t)(c * Np + j) * 16 + 16 <= b_split_bytes))
                    split_store_chunk<FORM, SB>(v, sB + (uint32_t)c * Np * 16 + j * 16, b_split_bytes);
            }
            // the tail columns continue the same recurrence
            for (int q = 0; q < P.tail; ++q) {
                const int k = Kp + q;
                float tk;
                if (k == 1) {
                    tk = xf.hi + xf.lo;
                } else {
                    const ff t2 = ff_cheb_step(x2, t1, t0);
                    t0 = t1;
                    t1 = t2;
                    tk = t2.hi + t2.lo;
                }
                if (CHEB_DCHECK(q * Np + j < kMaxTail * kMaxM)) sBt[q * Np + j] = j < m ? tk : 0.0f;
            }
        }
    }
    // from here on X (the previous kernel's output) is read
    if (!P.B) {
        griddep_launch_dependents();
        griddep_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const XT *X = static_cast<const XT *>(P.X);
    auto tile_full = [&](int64_t t) { return (t + 1) * kTileM <= P.R; };
    auto issue_load = [&](int64_t t, int buf) {
        const uint32_t bytes = (uint32_t)(kTileM * n * sizeof(XT));
        // a skipped copy leaves its barrier incomplete: the bounded wait gives up
        if (!CHEB_DCHECK((t + 1) * kTileM <= P.R && buf < kStages && bytes <= stage_bytes)) return;
        mbar_arrive_expect_tx(&bars[buf], bytes);
        bulk_g2s(sX + buf * stage_bytes, X + t * kTileM * (int64_t)n, bytes, &bars[buf]);
    };

    uint32_t load_phase = 0;     // bit b: parity of the next completion of load buffer b
    uint32_t load_pending = 0;   // bit b: a copy into buffer b is in flight
    uint32_t mma_phase = 0;
    uint32_t mma_pending = 0;    // the tile's MMAs were issued and not yet waited for
    int64_t tile = blockIdx.x;
    if (tid == 0 && tile < ntiles && tile_full(tile)) issue_load(tile, 0);
    if (tile < ntiles && tile_full(tile)) load_pending |= 1u;

    const uint32_t idesc = make_idesc(F::FMT, kTileM, Np);
    const int row = tid & (kTileM - 1);     // conversion: row of the tile
    const int chalf = tid >> 7;             // conversion: chunk parity
    const int quarter = warp & 3;           // epilogue: TMEM lane quarter
    const int ehalf = warp >> 2;            // epilogue: column-chunk parity
    int it = 0;
    for (; tile < ntiles; tile += gridDim.x, ++it) {
        const int buf = kStages == 2 ? (it & 1) : 0;
        const int64_t next = tile + gridDim.x;
        if (kStages == 2 && next < ntiles && tile_full(next)) {
            if (tid == 0) issue_load(next, buf ^ 1);
            load_pending |= 1u << (buf ^ 1);
        }
        const int rows = (int)((P.R - tile * kTileM) < kTileM ? (P.R - tile * kTileM) : kTileM);
        const XT *xs;
        if (load_pending & (1u << buf)) {
            // a copy whose wait gave up stays pending: the exit path waits for it
            if (mbar_wait_bounded(&bars[buf], (load_phase >> buf) & 1u, P.err, P.wait_limit)) {
                load_phase ^= 1u << buf;
                load_pending &= ~(1u << buf);
            } else {
                *abort_flag = 1;
            }
            xs = reinterpret_cast<const XT *>(sX + buf * stage_bytes);
        } else {
            // ragged last tile: plain loads straight from global memory
            xs = X + tile * kTileM * (int64_t)n;
        }
        // split row `row` of the tile into SA parts (zero beyond the data);
        // its tail columns stay in registers for the epilogue, which this
        // thread runs for the same row
        float xt[kMaxTail];
        {
            const bool valid = row < rows && CHEB_DCHECK(tile * kTileM + row < P.R);
            const XT *xr = xs + row * n;
#pragma unroll
            for (int q = 0; q < kMaxTail; ++q) xt[q] = (valid && q < P.tail) ? to_f32(xr[Kp + q]) : 0.0f;
            // two chunks per pass, loaded before anything is stored (the
            // stores could otherwise hold the loads back)
            for (int c0 = chalf; c0 < KC; c0 += 4) {
                const bool two = c0 + 2 < KC;
                float v0[E], v1[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = c0 * E + e;
                    v0[e] = (valid && k < n) ? to_f32(xr[k]) : 0.0f;
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = (c0 + 2) * E + e;
                    v1[e] = (valid && two && k < n) ? to_f32(xr[k]) : 0.0f;
                }
                if (!CHEB_DCHECK((uint32_t)((two ? c0 + 2 : c0) * kTileM + row) * 16 + 16 <= a_split_bytes)) break;
                split_store_chunk<FORM, SA>(v0, sA + (uint32_t)c0 * (kTileM * 16) + row * 16, a_split_bytes);
                if (two)
                    split_store_chunk<FORM, SA>(v1, sA + (uint32_t)(c0 + 2) * (kTileM * 16) + row * 16, a_split_bytes);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*abort_flag) break;
        // one slot: the rows are split, so the next tile's copy can start now
        if (kStages == 1 && next < ntiles && tile_full(next)) {
            if (tid == 0) issue_load(next, 0);
            load_pending |= 1u;
        }
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int p = 0; p < F::NPROD; ++p) {
                const uint32_t ab = a0 + F::pa(p) * a_split_bytes;
                const uint32_t bb = b0 + F::pb(p) * b_split_bytes;
                for (int ks = 0; ks < ksteps; ++ks) {
                    const uint64_t ad = make_sdesc(ab + ks * 2 * (kTileM * 16), kTileM * 16, 128);
                    const uint64_t bd = make_sdesc(bb + ks * 2 * (Np * 16), Np * 16, 128);
                    if constexpr (F::FMT == 2)
                        mma_tf32(tmem, ad, bd, idesc, (p | ks) != 0);
                    else
                        mma_bf16(tmem, ad, bd, idesc, (p | ks) != 0);
                }
            }
            mma_commit(&bars[2]);
        }
        mma_pending = 1;
        if (mbar_wait_bounded(&bars[2], mma_phase, P.err, P.wait_limit)) {
            mma_phase ^= 1;
            mma_pending = 0;
        } else {
            *abort_flag = 1;
        }
        tc_fence_after();
        // epilogue: rows 32*quarter + lane, column chunks ehalf, ehalf + 2, ...
        {
            const int r = quarter * 32 + lane;
            const bool valid = r < rows && CHEB_DCHECK(tile * kTileM + r < P.R);
            const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
            float *o = P.out + tile * kTileM + r;
            for (int c0 = ehalf * 16; c0 < Np; c0 += 32) {
                uint32_t v[16];
                tmem_ld16(lane_addr + c0, v);
                // B's first tail column for these 16 columns, in registers
                // before any store (the stores could otherwise order the loads)
                float bt[16];
                if (P.tail > 0) {
                    const float4 *s4 = reinterpret_cast<const float4 *>(sBt + c0);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 f = s4[q4];
                        bt[4 * q4] = f.x;
                        bt[4 * q4 + 1] = f.y;
                        bt[4 * q4 + 2] = f.z;
                        bt[4 * q4 + 3] = f.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) bt[q] = 0.0f;
                }
                tmem_ld_wait();
                if (valid) {
                    float y[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) y[q] = fmaf(xt[0], bt[q], __uint_as_float(v[q]));
                    if (P.tail > 1) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) y[q] = fmaf(xt[1], sBt[Np + c0 + q], y[q]);
                    }
                    float *oc = o + (int64_t)c0 * P.R;
                    const int lim = m - c0;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        if (q < lim && CHEB_DCHECK(c0 + q < m)) *oc = y[q];
                        oc += P.R;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
    }
    // drain copies and MMAs still in flight (abort path, full bound), then free TMEM
    for (int b = 0; b < 2; ++b)
        if (load_pending & (1u << b)) mbar_wait_bounded(&bars[b], (load_phase >> b) & 1u, P.err);
    if (mma_pending) mbar_wait_bounded(&bars[2], mma_phase, P.err);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)P.tmem_cols);
}

template <int FORM> constexpr int kAlignK = (Form<FORM>::EBYTES == 2) ? 16 : 8;

template <int FORM, typename XT>
cheb_status launch(const Params &P0, int num_sms, cudaStream_t st)
{
    using F = Form<FORM>;
    Params P = P0;
    // K on the tensor cores: n rounded down to the instruction K when at most
    // kMaxTail columns remain (n = 2^k + 1, the Lobatto sizes: one column),
    // else rounded up with zero padding
    P.Kp = P.n / kAlignK<FORM> * kAlignK<FORM>;
    P.tail = P.n - P.Kp;
    if (P.Kp == 0 || P.tail > kMaxTail) {
        P.Kp = round_up(P.n, kAlignK<FORM>);
        P.tail = 0;
    }
    P.Np = round_up(P.m, 16);
    int cols = 32;
    while (cols < P.Np) cols *= 2;
    P.tmem_cols = cols;
    const size_t a_bytes = (size_t)F::SA * kTileM * P.Kp * F::EBYTES;
    const size_t b_bytes = (size_t)F::SB * P.Np * P.Kp * F::EBYTES;
    const size_t stage = (size_t)round_up(kTileM * P.n * (int)sizeof(XT), 128);
    const size_t smem = a_bytes + b_bytes + kMaxTail * kMaxM * sizeof(float) + kStages * stage + 64;
    if (smem > 227 * 1024) return fail(CHEB_EUNSUPPORTED, "modeprod_tc: tile does not fit in shared memory");
    auto kern = modeprod_tc_kernel<FORM, XT>;
    // kernel attributes once per device; CTAs per SM from the shared-memory
    // budget (the occupancy query reports one CTA here although two fit),
    // capped by TMEM columns, threads and the registers per thread
    static PerDevice once;
    int regs = 0;
    cheb_status ra = per_device_once(once, [kern](int *v) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        CHEB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
        cudaFuncAttributes fa;
        CHEB_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        *v = std::max(1, (fa.numRegs + 7) / 8 * 8);
        return CHEB_OK;
    }, &regs);
    if (ra) return ra;
    int per_sm = (int)(228 * 1024 / (smem + 1024));
    per_sm = std::max(1, std::min({per_sm, 2048 / kThreads, 65536 / (regs * kThreads)}));
    while (per_sm > 1 && per_sm * P.tmem_cols > 512) --per_sm;
    const int64_t ntiles = (P.R + kTileM - 1) / kTileM;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms * per_sm);
    ProfScope prof("modeprod_tc R=" + std::to_string(P.R) + " n=" + std::to_string(P.n) +
                       " m=" + std::to_string(P.m) + (sizeof(XT) == 8 ? " x=f64" : " x=f32"),
                   st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CHEB_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, P));
    return CHEB_OK;
}

}  // namespace

cheb_status modeprod_tc_raw(const void *X, int x_f64, const double *B, float *out, int64_t R, int n,
                            int m, cheb_precision prec, int *err, int num_sms, cudaStream_t st,
                            const double *xpts, double ta, double tb, long long wait_limit)
{
    if (R <= 0 || m <= 0) return CHEB_OK;
    if (n < 1 || n > 64) return fail(CHEB_EUNSUPPORTED, "modeprod_tc: n must be in [1, 64]");
    if (m > kMaxM) return fail(CHEB_EUNSUPPORTED, "modeprod_tc: m must be <= 256");
    if ((reinterpret_cast<uintptr_t>(X) & 15) != 0)
        return fail(CHEB_EINVAL, "modeprod_tc: X must be 16-byte aligned");
    Params P{};
    if (!B && !xpts) return fail(CHEB_EINVAL, "modeprod_tc: need B or the points");
    P.X = X;
    P.B = B;
    P.xpts = xpts;
    P.xscale = 2.0 / (tb - ta);
    P.xshift = -(ta + tb) / (tb - ta);
    P.out = out;
    P.R = R;
    P.n = n;
    P.m = m;
    P.err = err;
    P.wait_limit = wait_limit;
    switch (prec) {
    case CHEB_BF16X3:
        return x_f64 ? launch<CHEB_BF16X3, double>(P, num_sms, st) : launch<CHEB_BF16X3, float>(P, num_sms, st);
    case CHEB_BF16X6:
        return x_f64 ? launch<CHEB_BF16X6, double>(P, num_sms, st) : launch<CHEB_BF16X6, float>(P, num_sms, st);
    case CHEB_TF32X3:
        return x_f64 ? launch<CHEB_TF32X3, double>(P, num_sms, st) : launch<CHEB_TF32X3, float>(P, num_sms, st);
    default:
        return fail(CHEB_EINVAL, "modeprod_tc: not a split precision");
    }
}

cheb_status modeprod_tc(cheb_ctx *ctx, const void *X, int x_f64, const double *B, float *out,
                        int64_t R, int n, int m, cheb_precision prec, cudaStream_t st,
                        const double *xpts, double ta, double tb)
{
    return modeprod_tc_raw(X, x_f64, B, out, R, n, m, prec, ctx->d_error, ctx->num_sms, st, xpts, ta, tb,
                           ctx->wait_limit);
}

}  // namespace cheb
