// Two successive mode products of the tensor-grid evaluation fused in one
// kernel on the tcgen05 tensor cores (Section 3.2: the values on the grid are
// the coefficient tensor multiplied along every mode by that mode's Chebyshev
// matrix B_s(j, l) = T_l(x_j); here two of those products per launch).
//
// On a row-major X of shape [P][n_a][n_b][Q] it computes
//     out[p][j_a][j_b][q] = sum_{k_a, k_b} T_a[j_a, k_a] T_b[j_b, k_b] X[p][k_a][k_b][q]
// into an FP32 out of shape [P][m_a][m_b][Q]: the products along modes a and b
// with every other index left in place. An evaluation with an even number d of
// modes is d / 2 such launches, on the mode pairs (0, 1), (2, 3), ... in this
// order; the last one has Q = 1.
//
// Work unit u = p Q + q: the n_a x n_b matrix X_u (entries Q apart). A tile is
// G = 4 consecutive units. Per tile (256 threads, up to two CTAs per SM):
//  1. split: the rows (k_a, g) of the tile's matrices (over k_b), rounded to
//     FP32 and split into BF16 (or TF32) parts in the K-major canonical layout,
//     operand B of MMA 1. With Q = 1 the tile is one contiguous block, brought
//     into shared memory by a bulk copy (TMA engine) issued while the previous
//     tile computes; with Q > 1 the entries are loaded directly, consecutive
//     threads reading consecutive q.
//  2. MMA 1: A = T_b (rows j_b; M = 128, rows >= m_b unused), N = K_a G,
//     K = k_b. TMEM lane j_b then holds H_g[k_a, j_b] = sum_{k_b} T_b[j_b, k_b]
//     X_g[k_a, k_b] for every (k_a, g) of the tile.
//  3. epilogue 1: each lane j_b adds the k_b tail columns (FP32) and writes its
//     H values as the rows (g, j_b) of operand A of MMA 2, split again; the
//     contraction index k_a is already contiguous along each lane, so the
//     intermediate never leaves the SM and needs no transpose.
//  4. MMA 2: A = those rows (in pieces of 128), B = T_a (N = m_a), K = k_a.
//  5. epilogue 2: TMEM lane (g, j_b) holds out_g[j_a][j_b] for every j_a; the
//     k_a tail rows are added in FP32 and the values stored (with Q = 1 the
//     32 lanes of a warp are 32 consecutive j_b, with Q > 1 consecutive q).
// K on the tensor cores is n rounded down to the instruction K when one or two
// columns remain (the Lobatto sizes n = 2^k + 1), else rounded up with zeros;
// the remaining columns are FP32 updates. The Chebyshev rows come from the
// three-term recurrence carried in double-float in the prologue (points are
// caller input, so the prologue overlaps the previous kernel of the stream).
// Every wait is bounded; a timeout records CHEB_ETIMEOUT, drains the copies
// and MMAs in flight with the default bound, frees TMEM and returns.
#include <algorithm>
#include <string>

#include "cheb_internal.cuh"
#include "tc_common.cuh"

namespace cheb {
namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kG = 4;          // units per tile
constexpr int kMaxTail = 2;

template <int FORM> struct PForm;
template <> struct PForm<CHEB_BF16X3> {
    static constexpr int S = 2, NPROD = 3, EB = 2, FMT = 1, KALIGN = 16;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};
template <> struct PForm<CHEB_BF16X6> {
    static constexpr int S = 3, NPROD = 6, EB = 2, FMT = 1, KALIGN = 16;
    __device__ static constexpr int pa(int p) { return p == 0 ? 2 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 2 : p == 3 ? 0 : p == 4 ? 1 : 0; }
};
template <> struct PForm<CHEB_TF32X3> {
    static constexpr int S = 2, NPROD = 3, EB = 4, FMT = 2, KALIGN = 8;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};

struct PairParams {
    const void *X;
    float *out;
    const double *xa, *xb;        // m_a and m_b points of modes a and b
    double sa, ha, sb, hb;        // reference coordinate x~ = s x + h
    int64_t Q, U;                 // units U = P Q
    int n_a, n_b, m_a, m_b;
    int Ka, ta, Kb, tb;           // tensor-core K and FP32 tail of modes a and b
    int Npa;                      // N of MMA 2: m_a padded to 16
    int MBp;                      // m_b padded to 32 (MMA 2 has kG * MBp rows)
    int pieces;                   // kG * MBp / 128
    int rowsA1;                   // T_b rows stored (m_b padded to 8)
    int NB1;                      // N of MMA 1: Ka * kG
    int tmem_cols;
    // shared-memory layout (byte offsets)
    uint32_t oA1, oB2, oR, oStage, oTb32, oXt, oXr, oGt, oTat, oTbt, oBar;
    uint32_t partA1, partB2, partB1, partA2;   // byte stride between split parts
    int *err;
    long long wait_limit;
};

__host__ __device__ constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

// 16 bytes worth of consecutive K elements (8 BF16 / 4 TF32) of one row,
// split into S parts in FP32 arithmetic; part s goes to dst + s * part_stride.
template <int FORM>
__device__ __forceinline__ void split16(const float *v, uint8_t *dst, uint32_t part_stride)
{
    using F = PForm<FORM>;
    if constexpr (F::EB == 2) {
        uint32_t w[F::S][4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float a = v[2 * p], b = v[2 * p + 1];
#pragma unroll
            for (int s = 0; s < F::S; ++s) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                w[s][p] = *reinterpret_cast<const uint32_t *>(&h);
                const float2 f = __bfloat1622float2(h);
                a -= f.x;
                b -= f.y;
            }
        }
#pragma unroll
        for (int s = 0; s < F::S; ++s)
            *reinterpret_cast<uint4 *>(dst + s * part_stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    } else {
        uint32_t w[F::S][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float r = v[e];
#pragma unroll
            for (int s = 0; s < F::S; ++s) {
                w[s][e] = tf32_rna(r);
                r -= __uint_as_float(w[s][e]);
            }
        }
#pragma unroll
        for (int s = 0; s < F::S; ++s)
            *reinterpret_cast<uint4 *>(dst + s * part_stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
    }
}

__device__ __forceinline__ float ld_f32(const float *p) { return *p; }
__device__ __forceinline__ float ld_f32(const double *p) { return (float)*p; }

// Chebyshev row T_0..T_{n-1}(x~) by the three-term recurrence in double-float,
// one value at a time: call next() n times.
struct ChebRow {
    ff x2, t0, t1, xf;
    int k;
    __device__ explicit ChebRow(double xr) : k(0)
    {
        xf = ff_from_double(xr);
        x2 = {2.0f * xf.hi, 2.0f * xf.lo};
        t0 = {1.0f, 0.0f};
        t1 = xf;
    }
    __device__ float next()
    {
        float v;
        if (k == 0) {
            v = 1.0f;
        } else if (k == 1) {
            v = xf.hi + xf.lo;
        } else {
            const ff t2 = ff_cheb_step(x2, t1, t0);
            t0 = t1;
            t1 = t2;
            v = t2.hi + t2.lo;
        }
        ++k;
        return v;
    }
};

template <int FORM, typename XT>
__global__ void __launch_bounds__(kThreads, 2)
modepair_tc_kernel(const PairParams P)
{
    using F = PForm<FORM>;
    constexpr int E = 16 / F::EB;            // K elements per 16-byte chunk
    const int KCa = P.Ka / E, KCb = P.Kb / E;
    const int NB1 = P.NB1;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA1 = smem + P.oA1;              // T_b split: parts x KCb chunks x rowsA1 rows x 16 B
    uint8_t *sB2 = smem + P.oB2;              // T_a split: parts x KCa chunks x Npa rows x 16 B
    uint8_t *sR = smem + P.oR;                // B1 (MMA 1 operand B) and later A2 (MMA 2 operand A)
    const XT *sStage = reinterpret_cast<const XT *>(smem + P.oStage);
    float *sTb32 = reinterpret_cast<float *>(smem + P.oTb32);   // [m_b][n_b] T_b in FP32 (k_a tails)
    float *sXt = reinterpret_cast<float *>(smem + P.oXt);       // [tb][NB1] X_g[k_a][Kb + t]
    float *sXr = reinterpret_cast<float *>(smem + P.oXr);       // [ta][kG][n_b] X_g[Ka + t][k]
    float *sGt = reinterpret_cast<float *>(smem + P.oGt);       // [kG][ta][MBp] tail rows of H
    float *sTat = reinterpret_cast<float *>(smem + P.oTat);     // [ta][Npa] T_a[j_a][Ka + t]
    float *sTbt = reinterpret_cast<float *>(smem + P.oTbt);     // [tb][128] T_b[j_b][Kb + t]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + P.oBar);   // [0] stage, [1] MMA 1, [2] MMA 2
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (P.U + kG - 1) / kG;
    const int64_t Q = P.Q;
    const int n_a = P.n_a, n_b = P.n_b, m_a = P.m_a, m_b = P.m_b;

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

    // ---- prologue: the two Chebyshev matrices, split (independent of X) ----
    if (tid < 128) {
        for (int j = tid; j < P.rowsA1; j += 128) {
            const bool valid = j < m_b;
            ChebRow row(valid ? fma(P.sb, P.xb[j], P.hb) : 0.0);
            for (int c = 0; c < KCb; ++c) {
                float v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = c * E + e;
                    const float t = row.next();
                    v[e] = (valid && k < n_b) ? t : 0.0f;
                    if (P.ta > 0 && valid && k < n_b) sTb32[j * n_b + k] = t;
                }
                split16<FORM>(v, sA1 + (uint32_t)c * P.rowsA1 * 16 + j * 16, P.partA1);
            }
            for (int k = P.Kb; k < n_b; ++k) {
                const float t = row.next();
                if (valid) {
                    sTbt[(k - P.Kb) * 128 + j] = t;
                    if (P.ta > 0) sTb32[j * n_b + k] = t;
                }
            }
            if (!valid)
                for (int t = 0; t < P.tb; ++t) sTbt[t * 128 + j] = 0.0f;
        }
    } else {
        for (int j = tid - 128; j < P.Npa; j += 128) {
            const bool valid = j < m_a;
            ChebRow row(valid ? fma(P.sa, P.xa[j], P.ha) : 0.0);
            for (int c = 0; c < KCa; ++c) {
                float v[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int k = c * E + e;
                    const float t = row.next();
                    v[e] = (valid && k < n_a) ? t : 0.0f;
                }
                split16<FORM>(v, sB2 + (uint32_t)c * P.Npa * 16 + j * 16, P.partB2);
            }
            for (int k = P.Ka; k < P.Ka + P.ta; ++k) {
                const float t = row.next();
                sTat[(k - P.Ka) * P.Npa + j] = valid ? t : 0.0f;
            }
        }
    }
    // from here on X, the previous kernel's output, is read
    griddep_launch_dependents();
    griddep_wait();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tmem2 = tmem + (uint32_t)NB1;     // MMA 2 accumulators, Npa columns per piece

    const XT *X = static_cast<const XT *>(P.X);
    const int64_t tile_elems = (int64_t)kG * n_a * n_b;       // a full tile with Q = 1
    const uint32_t stage_bytes = (uint32_t)(tile_elems * sizeof(XT));
    auto tile_staged = [&](int64_t t) { return Q == 1 && (t + 1) * kG <= P.U; };
    auto issue_stage = [&](int64_t t) {
        mbar_arrive_expect_tx(&bars[0], stage_bytes);
        bulk_g2s(smem + P.oStage, X + t * tile_elems, stage_bytes, &bars[0]);
    };

    uint32_t st_phase = 0, st_pending = 0;
    uint32_t mma1_phase = 0, mma1_pending = 0, mma2_phase = 0, mma2_pending = 0;
    int64_t tile = blockIdx.x;
    if (tile < ntiles && tile_staged(tile)) {
        if (tid == 0) issue_stage(tile);
        st_pending = 1;
    }
    const int qa = warp & 3, wh = warp >> 2;
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t u0 = tile * kG;
        const int units = (int)((P.U - u0) < kG ? (P.U - u0) : kG);
        const int64_t next = tile + gridDim.x;
        // ---- 1. split the tile's rows into operand B of MMA 1 ----
        bool staged = false;
        if (st_pending) {
            if (mbar_wait_bounded(&bars[0], st_phase, P.err, P.wait_limit)) {
                st_phase ^= 1u;
                st_pending = 0;
            } else {
                *abort_flag = 1;
            }
            staged = true;
        }
        // element (g, k_a, k_b) of the tile
        auto elem = [&](int g, int ka, int kb) -> float {
            if (g >= units || ka >= n_a || kb >= n_b) return 0.0f;
            if (staged) return ld_f32(sStage + ((int64_t)g * n_a + ka) * n_b + kb);
            const int64_t u = u0 + g;
            const int64_t p = u / Q, q = u - p * Q;
            return ld_f32(X + ((p * n_a + ka) * n_b + kb) * Q + q);
        };
        for (int idx = tid; idx < NB1 * KCb; idx += kThreads) {
            const int r = idx % NB1, c = idx / NB1;
            const int ka = r / kG, g = r - ka * kG;
            float v[E];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = elem(g, ka, c * E + e);
            split16<FORM>(v, sR + (uint32_t)c * NB1 * 16 + r * 16, P.partB1);
        }
        for (int idx = tid; idx < P.tb * NB1; idx += kThreads) {
            const int t = idx / NB1, r = idx - t * NB1;
            const int ka = r / kG, g = r - ka * kG;
            sXt[idx] = elem(g, ka, P.Kb + t);
        }
        for (int idx = tid; idx < P.ta * kG * n_b; idx += kThreads) {
            const int k = idx % n_b, g = (idx / n_b) % kG, t = idx / (n_b * kG);
            sXr[idx] = elem(g, P.Ka + t, k);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*abort_flag) break;
        // the stage slot is free: bring the next tile in while this one computes
        if (next < ntiles && tile_staged(next)) {
            if (tid == 0) issue_stage(next);
            st_pending = 1;
        }
        // ---- 2. MMA 1: H = T_b X^T ----
        if (tid == 0) {
            const uint32_t idesc = make_idesc(F::FMT, 128, NB1);
            const uint32_t a0 = smem_u32(sA1), b0 = smem_u32(sR);
#pragma unroll
            for (int p = 0; p < F::NPROD; ++p) {
                const uint32_t ab = a0 + F::pa(p) * P.partA1;
                const uint32_t bb = b0 + F::pb(p) * P.partB1;
                for (int ks = 0; ks < KCb / 2; ++ks) {
                    const uint64_t ad = make_sdesc(ab + ks * 2 * (P.rowsA1 * 16), P.rowsA1 * 16, 128);
                    const uint64_t bd = make_sdesc(bb + ks * 2 * (NB1 * 16), NB1 * 16, 128);
                    if constexpr (F::FMT == 2)
                        mma_tf32(tmem, ad, bd, idesc, (p | ks) != 0);
                    else
                        mma_bf16(tmem, ad, bd, idesc, (p | ks) != 0);
                }
            }
            mma_commit(&bars[1]);
        }
        mma1_pending = 1;
        // the k_a tail rows of H in FP32 while MMA 1 runs:
        // H_g[Ka + t, j_b] = sum_{k_b} T_b[j_b, k_b] X_g[Ka + t, k_b]
        for (int idx = tid; idx < kG * P.ta * m_b; idx += kThreads) {
            const int j = idx % m_b, t = (idx / m_b) % P.ta, g = idx / (m_b * P.ta);
            const float *xr = sXr + (t * kG + g) * n_b;
            const float *tr = sTb32 + j * n_b;
            float s = 0.0f;
            for (int k = 0; k < n_b; ++k) s = fmaf(xr[k], tr[k], s);
            sGt[(g * P.ta + t) * P.MBp + j] = s;
        }
        if (mbar_wait_bounded(&bars[1], mma1_phase, P.err, P.wait_limit)) {
            mma1_phase ^= 1u;
            mma1_pending = 0;
        } else {
            *abort_flag = 1;
        }
        tc_fence_after();
        // ---- 3. epilogue 1: lane j_b -> rows (g, j_b) of operand A of MMA 2 ----
        if (qa * 32 < P.MBp) {
            const int jb = qa * 32 + lane;
            const uint32_t lane_addr = tmem + ((uint32_t)(qa * 32) << 16);
            float tbt[kMaxTail];
#pragma unroll
            for (int t = 0; t < kMaxTail; ++t) tbt[t] = t < P.tb ? sTbt[t * 128 + jb] : 0.0f;
            for (int c = wh; c < KCa; c += 2) {
                float v[E * kG];
                {
                    uint32_t r0[16];
                    tmem_ld16(lane_addr + (uint32_t)(c * E * kG), r0);
                    if constexpr (E * kG == 32) {
                        uint32_t r1[16];
                        tmem_ld16(lane_addr + (uint32_t)(c * E * kG + 16), r1);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            v[i] = __uint_as_float(r0[i]);
                            v[16 + i] = __uint_as_float(r1[i]);
                        }
                    } else {
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r0[i]);
                    }
                }
#pragma unroll
                for (int t = 0; t < kMaxTail; ++t) {
                    if (t < P.tb) {
                        const float *xt = sXt + t * NB1 + c * E * kG;
#pragma unroll
                        for (int i = 0; i < E * kG; ++i) v[i] = fmaf(xt[i], tbt[t], v[i]);
                    }
                }
#pragma unroll
                for (int g = 0; g < kG; ++g) {
                    float w[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) w[e] = v[e * kG + g];
                    const int row = (Q == 1) ? g * P.MBp + jb : jb * kG + g;
                    const int pc = row >> 7, rin = row & 127;
                    split16<FORM>(w, sR + (uint32_t)(pc * KCa + c) * 2048 + rin * 16, P.partA2);
                }
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (*abort_flag) break;
        // ---- 4. MMA 2: out^T = H^T T_a^T, piece by piece ----
        if (tid == 0) {
            const uint32_t idesc = make_idesc(F::FMT, 128, P.Npa);
            const uint32_t a0 = smem_u32(sR), b0 = smem_u32(sB2);
            for (int pc = 0; pc < P.pieces; ++pc) {
#pragma unroll
                for (int p = 0; p < F::NPROD; ++p) {
                    const uint32_t ab = a0 + F::pa(p) * P.partA2 + (uint32_t)pc * KCa * 2048;
                    const uint32_t bb = b0 + F::pb(p) * P.partB2;
                    for (int ks = 0; ks < KCa / 2; ++ks) {
                        const uint64_t ad = make_sdesc(ab + ks * 2 * 2048, 2048, 128);
                        const uint64_t bd = make_sdesc(bb + ks * 2 * (P.Npa * 16), P.Npa * 16, 128);
                        const uint32_t d = tmem2 + (uint32_t)(pc * P.Npa);
                        if constexpr (F::FMT == 2)
                            mma_tf32(d, ad, bd, idesc, (p | ks) != 0);
                        else
                            mma_bf16(d, ad, bd, idesc, (p | ks) != 0);
                    }
                }
            }
            mma_commit(&bars[2]);
        }
        mma2_pending = 1;
        if (mbar_wait_bounded(&bars[2], mma2_phase, P.err, P.wait_limit)) {
            mma2_phase ^= 1u;
            mma2_pending = 0;
        } else {
            *abort_flag = 1;
        }
        tc_fence_after();
        // ---- 5. epilogue 2: k_a tail rows, then the stores ----
        for (int pc = wh; pc < P.pieces; pc += 2) {
            const int row = pc * 128 + qa * 32 + lane;
            const int g = (Q == 1) ? row / P.MBp : row % kG;
            const int jb = (Q == 1) ? row - g * P.MBp : row / kG;
            const bool valid = jb < m_b && g < units;
            int64_t obase = 0;
            if (valid) {
                const int64_t u = u0 + g;
                const int64_t p = u / Q, q = u - p * Q;
                obase = p * m_a * (int64_t)m_b * Q + q + (int64_t)jb * Q;
            }
            float gt[kMaxTail];
#pragma unroll
            for (int t = 0; t < kMaxTail; ++t)
                gt[t] = (t < P.ta && valid) ? sGt[(g * P.ta + t) * P.MBp + jb] : 0.0f;
            const uint32_t lane_addr = tmem2 + (uint32_t)(pc * P.Npa) + ((uint32_t)(qa * 32) << 16);
            const int64_t jstride = (int64_t)m_b * Q;
            for (int c0 = 0; c0 < P.Npa; c0 += 16) {
                uint32_t r[16];
                tmem_ld16(lane_addr + (uint32_t)c0, r);
                float ta[kMaxTail][16];
#pragma unroll
                for (int t = 0; t < kMaxTail; ++t)
#pragma unroll
                    for (int i = 0; i < 16; ++i) ta[t][i] = t < P.ta ? sTat[t * P.Npa + c0 + i] : 0.0f;
                tmem_ld_wait();
                if (valid) {
                    float y[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float s = __uint_as_float(r[i]);
#pragma unroll
                        for (int t = 0; t < kMaxTail; ++t) s = fmaf(gt[t], ta[t][i], s);
                        y[i] = s;
                    }
                    float *o = P.out + obase + (int64_t)c0 * jstride;
                    const int lim = m_a - c0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        if (i < lim) *o = y[i];
                        o += jstride;
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
    }
    // drain what is still in flight (abort path, default bound), then free TMEM
    if (st_pending) mbar_wait_bounded(&bars[0], st_phase, P.err);
    if (mma1_pending) mbar_wait_bounded(&bars[1], mma1_phase, P.err);
    if (mma2_pending) mbar_wait_bounded(&bars[2], mma2_phase, P.err);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)P.tmem_cols);
}

// Shape, TMEM and shared-memory plan of one launch; false if it does not fit.
template <int FORM>
bool plan(PairParams &P, int x_bytes, size_t *smem_out)
{
    using F = PForm<FORM>;
    constexpr int E = 16 / F::EB;
    auto kdim = [](int n, int *K, int *t) {
        *K = n / F::KALIGN * F::KALIGN;
        *t = n - *K;
        if (*K == 0 || *t > kMaxTail) {
            *K = round_up(n, F::KALIGN);
            *t = 0;
        }
    };
    kdim(P.n_a, &P.Ka, &P.ta);
    kdim(P.n_b, &P.Kb, &P.tb);
    if (P.m_b > 128 || P.m_a > 256 || P.n_a > 64 || P.n_b > 64) return false;
    P.Npa = round_up(P.m_a, 16);
    P.MBp = round_up(P.m_b, 32);
    P.pieces = kG * P.MBp / 128;
    P.rowsA1 = round_up(P.m_b, 8);
    P.NB1 = P.Ka * kG;
    if (P.NB1 > 256) return false;
    const int cols = P.NB1 + P.pieces * P.Npa;
    if (cols > 512) return false;
    int tc = 32;
    while (tc < cols) tc *= 2;
    P.tmem_cols = tc;
    const int KCa = P.Ka / E, KCb = P.Kb / E;
    auto al = [](size_t x) { return (x + 127) / 128 * 128; };
    size_t off = 0;
    P.oA1 = (uint32_t)off;
    P.partA1 = (uint32_t)(KCb * P.rowsA1 * 16);
    off = al(off + (size_t)F::S * P.partA1);
    P.oB2 = (uint32_t)off;
    P.partB2 = (uint32_t)(KCa * P.Npa * 16);
    off = al(off + (size_t)F::S * P.partB2);
    // MMA 1 reads 128 rows of T_b: rows >= rowsA1 of the last chunk fall past
    // the A1 block (into the blocks that follow, which exist), never past the end
    P.oR = (uint32_t)off;
    P.partB1 = (uint32_t)(KCb * P.NB1 * 16);
    P.partA2 = (uint32_t)(P.pieces * KCa * 2048);
    off = al(off + std::max((size_t)F::S * P.partB1, (size_t)F::S * P.partA2));
    P.oStage = (uint32_t)off;
    if (P.Q == 1) off = al(off + (size_t)kG * P.n_a * P.n_b * x_bytes);
    P.oTb32 = (uint32_t)off;
    if (P.ta > 0) off = al(off + sizeof(float) * (size_t)P.m_b * P.n_b);
    P.oXt = (uint32_t)off;
    off = al(off + sizeof(float) * (size_t)P.tb * P.NB1);
    P.oXr = (uint32_t)off;
    off = al(off + sizeof(float) * (size_t)P.ta * kG * P.n_b);
    P.oGt = (uint32_t)off;
    off = al(off + sizeof(float) * (size_t)kG * P.ta * P.MBp);
    P.oTat = (uint32_t)off;
    off = al(off + sizeof(float) * (size_t)P.ta * P.Npa);
    P.oTbt = (uint32_t)off;
    off = al(off + sizeof(float) * (size_t)P.tb * 128);
    P.oBar = (uint32_t)off;
    off += 64;
    // the overrun of MMA 1's A rows stays inside the allocation
    const size_t a1_reach = (size_t)P.oA1 + (size_t)(F::S - 1) * P.partA1 + (size_t)(KCb - 1) * P.rowsA1 * 16 +
                            128 * 16;
    if (a1_reach > off) return false;
    *smem_out = off;
    return off <= 227 * 1024;
}

template <int FORM, typename XT>
cheb_status launch_pair(PairParams P, int num_sms, cudaStream_t st)
{
    size_t smem = 0;
    if (!plan<FORM>(P, (int)sizeof(XT), &smem))
        return fail(CHEB_EUNSUPPORTED, "modepair_tc: shape outside the fused kernel's limits");
    auto kern = modepair_tc_kernel<FORM, XT>;
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
    per_sm = std::max(1, std::min({per_sm, 2, 65536 / (regs * kThreads), 512 / P.tmem_cols}));
    const int64_t ntiles = (P.U + kG - 1) / kG;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)num_sms * per_sm);
    ProfScope prof("modepair_tc U=" + std::to_string(P.U) + " Q=" + std::to_string(P.Q) + " n=" +
                       std::to_string(P.n_a) + "x" + std::to_string(P.n_b) + " m=" + std::to_string(P.m_a) + "x" +
                       std::to_string(P.m_b) + (sizeof(XT) == 8 ? " x=f64" : " x=f32"),
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

bool modepair_tc_fits(int n_a, int n_b, int m_a, int m_b, int x_f64, int64_t Q, cheb_precision prec)
{
    PairParams P{};
    P.n_a = n_a;
    P.n_b = n_b;
    P.m_a = m_a;
    P.m_b = m_b;
    P.Q = Q;
    size_t smem = 0;
    const int xb = x_f64 ? 8 : 4;
    switch (prec) {
    case CHEB_BF16X3: return plan<CHEB_BF16X3>(P, xb, &smem);
    case CHEB_BF16X6: return plan<CHEB_BF16X6>(P, xb, &smem);
    case CHEB_TF32X3: return plan<CHEB_TF32X3>(P, xb, &smem);
    default: return false;
    }
}

cheb_status modepair_tc(cheb_ctx *ctx, const void *X, int x_f64, float *out, int64_t Pn, int64_t Q, int n_a, int n_b,
                        int m_a, int m_b, const double *xa, double aa, double ba, const double *xb, double ab,
                        double bb, cheb_precision prec, cudaStream_t st)
{
    if (Pn <= 0 || Q <= 0 || m_a <= 0 || m_b <= 0) return CHEB_OK;
    if (Q == 1 && (reinterpret_cast<uintptr_t>(X) & 15) != 0)
        return fail(CHEB_EINVAL, "modepair_tc: X must be 16-byte aligned");
    PairParams P{};
    P.X = X;
    P.out = out;
    P.xa = xa;
    P.xb = xb;
    P.sa = 2.0 / (ba - aa);
    P.ha = -(aa + ba) / (ba - aa);
    P.sb = 2.0 / (bb - ab);
    P.hb = -(ab + bb) / (bb - ab);
    P.Q = Q;
    P.U = Pn * Q;
    P.n_a = n_a;
    P.n_b = n_b;
    P.m_a = m_a;
    P.m_b = m_b;
    P.err = ctx->d_error;
    P.wait_limit = ctx->wait_limit;
    const int sms = ctx->num_sms;
    switch (prec) {
    case CHEB_BF16X3:
        return x_f64 ? launch_pair<CHEB_BF16X3, double>(P, sms, st) : launch_pair<CHEB_BF16X3, float>(P, sms, st);
    case CHEB_BF16X6:
        return x_f64 ? launch_pair<CHEB_BF16X6, double>(P, sms, st) : launch_pair<CHEB_BF16X6, float>(P, sms, st);
    case CHEB_TF32X3:
        return x_f64 ? launch_pair<CHEB_TF32X3, double>(P, sms, st) : launch_pair<CHEB_TF32X3, float>(P, sms, st);
    default:
        return fail(CHEB_EINVAL, "modepair_tc: not a split precision");
    }
}

}  // namespace cheb
