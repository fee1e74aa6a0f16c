// Split-precision player update of the game iteration on the tcgen05 tensor
// cores (Section 3.4, Steps 1-3), J = 2, 3 or 4 players.
//
// For player i, its first other mode a, the remaining other modes ("rest"),
// node j and the next-state reference coordinates x(j), V_i^[r] along the next
// states is the series
//     w_j[k_i] = sum_{k_a, rest} C_i[k_i, k_a, rest] T_{k_a}(x_a(j)) prod_rest T(x(j)),
// a dense contraction: Y[j, (k_i, rest)] = sum_{k_a} T_{k_a}(x_a(j)) C_i[k_i, k_a, rest]
// is a GEMM (M = nodes, K = n, N = n^(J-1)) and w_j[k_i] is the row-wise
// reduction of Y over the rest modes with their Chebyshev rows (J = 2: no rest,
// w is the GEMM itself; J = 3: one mode b; J = 4: modes b, c with the products
// T_{k_b} T_{k_c} as weights). One fused kernel does both for a 128-node tile
// (described below for J = 3; the others differ only in the reduction):
//  - the A operand T_{k_a}(x_a(j)) is formed in the kernel (double-float
//    three-term recurrence, rounded to FP32, split into BF16/TF32 parts);
//  - the B operand (C_i, columns (k_i, k_b) with k_b padded to a multiple of
//    16) is split once per iteration by game_bprep_kernel into the canonical
//    shared-memory layout, chunk by chunk (<= 256 columns), and each chunk is
//    brought in by one bulk copy (TMA engine), double-buffered;
//  - for n = 16 q + 1 (17, 33) the tensor cores take k_a, k_b < n - 1 with no
//    padding (a third of the MMA work at n = 33, half at n = 17); the
//    k_b = n - 1 column of C_i rides along as 16 extra B columns per chunk
//    (one per k_i of the chunk), and the k_a = n - 1 row is one FP32 dot
//    product per (node, k_i) in the epilogue, its coefficients read from
//    shared memory by 16-byte broadcast loads;
//  - tcgen05.mma accumulates the split products of a chunk in TMEM (FP32);
//  - the epilogue reads TMEM, multiplies by T_{k_b}(x_b(j)) (kept in
//    registers) and writes w_j[k_i] to shared memory;
//  - after the last chunk, one thread per node of the lower 128 maximises
//    over its control (Newton in FP32 from the previous control, the value at
//    the maximiser in double-float and FP64) and writes the new control, value
//    and the FP64 residual, while the upper 128 threads run the next tile's
//    prologue (A operand, T_{k_b} rows staged in shared memory, first B
//    copies, first MMA); the first thread of the upper half issues every bulk
//    copy and MMA.
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "game_internal.cuh"
#include "tc_common.cuh"

namespace cheb {
namespace game {
namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kThreads = 256;
constexpr int kProducer = kTile;    // issues the bulk copies and the MMAs (first thread of the upper half)
constexpr int kPairs = 32;          // (instance, player) pairs interleaved in the work order
// Step 3 inputs of a node, copied into shared memory at the start of its tile
// (the copies complete during the column chunks): u_i, X_i, the old value and
// the node's own Chebyshev node
constexpr int kStep3 = 4;

template <int FORM> struct GForm;
template <> struct GForm<CHEB_BF16X3> {
    static constexpr int SA = 2, SB = 2, NPROD = 3, EB = 2, FMT = 1, KALIGN = 16;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};
template <> struct GForm<CHEB_BF16X6> {
    static constexpr int SA = 3, SB = 3, NPROD = 6, EB = 2, FMT = 1, KALIGN = 16;
    __device__ static constexpr int pa(int p) { return p == 0 ? 2 : p == 1 ? 1 : p == 2 ? 0 : p == 3 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 0 ? 0 : p == 1 ? 1 : p == 2 ? 2 : p == 3 ? 0 : p == 4 ? 1 : 0; }
};
template <> struct GForm<CHEB_TF32X3> {
    static constexpr int SA = 2, SB = 2, NPROD = 3, EB = 4, FMT = 2, KALIGN = 8;
    __device__ static constexpr int pa(int p) { return p == 0 ? 1 : 0; }
    __device__ static constexpr int pb(int p) { return p == 1 ? 1 : 0; }
};

// The column chunk (k_i values per chunk, CH) is the tuned tile shape: it sets
// the MMA N (CH x NBP <= 256), the shared memory of the two B stages and the
// TMEM columns, hence how many CTAs fit on an SM.
template <int FORM, int JJ, int NN, int CH> struct Shape {
    using F = GForm<FORM>;
    // J = 3 and n = 16 q + 1 (the Lobatto sizes 17, 33): the tensor cores take
    // k_a, k_b < n - 1 with no padding, plus the k_b = n - 1 column of C_i as
    // a group of TCOL extra B columns at the front of each chunk (column k_l
    // holds C[k_i, k_a, n-1]); the k_a = n - 1 row is one FP32 dot product per
    // (node, k_i) in the epilogue. Other J pad k_a to the instruction K.
    static constexpr int TAIL = (JJ == 3 && NN > 16 && (NN - 1) % 16 == 0) ? 1 : 0;
    static constexpr int NM = NN - TAIL;                              // k_a (and k_b, J = 3) on the tensor cores
    static constexpr int NPOW = JJ == 2 ? NN * NN : JJ == 3 ? NN * NN * NN : NN * NN * NN * NN;   // n^J
    // rest columns per k_i: J = 2 none (the k_i are the columns), J = 3 the k_b
    // (padded), J = 4 the (k_b, k_c) pairs (padded)
    static constexpr int RESTN = JJ == 2 ? 1 : JJ == 3 ? NM : NN * NN;
    static constexpr int NBP = JJ == 2 ? 1 : (RESTN + 15) / 16 * 16;
    static constexpr int KP = (NM + F::KALIGN - 1) / F::KALIGN * F::KALIGN;   // k_a padded
    static constexpr int E = 16 / F::EB;                            // K elements per 16 bytes
    static constexpr int KC = KP / E;                               // 16-byte chunks along K
    static constexpr int CHKI = CH;                                 // k_i per column chunk
    static constexpr int TCOL = TAIL ? 16 : 0;                      // tail columns per chunk
    static constexpr int NCH = (NN + CHKI - 1) / CHKI;              // column chunks
    static constexpr int NC = JJ == 2 ? (CHKI + 15) / 16 * 16 : TCOL + CHKI * NBP;   // columns of a stored chunk
    static_assert(CH >= 1 && CH <= NN && NC <= 256 && (JJ == 2 || CH <= 16), "column chunk out of range");
    static_assert(NC % 16 == 0 && (JJ == 2 || NBP % 16 == 0), "MMA N must be a multiple of 16");
    static constexpr int SPLIT_BYTES = NC * KP * F::EB;             // one split part of a chunk
    static constexpr int CHUNK_BYTES = F::SB * SPLIT_BYTES;
    static constexpr int A_SPLIT = kTile * KP * F::EB;
    static constexpr int TMEM_COLS = NC <= 32 ? 32 : NC <= 64 ? 64 : NC <= 128 ? 128 : 256;   // one buffer
    static constexpr int TMEM_ALLOC = 2 * TMEM_COLS;                // two accumulators (<= 512)
    // FP32 tail coefficients per player, Ca[k_i][k_b] = C[k_i, n-1, k_b]
    // (k_b < n), rows padded to CAP floats for 16-byte loads
    static constexpr int CAP = (NN + 3) / 4 * 4;
    static constexpr int TAIL_FLOATS = TAIL ? NN * CAP : 0;
    static constexpr size_t PLAYER_BYTES =     // a multiple of 128: every chunk starts 16-byte aligned
        ((size_t)NCH * CHUNK_BYTES + (size_t)TAIL_FLOATS * sizeof(float) + 127) / 128 * 128;
    // rows staged by the prologue for the epilogue: J = 3 T_{k_b} (k_b < NM),
    // and T_{n-1}(x_a), T_{n-1}(x_b) (TAIL); J = 4 T_{k_b} and T_{k_c}
    static constexpr int STG = JJ == 2 ? 0 : JJ == 3 ? NM + 2 * TAIL : 2 * NN;
    static constexpr size_t SMEM = (size_t)F::SA * A_SPLIT + 2 * (size_t)CHUNK_BYTES +
                                   (size_t)NN * kTile * sizeof(float) +              // w
                                   (size_t)TAIL_FLOATS * sizeof(float) +
                                   (size_t)STG * kTile * sizeof(float) +
                                   (size_t)kStep3 * kTile * sizeof(double) + 128;     // Step 3 inputs
    // CTAs per SM that shared memory and TMEM allow, at most 2: the register
    // budget the kernel is compiled to (128 per thread at 2)
    static constexpr int MINB = (2 * (SMEM + 1024) <= 228 * 1024 && 2 * TMEM_ALLOC <= 512) ? 2 : 1;
};

// Column chunks the tuner tries for each player count and node count; the
// first is the default (the widest chunk: fewest MMA rounds, one CTA per SM).
template <int JJ, int NN> struct Chunks;
template <int NN> struct Chunks<2, NN> { static constexpr int count = 1, v0 = NN, v1 = NN, v2 = NN; };  // N = n padded
template <> struct Chunks<3, 5> { static constexpr int count = 2, v0 = 5, v1 = 2, v2 = 2; };
template <> struct Chunks<3, 9> { static constexpr int count = 2, v0 = 9, v1 = 3, v2 = 3; };
template <> struct Chunks<3, 17> { static constexpr int count = 3, v0 = 9, v1 = 6, v2 = 3; };    // N = 160, 112, 64
template <> struct Chunks<3, 33> { static constexpr int count = 3, v0 = 7, v1 = 5, v2 = 3; };    // N = 240, 176, 112
template <> struct Chunks<4, 5> { static constexpr int count = 2, v0 = 5, v1 = 2, v2 = 2; };     // N = 160, 64
template <> struct Chunks<4, 9> { static constexpr int count = 2, v0 = 2, v1 = 1, v2 = 1; };     // N = 192, 96

// ---- helpers -------------------------------------------------------------------
// T_0..T_{NN-1}(x) rounded to FP32, by the three-term recurrence carried in
// double-float (the plain FP32 recurrence loses up to k^2 ulp near |x| = 1).
template <int NN>
__device__ __forceinline__ void cheb_row_f32(double x, float (&T)[NN])
{
    const ff xf = ff_from_double(x);
    const ff x2 = {2.0f * xf.hi, 2.0f * xf.lo};
    ff t0 = {1.0f, 0.0f}, t1 = xf;
    T[0] = 1.0f;
    if (NN > 1) T[1] = xf.hi + xf.lo;
#pragma unroll
    for (int k = 2; k < NN; ++k) {
        const ff t2 = ff_cheb_step(x2, t1, t0);
        T[k] = t2.hi + t2.lo;
        t0 = t1;
        t1 = t2;
    }
}

template <int FORM, int S>
__device__ __forceinline__ void split_store16(const float *v, uint8_t *dst, uint32_t split_stride)
{
    if constexpr (GForm<FORM>::EB == 2) {
        uint32_t w[S][4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float a = v[2 * p], b = v[2 * p + 1];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
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

// the other modes of player i in a J-player game, ascending: o[0] = a, then the rest
template <int JJ>
__device__ __forceinline__ void other_modes(int i, int (&o)[3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = k < i ? k : k + 1;     // k-th mode other than i
}

// stride of mode s in a row-major tensor of J modes with NN entries each
template <int JJ, int NN>
__host__ __device__ constexpr int mode_stride(int s)
{
    int r = 1;
    for (int t = s + 1; t < JJ; ++t) r *= NN;
    return r;
}

// ---- B operand: split C_i once per iteration -----------------------------------
// Thread per (instance, player, chunk, row of the chunk, 16-byte K chunk).
template <int FORM, int JJ, int NN, int CH>
__global__ void game_bprep_kernel(const GameDev *__restrict__ insts, const GameStat *__restrict__ stats, int B)
{
    using S = Shape<FORM, JJ, NN, CH>;
    using F = GForm<FORM>;
    const int per_item = S::NC * S::KC;
    const int64_t total = (int64_t)B * JJ * S::NCH * per_item;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(t % per_item);
        const int64_t it = t / per_item;
        const int c = (int)(it % S::NCH);
        const int i = (int)((it / S::NCH) % JJ);
        const int q = (int)(it / (S::NCH * JJ));
        if (stats[q].done || stats[q].mode != 1) continue;
        const GameDev &g = insts[q];
        const int row = e / S::KC, kc = e - row * S::KC;
        int o[3] = {0, 0, 0};
        other_modes<JJ>(i, o);
        const int si = mode_stride<JJ, NN>(i), sa = mode_stride<JJ, NN>(o[0]);
        const double *C = g.C + (size_t)i * g.NP;
        float v[S::E];
        if (row < S::TCOL) {
            // tail column k_l (J = 3): C[k_i, k_a, n-1]
            const int sb = mode_stride<JJ, NN>(o[1]);
            const int ki = c * S::CHKI + row;
#pragma unroll
            for (int k = 0; k < S::E; ++k) {
                const int ka = kc * S::E + k;
                v[k] = (row < S::CHKI && ki < NN && ka < S::NM) ? (float)C[ki * si + ka * sa + (NN - 1) * sb]
                                                                : 0.0f;
            }
        } else {
            const int mrow = row - S::TCOL;
            int ki, roff;
            bool ok;
            if constexpr (JJ == 2) {
                ki = c * S::CHKI + mrow;
                roff = 0;
                ok = mrow < S::CHKI && ki < NN;
            } else if constexpr (JJ == 3) {
                const int kl = mrow / S::NBP, kb = mrow - kl * S::NBP;
                ki = c * S::CHKI + kl;
                roff = kb * mode_stride<JJ, NN>(o[1]);
                ok = ki < NN && kb < S::NM;
            } else {
                const int kl = mrow / S::NBP, rr = mrow - kl * S::NBP;
                ki = c * S::CHKI + kl;
                const int kb = rr / NN, kcc = rr - kb * NN;
                roff = kb * mode_stride<JJ, NN>(o[1]) + kcc * mode_stride<JJ, NN>(o[2]);
                ok = ki < NN && rr < NN * NN;
            }
#pragma unroll
            for (int k = 0; k < S::E; ++k) {
                const int ka = kc * S::E + k;
                v[k] = (ok && ka < S::NM && CHEB_DCHECK(ki * si + ka * sa + roff < S::NPOW))
                           ? (float)C[ki * si + ka * sa + roff]
                           : 0.0f;
            }
        }
        const size_t off = (size_t)c * S::CHUNK_BYTES + (size_t)kc * (S::NC * 16) + (size_t)row * 16;
        if (!CHEB_DCHECK(off + (size_t)(F::SB - 1) * S::SPLIT_BYTES + 16 <= (size_t)S::NCH * S::CHUNK_BYTES)) continue;
        uint8_t *dst = static_cast<uint8_t *>(g.bsplit) + (size_t)i * S::PLAYER_BYTES + off;
        split_store16<FORM, F::SB>(v, dst, S::SPLIT_BYTES);
    }
    if constexpr (S::TAIL) {
        // the FP32 tail coefficients (J = 3), after each player's chunks
        const int64_t ttot = (int64_t)B * JJ * S::TAIL_FLOATS;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ttot;
             t += (int64_t)gridDim.x * blockDim.x) {
            const int e = (int)(t % S::TAIL_FLOATS);
            const int i = (int)((t / S::TAIL_FLOATS) % JJ);
            const int q = (int)(t / (S::TAIL_FLOATS * JJ));
            if (stats[q].done || stats[q].mode != 1) continue;
            const GameDev &g = insts[q];
            int o[3] = {0, 0, 0};
            other_modes<JJ>(i, o);
            const int si = mode_stride<JJ, NN>(i), sa = mode_stride<JJ, NN>(o[0]), sb = mode_stride<JJ, NN>(o[1]);
            const double *C = g.C + (size_t)i * g.NP;
            const int ki = e / S::CAP, k = e - ki * S::CAP;
            const float v = (k < NN && CHEB_DCHECK(ki * si + (NN - 1) * sa + k * sb < S::NPOW))
                                ? (float)C[ki * si + (NN - 1) * sa + k * sb]
                                : 0.0f;   // Ca[ki][kb = k]
            float *dst = reinterpret_cast<float *>(static_cast<uint8_t *>(g.bsplit) + (size_t)i * S::PLAYER_BYTES +
                                                   (size_t)S::NCH * S::CHUNK_BYTES);
            dst[e] = v;
        }
    }
}

// ---- the fused player kernel ----------------------------------------------------
template <int NN>
__device__ __forceinline__ void objective_f32(const float (&w)[NN], float xc, float slope, float hA, float h,
                                              float delta, float u, float &W, float &W1, float &W2)
{
    const float x = xc + slope * u;
    float t0 = 1.f, t1 = x, d0 = 0.f, d1 = 1.f, e0 = 0.f, e1 = 0.f;
    float s = w[0] + w[1] * x, s1 = w[1], s2 = 0.f;
#pragma unroll
    for (int m = 2; m < NN; ++m) {
        const float t2 = 2.f * x * t1 - t0;
        const float d2 = 2.f * t1 + 2.f * x * d1 - d0;
        const float e2 = 4.f * d1 + 2.f * x * e1 - e0;
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

template <int FORM, int JJ, int NN, int CH>
__global__ void __launch_bounds__(kThreads, (Shape<FORM, JJ, NN, CH>::MINB))
game_player_tc_kernel(const GameDev *__restrict__ insts, GameStat *__restrict__ stats, int B, int *err)
{
    using S = Shape<FORM, JJ, NN, CH>;
    using F = GForm<FORM>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;                                         // SA x [128 x KP]
    uint8_t *sB = sA + F::SA * S::A_SPLIT;                      // 2 stages x CHUNK_BYTES
    float *w_s = reinterpret_cast<float *>(sB + 2 * S::CHUNK_BYTES);   // [NN][128]
    float *ct_s = w_s + NN * kTile;                                   // tail coefficients Ca (TAIL)
    float *tb_s = ct_s + S::TAIL_FLOATS;                              // [STG][128] staged T_{k_b}, T_{n-1}
    double *s3_s = reinterpret_cast<double *>(tb_s + S::STG * kTile);   // [kStep3][128] Step 3 inputs
    uint64_t *bars = reinterpret_cast<uint64_t *>(s3_s + kStep3 * kTile);   // [0,1] B loads, [2,3] mma per accumulator
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 4);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the carve-up above fits the dynamic shared memory (uniform: all or none return)
    if (!CHEB_DCHECK((uint32_t)(reinterpret_cast<uint8_t *>(abort_flag + 1) - smem) <= dyn_smem_bytes())) return;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_init(&bars[3], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, S::TMEM_ALLOC);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    constexpr int NP = S::NPOW;
    const int tiles = (NP + kTile - 1) / kTile;
    const int64_t items = (int64_t)B * JJ * tiles;
    // producer-thread state (tid == kProducer)
    uint32_t ld_phase = 0;     // bit s: parity of B stage s
    uint32_t pending = 0;      // bit s: a copy into stage s is in flight
    uint32_t mma_out = 0;      // bit s: an MMA commit on accumulator s not yet waited for
    uint32_t mma_phase = 0;    // bit s: parity of accumulator s (every thread)

    const int row = tid & (kTile - 1);
    const int half = tid >> 7;
    const int quarter = warp & 3, ehalf = warp >> 2;

    // Work items are (instance q, player i, tile t). They are ordered in blocks
    // of kPairs (q, i) pairs with the pair fastest inside a block, so the CTAs
    // working at one time spread over kPairs coefficient tensors (each read by
    // a few CTAs, all of them resident in L2) instead of all streaming the same
    // one; a contiguous tile order made every CTA fetch the same bytes at once
    // and the bulk copies of B waited on that contention.
    const int npair = B * JJ;
    auto decode = [&](int64_t it, int &t, int &i, int &q) {
        const int64_t blk = it / ((int64_t)kPairs * tiles);
        const int rem = (int)(it - blk * kPairs * tiles);
        const int64_t left = npair - blk * kPairs;
        const int pb = left < kPairs ? (int)left : kPairs;
        t = rem / pb;
        const int pair = (int)(blk * kPairs) + rem % pb;
        i = pair % JJ;
        q = pair / JJ;
    };
    // the next work item at or after `from` whose instance is still iterating
    // in split precision (uniform across the block)
    auto next_item = [&](int64_t from) {
        for (int64_t it = from; it < items; it += gridDim.x) {
            int t, i, q;
            decode(it, t, i, q);
            if (!stats[q].done && stats[q].mode == 1) return it;
        }
        return items;
    };
    // MMA of chunk c into accumulator c & 1 (producer thread); the accumulator
    // of chunk c + 1 is filled while the epilogue drains chunk c
    auto issue_mma = [&](int c) {
        const int stage = c & 1;
        const int kis = (c == S::NCH - 1) ? NN - c * S::CHKI : S::CHKI;
        // MMA N: a multiple of 16 (J = 2 stores the k_i of its one chunk padded to NC)
        const int N = JJ == 2 ? S::NC : S::TCOL + kis * S::NBP;
        // a copy whose wait gave up stays pending: the exit path waits for it
        if (mbar_wait_bounded(&bars[stage], (ld_phase >> stage) & 1u, err)) {
            ld_phase ^= 1u << stage;
            pending &= ~(1u << stage);
        } else {
            *abort_flag = 1;
        }
        tc_fence_after();
        const uint32_t idesc = make_idesc(F::FMT, kTile, N);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + stage * S::CHUNK_BYTES);
        const uint32_t acc = tmem + (uint32_t)(stage * S::TMEM_COLS);
#pragma unroll
        for (int p = 0; p < F::NPROD; ++p) {
            const uint32_t ab = a0 + F::pa(p) * S::A_SPLIT;
            const uint32_t bb = b0 + F::pb(p) * S::SPLIT_BYTES;
#pragma unroll
            for (int ks = 0; ks < S::KC / 2; ++ks) {
                const uint64_t ad = make_sdesc(ab + ks * 2 * (kTile * 16), kTile * 16, 128);
                const uint64_t bd = make_sdesc(bb + ks * 2 * (S::NC * 16), S::NC * 16, 128);
                if constexpr (F::FMT == 2)
                    mma_tf32(acc, ad, bd, idesc, (p | ks) != 0);
                else
                    mma_bf16(acc, ad, bd, idesc, (p | ks) != 0);
            }
        }
        mma_commit(&bars[2 + stage]);
        mma_out |= 1u << stage;
    };
    // Prologue of a tile, run by the upper 128 threads (one per node of the
    // tile) while the lower 128 finish the previous tile's Step 3: the tail
    // coefficients and the first two B chunks are brought in, the A operand
    // T_{k_a}(x_a(j)) is formed and split, T_{k_b}(x_b(j)) is staged for the
    // epilogue, and chunk 0's MMA is issued.
    auto prologue = [&](int64_t it) {
        int t, i, q;
        decode(it, t, i, q);
        const GameDev &g = insts[q];
        int o[3] = {0, 0, 0};
        other_modes<JJ>(i, o);
        const int a = o[0];
        const uint8_t *bsrc = static_cast<const uint8_t *>(g.bsplit) + (size_t)i * S::PLAYER_BYTES;
        if (tid == kProducer)
            for (int c = 0; c < 2 && c < S::NCH; ++c) {
                mbar_arrive_expect_tx(&bars[c], S::CHUNK_BYTES);
                bulk_g2s(sB + c * S::CHUNK_BYTES, bsrc + (size_t)c * S::CHUNK_BYTES, S::CHUNK_BYTES, &bars[c]);
                pending |= 1u << c;
            }
        if constexpr (S::TAIL) {
            const float *tsrc = reinterpret_cast<const float *>(bsrc + (size_t)S::NCH * S::CHUNK_BYTES);
            for (int e = row; e < S::TAIL_FLOATS / 4; e += kTile)
                reinterpret_cast<float4 *>(ct_s)[e] = reinterpret_cast<const float4 *>(tsrc)[e];
        }
        const int j = t * kTile + row;
        const bool valid = j < NP;
        float Ta[NN];
        const double xa = valid ? g.X[a * NP + j] : 0.0;
        cheb_row_f32<NN>(xa, Ta);
        if constexpr (JJ == 3) {
            float Tbn[NN];
            const double xb = valid ? g.X[o[1] * NP + j] : 0.0;
            cheb_row_f32<NN>(xb, Tbn);
#pragma unroll
            for (int k = 0; k < S::NM; ++k) tb_s[k * kTile + row] = valid ? Tbn[k] : 0.0f;
            if constexpr (S::TAIL) {
                tb_s[S::NM * kTile + row] = valid ? Ta[NN - 1] : 0.0f;
                tb_s[(S::NM + 1) * kTile + row] = valid ? Tbn[NN - 1] : 0.0f;
            }
        } else if constexpr (JJ == 4) {
            float Tbn[NN], Tcn[NN];
            const double xb = valid ? g.X[o[1] * NP + j] : 0.0;
            const double xc = valid ? g.X[o[2] * NP + j] : 0.0;
            cheb_row_f32<NN>(xb, Tbn);
            cheb_row_f32<NN>(xc, Tcn);
#pragma unroll
            for (int k = 0; k < NN; ++k) {
                tb_s[k * kTile + row] = valid ? Tbn[k] : 0.0f;
                tb_s[(NN + k) * kTile + row] = valid ? Tcn[k] : 0.0f;
            }
        }
#pragma unroll
        for (int kc = 0; kc < S::KC; ++kc) {
            float v[S::E];
#pragma unroll
            for (int e = 0; e < S::E; ++e) {
                const int k = kc * S::E + e;
                v[e] = (valid && k < S::NM) ? Ta[k < S::NM ? k : 0] : 0.0f;
            }
            split_store16<FORM, F::SA>(v, sA + (uint32_t)kc * (kTile * 16) + row * 16, S::A_SPLIT);
        }
        fence_async_smem();
        named_barrier_sync(1, kTile);
        if (tid == kProducer) issue_mma(0);
    };

    int64_t item = next_item(blockIdx.x);
    if (item < items && half == 1) prologue(item);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    while (item < items) {
        int t, i, q;
        decode(item, t, i, q);
        if (!CHEB_DCHECK(q < B && i < JJ && t < tiles)) break;   // uniform across the block
        GameStat *st = &stats[q];
        const GameDev &g = insts[q];
        const uint8_t *bsrc = static_cast<const uint8_t *>(g.bsplit) + (size_t)i * S::PLAYER_BYTES;
        const int j = t * kTile + row;
        const bool valid = j < NP;
        // Step 3's global inputs of this thread's node, in flight while the
        // column chunks run (the lower half reads them after the chunks)
        if (half == 0) {
            if (valid) {
                const int ki = (j / mode_stride<JJ, NN>(i)) % NN;
                cp_async8(&s3_s[0 * kTile + tid], g.u + i * NP + j);
                cp_async8(&s3_s[1 * kTile + tid], g.X + i * NP + j);
                cp_async8(&s3_s[2 * kTile + tid], g.Vn + i * NP + j);
                cp_async8(&s3_s[3 * kTile + tid], g.nodes + ki);
            }
            cp_async_commit();
        }
        // the epilogue factors of this thread's row, from the stage: J = 3
        // T_{k_b}(x_b(j)); J = 4 T_{k_b}(x_b(j)) and T_{k_c}(x_c(j))
        constexpr int NTB = JJ == 3 ? S::NBP : 1;
        float Tb[NTB];
#pragma unroll
        for (int k = 0; k < NTB; ++k) Tb[k] = (JJ == 3 && k < S::NM) ? tb_s[k * kTile + row] : 0.0f;
        constexpr int N4 = JJ == 4 ? NN : 1;
        float Tb4[N4], Tc4[N4];
#pragma unroll
        for (int k = 0; k < N4; ++k) {
            Tb4[k] = JJ == 4 ? tb_s[k * kTile + row] : 0.0f;
            Tc4[k] = JJ == 4 ? tb_s[(NN + k) * kTile + row] : 0.0f;
        }
        float ta_last = 0.0f, tb_last = 0.0f;    // T_{n-1}(x_a), T_{n-1}(x_b) (TAIL)
        if constexpr (S::TAIL) {
            ta_last = tb_s[S::NM * kTile + row];
            tb_last = tb_s[(S::NM + 1) * kTile + row];
        }
        for (int c = 0; c < S::NCH; ++c) {
            const int buf = c & 1;
            const int kis = (c == S::NCH - 1) ? NN - c * S::CHKI : S::CHKI;   // k_i in this chunk
            if (mbar_wait_bounded(&bars[2 + buf], (mma_phase >> buf) & 1u, err)) {
                mma_phase ^= 1u << buf;
                mma_out &= ~(1u << buf);
            } else {
                *abort_flag = 1;
            }
            tc_fence_after();
            // chunk c + 1 goes to the tensor cores as soon as chunk c is done (its
            // accumulator was drained before the last barrier); issued earlier, the
            // MMAs queue behind chunk c and hold the producer's warp back from
            // its share of the epilogue
            if (tid == kProducer && c + 1 < S::NCH) issue_mma(c + 1);
            // the B stage of chunk c is free again: prefetch chunk c + 2 into it
            // (not while a copy into it is still pending after a timeout)
            if (tid == kProducer && c + 2 < S::NCH && !(pending & (1u << buf))) {
                mbar_arrive_expect_tx(&bars[buf], S::CHUNK_BYTES);
                bulk_g2s(sB + buf * S::CHUNK_BYTES, bsrc + (size_t)(c + 2) * S::CHUNK_BYTES, S::CHUNK_BYTES,
                         &bars[buf]);
                pending |= 1u << buf;
            }
            // epilogue: rows 32 quarter + lane (the row whose T_b this thread
            // holds), k_i of this chunk alternating between the two halves
            if constexpr (JJ == 2) {
                // the columns are the k_i themselves
                const int r = quarter * 32 + lane;
                const uint32_t lane_addr = tmem + (uint32_t)(buf * S::TMEM_COLS) + ((uint32_t)(quarter * 32) << 16);
                for (int g16 = ehalf; g16 < S::NC / 16; g16 += 2) {
                    uint32_t v[16];
                    tmem_ld16(lane_addr + g16 * 16, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int col = g16 * 16 + e;
                        if (col < kis && CHEB_DCHECK(c * S::CHKI + col < NN))
                            w_s[(c * S::CHKI + col) * kTile + r] = __uint_as_float(v[e]);
                    }
                }
            } else if constexpr (JJ == 4) {
                // w[k_i] = sum_{k_b, k_c} Y[(k_i, k_b, k_c)] T_{k_b}(x_b) T_{k_c}(x_c)
                const int r = quarter * 32 + lane;
                const uint32_t lane_addr = tmem + (uint32_t)(buf * S::TMEM_COLS) + ((uint32_t)(quarter * 32) << 16);
                for (int kl = ehalf; kl < kis; kl += 2) {
                    float acc = 0.0f;
#pragma unroll
                    for (int g16 = 0; g16 < S::NBP / 16; ++g16) {
                        uint32_t v[16];
                        tmem_ld16(lane_addr + kl * S::NBP + g16 * 16, v);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int rr = g16 * 16 + e;
                            if (rr < NN * NN) acc = fmaf(__uint_as_float(v[e]), Tb4[rr / N4] * Tc4[rr % N4], acc);
                        }
                    }
                    if (CHEB_DCHECK(c * S::CHKI + kl < NN)) w_s[(c * S::CHKI + kl) * kTile + r] = acc;
                }
            } else {
                const int r = quarter * 32 + lane;
                const uint32_t lane_addr = tmem + (uint32_t)(buf * S::TMEM_COLS) + ((uint32_t)(quarter * 32) << 16);
                for (int kl = ehalf; kl < kis; kl += 2) {
                    uint32_t v[S::NBP / 16][16];
#pragma unroll
                    for (int g16 = 0; g16 < S::NBP / 16; ++g16)
                        tmem_ld16(lane_addr + S::TCOL + kl * S::NBP + g16 * 16, v[g16]);
                    uint32_t vt = 0;
                    if constexpr (S::TAIL) tmem_ld1(lane_addr + kl, vt);
                    tmem_ld_wait();
                    float acc = 0.0f;
#pragma unroll
                    for (int g16 = 0; g16 < S::NBP / 16; ++g16)
#pragma unroll
                        for (int e = 0; e < 16; ++e) acc = fmaf(__uint_as_float(v[g16][e]), Tb[g16 * 16 + e], acc);
                    if constexpr (S::TAIL) {
                        // + T_{n-1}(x_b) sum_{k_a < n-1} C[k_i, k_a, n-1] T_{k_a}(x_a)   (tail column)
                        //   + T_{n-1}(x_a) sum_{k_b} C[k_i, n-1, k_b] T_{k_b}(x_b)      (FP32)
                        const float4 *ca = reinterpret_cast<const float4 *>(ct_s + (c * S::CHKI + kl) * S::CAP);
                        float ta_dot = ct_s[(c * S::CHKI + kl) * S::CAP + NN - 1] * tb_last;
#pragma unroll
                        for (int k4 = 0; k4 < S::NM / 4; ++k4) {
                            const float4 cv = ca[k4];
                            ta_dot = fmaf(cv.x, Tb[4 * k4], ta_dot);
                            ta_dot = fmaf(cv.y, Tb[4 * k4 + 1], ta_dot);
                            ta_dot = fmaf(cv.z, Tb[4 * k4 + 2], ta_dot);
                            ta_dot = fmaf(cv.w, Tb[4 * k4 + 3], ta_dot);
                        }
                        acc = fmaf(ta_last, ta_dot, fmaf(tb_last, __uint_as_float(vt), acc));
                    }
                    if (CHEB_DCHECK(c * S::CHKI + kl < NN)) w_s[(c * S::CHKI + kl) * kTile + r] = acc;
                }
            }
            tc_fence_before();
            __syncthreads();
            if (*abort_flag) break;
        }
        if (*abort_flag) break;
        const int64_t next = next_item(item + gridDim.x);
        if (half == 0) {
            // Step 3 for each node of the tile: one thread per node
            if (valid) {
                float w[NN];
#pragma unroll
                for (int k = 0; k < NN; ++k) w[k] = w_s[k * kTile + tid];
                // the node's own coordinate (row-major multi-index, last player
                // fastest; its Chebyshev node came with the other inputs) and
                // the per-player constants formed on the host
                cp_async_wait_all();
                const double pbi = 0.5 * g.P_M * (s3_s[3 * kTile + tid] + 1.0);
                const double ui = s3_s[0 * kTile + tid];
                const double slope = g.slope[i];
                const double xc = s3_s[1 * kTile + tid] - slope * ui;
                const double hA = g.hA[i];
                const double hG0 = g.hphi2[i] * pbi * pbi;
                const float U_M = (float)g.U_M;
                float u = fminf(fmaxf((float)ui, 0.0f), U_M);
                // Newton on W'(u) = 0; W'' of the last iterate decides below
                // whether the stationary point is a concave interior maximiser
                // (the final step is below 1e-7 U_M)
                float W, W1, W2;
                for (int itn = 0; itn < 12; ++itn) {
                    objective_f32<NN>(w, (float)xc, (float)slope, (float)hA, (float)g.h, (float)g.delta, u, W, W1, W2);
                    float un = (W2 < 0.0f) ? u - W1 / W2 : (W1 > 0.0f ? 0.5f * (u + U_M) : 0.5f * u);
                    un = fminf(fmaxf(un, 0.0f), U_M);
                    const float step = fabsf(un - u);
                    u = un;
                    if (step <= 1e-7f * U_M) break;
                }
                // W at a control: the series sum_m w_m T_m(x) in double-float
                // (T by the recurrence in double-float, products and sums
                // error-free), the rest in FP64
                auto value64 = [&](double uu) {
                    const double x = xc + slope * uu;
                    const ff xf = ff_from_double(x);
                    const ff x2 = {2.0f * xf.hi, 2.0f * xf.lo};
                    ff t0 = {1.0f, 0.0f}, t1 = xf;
                    double s = (double)w[0] + (double)w[1] * ((double)xf.hi + (double)xf.lo);
                    ff acc = {0.0f, 0.0f};
#pragma unroll
                    for (int m = 2; m < NN; ++m) {
                        const ff t2 = ff_cheb_step(x2, t1, t0);
                        // acc += w_m * t2 (error-free product, compensated sum)
                        const float p = w[m] * t2.hi;
                        float e = fmaf(w[m], t2.hi, -p);
                        e = fmaf(w[m], t2.lo, e);
                        const float sh = acc.hi + p;
                        const float bb = sh - acc.hi;
                        const float er = (acc.hi - (sh - bb)) + (p - bb);
                        float lo = acc.lo + e + er;
                        acc.hi = sh + lo;
                        acc.lo = lo - (acc.hi - sh);
                        t0 = t1;
                        t1 = t2;
                    }
                    s += (double)acc.hi + (double)acc.lo;
                    return hA * uu - 0.5 * g.h * uu * uu + hG0 + g.delta * s;
                };
                // the same at three controls, the three recurrences interleaved
                // (independent chains: one evaluation's latency for all three)
                auto value64x3 = [&](const double (&uu)[3], double (&out)[3]) {
                    ff xf[3], x2[3], t0[3], t1[3], acc[3];
                    double s[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        xf[c] = ff_from_double(xc + slope * uu[c]);
                        x2[c] = {2.0f * xf[c].hi, 2.0f * xf[c].lo};
                        t0[c] = {1.0f, 0.0f};
                        t1[c] = xf[c];
                        acc[c] = {0.0f, 0.0f};
                        s[c] = (double)w[0] + (double)w[1] * ((double)xf[c].hi + (double)xf[c].lo);
                    }
#pragma unroll
                    for (int m = 2; m < NN; ++m) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const ff t2 = ff_cheb_step(x2[c], t1[c], t0[c]);
                            const float p = w[m] * t2.hi;
                            float e = fmaf(w[m], t2.hi, -p);
                            e = fmaf(w[m], t2.lo, e);
                            const float sh = acc[c].hi + p;
                            const float bb = sh - acc[c].hi;
                            const float er = (acc[c].hi - (sh - bb)) + (p - bb);
                            float lo = acc[c].lo + e + er;
                            acc[c].hi = sh + lo;
                            acc[c].lo = lo - (acc[c].hi - sh);
                            t0[c] = t1[c];
                            t1[c] = t2;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        s[c] += (double)acc[c].hi + (double)acc[c].lo;
                        out[c] = hA * uu[c] - 0.5 * g.h * uu[c] * uu[c] + hG0 + g.delta * s[c];
                    }
                };
                double us = (double)u;
                double V;
                if (u > 0.0f && u < U_M && W2 < 0.0f) {
                    // a concave stationary point inside (0, U_M): the maximiser
                    V = value64(us);
                } else {
                    // at a bound or not concave: the bounds and the Newton point
                    // compete in FP64 (differences of W near a bound are far below
                    // FP32 resolution), ties to the smaller control
                    const double cu[3] = {0.0, us, g.U_M};
                    double cv[3];
                    value64x3(cu, cv);
                    double bu = 0.0, bv = cv[0];
                    if (cv[1] > bv) { bv = cv[1]; bu = us; }
                    if (cv[2] > bv) { bv = cv[2]; bu = g.U_M; }
                    us = bu;
                    V = bv;
                }
                g.u_new[i * NP + j] = us;
                store_vn_new(g, i * NP + j, V);
                const double d = fabs(V - s3_s[2 * kTile + tid]);
                atomicMax(&st->res_bits, (unsigned long long)__double_as_longlong(d));
            }
        } else if (next < items) {
            prologue(next);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        item = next;
    }
    // drain copies and MMAs in flight (abort path), free TMEM
    cp_async_wait_all();
    if (tid == kProducer) {
        for (int s2 = 0; s2 < 2; ++s2)
            if (pending & (1u << s2)) mbar_wait_bounded(&bars[s2], (ld_phase >> s2) & 1u, err);
        for (int s2 = 0; s2 < 2; ++s2)
            if (mma_out & (1u << s2)) mbar_wait_bounded(&bars[2 + s2], (mma_phase >> s2) & 1u, err);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, S::TMEM_ALLOC);
}

// Most CTAs of one variant that fit on an SM (shared memory, registers, TMEM).
template <int FORM, int JJ, int NN, int CH>
cheb_status max_ctas(int *out)
{
    using S = Shape<FORM, JJ, NN, CH>;
    auto kern = game_player_tc_kernel<FORM, JJ, NN, CH>;
    static PerDevice cache;
    return per_device_once(cache, [kern](int *v) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM));
        CHEB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
        cudaFuncAttributes fa;
        CHEB_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
        const int regs = std::max(8, (fa.numRegs + 7) / 8 * 8);
        int k = (int)(228 * 1024 / (S::SMEM + 1024));
        k = std::min({k, 65536 / (regs * kThreads), 512 / S::TMEM_ALLOC, 2048 / kThreads, 3});
        *v = std::max(1, k);
        return CHEB_OK;
    }, out);
}

template <int FORM, int JJ, int NN, int CH>
cheb_status launch_player(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int per_sm, cudaStream_t st)
{
    using S = Shape<FORM, JJ, NN, CH>;
    static_assert(S::SMEM <= 227 * 1024, "game player tile does not fit in shared memory");
    int kmax = 1;
    cheb_status r = max_ctas<FORM, JJ, NN, CH>(&kmax);
    if (r) return r;
    per_sm = std::max(1, std::min(per_sm, kmax));
    const std::string shape = "J=" + std::to_string(JJ) + " n=" + std::to_string(NN) + " chunk=" + std::to_string(CH);
    {
        const int64_t total = (int64_t)B * JJ * S::NCH * S::NC * S::KC;
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
        ProfScope prof("game_bprep " + shape, st);
        game_bprep_kernel<FORM, JJ, NN, CH><<<blocks, 256, 0, st>>>(d_inst, d_stat, B);
        CHEB_CUDA_TRY(cudaGetLastError());
    }
    const int tiles = (S::NPOW + kTile - 1) / kTile;
    const int64_t items = (int64_t)B * JJ * tiles;
    const int grid = (int)std::min<int64_t>(items, (int64_t)ctx->num_sms * per_sm);
    ProfScope prof("game_player_tc " + shape + " ctas/SM=" + std::to_string(per_sm), st);
    game_player_tc_kernel<FORM, JJ, NN, CH><<<grid, kThreads, S::SMEM, st>>>(d_inst, d_stat, B, ctx->d_error);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

// A tile configuration: chunk variant c (index into Chunks<NN>) and CTAs per SM k.
constexpr int cfg_of(int c, int k) { return c * 4 + k; }

template <int FORM, int JJ, int NN>
cheb_status run_cfg(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int cfg, cudaStream_t st)
{
    using C = Chunks<JJ, NN>;
    const int c = cfg / 4, k = cfg % 4;
    if constexpr (C::count > 1)
        if (c == 1) return launch_player<FORM, JJ, NN, C::v1>(ctx, d_inst, d_stat, B, k, st);
    if constexpr (C::count > 2)
        if (c == 2) return launch_player<FORM, JJ, NN, C::v2>(ctx, d_inst, d_stat, B, k, st);
    return launch_player<FORM, JJ, NN, C::v0>(ctx, d_inst, d_stat, B, k, st);
}

// The configurations the tuner tries for NN: every chunk variant at every CTA
// count from 1 to what fits.
template <int FORM, int JJ, int NN>
cheb_status candidates(std::vector<int> *out)
{
    using C = Chunks<JJ, NN>;
    int k[3] = {1, 1, 1};
    cheb_status r = max_ctas<FORM, JJ, NN, C::v0>(&k[0]);
    if constexpr (C::count > 1)
        if (!r) r = max_ctas<FORM, JJ, NN, C::v1>(&k[1]);
    if constexpr (C::count > 2)
        if (!r) r = max_ctas<FORM, JJ, NN, C::v2>(&k[2]);
    if (r) return r;
    out->clear();
    for (int c = 0; c < C::count; ++c)
        for (int kk = 1; kk <= k[c]; ++kk) out->push_back(cfg_of(c, kk));
    return CHEB_OK;
}

template <int FORM, int JJ, int NN>
std::string describe(int cfg)
{
    using C = Chunks<JJ, NN>;
    const int c = cfg / 4, chunk = c == 0 ? C::v0 : c == 1 ? C::v1 : C::v2;
    const int N = c == 0 ? Shape<FORM, JJ, NN, C::v0>::NC : c == 1 ? Shape<FORM, JJ, NN, C::v1>::NC
                                                                   : Shape<FORM, JJ, NN, C::v2>::NC;
    return "chunk=" + std::to_string(chunk) + " (N=" + std::to_string(N) + ") ctas/SM=" + std::to_string(cfg % 4);
}

// the (J, n) combinations of the split player update
#define CHEB_GAME_TC_SHAPES(X) X(2, 5) X(2, 9) X(2, 17) X(2, 33) X(3, 5) X(3, 9) X(3, 17) X(3, 33) X(4, 5) X(4, 9)

bool shape_ok(int J, int n)
{
#define CHEB_X(JJ, NN) if (J == JJ && n == NN) return true;
    CHEB_GAME_TC_SHAPES(CHEB_X)
#undef CHEB_X
    return false;
}

template <int FORM>
cheb_status dispatch_n(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int J, int n, int cfg,
                       cudaStream_t st)
{
#define CHEB_X(JJ, NN) if (J == JJ && n == NN) return run_cfg<FORM, JJ, NN>(ctx, d_inst, d_stat, B, cfg, st);
    CHEB_GAME_TC_SHAPES(CHEB_X)
#undef CHEB_X
    return fail(CHEB_EUNSUPPORTED, "game_solve: no split player update for this (J, n)");
}

template <int FORM>
cheb_status candidates_n(int J, int n, std::vector<int> *out)
{
#define CHEB_X(JJ, NN) if (J == JJ && n == NN) return candidates<FORM, JJ, NN>(out);
    CHEB_GAME_TC_SHAPES(CHEB_X)
#undef CHEB_X
    return fail(CHEB_EUNSUPPORTED, "game_solve: no split player update for this (J, n)");
}

template <int FORM>
std::string describe_n(int J, int n, int cfg)
{
#define CHEB_X(JJ, NN) if (J == JJ && n == NN) return describe<FORM, JJ, NN>(cfg);
    CHEB_GAME_TC_SHAPES(CHEB_X)
#undef CHEB_X
    return "?";
}

template <int FORM, int JJ, int NN> constexpr size_t max_bytes()
{
    using C = Chunks<JJ, NN>;
    size_t b = Shape<FORM, JJ, NN, C::v0>::PLAYER_BYTES;
    b = std::max(b, Shape<FORM, JJ, NN, C::v1>::PLAYER_BYTES);
    return std::max(b, Shape<FORM, JJ, NN, C::v2>::PLAYER_BYTES);
}

// B-operand bytes per player, the largest over the chunk variants (the
// workspace serves whichever variant runs)
template <int FORM>
size_t bsplit_bytes_form(int J, int n)
{
#define CHEB_X(JJ, NN) if (J == JJ && n == NN) return max_bytes<FORM, JJ, NN>();
    CHEB_GAME_TC_SHAPES(CHEB_X)
#undef CHEB_X
    return 0;
}

size_t bsplit_bytes(int J, int n, int prec)
{
    switch (prec) {
    case CHEB_BF16X3: return bsplit_bytes_form<CHEB_BF16X3>(J, n);
    case CHEB_BF16X6: return bsplit_bytes_form<CHEB_BF16X6>(J, n);
    case CHEB_TF32X3: return bsplit_bytes_form<CHEB_TF32X3>(J, n);
    default: return 0;
    }
}

cheb_status run_any(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int J, int n, int prec, int cfg,
                    cudaStream_t st)
{
    switch (prec) {
    case CHEB_BF16X3: return dispatch_n<CHEB_BF16X3>(ctx, d_inst, d_stat, B, J, n, cfg, st);
    case CHEB_BF16X6: return dispatch_n<CHEB_BF16X6>(ctx, d_inst, d_stat, B, J, n, cfg, st);
    case CHEB_TF32X3: return dispatch_n<CHEB_TF32X3>(ctx, d_inst, d_stat, B, J, n, cfg, st);
    default: return fail(CHEB_EINVAL, "game_solve: bad precision");
    }
}

cheb_status candidates_any(int J, int n, int prec, std::vector<int> *out)
{
    switch (prec) {
    case CHEB_BF16X3: return candidates_n<CHEB_BF16X3>(J, n, out);
    case CHEB_BF16X6: return candidates_n<CHEB_BF16X6>(J, n, out);
    case CHEB_TF32X3: return candidates_n<CHEB_TF32X3>(J, n, out);
    default: return fail(CHEB_EINVAL, "game_solve: bad precision");
    }
}

std::string describe_any(int J, int n, int prec, int cfg)
{
    switch (prec) {
    case CHEB_BF16X3: return describe_n<CHEB_BF16X3>(J, n, cfg);
    case CHEB_BF16X6: return describe_n<CHEB_BF16X6>(J, n, cfg);
    default: return describe_n<CHEB_TF32X3>(J, n, cfg);
    }
}

const char *form_name(int prec)
{
    return prec == CHEB_BF16X3 ? "bf16x3" : prec == CHEB_BF16X6 ? "bf16x6" : "tf32x3";
}

// batch-size class of a tuning entry: 0 for B = 1, then one class per factor 4
int batch_class(int B)
{
    int c = 0;
    while (B > 1 && c < 8) {
        B = (B + 3) / 4;
        ++c;
    }
    return c;
}

std::string tune_key(int prec, int J, int n, int B)
{
    return std::string(form_name(prec)) + " J=" + std::to_string(J) + " n=" + std::to_string(n) + " batch class " +
           std::to_string(batch_class(B));
}

}  // namespace

bool tc_shape_supported(int J, int n) { return shape_ok(J, n); }

size_t game_tc_workspace_bytes(int J, int n, int NP, int B, int prec)
{
    (void)NP;
    if (prec == CHEB_FP64 || prec == CHEB_DF64 || !shape_ok(J, n)) return 0;
    return (size_t)B * J * ((bsplit_bytes(J, n, prec) + 255) & ~size_t(255));
}

void game_tc_bind(GameDev *hinst, int B, int J, int n, int NP, int prec, uint8_t *ws)
{
    (void)NP;
    if (prec == CHEB_FP64 || prec == CHEB_DF64 || !shape_ok(J, n)) return;
    const size_t per = J * ((bsplit_bytes(J, n, prec) + 255) & ~size_t(255));
    for (int q = 0; q < B; ++q) hinst[q].bsplit = ws + per * q;
}

cheb_status game_tc_player(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, const GameDev *hinst, int B,
                           int J, int n, int NP, int prec, uint8_t *ws, cudaStream_t st)
{
    (void)hinst;
    (void)NP;
    (void)ws;
    if (!tc_shape_supported(J, n)) return fail(CHEB_EUNSUPPORTED, "game_solve: no split player update for this (J, n)");
    int cfg = cfg_of(0, 1);   // the default shape
    if (ctx->tune_mode >= 2) {
        std::vector<int> cands;
        cheb_status r = candidates_any(J, n, prec, &cands);
        if (r) return r;
        cfg = ctx->tune_mode - 2;
        if (std::find(cands.begin(), cands.end(), cfg) == cands.end())
            return fail(CHEB_EINVAL, "game_solve: the forced tile configuration does not exist for n = " +
                                         std::to_string(n));
    } else if (ctx->tune_mode == 0) {
        auto it = ctx->game_tune.find(tune_key(prec, J, n, B));
        if (it != ctx->game_tune.end()) cfg = it->second.first;
    }
    return run_any(ctx, d_inst, d_stat, B, J, n, prec, cfg, st);
}

cheb_status game_tc_tune(cheb_ctx *ctx, const GameDev *d_inst, GameStat *d_stat, int B, int J, int n, int prec,
                         cudaStream_t st)
{
    if (prec == CHEB_FP64 || !tc_shape_supported(J, n) || ctx->tune_mode != 0) return CHEB_OK;
    const std::string key = tune_key(prec, J, n, B);
    if (ctx->game_tune.count(key)) return CHEB_OK;
    std::vector<int> cands;
    cheb_status r = candidates_any(J, n, prec, &cands);
    if (r) return r;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CHEB_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return CHEB_OK;   // cannot time inside a capture: default shape
    cudaEvent_t e0, e1;
    CHEB_CUDA_TRY(cudaEventCreate(&e0));
    CHEB_CUDA_TRY(cudaEventCreate(&e1));
    int best = cands[0];
    float best_ms = 0.0f;
    std::string times;
    for (size_t c = 0; c < cands.size() && r == CHEB_OK; ++c) {
        const int cfg = cands[c];
        if ((r = run_any(ctx, d_inst, d_stat, B, J, n, prec, cfg, st))) break;   // warm-up
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3 && r == CHEB_OK; ++rep) r = run_any(ctx, d_inst, d_stat, B, J, n, prec, cfg, st);
        cudaEventRecord(e1, st);
        if (r) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
            r = cuda_fail(ce, "game tile tuning");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= 3.0f;
        char buf[64];
        std::snprintf(buf, sizeof(buf), " %.1f us", 1000.0f * ms);
        times += (c ? ", " : "") + describe_any(J, n, prec, cfg) + buf;
        if (c == 0 || ms < best_ms) {
            best_ms = ms;
            best = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    ctx->game_tune[key] = {best, describe_any(J, n, prec, best) + " [tried: " + times + "]"};
    return CHEB_OK;
}

}  // namespace game
}  // namespace cheb
