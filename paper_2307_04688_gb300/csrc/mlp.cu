// The learned warm start: a multilayer perceptron in -> width (x depth) -> out,
// GELU between layers, BF16 operands with FP32 accumulation on the tcgen05
// tensor cores, FP32 master weights, Adam, mean-squared error on normalised
// targets. It maps game parameters to the coefficient tensor of one player's
// value function and warm-starts the iteration (the paper leaves the initial
// guess V^[0] free, Section 2.1 Step 0).
//
// One GEMM kernel serves the forward and backward passes, C = epi(A B^T), on
// operands that the producing kernels have already written as packed BF16
// tiles in the tensor cores' K-major layout (see tile_base): the forward
// epilogue writes the next layer's input in both orientations (K-major for the
// next forward product, transposed for the weight gradient), the loss kernel
// and the backward epilogue do the same for the gradients, and the weights are
// packed in both orientations after each update. The GEMM streams 16 KB tiles
// with bulk copies through a three-stage mbarrier ring, one thread issues
// tcgen05.mma (M = N = 128, K = 16 steps) into TMEM, and the epilogue stages
// the accumulator through shared memory for coalesced stores and applies
// bias, GELU or the GELU derivative. Products with few output tiles and a long
// K (the hidden-layer gradient of a wide output layer) split K across CTAs and
// sum the partials in a fixed order.
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

constexpr int kTM = 128, kTN = 128, kTK = 64;      // output tile (M x N) and K tile of the GEMM
constexpr int kStages = 3;                          // operand pipeline depth
constexpr int kGemmThreads = 256;                   // 8 warps: two per TMEM lane quadrant in the epilogue
constexpr int kTileBytes = kTM * kTK * 2;           // one packed operand tile: 16 KB
constexpr int kLdT = kTN + 4;                       // row stride (floats) of a staged FP32 slab
static_assert(kTM == kTN && kGemmThreads == 256, "the epilogue maps warps w and w + 4 to one TMEM lane quadrant");

enum Epi { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

inline int cdiv(int64_t a, int b) { return (int)((a + b - 1) / b); }

// A packed operand holds a logical matrix X (R rows x K) in BF16 as tiles of
// 128 rows x 64 K. Tile (rt, kt) starts at (rt * kt_count + kt) * 16 KB, and
// element (r, k) of it sits at (k / 8) * 2048 + r * 16 + (k % 8) * 2 bytes:
// the no-swizzle K-major layout that tcgen05.mma reads (core rows of 8
// elements = 16 bytes, 8-row groups 128 bytes apart, K-adjacent core
// matrices 2048 bytes apart), so one bulk copy moves a tile into shared
// memory. Entries outside R x K are zero. The producers of the operands (the
// GEMM epilogue, the loss kernel, the input and weight packing) write them
// in this form, so the GEMM itself never converts or transposes.
__host__ __device__ inline int64_t tile_base(int rt, int kt, int kt_count)
{
    return ((int64_t)rt * kt_count + kt) * kTileBytes;
}

inline int64_t packed_bytes(int R, int K) { return (int64_t)cdiv(R, kTM) * cdiv(K, kTK) * kTileBytes; }

// Where a finished 128 x 128 FP32 tile of C[m, n] goes, and what is applied to it.
struct OutSpec {
    float *C;               // row-major FP32 result C[m * ldc + n], or null
    float *Z;               // EPI_BIAS_GELU: the pre-activation, same layout, or null
    int64_t ldc;
    const float *bias;      // EPI_BIAS, EPI_BIAS_GELU: bias[n]
    const float *aux;       // EPI_GELU_BWD: the pre-activation Z[m * ldc + n]
    uint8_t *pk;            // packed copy with rows = m, K = n, or null
    int pk_kt;              //   its K tiles per row tile
    uint8_t *pt;            // packed copy with rows = n, K = m (the transpose), or null
    int pt_kt;
    int M, N, epi;
};

struct GemmP {
    const uint8_t *A;       // packed, rows = m
    const uint8_t *B;       // packed, rows = n
    int a_kt, b_kt;         // K tiles per row tile of A and of B
    int kt_total;           // K tiles of the product
    int kt_per;             // K tiles per split (gridDim.z splits)
    float *ws;              // partial tiles: (z, mt, nt) at ((z * gridDim.y + mt) * gridDim.x + nt) * 128 * 128
    int use_ws;             // write raw partials to ws (finished by splitk_reduce_kernel)
    OutSpec o;
    int *err;
    long long wait_limit;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float Phi = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
    return Phi + z * 0.3989422804014327f * __expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Applies the epilogue to a staged slab of `rows` rows (a multiple of 8) of an
// output tile: rows m0 + [0, rows), columns n0 + [0, 128), row stride kLdT,
// with n0 a multiple of 128 and m0 a multiple of 8. Writes every form of the
// result that `o` asks for; all kGemmThreads threads of the block take part.
// Entries outside M x N become zero in the slab, so that the packed copies
// carry their zero padding. The loads of the epilogue (bias, and the
// pre-activation for the GELU derivative) are issued eight rows at a time
// before any store, so that a warp waits for one memory round trip per eight
// rows, not per row.
__device__ void finish_tile(float *tile, int m0, int n0, int rows, const OutSpec &o)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kWarps = kGemmThreads / 32;
    float *__restrict__ C = o.C;
    float *__restrict__ Z = o.Z;
    const float *__restrict__ aux = o.aux;
    const bool has_bias = o.epi == EPI_BIAS || o.epi == EPI_BIAS_GELU;
    float bv[kTN / 32];
#pragma unroll
    for (int j = 0; j < kTN / 32; ++j) {
        const int n = n0 + lane + 32 * j;
        bv[j] = (has_bias && n < o.N) ? __ldg(o.bias + n) : 0.0f;
    }
    // row r = rb + kWarps u (u = 0..7) of this warp's batch, column lane + 32 j
    for (int rb = warp; rb < rows; rb += 8 * kWarps) {
        float av[8][kTN / 32];
        if (o.epi == EPI_GELU_BWD) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int j = 0; j < kTN / 32; ++j) {
                    const int r = rb + kWarps * u, m = m0 + r, n = n0 + lane + 32 * j;
                    av[u][j] = (r < rows && m < o.M && n < o.N) ? __ldg(aux + (int64_t)m * o.ldc + n) : 0.0f;
                }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = rb + kWarps * u, m = m0 + r;
            if (r >= rows) break;
#pragma unroll
            for (int j = 0; j < kTN / 32; ++j) {
                const int c = lane + 32 * j, n = n0 + c;
                float v = 0.0f;
                if (m < o.M && n < o.N) {
                    v = tile[r * kLdT + c] + bv[j];
                    const int64_t off = (int64_t)m * o.ldc + n;
                    if (o.epi == EPI_BIAS_GELU) {
                        if (Z) Z[off] = v;
                        v = gelu_f(v);
                    } else if (o.epi == EPI_GELU_BWD) {
                        v *= gelu_grad_f(av[u][j]);
                    }
                    if (C) C[off] = v;
                }
                tile[r * kLdT + c] = v;
            }
        }
    }
    if (!o.pk && !o.pt) return;
    __syncthreads();
    if (o.pk) {
        // chunk (row r, 8 consecutive n from q * 8): one 16-byte store; consecutive
        // threads store consecutive rows of one core-matrix column
        for (int t = tid; t < rows * (kTN / 8); t += kGemmThreads) {
            const int r = t % rows, q = t / rows;
            const int m = m0 + r, n = n0 + q * 8, kt = n / kTK;
            if (kt >= o.pk_kt) continue;
            const float4 a = *reinterpret_cast<const float4 *>(tile + r * kLdT + q * 8);
            const float4 b = *reinterpret_cast<const float4 *>(tile + r * kLdT + q * 8 + 4);
            const uint4 w = make_uint4(bf16x2(a.x, a.y), bf16x2(a.z, a.w), bf16x2(b.x, b.y), bf16x2(b.z, b.w));
            *reinterpret_cast<uint4 *>(o.pk + tile_base(m / kTM, kt, o.pk_kt) + ((n % kTK) / 8) * 2048 + (m % kTM) * 16) = w;
        }
    }
    if (o.pt) {
        // chunk (column c, 8 consecutive m from g * 8)
        for (int t = tid; t < kTN * (rows / 8); t += kGemmThreads) {
            const int c = t % kTN, g = t / kTN;
            const int n = n0 + c, m = m0 + g * 8, kt = m / kTK;
            if (kt >= o.pt_kt) continue;
            float e[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) e[u] = tile[(g * 8 + u) * kLdT + c];
            const uint4 w = make_uint4(bf16x2(e[0], e[1]), bf16x2(e[2], e[3]), bf16x2(e[4], e[5]), bf16x2(e[6], e[7]));
            *reinterpret_cast<uint4 *>(o.pt + tile_base(n / kTM, kt, o.pt_kt) + ((m % kTK) / 8) * 2048 + (n % kTM) * 16) = w;
        }
    }
}

constexpr int kStLd = 36;                           // row stride (floats) of a warp's 32 x 32 staging block
constexpr int kEpiSmem = 4 * kTileBytes + (kGemmThreads / 32) * 32 * kStLd * 4;
// operand stages, reused by the epilogue once the MMAs are done
constexpr int kGemmSmem = kStages * 2 * kTileBytes > kEpiSmem ? kStages * 2 * kTileBytes : kEpiSmem;

// Epilogue of the 128 x 128 accumulator tile (mt, nt) of a GEMM CTA. Warp w
// takes the 32 TMEM lanes of quadrant w % 4 (rows 32 (w % 4) + lane) and the
// column half w / 4, and moves them 32 columns at a time into a warp-private
// staging block in shared memory; then lane = column, so every
// global load and store of the epilogue (bias, pre-activation, C, Z, or the
// raw split partial) is a coalesced 128-byte row segment, and the 32 rows of
// a chunk are independent work for the scheduler. The packed copies are
// assembled in shared memory in their final tile layout (two 16 KB tiles per
// form, rows or K zero outside M x N) and written with bulk copies.
__device__ void epilogue_direct(uint32_t tmem, uint8_t *smem, const GemmP &p, int mt, int nt)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const OutSpec &o = p.o;
    uint8_t *spk = smem, *spt = smem + 2 * kTileBytes;
    float *stg = reinterpret_cast<float *>(smem + 4 * kTileBytes) + warp * 32 * kStLd;
    const int m0 = mt * kTM, n0 = nt * kTN, rw0 = (warp & 3) * 32, ch0 = (warp >> 2) * (kTN / 2);
    const bool raw = p.use_ws != 0;
    const bool want_pk = !raw && o.pk, want_pt = !raw && o.pt;
    float *__restrict__ part =
        raw ? p.ws + (((int64_t)blockIdx.z * gridDim.y + mt) * gridDim.x + nt) * (kTM * kTN) : nullptr;
    float *__restrict__ C = o.C;
    float *__restrict__ Z = o.Z;
    const float *__restrict__ aux = o.aux;
    const bool has_bias = o.epi == EPI_BIAS || o.epi == EPI_BIAS_GELU;
    const uint32_t lane_addr = tmem + ((uint32_t)rw0 << 16);
    for (int c0 = ch0; c0 < ch0 + kTN / 2; c0 += 32) {
        uint32_t va[16], vb[16];
        tmem_ld16(lane_addr + c0, va);
        tmem_ld16(lane_addr + c0 + 16, vb);
        tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; e += 4) {
            *reinterpret_cast<float4 *>(stg + lane * kStLd + e) =
                make_float4(__uint_as_float(va[e]), __uint_as_float(va[e + 1]), __uint_as_float(va[e + 2]),
                            __uint_as_float(va[e + 3]));
            *reinterpret_cast<float4 *>(stg + lane * kStLd + 16 + e) =
                make_float4(__uint_as_float(vb[e]), __uint_as_float(vb[e + 1]), __uint_as_float(vb[e + 2]),
                            __uint_as_float(vb[e + 3]));
        }
        __syncwarp();
        const int c = c0 + lane, n = n0 + c;
        if (raw) {
#pragma unroll 8
            for (int rr = 0; rr < 32; ++rr) part[(rw0 + rr) * kTN + c] = stg[rr * kStLd + lane];
        } else {
            const bool col_ok = n < o.N;
            const float bv = (has_bias && col_ok) ? __ldg(o.bias + n) : 0.0f;
            // eight rows at a time: all loads, then the arithmetic, then all stores
            for (int rb = 0; rb < 32; rb += 8) {
                float x[8], a8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = stg[(rb + u) * kStLd + lane] + bv;
                if (o.epi == EPI_GELU_BWD) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int m = m0 + rw0 + rb + u;
                        a8[u] = (col_ok && m < o.M) ? __ldg(aux + (int64_t)m * o.ldc + n) : 0.0f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int m = m0 + rw0 + rb + u;
                    const bool ok = col_ok && m < o.M;
                    float y = x[u];
                    if (o.epi == EPI_BIAS_GELU) {
                        if (ok && Z) Z[(int64_t)m * o.ldc + n] = y;
                        y = gelu_f(y);
                    } else if (o.epi == EPI_GELU_BWD) {
                        y *= gelu_grad_f(a8[u]);
                    }
                    y = ok ? y : 0.0f;
                    if (ok && C) C[(int64_t)m * o.ldc + n] = y;
                    x[u] = y;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) stg[(rb + u) * kStLd + lane] = x[u];
            }
        }
        __syncwarp();
        if (want_pk) {
            // row rw0 + lane, four chunks of 8 consecutive columns
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int col = c0 + 8 * q;
                const float4 a = *reinterpret_cast<const float4 *>(stg + lane * kStLd + 8 * q);
                const float4 b = *reinterpret_cast<const float4 *>(stg + lane * kStLd + 8 * q + 4);
                *reinterpret_cast<uint4 *>(spk + (col / kTK) * kTileBytes + ((col % kTK) / 8) * 2048 + (rw0 + lane) * 16) =
                    make_uint4(bf16x2(a.x, a.y), bf16x2(a.z, a.w), bf16x2(b.x, b.y), bf16x2(b.z, b.w));
            }
        }
        if (want_pt) {
            // column c0 + lane, four groups of 8 consecutive rows
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int r8 = rw0 + 8 * g;
                float e[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) e[u] = stg[(8 * g + u) * kStLd + lane];
                *reinterpret_cast<uint4 *>(spt + (r8 / kTK) * kTileBytes + ((r8 % kTK) / 8) * 2048 + (c0 + lane) * 16) =
                    make_uint4(bf16x2(e[0], e[1]), bf16x2(e[2], e[3]), bf16x2(e[4], e[5]), bf16x2(e[6], e[7]));
            }
        }
        __syncwarp();
    }
    if (want_pk || want_pt) {
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            for (int sel = 0; sel < 2; ++sel) {
                const int kk = n0 / kTK + sel, km = m0 / kTK + sel;
                if (want_pk && kk < o.pk_kt) bulk_s2g(o.pk + tile_base(mt, kk, o.pk_kt), spk + sel * kTileBytes, kTileBytes);
                if (want_pt && km < o.pt_kt) bulk_s2g(o.pt + tile_base(nt, km, o.pt_kt), spt + sel * kTileBytes, kTileBytes);
            }
            bulk_commit();
            bulk_wait_all();
        }
    }
}

// C = epi(A B^T) on one 128 x 128 output tile per CTA (blockIdx.x: n tile,
// blockIdx.y: m tile, blockIdx.z: K split). Thread 0 streams the K tiles of
// both packed operands into a kStages-deep ring of shared-memory stages with
// bulk copies (full[s] counts their bytes); thread 32 issues four
// tcgen05.mma (K = 16 each) per stage into a TMEM accumulator and commits to
// empty[s], which frees the stage for the next copy. After the last MMA all
// four warps read their 32 accumulator rows from TMEM into a shared-memory
// tile (the stages are idle by then) and finish it: the epilogue and the
// stores (one split), or the raw partial into the split workspace.
__global__ void __launch_bounds__(kGemmThreads, 2) gemm_tc_kernel(const GemmP p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    __shared__ int n_issued, n_consumed, done_issued;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = blockIdx.x, mt = blockIdx.y, z = blockIdx.z;
    const int kt0 = z * p.kt_per;
    const int nk = min(p.kt_per, p.kt_total - kt0);
    // the operand stages fit the dynamic shared memory, the tile lies in the
    // output, the K tiles in both packed operands (uniform: all or none return)
    if (!CHEB_DCHECK(kGemmSmem <= (int)dyn_smem_bytes() && mt * kTM < p.o.M && nt * kTN < p.o.N &&
                     kt0 + nk <= p.a_kt && kt0 + nk <= p.b_kt))
        return;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        n_issued = 0;
        n_consumed = 0;
        done_issued = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, kTN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        // producer: stage s = i % kStages is free once the MMAs of K tile i - kStages are done
        const uint8_t *a = p.A + tile_base(mt, kt0, p.a_kt);
        const uint8_t *b = p.B + tile_base(nt, kt0, p.b_kt);
        int i = 0;
        for (; i < nk; ++i) {
            const int s = i % kStages;
            if (abort_flag) break;
            if (i >= kStages && !mbar_wait_bounded(&empty[s], ((i / kStages) - 1) & 1u, p.err, p.wait_limit)) {
                abort_flag = 1;
                break;
            }
            uint8_t *sa = smem + s * 2 * kTileBytes;
            mbar_arrive_expect_tx(&full[s], 2 * kTileBytes);
            bulk_g2s(sa, a + (int64_t)i * kTileBytes, kTileBytes, &full[s]);
            bulk_g2s(sa + kTileBytes, b + (int64_t)i * kTileBytes, kTileBytes, &full[s]);
        }
        n_issued = i;
    } else if (tid == 32) {
        // MMA issuer
        const uint32_t idesc = make_idesc(1, kTM, kTN);
        int i = 0;
        for (; i < nk; ++i) {
            const int s = i % kStages;
            if (abort_flag) break;
            if (!mbar_wait_bounded(&full[s], (i / kStages) & 1u, p.err, p.wait_limit)) {
                abort_flag = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * 2 * kTileBytes), b0 = a0 + kTileBytes;
#pragma unroll
            for (int ks = 0; ks < kTK / 16; ++ks)
                mma_bf16(tmem, make_sdesc(a0 + ks * 2 * 2048, 2048, 128), make_sdesc(b0 + ks * 2 * 2048, 2048, 128),
                         idesc, (i | ks) != 0);
            mma_commit(&empty[s]);
        }
        n_consumed = i;
        if (i == nk) {
            mma_commit(&done);
            done_issued = 1;
        }
    }
    __syncthreads();
    if (tid == 0 && !abort_flag && !mbar_wait_bounded(&done, 0, p.err, p.wait_limit)) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
        // drain with the full bound: copies still landing, then the MMAs, before TMEM is freed
        if (tid == 0) {
            for (int i = n_consumed; i < n_issued; ++i) mbar_wait_bounded(&full[i % kStages], (i / kStages) & 1u, p.err);
            if (done_issued) {
                mbar_wait_bounded(&done, 0, p.err);
            } else if (n_consumed > 0) {
                const int j = n_consumed - 1;
                mbar_wait_bounded(&empty[j % kStages], (j / kStages) & 1u, p.err);
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tmem_dealloc(tmem, kTN);
        return;
    }
    tc_fence_after();
    epilogue_direct(tmem, smem, p, mt, nt);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTN);
}

// The reduce, pack and loss kernels work on slabs of kSlab rows x 128 columns
// (16 slabs per 128 x 128 tile), so that many CTAs share the memory traffic.
constexpr int kSlab = 8;

// Sums the split partials of one slab of an output tile in split order
// (deterministic) and finishes it. Grid: (n tiles, m tiles, 128 / kSlab).
__global__ void __launch_bounds__(kGemmThreads) splitk_reduce_kernel(const float *__restrict__ ws, int splits,
                                                                     const OutSpec o)
{
    __shared__ __align__(16) float stile[kSlab * kLdT];
    const int nt = blockIdx.x, mt = blockIdx.y, r0 = blockIdx.z * kSlab;
    const int64_t zstride = (int64_t)gridDim.y * gridDim.x * (kTM * kTN / 4);
    const float4 *src = reinterpret_cast<const float4 *>(ws) + ((int64_t)mt * gridDim.x + nt) * (kTM * kTN / 4) +
                        r0 * (kTN / 4);
    for (int q = threadIdx.x; q < kSlab * kTN / 4; q += kGemmThreads) {
        float4 s = src[q];
#pragma unroll 8
        for (int zz = 1; zz < splits; ++zz) {
            const float4 t = src[q + zz * zstride];
            s.x += t.x;
            s.y += t.y;
            s.z += t.z;
            s.w += t.w;
        }
        const int rr = q / (kTN / 4), c4 = q % (kTN / 4);
        *reinterpret_cast<float4 *>(stile + rr * kLdT + c4 * 4) = s;
    }
    __syncthreads();
    finish_tile(stile, mt * kTM + r0, nt * kTN, kSlab, o);
}

// Packs the slab at rows m0 + [0, kSlab), columns n0 + [0, 128) of an FP32
// row-major matrix src (R x K, row stride ld) into the packed forms that `o`
// asks for (o.M = R, o.N = K, o.epi = EPI_NONE, o.C = null).
__device__ __forceinline__ void pack_slab(float *stile, const float *__restrict__ src, int64_t ld, int m0, int n0,
                                          const OutSpec &o)
{
    float v[kSlab * kTN / kGemmThreads];
#pragma unroll
    for (int u = 0; u < kSlab * kTN / kGemmThreads; ++u) {
        const int q = threadIdx.x + u * kGemmThreads, rr = q / kTN, c = q % kTN;
        const int m = m0 + rr, n = n0 + c;
        v[u] = (m < o.M && n < o.N) ? __ldg(src + (int64_t)m * ld + n) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kSlab * kTN / kGemmThreads; ++u) {
        const int q = threadIdx.x + u * kGemmThreads;
        stile[(q / kTN) * kLdT + q % kTN] = v[u];
    }
    __syncthreads();
    finish_tile(stile, m0, n0, kSlab, o);
}

// Grid: (column tiles, row slabs).
__global__ void __launch_bounds__(kGemmThreads) pack_kernel(const float *__restrict__ src, int64_t ld, const OutSpec o)
{
    __shared__ __align__(16) float stile[kSlab * kLdT];
    pack_slab(stile, src, ld, blockIdx.y * kSlab, blockIdx.x * kTN, o);
}

// One matrix of a multi-matrix pack: its blocks are first_block ..
// first_block + col_tiles * slabs - 1 of the launch.
struct PackJob {
    const float *src;
    int64_t ld;
    OutSpec o;
    int col_tiles, first_block;
};

// Packs every weight matrix of a network in one launch (1-D grid over the
// jobs' blocks; a block finds its job by the jobs' first blocks).
__global__ void __launch_bounds__(kGemmThreads) pack_multi_kernel(const PackJob *__restrict__ jobs, int njobs)
{
    __shared__ __align__(16) float stile[kSlab * kLdT];
    int j = 0;
    while (j + 1 < njobs && (int)blockIdx.x >= jobs[j + 1].first_block) ++j;
    const PackJob jb = jobs[j];
    const int local = (int)blockIdx.x - jb.first_block;
    pack_slab(stile, jb.src, jb.ld, (local / jb.col_tiles) * kSlab, (local % jb.col_tiles) * kTN, jb.o);
}

// The mean-squared-error gradient dY = 2 (Y - T) / (B F) on one slab (Y, T
// row-major B x F), the block's share of the loss into part[block] (summed in a
// fixed order by loss_sum_kernel), and dY finished through `o` (FP32 copy and
// the two packed forms for backpropagation). Grid: (column tiles, row slabs).
__global__ void __launch_bounds__(kGemmThreads) mse_tile_kernel(const float *__restrict__ Y, const float *__restrict__ T,
                                                                float scale, float *__restrict__ part, const OutSpec o)
{
    __shared__ __align__(16) float stile[kSlab * kLdT];
    __shared__ float wsum[kGemmThreads / 32];
    const int m0 = blockIdx.y * kSlab, n0 = blockIdx.x * kTN;
    constexpr int kPer = kSlab * kTN / kGemmThreads;
    float y[kPer], t[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int q = threadIdx.x + u * kGemmThreads, m = m0 + q / kTN, n = n0 + q % kTN;
        const bool in = m < o.M && n < o.N;
        y[u] = in ? __ldg(Y + (int64_t)m * o.N + n) : 0.0f;
        t[u] = in ? __ldg(T + (int64_t)m * o.N + n) : 0.0f;
    }
    float local = 0.0f;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int q = threadIdx.x + u * kGemmThreads;
        const float d = y[u] - t[u];
        local += d * d * scale;
        stile[(q / kTN) * kLdT + q % kTN] = 2.0f * d * scale;
    }
    for (int s = 16; s > 0; s >>= 1) local += __shfl_xor_sync(0xffffffffu, local, s);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < kGemmThreads / 32; ++w) t += wsum[w];
        part[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
    finish_tile(stile, m0, n0, kSlab, o);
}

// *loss += sum of part[0 .. n) in a fixed order (one block).
__global__ void __launch_bounds__(256) loss_sum_kernel(const float *__restrict__ part, int n, float *__restrict__ loss)
{
    __shared__ float red[256];
    float t = 0.0f;
    for (int i = threadIdx.x; i < n; i += 256) t += part[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss += red[0];
}

// Launch through cudaLaunchKernelEx (typed arguments, error returned as a status).
// No programmatic dependent launch here: inside the captured training graph
// an early-started kernel of this chain produced wrong weights, so every
// kernel waits for the previous one in full.
template <class... Params, class... Args>
cheb_status launch(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    CHEB_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    return CHEB_OK;
}

cheb_status set_kernel_attrs()
{
    static PerDevice attr;
    return per_device_once(attr, [](int *) -> cheb_status {
        CHEB_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
        return CHEB_OK;
    }, nullptr);
}

// C = epi(A B^T) with K = the product's inner size. An output with few tiles
// (at most half the SM count) goes through the workspace: K is split across
// up to num_sms / tiles CTAs per tile, and splitk_reduce_kernel sums the
// partials and runs the epilogue on 8-row slabs, 16 CTAs per tile, so that
// neither the products nor the epilogue (GELU, packing) run on a handful of
// SMs. tiles x splits <= the SM count bounds the workspace `ws` (num_sms
// tiles of 128 x 128 FP32).
cheb_status gemm(cheb_ctx *ctx, const uint8_t *A, int a_kt, const uint8_t *B, int b_kt, int K, const OutSpec &o,
                 float *ws, cudaStream_t st)
{
    if (o.M <= 0 || o.N <= 0) return CHEB_OK;
    if (K <= 0) return fail(CHEB_EINVAL, "surrogate GEMM with K = 0");
    cheb_status r = set_kernel_attrs();
    if (r) return r;
    const int mt = cdiv(o.M, kTM), nt = cdiv(o.N, kTN), kt = cdiv(K, kTK), tiles = mt * nt;
    int per = kt, splits = 1;
    const bool use_ws = ws && 2 * tiles <= ctx->num_sms;
    if (use_ws) {
        per = cdiv(kt, std::min(kt, ctx->num_sms / tiles));
        splits = cdiv(kt, per);
    }
    GemmP p;
    p.A = A;
    p.B = B;
    p.a_kt = a_kt;
    p.b_kt = b_kt;
    p.kt_total = kt;
    p.kt_per = per;
    p.ws = ws;
    p.use_ws = use_ws ? 1 : 0;
    p.o = o;
    p.err = ctx->d_error;
    p.wait_limit = ctx->wait_limit;
    ProfScope prof("mlp_gemm M=" + std::to_string(o.M) + " N=" + std::to_string(o.N) + " K=" + std::to_string(K), st);
    if ((r = launch(gemm_tc_kernel, dim3((unsigned)nt, (unsigned)mt, (unsigned)splits), dim3(kGemmThreads),
                        kGemmSmem, st, p)))
        return r;
    if (use_ws &&
        (r = launch(splitk_reduce_kernel, dim3((unsigned)nt, (unsigned)mt, kTM / kSlab), dim3(kGemmThreads), 0, st,
                        (const float *)ws, splits, o)))
        return r;
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

// per-column mean and std of an S x F FP64 matrix (row stride sx): a block of
// 32 columns x 32 row groups; thread (c, g) sums rows r = g (mod 32) of its
// column in FP64, and the 32 partial sums are combined in the order g = 0..31
__global__ void __launch_bounds__(1024) column_stats_kernel(const double *__restrict__ X, int64_t sx, int64_t S, int F,
                                                            float *__restrict__ mean, float *__restrict__ std_out)
{
    __shared__ double ps[32][33], ps2[32][33];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int f = blockIdx.x * 32 + c;
    double s = 0.0, s2 = 0.0;
    if (f < F) {
#pragma unroll 4
        for (int64_t r = g; r < S; r += 32) {
            const double v = __ldg(X + r * sx + f);
            s += v;
            s2 += v * v;
        }
    }
    ps[g][c] = s;
    ps2[g][c] = s2;
    __syncthreads();
    if (g == 0 && f < F) {
        double t = 0.0, t2 = 0.0;
        for (int k = 0; k < 32; ++k) {
            t += ps[k][c];
            t2 += ps2[k][c];
        }
        const double mu = t / (double)S;
        const double var = fmax(t2 / (double)S - mu * mu, 0.0);
        mean[f] = (float)mu;
        std_out[f] = (float)sqrt(var);
    }
}

__global__ void finish_inv_std_kernel(const float *__restrict__ std_in, int F, float floor_abs, float *__restrict__ inv_std)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F) return;
    inv_std[f] = 1.0f / fmaxf(std_in[f], floor_abs);
}

// gb[n] = sum_b dZ[b, n] (dZ row-major B x N): a block of 32 x 8 threads takes 32
// columns; thread (c, g) sums the rows b = g (mod 8) of its column, and the
// eight partial sums are added in the order g = 0..7 (deterministic).
__global__ void __launch_bounds__(256) bias_grad_kernel(const float *__restrict__ dZ, int B, int N, float *__restrict__ gb)
{
    __shared__ float part[8][33];
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float s = 0.0f;
    if (n < N) {
#pragma unroll 8
        for (int b = g; b < B; b += 8) s += __ldg(dZ + (int64_t)b * N + n);
    }
    part[g][c] = s;
    __syncthreads();
    if (g == 0 && n < N) {
        float t = part[0][c];
        for (int k = 1; k < 8; ++k) t += part[k][c];
        gb[n] = t;
    }
}

// Adam; with `sched` non-null the step's lr, 1 - b1^t and 1 - b2^t are read from
// sched[0..2] (a graph-captured step reads its own row of a per-epoch table)
__global__ void adam_kernel(int64_t nparam, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                            const float *__restrict__ sched)
{
    if (sched) {
        lr = sched[0];
        c1 = sched[1];
        c2 = sched[2];
    }
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
    // packed BF16 weights: wk[l] rows = out, K = in (forward); wt[l] rows = in, K = out (backward)
    std::vector<uint8_t *> wk, wt;
    bool wpack_valid = false;        // the packed weights match w
    PackJob *d_jobs = nullptr;       // the weight-packing jobs (device), one per layer
    int pack_blocks = 0;
    // a second stream for the weight and bias gradients (concurrent with the
    // input-gradient chain), and the events that fork and join it
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_t = nullptr, ev_w = nullptr;
    bool wpack_pending = false;      // packing on the side stream; wait for ev_w before the first GEMM
    // normalisation (inputs and targets)
    float *x_mean = nullptr, *x_inv = nullptr, *x_std = nullptr;
    float *y_mean = nullptr, *y_inv = nullptr, *y_std = nullptr;
    bool normalised = false;
    // batch workspace (sized for ws_batch rows)
    int ws_batch = 0;
    // Z: pre-activations, dZ: their gradients, level l (1..L) at act_off(l) of each
    float *Z = nullptr, *dZ = nullptr, *X = nullptr, *T = nullptr, *loss = nullptr;
    int *rows = nullptr;
    float *split_ws = nullptr;       // split-K partial tiles (num_sms of them), main stream
    float *split_ws2 = nullptr;      // the same for the side stream
    float *loss_part = nullptr;      // per-block loss sums of the loss kernel
    // packed activations per level l = 0..L: hk (rows = batch, K = width), ht (rows = width,
    // K = batch); packed pre-activation gradients dzk, dzt (levels 1..L), same two forms
    std::vector<uint8_t *> hk, ht, dzk, dzt;
    std::vector<void *> batch_bufs;  // everything above that depends on ws_batch
};

namespace {

void free_batch(cheb_mlp *net)
{
    for (void *p : net->batch_bufs) cudaFree(p);
    net->batch_bufs.clear();
    net->Z = net->dZ = net->X = net->T = net->split_ws = net->split_ws2 = net->loss_part = nullptr;
    net->rows = nullptr;
    net->hk.assign(net->L + 1, nullptr);
    net->ht.assign(net->L + 1, nullptr);
    net->dzk.assign(net->L + 1, nullptr);
    net->dzt.assign(net->L + 1, nullptr);
    net->ws_batch = 0;
}

cheb_status net_ws(cheb_ctx *ctx, cheb_mlp *net, int B)
{
    if (B <= net->ws_batch) return CHEB_OK;
    free_batch(net);
    int64_t act = 0;
    for (int l = 1; l <= net->L; ++l) act += (int64_t)B * net->dims[l];
    bool ok = true;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (!ok || cudaMalloc(&p, bytes) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        net->batch_bufs.push_back(p);
        cudaMemset(p, 0, bytes);
        return p;
    };
    net->Z = static_cast<float *>(alloc(sizeof(float) * act));
    net->dZ = static_cast<float *>(alloc(sizeof(float) * act));
    net->X = static_cast<float *>(alloc(sizeof(float) * B * net->dims[0]));
    net->T = static_cast<float *>(alloc(sizeof(float) * B * net->dims[net->L]));
    net->rows = static_cast<int *>(alloc(sizeof(int) * B));
    net->split_ws = static_cast<float *>(alloc(sizeof(float) * kTM * kTN * (size_t)std::max(ctx->num_sms, 1)));
    net->split_ws2 = static_cast<float *>(alloc(sizeof(float) * kTM * kTN * (size_t)std::max(ctx->num_sms, 1)));
    net->loss_part = static_cast<float *>(
        alloc(sizeof(float) * (size_t)cdiv(net->dims[net->L], kTN) * cdiv(B, kTK) * (kTK / kSlab)));
    for (int l = 0; l <= net->L; ++l) {
        net->hk[l] = static_cast<uint8_t *>(alloc(packed_bytes(B, net->dims[l])));
        net->ht[l] = static_cast<uint8_t *>(alloc(packed_bytes(net->dims[l], B)));
        if (l > 0) {
            net->dzk[l] = static_cast<uint8_t *>(alloc(packed_bytes(B, net->dims[l])));
            net->dzt[l] = static_cast<uint8_t *>(alloc(packed_bytes(net->dims[l], B)));
        }
    }
    if (!ok) {
        free_batch(net);
        return fail(CHEB_ENOMEM, "surrogate workspace allocation failed");
    }
    net->ws_batch = B;
    return CHEB_OK;
}

// pre-activations Z of level l (l = 1..L) inside net->Z
int64_t act_off(const cheb_mlp *net, int l, int B)
{
    int64_t o = 0;
    for (int t = 1; t < l; ++t) o += (int64_t)B * net->dims[t];
    return o;
}

OutSpec no_out(int M, int N)
{
    OutSpec o;
    std::memset(&o, 0, sizeof(o));
    o.M = M;
    o.N = N;
    o.ldc = N;
    o.epi = EPI_NONE;
    return o;
}

// FP32 row-major src (R x K) -> packed forms pk (rows = R) and pt (rows = K)
cheb_status pack(const float *src, int64_t ld, int R, int K, uint8_t *pk, uint8_t *pt, cudaStream_t st)
{
    cheb_status r = set_kernel_attrs();
    if (r) return r;
    OutSpec o = no_out(R, K);
    o.pk = pk;
    o.pk_kt = cdiv(K, kTK);
    o.pt = pt;
    o.pt_kt = cdiv(R, kTK);
    ProfScope prof("mlp_pack", st);
    // row slabs up to the next multiple of 64 rows: the transposed copy's last K tile is written whole
    return launch(pack_kernel, dim3((unsigned)cdiv(K, kTN), (unsigned)(cdiv(R, kTK) * (kTK / kSlab))),
                      dim3(kGemmThreads), 0, st, src, ld, o);
}

cheb_status pack_weights(cheb_mlp *net, cudaStream_t st)
{
    cheb_status r = set_kernel_attrs();
    if (r) return r;
    {
        ProfScope prof("mlp_pack_weights", st);
        if ((r = launch(pack_multi_kernel, dim3((unsigned)net->pack_blocks), dim3(kGemmThreads), 0, st,
                        (const PackJob *)net->d_jobs, net->L)))
            return r;
    }
    net->wpack_valid = true;
    return CHEB_OK;
}

// pack the weights on the side stream; the first GEMM of the next forward pass
// waits for them (ev_w)
cheb_status fork_weight_pack(cheb_mlp *net, cudaStream_t st)
{
    CHEB_CUDA_TRY(cudaEventRecord(net->ev_fork, st));
    CHEB_CUDA_TRY(cudaStreamWaitEvent(net->side, net->ev_fork, 0));
    cheb_status r = pack_weights(net, net->side);
    if (r) return r;
    CHEB_CUDA_TRY(cudaEventRecord(net->ev_w, net->side));
    net->wpack_pending = true;
    return CHEB_OK;
}

// forward pass of a batch whose (normalised) inputs are in net->X; with
// `train` the transposed packed activations for backpropagation are written too
cheb_status forward(cheb_ctx *ctx, cheb_mlp *net, int B, bool train, cudaStream_t st)
{
    cheb_status r;
    if (!net->wpack_valid && (r = fork_weight_pack(net, st))) return r;
    if ((r = pack(net->X, net->dims[0], B, net->dims[0], net->hk[0], train ? net->ht[0] : nullptr, st))) return r;
    if (net->wpack_pending) {
        CHEB_CUDA_TRY(cudaStreamWaitEvent(st, net->ev_w, 0));
        net->wpack_pending = false;
    }
    for (int l = 0; l < net->L; ++l) {
        const int ni = net->dims[l], no = net->dims[l + 1];
        const bool last = (l == net->L - 1);
        float *Zl = net->Z + act_off(net, l + 1, B);
        OutSpec o = no_out(B, no);
        o.bias = net->w + net->boff[l];
        if (last) {
            o.C = Zl;
            o.epi = EPI_BIAS;
        } else {
            o.Z = Zl;
            o.epi = EPI_BIAS_GELU;
            o.pk = net->hk[l + 1];
            o.pk_kt = cdiv(no, kTK);
            if (train) {
                o.pt = net->ht[l + 1];
                o.pt_kt = cdiv(B, kTK);
            }
        }
        if ((r = gemm(ctx, net->hk[l], cdiv(ni, kTK), net->wk[l], cdiv(ni, kTK), ni, o, net->split_ws, st))) return r;
    }
    return CHEB_OK;
}

// output of the last layer (FP32, B x out)
float *output(cheb_mlp *net, int B) { return net->Z + act_off(net, net->L, B); }

// loss gradient of the last layer from the normalised targets in T: FP32 into
// level L of net->dZ and the packed forms of level L
cheb_status loss_grad(cheb_mlp *net, int B, const float *T, float *loss, cudaStream_t st)
{
    cheb_status r = set_kernel_attrs();
    if (r) return r;
    const int O = net->dims[net->L];
    OutSpec o = no_out(B, O);
    o.C = net->dZ + act_off(net, net->L, B);
    o.pk = net->dzk[net->L];
    o.pk_kt = cdiv(O, kTK);
    o.pt = net->dzt[net->L];
    o.pt_kt = cdiv(B, kTK);
    const dim3 grid((unsigned)cdiv(O, kTN), (unsigned)(cdiv(B, kTK) * (kTK / kSlab)));
    {
        ProfScope prof("mlp_loss_grad", st);
        if ((r = launch(mse_tile_kernel, grid, dim3(kGemmThreads), 0, st, (const float *)output(net, B), T,
                        1.0f / ((float)B * O), net->loss_part, o)))
            return r;
    }
    // the loss itself is only reported: summed on the side stream (joined at the end of backward)
    CHEB_CUDA_TRY(cudaEventRecord(net->ev_fork, st));
    CHEB_CUDA_TRY(cudaStreamWaitEvent(net->side, net->ev_fork, 0));
    return launch(loss_sum_kernel, dim3(1), dim3(256), 0, net->side, (const float *)net->loss_part,
                  (int)(grid.x * grid.y), loss);
}

// backward pass from the level-L gradient (FP32 and packed) to net->grad. The
// input-gradient chain (dZ of level l from dZ of level l + 1) runs on `st`;
// each layer's weight and bias gradients fork to the side stream as soon as
// their inputs exist and join `st` at the end, so they overlap the chain.
cheb_status backward(cheb_ctx *ctx, cheb_mlp *net, int B, cudaStream_t st)
{
    cheb_status r;
    for (int l = net->L - 1; l >= 0; --l) {
        const int ni = net->dims[l], no = net->dims[l + 1];
        const float *dZo = net->dZ + act_off(net, l + 1, B);
        CHEB_CUDA_TRY(cudaEventRecord(net->ev_fork, st));
        CHEB_CUDA_TRY(cudaStreamWaitEvent(net->side, net->ev_fork, 0));
        // dW_l[o, i] = sum_b dZ[b, o] in[b, i]
        OutSpec g = no_out(no, ni);
        g.C = net->grad + net->woff[l];
        if ((r = gemm(ctx, net->dzt[l + 1], cdiv(B, kTK), net->ht[l], cdiv(B, kTK), B, g, net->split_ws2, net->side)))
            return r;
        {
            ProfScope prof("mlp_bias_grad", net->side);
            if ((r = launch(bias_grad_kernel, dim3((unsigned)cdiv(no, 32)), dim3(256), 0, net->side, dZo, B, no,
                            net->grad + net->boff[l])))
                return r;
        }
        if (l > 0) {
            // dZ_{l-1}[b, i] = (sum_o dZ[b, o] W_l[o, i]) GELU'(Z_{l-1}[b, i])
            OutSpec h = no_out(B, ni);
            h.C = net->dZ + act_off(net, l, B);
            h.aux = net->Z + act_off(net, l, B);
            h.epi = EPI_GELU_BWD;
            h.pk = net->dzk[l];
            h.pk_kt = cdiv(ni, kTK);
            h.pt = net->dzt[l];
            h.pt_kt = cdiv(B, kTK);
            if ((r = gemm(ctx, net->dzk[l + 1], cdiv(no, kTK), net->wt[l], cdiv(no, kTK), no, h, net->split_ws, st)))
                return r;
        }
    }
    CHEB_CUDA_TRY(cudaEventRecord(net->ev_join, net->side));
    CHEB_CUDA_TRY(cudaStreamWaitEvent(st, net->ev_join, 0));
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
    NvtxRange nvtx_range("surrogate_create");
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
        surrogate_destroy(net);
        return fail(CHEB_ENOMEM, "surrogate allocation failed");
    }
    net->wk.assign(net->L, nullptr);
    net->wt.assign(net->L, nullptr);
    for (int l = 0; l < net->L; ++l) {
        const int ni = net->dims[l], no = net->dims[l + 1];
        if (cudaMalloc(&net->wk[l], packed_bytes(no, ni)) || cudaMalloc(&net->wt[l], packed_bytes(ni, no))) {
            surrogate_destroy(net);
            return fail(CHEB_ENOMEM, "surrogate allocation failed");
        }
        cudaMemset(net->wk[l], 0, packed_bytes(no, ni));
        cudaMemset(net->wt[l], 0, packed_bytes(ni, no));
    }
    {
        std::vector<PackJob> jobs(net->L);
        int first = 0;
        for (int l = 0; l < net->L; ++l) {
            const int ni = net->dims[l], no = net->dims[l + 1];
            PackJob &j = jobs[l];
            std::memset(&j, 0, sizeof(j));
            j.src = net->w + net->woff[l];
            j.ld = ni;
            j.o = no_out(no, ni);
            j.o.pk = net->wk[l];
            j.o.pk_kt = cdiv(ni, kTK);
            j.o.pt = net->wt[l];
            j.o.pt_kt = cdiv(no, kTK);
            j.col_tiles = cdiv(ni, kTN);
            j.first_block = first;
            first += j.col_tiles * cdiv(no, kTK) * (kTK / kSlab);   // row slabs up to a multiple of 64 rows
        }
        net->pack_blocks = first;
        if (cudaMalloc(&net->d_jobs, sizeof(PackJob) * net->L) ||
            cudaMemcpy(net->d_jobs, jobs.data(), sizeof(PackJob) * net->L, cudaMemcpyHostToDevice) ||
            cudaStreamCreateWithFlags(&net->side, cudaStreamNonBlocking) ||
            cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming) ||
            cudaEventCreateWithFlags(&net->ev_join, cudaEventDisableTiming) ||
            cudaEventCreateWithFlags(&net->ev_t, cudaEventDisableTiming) ||
            cudaEventCreateWithFlags(&net->ev_w, cudaEventDisableTiming)) {
            surrogate_destroy(net);
            return fail(CHEB_ENOMEM, "surrogate allocation failed");
        }
    }
    free_batch(net);
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
    NvtxRange nvtx_range("surrogate_destroy");
    if (!net) return CHEB_OK;
    cudaSetDevice(net->device);
    cudaDeviceSynchronize();
    for (void *p : {(void *)net->w, (void *)net->grad, (void *)net->m, (void *)net->v, (void *)net->x_mean,
                    (void *)net->x_inv, (void *)net->x_std, (void *)net->y_mean, (void *)net->y_inv,
                    (void *)net->y_std, (void *)net->loss})
        if (p) cudaFree(p);
    for (uint8_t *p : net->wk)
        if (p) cudaFree(p);
    for (uint8_t *p : net->wt)
        if (p) cudaFree(p);
    for (void *p : net->batch_bufs) cudaFree(p);
    if (net->d_jobs) cudaFree(net->d_jobs);
    if (net->side) cudaStreamDestroy(net->side);
    for (cudaEvent_t e : {net->ev_fork, net->ev_join, net->ev_t, net->ev_w})
        if (e) cudaEventDestroy(e);
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
        net->wpack_valid = false;
    }
    if (get) CHEB_CUDA_TRY(cudaMemcpy(get, net->w, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost));
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_loss_grad(cheb_ctx *ctx, cheb_mlp *net, const float *X, const float *T, int32_t B,
                                         float *loss, float *grad, void *stream)
{
    NvtxRange nvtx_range("surrogate_loss_grad");
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    if (B < 1 || !X || !T) return fail(CHEB_EINVAL, "surrogate_loss_grad: bad batch");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = net_ws(ctx, net, B))) return r;
    const int F = net->dims[0];
    CHEB_CUDA_TRY(cudaMemcpyAsync(net->X, X, sizeof(float) * B * F, cudaMemcpyDeviceToDevice, st));
    if ((r = forward(ctx, net, B, true, st))) return r;
    CHEB_CUDA_TRY(cudaMemsetAsync(net->loss, 0, sizeof(float), st));
    if ((r = loss_grad(net, B, T, net->loss, st))) return r;
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
    NvtxRange nvtx_range("surrogate_adam_step");
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    if (!(lr > 0)) return fail(CHEB_EINVAL, "surrogate_adam_step: lr must be > 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    net->adam_t += 1;
    const float c1 = 1.0f - std::pow(b1, (float)net->adam_t), c2 = 1.0f - std::pow(b2, (float)net->adam_t);
    {
        ProfScope prof("mlp_adam", st);
        if ((r = launch(adam_kernel, dim3(blocks_for(net->nparam)), dim3(256), 0, st, net->nparam, net->w,
                            (const float *)(grad ? grad : net->grad), net->m, net->v, lr, b1, b2, eps, c1, c2,
                            (const float *)nullptr)))
            return r;
    }
    net->wpack_valid = false;
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}

CHEB_API cheb_status surrogate_train(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride,
                                     const double *Y, int64_t y_stride, int64_t S, int32_t epochs, int32_t batch,
                                     float lr, uint64_t seed, float *loss_per_epoch, void *stream)
{
    NvtxRange nvtx_range("surrogate_train");
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    const int F = net->dims[0], O = net->dims[net->L];
    if (!X || !Y || S < 1 || epochs < 0 || batch < 1 || x_stride < F || y_stride < O || !(lr > 0))
        return fail(CHEB_EINVAL, "surrogate_train: bad arguments");
    if (epochs > 4096) return fail(CHEB_EINVAL, "surrogate_train: at most 4096 epochs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = (int)std::min<int64_t>(batch, S);
    if ((r = net_ws(ctx, net, B))) return r;
    // normalisation from the training set: inputs and targets to zero mean, unit std
    column_stats_kernel<<<(unsigned)cdiv(F, 32), 1024, 0, st>>>(X, x_stride, S, F, net->x_mean, net->x_std);
    column_stats_kernel<<<(unsigned)cdiv(O, 32), 1024, 0, st>>>(Y, y_stride, S, O, net->y_mean, net->y_std);
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
    const int64_t steps = S / B;      // full batches per epoch
    if (epochs == 0 || steps == 0) return CHEB_OK;
    if ((r = set_kernel_attrs())) return r;
    // device side of one epoch: the permutation, the per-step (lr, 1 - b1^t, 1 - b2^t)
    // and the epoch's loss sum
    std::vector<int> perm(S);
    std::vector<float> sched(3 * steps);
    int *d_perm = nullptr;
    float *d_sched = nullptr;
    CHEB_CUDA_TRY(cudaMalloc(&d_perm, sizeof(int) * S));
    if (cudaMalloc(&d_sched, sizeof(float) * (3 * steps + 1)) != cudaSuccess) {
        cudaFree(d_perm);
        return fail(CHEB_ENOMEM, "surrogate_train: allocation failed");
    }
    float *d_acc = d_sched + 3 * steps;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    auto enqueue_epoch = [&](cudaStream_t s) -> cheb_status {
        cheb_status e;
        CHEB_CUDA_TRY(cudaMemsetAsync(d_acc, 0, sizeof(float), s));
        net->wpack_valid = false;
        for (int64_t k = 0; k < steps; ++k) {
            const int *rows = d_perm + k * B;
            // the weights are packed and the targets gathered on the side stream,
            // concurrently with the input gather and the start of the forward pass
            if ((e = fork_weight_pack(net, s))) return e;
            if ((e = launch(gather_norm_kernel, dim3(blocks_for((int64_t)B * O)), dim3(256), 0, net->side, Y, y_stride,
                            rows, B, O, (const float *)net->y_mean, (const float *)net->y_inv, net->T)))
                return e;
            CHEB_CUDA_TRY(cudaEventRecord(net->ev_t, net->side));
            if ((e = launch(gather_norm_kernel, dim3(blocks_for((int64_t)B * F)), dim3(256), 0, s, X, x_stride,
                            rows, B, F, (const float *)net->x_mean, (const float *)net->x_inv, net->X)))
                return e;
            if ((e = forward(ctx, net, B, true, s))) return e;
            CHEB_CUDA_TRY(cudaStreamWaitEvent(s, net->ev_t, 0));
            if ((e = loss_grad(net, B, net->T, d_acc, s))) return e;
            if ((e = backward(ctx, net, B, s))) return e;
            if ((e = launch(adam_kernel, dim3(blocks_for(net->nparam)), dim3(256), 0, s, net->nparam, net->w,
                                (const float *)net->grad, net->m, net->v, 0.0f, b1, b2, eps, 1.0f, 1.0f,
                                (const float *)(d_sched + 3 * k))))
                return e;
            net->wpack_valid = false;
        }
        return CHEB_OK;
    };
    // one epoch is captured once into a CUDA graph; with kernel timing on, the
    // timing events are captured as event-record nodes, so each kernel is timed
    // where it runs, inside the graph (the last replay's times are read)
    cudaGraphExec_t exec = nullptr;
    {
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            r = enqueue_epoch(cs);
            ce = cudaStreamEndCapture(cs, &graph);
            if (r == CHEB_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        if (cs) cudaStreamDestroy(cs);
        if (r == CHEB_OK && ce != cudaSuccess) r = cuda_fail(ce, "surrogate_train: epoch graph");
    }
    for (int e = 0; e < epochs && r == CHEB_OK; ++e) {
        // Fisher-Yates shuffle driven by SplitMix64(seed), counter = (epoch, position)
        for (int64_t i = 0; i < S; ++i) perm[i] = (int)i;
        for (int64_t i = S - 1; i > 0; --i) {
            const uint64_t z = splitmix64(seed, ((uint64_t)e << 32) + (uint64_t)i);
            const int64_t j = (int64_t)(z % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        for (int64_t k = 0; k < steps; ++k) {
            const int64_t t = net->adam_t + 1 + k;
            // cosine decay of the learning rate over the run
            const double prog = (double)(e * steps + k) / (double)std::max<int64_t>(1, (int64_t)epochs * steps);
            sched[3 * k] = (float)(0.5 * lr * (1.0 + std::cos(M_PI * prog)));
            sched[3 * k + 1] = 1.0f - std::pow(b1, (float)t);
            sched[3 * k + 2] = 1.0f - std::pow(b2, (float)t);
        }
        cudaError_t ce = cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(d_sched, sched.data(), sizeof(float) * 3 * steps, cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess) {
            if (exec) {
                ce = cudaGraphLaunch(exec, st);
            } else {
                r = enqueue_epoch(st);
            }
        }
        if (ce == cudaSuccess && r == CHEB_OK)
            ce = cudaMemcpyAsync(net->loss + e, d_acc, sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (ce != cudaSuccess && r == CHEB_OK) r = cuda_fail(ce, "surrogate_train");
        net->adam_t += steps;
        net->wpack_valid = false;
    }
    if (loss_per_epoch && r == CHEB_OK) {
        std::vector<float> l(epochs);
        CHEB_CUDA_TRY(cudaMemcpyAsync(l.data(), net->loss, sizeof(float) * epochs, cudaMemcpyDeviceToHost, st));
        CHEB_CUDA_TRY(cudaStreamSynchronize(st));
        for (int e = 0; e < epochs; ++e) loss_per_epoch[e] = l[e] / (float)steps;
    }
    cudaStreamSynchronize(st);
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(d_perm);
    cudaFree(d_sched);
    return r;
}

CHEB_API cheb_status surrogate_predict(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride, int64_t P,
                                       double *Y, int64_t y_stride, void *stream)
{
    NvtxRange nvtx_range("surrogate_predict");
    cheb_status r = check_net(ctx, net);
    if (r) return r;
    const int F = net->dims[0], O = net->dims[net->L];
    if (P < 0 || (P > 0 && (!X || !Y)) || x_stride < F || y_stride < O)
        return fail(CHEB_EINVAL, "surrogate_predict: bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = std::max(net->ws_batch, 256);
    if ((r = net_ws(ctx, net, B))) return r;
    for (int64_t p0 = 0; p0 < P; p0 += B) {
        const int nb = (int)std::min<int64_t>(B, P - p0);
        gather_norm_kernel<<<blocks_for((int64_t)nb * F), 256, 0, st>>>(X + p0 * x_stride, x_stride, nullptr, nb, F,
                                                                        net->x_mean, net->x_inv, net->X);
        if ((r = forward(ctx, net, nb, false, st))) return r;
        denorm_kernel<<<blocks_for((int64_t)nb * O), 256, 0, st>>>(output(net, nb), nb, O, net->y_mean, net->y_inv,
                                                                   Y + p0 * y_stride, y_stride);
        CHEB_CUDA_TRY(cudaGetLastError());
    }
    return CHEB_OK;
}

}  // extern "C"
