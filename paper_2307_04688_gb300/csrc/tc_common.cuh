// Inline-PTX helpers for sm_103a: mbarriers, bulk copies (TMA engine),
// tcgen05 MMA with TMEM accumulators, and the operand splits used by the
// split-precision forms. Used by the tensor-core kernels of libcheb.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace cheb {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One try: the thread is suspended until the phase completes or about a
// millisecond passes (the suspend-time hint), so a waiting warp does not spin
// through issue slots that the other warps of the SM need.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Default bound of a device-side wait: 2^32 SM cycles (about 2 s).
constexpr long long kWaitCycles = 1ll << 32;

// Wait for phase `parity` of `bar` to complete, giving up once `limit` SM
// cycles have passed (the limit is checked before every try, so a limit of 0
// gives up at once). Returns false on timeout and records CHEB_ETIMEOUT (6)
// in the device error word `err`. A caller that gives up must still wait, with
// the default bound, for the copies and MMAs that signal `bar` before its CTA
// frees TMEM or exits.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  long long limit = kWaitCycles)
{
    const long long t0 = clock64();
    for (uint32_t it = 0; it < (1u << 28); ++it) {
        if (clock64() - t0 >= limit) break;
        if (mbar_try_wait(bar, parity)) return true;
    }
    atomicCAS(err, 0, 6);
    return false;
}

// ---- bulk copy global -> shared (TMA engine, non-tensor form) ---------------
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- per-thread asynchronous copy global -> shared (8 bytes) -----------------
// Completes for the issuing thread at its cp_async_wait_all(); both addresses
// 8-byte aligned.
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---- bulk copy shared -> global (TMA engine, non-tensor form) ---------------
// dst and src 16-byte aligned, bytes a multiple of 16; tracked in bulk groups
// of the issuing thread.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until every committed bulk group of this thread has completed (its
// writes performed, its shared-memory sources free).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Make generic-proxy writes to shared memory visible to the async proxy
// (tensor-core operand reads).
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---- programmatic dependent launch --------------------------------------------
// Let the next kernel in the stream start its prologue now (it still waits for
// this grid's completion at its own griddep_wait).
__device__ __forceinline__ void griddep_launch_dependents()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Wait until the grids this one depends on have completed and their memory
// is visible (returns at once when launched without a programmatic edge).
__device__ __forceinline__ void griddep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- TMEM -------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 16 consecutive 32-bit columns; thread i of the warp receives
// lane (32 * (warp % 4) + i) of TMEM.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Barrier `id` (1..15) over the first `count` threads that reach it (a
// multiple of 32; every warp of the group must arrive).
__device__ __forceinline__ void named_barrier_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// One 32-bit column: thread i of the warp receives lane (32 * (warp % 4) + i).
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t &r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- MMA ----------------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// core matrices of 8 rows x 16 bytes (128 contiguous bytes); `lbo` = byte
// distance between core matrices adjacent along K, `sbo` = between core
// matrices adjacent along M/N. Bits 46-47 hold the descriptor version (1).
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor for kind::f16 (BF16 inputs) and kind::tf32: FP32
// accumulator, both operands K-major, dense.
//   bits 4-5 D format (1 = F32), 7-9 A format, 10-12 B format
//   (BF16 = 1, TF32 = 2), 17-22 N >> 3, 24-28 M >> 4.
__host__ __device__ constexpr uint32_t make_idesc(int ab_format, int M, int N)
{
    return (1u << 4) | ((uint32_t)ab_format << 7) | ((uint32_t)ab_format << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on `bar` when every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// ---- operand splits -----------------------------------------------------------
// x = x_0 + x_1 + ... + x_{S-1} + residual, each x_s the nearest BF16 (or TF32)
// to what is left; the residual is formed exactly in the input's precision.
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

template <int S>
__device__ __forceinline__ void split_bf16(double x, uint16_t (&o)[S])
{
    double r = x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        __nv_bfloat16 h = __double2bfloat16(r);
        o[s] = __bfloat16_as_ushort(h);
        r -= (double)__bfloat162float(h);
    }
}

template <int S>
__device__ __forceinline__ void split_bf16(float x, uint16_t (&o)[S])
{
    float r = x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        __nv_bfloat16 h = __float2bfloat16_rn(r);
        o[s] = __bfloat16_as_ushort(h);
        r -= __bfloat162float(h);
    }
}

template <int S>
__device__ __forceinline__ void split_tf32(double x, uint32_t (&o)[S])
{
    double r = x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        o[s] = tf32_rna((float)r);
        r -= (double)__uint_as_float(o[s]);
    }
}

template <int S>
__device__ __forceinline__ void split_tf32(float x, uint32_t (&o)[S])
{
    float r = x;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        o[s] = tf32_rna(r);
        r -= __uint_as_float(o[s]);
    }
}

// ---- double-float (an FP32 pair hi + lo) -------------------------------------
// GB300 runs FP64 at a small fraction of its FP32 rate; values that need more
// than FP32 precision but are only ever rounded to FP32 are carried as pairs.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_from_double(double x)
{
    ff r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

// 2 x t1 - t0 in double-float arithmetic (error-free products and sums)
__device__ __forceinline__ ff ff_cheb_step(ff x2, ff t1, ff t0)
{
    float p = x2.hi * t1.hi;
    float e = fmaf(x2.hi, t1.hi, -p);
    e = fmaf(x2.hi, t1.lo, e);
    e = fmaf(x2.lo, t1.hi, e);
    // (p + e) - (t0.hi + t0.lo)
    const float s = p - t0.hi;
    const float bb = s - p;
    const float err = (p - (s - bb)) + (-t0.hi - bb);
    float lo = err + e - t0.lo;
    float hi = s + lo;
    lo = lo - (hi - s);
    return {hi, lo};
}

}  // namespace tc

}  // namespace cheb
