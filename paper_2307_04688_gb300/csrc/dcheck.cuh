// Device bounds checks of the checked build, and NVTX ranges.
//
// Compiled with -DCHEB_CHECK (libcheb_check.so), CHEB_DCHECK(cond) tests an
// index or an offset against the extent of the buffer it addresses. A failed
// test records its source line in the check word of its translation unit
// (first failure wins) and evaluates to false, so the guarded access is
// skipped: nothing traps and the context stays usable. cheb_device_status
// reads and clears the words of every translation unit and returns
// CHEB_EBOUNDS with the file and line in cheb_last_error(). In the default
// build CHEB_DCHECK(cond) is the constant true and `cond` is not compiled.
//
// NvtxRange pushes a named NVTX range for its lifetime (header-only NVTX 3:
// without a tool attached the calls return at once).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace cheb {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Dynamic shared memory of the running kernel, in bytes.
__device__ __forceinline__ unsigned dyn_smem_bytes()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

#ifdef CHEB_CHECK
namespace dcheck {

// Reads this translation unit's check word on the current device and clears
// it; returns a cudaError_t, the line (0: no failure) in *line.
using Reader = int (*)(int *line);
void register_reader(const char *file, Reader r);
// Reads and clears every translation unit's word on the current device:
// CHEB_EBOUNDS (file and line in the last error) if any check failed.
cheb_status report();

namespace {
__device__ int g_check_line;

__device__ __noinline__ bool failed_at(int line)
{
    atomicCAS(&g_check_line, 0, line);
    return false;
}

int read_and_clear(int *line)
{
    *line = 0;
    cudaError_t e = cudaMemcpyFromSymbol(line, g_check_line, sizeof(int));
    if (e == cudaSuccess && *line != 0) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_check_line, &zero, sizeof(int));
    }
    return (int)e;
}

struct Registration {
    Registration() { register_reader(__BASE_FILE__, &read_and_clear); }
};
Registration g_registration;
}  // namespace

}  // namespace dcheck
#define CHEB_DCHECK(cond) ((cond) || ::cheb::dcheck::failed_at(__LINE__))
#else
#define CHEB_DCHECK(cond) true
#endif

}  // namespace cheb
