// cheb_eval_grid_noalloc: the split-precision tensor-grid evaluation with all
// of its scratch memory in one file-scope device array, for callers that must
// not allocate device memory.
//
// Who needs it: callers that cannot call cudaMalloc or own a libcheb context.
// A host framework may have reserved all device memory in its own pool, so a
// cudaMalloc from inside its hot path fails; cudaMalloc and cudaFree can also
// synchronise the device and stall unrelated streams, which latency-bound
// callers cannot accept; and a context (cheb_create) itself allocates. This
// entry point takes no context, makes no allocation of any kind and only
// enqueues kernels, a memset of its error word and nothing else.
//
// Scratch: kScratchBytes of FP32 intermediates (the two largest consecutive
// intermediates of the mode-product chain must fit together), kTmatBytes for
// the Chebyshev matrices T_l(x_j) and one error word. The array lives in every
// GPU that loads the library until the process exits. Its device address is
// looked up once per device with cudaGetSymbolAddress, the first time this
// entry point runs with that device current (so that first call should come
// before any stream capture), and handed to the kernels; host code never
// dereferences the symbol itself. Every call reuses the same array and it
// keeps the previous call's contents: the error word is cleared at the start
// of every call, everything else is written before it is read. Two calls that
// overlap on the GPU (different streams, or different host threads) race on
// the array and corrupt each other's results: serialise them.
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>

#include "cheb_internal.cuh"

namespace cheb {
namespace {

constexpr size_t kScratchBytes = 64ull << 20;   // FP32 intermediates
constexpr size_t kTmatBytes = 1ull << 20;       // FP64 T matrices
constexpr size_t kTotalBytes = kScratchBytes + kTmatBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kTotalBytes];
// bound, in SM cycles, of the device-side waits of this entry point (process-wide)
static std::atomic<long long> g_noalloc_wait_limit{kDefaultWaitCycles};

struct DeviceSlot {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch
    int num_sms = 0;
};

std::mutex g_slot_mutex;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: the symbol's device address.
cheb_status device_slot(int device, DeviceSlot **out)
{
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    DeviceSlot &s = g_slots[device];
    if (!s.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(multiProcessorCount)");
        s.base = static_cast<unsigned char *>(ptr);
        s.num_sms = sms;
        s.ready = true;
    }
    *out = &s;
    return CHEB_OK;
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" CHEB_API cheb_status cheb_eval_grid_noalloc(int d, const int32_t *n, const double *coeffs,
                                                       const double *a, const double *b,
                                                       const int32_t *m, const double *const *x,
                                                       float *out, cheb_precision prec, void *stream)
{
    NvtxRange nvtx_range("cheb_eval_grid_noalloc");
    tl_ctx = nullptr;
    if (prec != CHEB_TF32X3 && prec != CHEB_BF16X3 && prec != CHEB_BF16X6)
        return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: prec must be a split form");
    if (d < 1 || d > 6 || !n || !m || !x || !a || !b || !coeffs || !out)
        return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: bad d or null argument");
    int64_t total = 1, out_total = 1;
    size_t tmat = 0;
    for (int s = 0; s < d; ++s) {
        if (n[s] < 2 || n[s] > 64) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: n[s] must be in [2, 64]");
        if (m[s] < 1 || m[s] > 256) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: m[s] must be in [1, 256]");
        if (!x[s]) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: null point array");
        if (!(a[s] < b[s])) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: need a[s] < b[s]");
        total *= n[s];
        out_total *= m[s];
        tmat += sizeof(double) * (size_t)m[s] * n[s];
    }
    if (tmat > kTmatBytes)
        return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: the T matrices need " + std::to_string(tmat) +
                                     " bytes, above the fixed maximum of " + std::to_string(kTmatBytes));
    // sizes of the chain's FP32 intermediates (outputs of steps 0..d-2)
    int64_t sizes[6] = {0, 0, 0, 0, 0, 0};
    {
        int64_t cur = total;
        for (int t = 0; t < d - 1; ++t) {
            const int mode = d - 1 - t;
            cur = cur / n[mode] * m[mode];
            sizes[t] = cur;
        }
        for (int t = 0; t < d - 1; ++t) {
            const size_t need = sizeof(float) * (size_t)(sizes[t] + (t > 0 ? sizes[t - 1] : 0)) + 16;
            if (need > kScratchBytes)
                return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc: intermediates need " + std::to_string(need) +
                                             " bytes, above the fixed maximum of " +
                                             std::to_string(kScratchBytes));
        }
    }
    int device = 0;
    CHEB_CUDA_TRY(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) return fail(CHEB_EUNSUPPORTED, "device ordinal too large");
    DeviceSlot *slot = nullptr;
    cheb_status st = device_slot(device, &slot);
    if (st) return st;
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    unsigned char *base = slot->base;
    double *T = reinterpret_cast<double *>(base + kScratchBytes);
    int *err = reinterpret_cast<int *>(base + kScratchBytes + kTmatBytes);
    CHEB_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), sm));
    double *Ts[6];
    size_t toff = 0;
    for (int s = 0; s < d; ++s) {
        Ts[s] = T + toff;
        toff += (size_t)m[s] * n[s];
    }
    if ((st = cheb_matrices(d, x, m, n, a, b, Ts, sm))) return st;
    // intermediates alternate between the two ends of the scratch area, so
    // a step's input and output never overlap
    const void *src = coeffs;
    int64_t cur = total;
    for (int t = 0; t < d; ++t) {
        const int mode = d - 1 - t;
        float *dst;
        if (t == d - 1)
            dst = out;
        else if ((t & 1) == 0)
            dst = reinterpret_cast<float *>(base);
        else  // the next step bulk-copies from here: round down to 16 bytes
            dst = reinterpret_cast<float *>(
                reinterpret_cast<uintptr_t>(reinterpret_cast<float *>(base + kScratchBytes) - sizes[t]) &
                ~uintptr_t(15));
        const int64_t R = cur / n[mode];
        if ((st = modeprod_tc_raw(src, t == 0, Ts[mode], dst, R, n[mode], m[mode], prec, err, slot->num_sms, sm,
                                  nullptr, -1.0, 1.0, g_noalloc_wait_limit.load())))
            return st;
        cur = R * m[mode];
        src = dst;
    }
    return CHEB_OK;
}

extern "C" CHEB_API cheb_status cheb_eval_grid_noalloc_set_wait_limit(int64_t cycles)
{
    tl_ctx = nullptr;
    if (cycles < 0) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc_set_wait_limit: cycles must be >= 0");
    g_noalloc_wait_limit.store(cycles);
    return CHEB_OK;
}

extern "C" CHEB_API cheb_status cheb_eval_grid_noalloc_status(void *stream)
{
    tl_ctx = nullptr;
    int device = 0;
    CHEB_CUDA_TRY(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) return fail(CHEB_EUNSUPPORTED, "device ordinal too large");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_slot_mutex);
        if (g_slots[device].ready) base = g_slots[device].base;
    }
    if (!base) return fail(CHEB_EINVAL, "cheb_eval_grid_noalloc_status: no call ran on this device");
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    const int *err = reinterpret_cast<const int *>(base + kScratchBytes + kTmatBytes);
    int v = 0;
    CHEB_CUDA_TRY(cudaStreamSynchronize(sm));
    CHEB_CUDA_TRY(cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) return fail((cheb_status)v, "cheb_eval_grid_noalloc: a device-side wait ran out of time");
#ifdef CHEB_CHECK
    return dcheck::report();
#else
    return CHEB_OK;
#endif
}
