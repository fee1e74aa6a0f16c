// Internal declarations shared by the translation units of libcheb.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cheb.h"
#include "dcheck.cuh"

namespace cheb {

// Record `msg` as the calling thread's last error and return `st`.
cheb_status fail(cheb_status st, const std::string &msg);
cheb_status cuda_fail(cudaError_t e, const char *what);

#define CHEB_CUDA_TRY(expr)                                                  \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) return ::cheb::cuda_fail(e_, #expr);          \
    } while (0)

// Bound of a device-side wait in SM cycles (about 2 s at 2 GHz); must equal
// the kernels' own default (tc_common.cuh) and CHEB_WAIT_LIMIT_DEFAULT.
constexpr long long kDefaultWaitCycles = 1ll << 32;

// One-time set-up per device (kernel attributes such as the dynamic shared
// memory limit apply to the device that is current when they are set): the
// first call on a device runs `init` with that device current and caches the
// int it produces; later calls on the same device return the cached value.
// Thread-safe. A failed `init` is retried by the next call.
constexpr int kMaxDevices = 64;
struct PerDevice {
    std::mutex mu;
    bool set[kMaxDevices] = {};
    int val[kMaxDevices] = {};
};

template <class Init>
cheb_status per_device_once(PerDevice &pd, Init init, int *out)
{
    int dev = 0;
    CHEB_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CHEB_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(pd.mu);
    if (!pd.set[dev]) {
        int v = 0;
        const cheb_status st = init(&v);
        if (st != CHEB_OK) return st;
        pd.val[dev] = v;
        pd.set[dev] = true;
    }
    if (out) *out = pd.val[dev];
    return CHEB_OK;
}

// A device buffer owned by the context that only grows.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cheb_status reserve(size_t want);
    void release();
};

// The context of the ABI call in progress on this host thread (set by the
// entry points; read by the launch helpers for profiling and error words).
extern thread_local cheb_ctx *tl_ctx;

// Records CUDA events around one kernel launch when profiling is on.
struct ProfScope {
    cheb_ctx *ctx;
    std::string name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    unsigned record_flags = 0;   // cudaEventRecordExternal while `st` is being captured into a graph
    ProfScope(std::string nm, cudaStream_t s);
    ~ProfScope();
};

}  // namespace cheb

struct cheb_ctx {
    int device = 0;
    int num_sms = 0;
    cheb::DevBuf ws[2];                 // ping-pong intermediates of mode-product chains
    cheb::DevBuf tmats;                 // Chebyshev matrices T_l(x_j) of one call
    cheb::DevBuf xbuf;                  // a copy of the fit input for in-place fits
    std::map<int, double *> dct;        // n -> device n x n DCT-I matrix (FP64)
    cheb::DevBuf game;                  // game state of one game_solve call
    cheb::DevBuf game_aux;
    cheb::DevBuf paths;                 // control coefficients of one game_paths call
    // cheb_eval_grid_host: device copies of the host inputs and of the
    // result, and a page-locked host buffer that gathers the point arrays
    // into one copy
    cheb::DevBuf io_in, io_out;
    void *pts_host = nullptr;
    size_t pts_host_bytes = 0;
    cudaEvent_t pts_done = nullptr;     // the last copy out of pts_host has finished
    // tile-shape tuning (cheb_set_tuning): 0 tune on first use, 1 default
    // shapes, 2 + k force configuration k; tuned choices by shape key
    int tune_mode = 0;
    std::map<std::string, std::pair<int, std::string>> game_tune;
    int *d_error = nullptr;             // device error word written by bounded waits
    long long wait_limit = cheb::kDefaultWaitCycles;   // SM cycles a main-loop device wait may take
    // kernel timing (cheb_profile): events around every library launch
    bool prof_on = false;
    struct ProfEvent {
        std::string name;
        cudaEvent_t a, b;
    };
    std::vector<ProfEvent> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    std::map<std::string, std::pair<int64_t, double>> prof_totals;
};

namespace cheb {

// ---- kernels (fp64_kernels.cu) ----------------------------------------------

// out[j * R + r] = sum_k B[j * n + k] * X[r * n + k]   (j < m, r < R)
// One product along the trailing mode of a row-major [R x n] view, with the
// new mode written in front: applied d times it visits every mode and leaves
// the modes in their original order.
cheb_status modeprod_f64(const double *X, const double *B, double *out, int64_t R, int n, int m,
                         cudaStream_t st);

// Slabs to leave alone in modeprod_f64_slabs: slab g is skipped when
// flags[(g / per_flag) * stride] != 0 (no flags: none is).
struct SlabSkip {
    const int *flags = nullptr;
    int64_t stride = 0;      // in ints
    int64_t per_flag = 1;    // slabs per flag
};

// The same product on G slabs of R rows each, every slab moving its new mode
// to its own front: out[(g m + j) R + r] = sum_k B[j * n + k] X[(g R + r) n + k].
// Applied d times it takes each slab's tensor through all its modes and back
// to their original order, slab by slab. Rows of skipped slabs are neither
// computed nor written.
// All J mode products of G slabs (each an n^J tensor, row-major) with the same
// n x n matrix B in one launch, for small problems: one CTA per (slab, last
// output index) keeps the intermediate tensors in shared memory. Bit-identical
// to J successive modeprod_f64_slabs calls (same order of every sum). Returns
// CHEB_EUNSUPPORTED (and launches nothing) when n^(J-1) > 4913.
cheb_status modeprod_f64_chain(const double *X, const double *B, double *out, int64_t G, int J, int n,
                               const SlabSkip &skip, cudaStream_t st);
cheb_status modeprod_f64_slabs(const double *X, const double *B, double *out, int64_t G, int64_t R, int n, int m,
                               const SlabSkip &skip, cudaStream_t st);

// T[j * n + l] = T_l(x~_j), x~_j = (2 x[j * stride] - a - b) / (b - a), j < m, l < n.
cheb_status cheb_matrix(const double *x, int64_t stride, int64_t m, int n, double a, double b,
                        double *T, cudaStream_t st);

// The d matrices T_s[j * n_s + l] = T_l(x~_{s,j}) of a tensor grid, one launch.
cheb_status cheb_matrices(int d, const double *const *x, const int32_t *m, const int32_t *n,
                          const double *a, const double *b, double *const *T, cudaStream_t st);

// Split-precision point evaluation: the trailing mode on the tensor cores
// (modeprod_tc with the T rows as the A operand), the rest per point in FP64.
cheb_status eval_points_tc(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                           const double *a, const double *b, int64_t P, const double *x, float *out,
                           cheb_precision prec, cudaStream_t st);

// c[k] *= prod_s exp(-alpha (k_s / N_s)^(2 order)), in place.
cheb_status spectral_filter(int d, const int32_t *n, double *coeffs, double alpha, int order, cudaStream_t st);

// FP64 point evaluation: out[j] = sum_l c_l prod_s T_{l_s}(x~_{j,s}).
cheb_status eval_points_f64(int d, const int32_t *n, const double *coeffs, const double *a,
                            const double *b, int64_t P, const double *x, double *out,
                            cudaStream_t st);

// ---- tensor-core split-precision mode product (tc_modeprod.cu) -------------

// The same product as modeprod_f64 on the tensor cores. X is FP64 when
// x_f64 != 0 and FP32 otherwise; B is FP64 (split on the fly); out is FP32.
// With B null, B[j][k] = T_k(x~_j) is formed in the kernel from the m points
// xpts on [ta, tb]. Launched with programmatic stream serialization: the
// prologue overlaps the previous kernel's tail.
cheb_status modeprod_tc(cheb_ctx *ctx, const void *X, int x_f64, const double *B, float *out,
                        int64_t R, int n, int m, cheb_precision prec, cudaStream_t st,
                        const double *xpts = nullptr, double ta = -1.0, double tb = 1.0);

// modeprod_tc without a context: `err` is the device error word to use and
// `num_sms` the SM count of the current device.
cheb_status modeprod_tc_raw(const void *X, int x_f64, const double *B, float *out, int64_t R, int n,
                            int m, cheb_precision prec, int *err, int num_sms, cudaStream_t st,
                            const double *xpts = nullptr, double ta = -1.0, double tb = 1.0,
                            long long wait_limit = kDefaultWaitCycles);

// Evaluation at the Lobatto nodes E[k, l] = cos(pi l k / N), cached per n.
cheb_status node_eval_matrix(cheb_ctx *ctx, int n, const double **out);

// Host-side DCT-I matrix of eq. (forcoef), cached per n on the context.
cheb_status dct_matrix(cheb_ctx *ctx, int n, const double **out);

}  // namespace cheb
