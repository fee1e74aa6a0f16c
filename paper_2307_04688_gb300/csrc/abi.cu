// C ABI of libcheb: argument checking, workspaces and the mode-product
// chains behind cheb_fit, cheb_eval_grid and cheb_eval_points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cheb_internal.cuh"

namespace cheb {

static thread_local std::string g_last_error;
thread_local cheb_ctx *tl_ctx = nullptr;

static cudaEvent_t prof_event(cheb_ctx *c)
{
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(std::string nm, cudaStream_t s) : ctx(tl_ctx), name(std::move(nm)), st(s)
{
    if (ctx && ctx->prof_on) {
        a = prof_event(ctx);
        b = prof_event(ctx);
        // inside a stream capture the pair becomes two event-record nodes of the
        // graph, so the kernel is timed where the graph runs it
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            record_flags = cudaEventRecordExternal;
        cudaEventRecordWithFlags(a, st, record_flags);
    }
}

ProfScope::~ProfScope()
{
    if (a) {
        cudaEventRecordWithFlags(b, st, record_flags);
        ctx->prof_pending.push_back({name, a, b});
    }
}

static void prof_drain(cheb_ctx *c)
{
    for (auto &e : c->prof_pending) {
        float ms = 0.f;
        cudaEventSynchronize(e.b);
        cudaEventElapsedTime(&ms, e.a, e.b);
        auto &t = c->prof_totals[e.name];
        t.first += 1;
        t.second += ms;
        c->prof_pool.push_back(e.a);
        c->prof_pool.push_back(e.b);
    }
    c->prof_pending.clear();
}

#ifdef CHEB_CHECK
namespace dcheck {
namespace {
struct ReaderEntry {
    const char *file;
    Reader read;
};
std::mutex &registry_mutex()
{
    static std::mutex mu;
    return mu;
}
std::vector<ReaderEntry> &registry()
{
    static std::vector<ReaderEntry> r;
    return r;
}
}  // namespace

void register_reader(const char *file, Reader r)
{
    std::lock_guard<std::mutex> lock(registry_mutex());
    registry().push_back({file, r});
}

// Reads and clears every translation unit's check word on the current device;
// the first failure found (in registration order) is reported.
cheb_status report()
{
    std::lock_guard<std::mutex> lock(registry_mutex());
    std::string where;
    for (const ReaderEntry &e : registry()) {
        int line = 0;
        const int ce = e.read(&line);
        if (ce != 0) return cuda_fail((cudaError_t)ce, "reading a bounds check word");
        if (line != 0 && where.empty()) where = std::string(e.file) + ":" + std::to_string(line);
    }
    if (!where.empty()) return fail(CHEB_EBOUNDS, "device bounds check failed at " + where);
    return CHEB_OK;
}

namespace {
__global__ void selftest_kernel(int flag)
{
    // fails when flag == 0 (always, as launched); touches no memory
    if (!CHEB_DCHECK(flag != 0)) return;
}
}  // namespace
}  // namespace dcheck
#endif

cheb_status fail(cheb_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

cheb_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return CHEB_ECUDA;
}

cheb_status DevBuf::reserve(size_t want)
{
    if (want <= bytes) return CHEB_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    size_t sz = want < 256 ? 256 : want;
    cudaError_t e = cudaMalloc(&ptr, sz);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return fail(CHEB_ENOMEM, std::string("workspace allocation failed: ") + cudaGetErrorString(e));
    }
    bytes = sz;
    return CHEB_OK;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

// DCT-I matrix of eq. (forcoef): M[l,k] = (c_l / N) w_k cos(pi l k / N) with
// c_l = 1 for l in {0, N} else 2 and w_k = 1/2 for k in {0, N} else 1, so
// that p = M F gives the interpolation coefficients. The integer l*k is
// reduced modulo 2N before the cosine.
cheb_status dct_matrix(cheb_ctx *ctx, int n, const double **out)
{
    auto it = ctx->dct.find(n);
    if (it != ctx->dct.end()) {
        *out = it->second;
        return CHEB_OK;
    }
    const int N = n - 1;
    std::vector<double> M((size_t)n * n);
    for (int l = 0; l < n; ++l)
        for (int k = 0; k < n; ++k) {
            const long t = ((long)l * k) % (2L * N);
            const double cl = (l == 0 || l == N) ? 1.0 : 2.0;
            const double wk = (k == 0 || k == N) ? 0.5 : 1.0;
            M[(size_t)l * n + k] = cl / N * wk * std::cos(M_PI * (double)t / (double)N);
        }
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * M.size());
    if (e != cudaSuccess) return fail(CHEB_ENOMEM, "dct matrix allocation failed");
    e = cudaMemcpy(d, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "dct matrix upload");
    }
    ctx->dct[n] = d;
    *out = d;
    return CHEB_OK;
}

// Evaluation at the Lobatto nodes, E[k, l] = T_l(alpha^k) = cos(pi l k / N),
// cached per n on the context (key -n).
cheb_status node_eval_matrix(cheb_ctx *ctx, int n, const double **out)
{
    auto it = ctx->dct.find(-n);
    if (it != ctx->dct.end()) {
        *out = it->second;
        return CHEB_OK;
    }
    const int N = n - 1;
    std::vector<double> E((size_t)n * n);
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            const long t = ((long)l * k) % (2L * N);
            E[(size_t)k * n + l] = std::cos(M_PI * (double)t / (double)N);
        }
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * E.size());
    if (e != cudaSuccess) return fail(CHEB_ENOMEM, "node matrix allocation failed");
    e = cudaMemcpy(d, E.data(), sizeof(double) * E.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "node matrix upload");
    }
    ctx->dct[-n] = d;
    *out = d;
    return CHEB_OK;
}

namespace {

cheb_status check_ctx(cheb_ctx *ctx)
{
    tl_ctx = ctx;
    if (!ctx) return fail(CHEB_EINVAL, "null context");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != ctx->device) CHEB_CUDA_TRY(cudaSetDevice(ctx->device));
    return CHEB_OK;
}

cheb_status check_shape(int d, const int32_t *n, int nmax, int64_t *total)
{
    if (d < 1 || d > 6) return fail(CHEB_EINVAL, "d must be in [1, 6]");
    if (!n) return fail(CHEB_EINVAL, "null n");
    int64_t t = 1;
    for (int s = 0; s < d; ++s) {
        if (n[s] < 2 || n[s] > nmax)
            return fail(CHEB_EINVAL, "n[" + std::to_string(s) + "] must be in [2, " + std::to_string(nmax) + "]");
        t *= n[s];
        if (t > (int64_t)1 << 34) return fail(CHEB_EINVAL, "tensor too large");
    }
    *total = t;
    return CHEB_OK;
}

cheb_status check_domain(int d, const double *a, const double *b)
{
    if (!a || !b) return fail(CHEB_EINVAL, "null domain");
    for (int s = 0; s < d; ++s)
        if (!(std::isfinite(a[s]) && std::isfinite(b[s]) && a[s] < b[s]))
            return fail(CHEB_EINVAL, "domain must satisfy a[s] < b[s], finite");
    return CHEB_OK;
}

}  // namespace
}  // namespace cheb

using namespace cheb;

extern "C" {

const char *cheb_last_error(void) { return g_last_error.c_str(); }

#ifdef CHEB_CHECK
const char *cheb_version(void) { return "0.1.0+check"; }
#else
const char *cheb_version(void) { return "0.1.0"; }
#endif

cheb_status cheb_create(cheb_ctx **ctx, int device)
{
    NvtxRange nvtx_range("cheb_create");
    if (!ctx) return fail(CHEB_EINVAL, "null ctx pointer");
    *ctx = nullptr;
    int count = 0;
    CHEB_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(CHEB_EINVAL, "bad device ordinal");
    CHEB_CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    CHEB_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(CHEB_EUNSUPPORTED, "libcheb needs a Blackwell (sm_10x) GPU");
    cheb_ctx *c = new cheb_ctx();
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    cudaError_t e = cudaMalloc(&c->d_error, sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return fail(CHEB_ENOMEM, "error word allocation failed");
    }
    cudaMemset(c->d_error, 0, sizeof(int));
    *ctx = c;
    return CHEB_OK;
}

cheb_status cheb_destroy(cheb_ctx *ctx)
{
    NvtxRange nvtx_range("cheb_destroy");
    if (!ctx) return CHEB_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->dct) cudaFree(kv.second);
    ctx->ws[0].release();
    ctx->ws[1].release();
    ctx->tmats.release();
    ctx->xbuf.release();
    ctx->game.release();
    ctx->game_aux.release();
    ctx->paths.release();
    ctx->io_in.release();
    ctx->io_out.release();
    if (ctx->pts_host) cudaFreeHost(ctx->pts_host);
    if (ctx->pts_done) cudaEventDestroy(ctx->pts_done);
    if (ctx->d_error) cudaFree(ctx->d_error);
    prof_drain(ctx);
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    if (tl_ctx == ctx) tl_ctx = nullptr;
    delete ctx;
    return CHEB_OK;
}

cheb_status cheb_device_status(cheb_ctx *ctx)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    CHEB_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    CHEB_CUDA_TRY(cudaMemcpy(&v, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        CHEB_CUDA_TRY(cudaMemset(ctx->d_error, 0, sizeof(int)));
#ifdef CHEB_CHECK
        (void)dcheck::report();
#endif
        return fail((cheb_status)v, "a device-side wait ran out of time");
    }
#ifdef CHEB_CHECK
    return dcheck::report();
#else
    return CHEB_OK;
#endif
}

#ifdef CHEB_CHECK
cheb_status cheb_check_selftest(cheb_ctx *ctx)
{
    NvtxRange nvtx_range("cheb_check_selftest");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    dcheck::selftest_kernel<<<1, 1>>>(0);
    CHEB_CUDA_TRY(cudaGetLastError());
    return CHEB_OK;
}
#endif

cheb_status cheb_set_wait_limit(cheb_ctx *ctx, int64_t cycles)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    if (cycles < 0) return fail(CHEB_EINVAL, "cheb_set_wait_limit: cycles must be >= 0");
    ctx->wait_limit = (long long)cycles;
    return CHEB_OK;
}

cheb_status cheb_profile(cheb_ctx *ctx, int enable)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    prof_drain(ctx);
    ctx->prof_totals.clear();
    ctx->prof_on = enable != 0;
    return CHEB_OK;
}

int cheb_profile_count(cheb_ctx *ctx)
{
    if (check_ctx(ctx)) return -1;
    prof_drain(ctx);
    return (int)ctx->prof_totals.size();
}

cheb_status cheb_profile_get(cheb_ctx *ctx, int idx, char *name, int name_len, int64_t *launches,
                             double *total_ms)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    prof_drain(ctx);
    if (idx < 0 || idx >= (int)ctx->prof_totals.size()) return fail(CHEB_EINVAL, "bad profile index");
    auto it = ctx->prof_totals.begin();
    std::advance(it, idx);
    if (name && name_len > 0) {
        std::strncpy(name, it->first.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = it->second.first;
    if (total_ms) *total_ms = it->second.second;
    return CHEB_OK;
}

cheb_status cheb_set_tuning(cheb_ctx *ctx, int mode)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    if (mode < 0 || mode > 2 + 4 * 3) return fail(CHEB_EINVAL, "cheb_set_tuning: mode must be 0, 1 or 2 + a configuration");
    ctx->tune_mode = mode;
    return CHEB_OK;
}

cheb_status cheb_tuning_report(cheb_ctx *ctx, char *buf, int64_t buf_len)
{
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    if (!buf || buf_len < 1) return fail(CHEB_EINVAL, "cheb_tuning_report: need a buffer");
    std::string out;
    for (const auto &kv : ctx->game_tune) out += "game_player_tc " + kv.first + ": " + kv.second.second + "\n";
    const size_t nb = std::min<size_t>(out.size(), (size_t)buf_len - 1);
    std::memcpy(buf, out.data(), nb);
    buf[nb] = 0;
    return CHEB_OK;
}

cheb_status cheb_fit(cheb_ctx *ctx, int d, const int32_t *n, const double *values, double *coeffs,
                     void *stream)
{
    NvtxRange nvtx_range("cheb_fit");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    int64_t total = 0;
    if ((st = check_shape(d, n, 64, &total))) return st;
    if (!values || !coeffs) return fail(CHEB_EINVAL, "null values/coeffs");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * (size_t)total;
    if ((st = ctx->ws[0].reserve(bytes))) return st;
    if ((st = ctx->ws[1].reserve(bytes))) return st;
    const double *src = values;
    if (d == 1 && values == coeffs) {
        CHEB_CUDA_TRY(cudaMemcpyAsync(ctx->ws[1].ptr, values, bytes, cudaMemcpyDeviceToDevice, s));
        src = static_cast<const double *>(ctx->ws[1].ptr);
    }
    // Rotating products: step t contracts mode d-1-t (the trailing mode of
    // the current layout) and moves the new index to the front.
    for (int t = 0; t < d; ++t) {
        const int mode = d - 1 - t;
        const double *M = nullptr;
        if ((st = dct_matrix(ctx, n[mode], &M))) return st;
        double *dst = (t == d - 1) ? coeffs : static_cast<double *>(ctx->ws[t & 1].ptr);
        if ((st = modeprod_f64(src, M, dst, total / n[mode], n[mode], n[mode], s))) return st;
        src = dst;
    }
    return CHEB_OK;
}

cheb_status cheb_filter(cheb_ctx *ctx, int d, const int32_t *n, double *coeffs, double alpha, int32_t order,
                        void *stream)
{
    NvtxRange nvtx_range("cheb_filter");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    int64_t total = 0;
    if ((st = check_shape(d, n, 64, &total))) return st;
    if (!coeffs) return fail(CHEB_EINVAL, "null coeffs");
    if (!(alpha >= 0) || order < 1 || order > 32) return fail(CHEB_EINVAL, "cheb_filter: need alpha >= 0, 1 <= order <= 32");
    return spectral_filter(d, n, coeffs, alpha, order, static_cast<cudaStream_t>(stream));
}

cheb_status cheb_smooth(cheb_ctx *ctx, int d, const int32_t *n, double *values, double alpha, int32_t order,
                        void *stream)
{
    NvtxRange nvtx_range("cheb_smooth");
    cheb_status st = cheb_fit(ctx, d, n, values, values, stream);
    if (st) return st;
    if ((st = cheb_filter(ctx, d, n, values, alpha, order, stream))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t total = 1;
    for (int t = 0; t < d; ++t) total *= n[t];
    if ((st = ctx->ws[0].reserve(sizeof(double) * total))) return st;
    if ((st = ctx->ws[1].reserve(sizeof(double) * total))) return st;
    // back to the nodes: T_l(alpha^k) = cos(pi l k / N), one product per mode
    const double *src = values;
    for (int t = 0; t < d; ++t) {
        const int mode = d - 1 - t;
        const double *E = nullptr;
        if ((st = node_eval_matrix(ctx, n[mode], &E))) return st;
        double *dst = (t == d - 1) ? values : static_cast<double *>(ctx->ws[t & 1].ptr);
        if (t == d - 1 && d == 1) {
            CHEB_CUDA_TRY(cudaMemcpyAsync(ctx->ws[1].ptr, values, sizeof(double) * total, cudaMemcpyDeviceToDevice, s));
            src = static_cast<const double *>(ctx->ws[1].ptr);
        }
        if ((st = modeprod_f64(src, E, dst, total / n[mode], n[mode], n[mode], s))) return st;
        src = dst;
    }
    return CHEB_OK;
}

cheb_status cheb_eval_grid(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                           const double *a, const double *b, const int32_t *m,
                           const double *const *x, void *out, cheb_precision prec, void *stream)
{
    NvtxRange nvtx_range("cheb_eval_grid");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    int64_t total = 0;
    if ((st = check_shape(d, n, 64, &total))) return st;
    if ((st = check_domain(d, a, b))) return st;
    if (!coeffs || !out || !m || !x) return fail(CHEB_EINVAL, "null argument");
    if (prec < CHEB_FP64 || prec > CHEB_BF16X6) return fail(CHEB_EINVAL, "bad precision");
    int64_t out_total = 1;
    for (int s = 0; s < d; ++s) {
        if (m[s] < 1 || m[s] > 4096) return fail(CHEB_EINVAL, "m[s] must be in [1, 4096]");
        if (!x[s]) return fail(CHEB_EINVAL, "null point array");
        out_total *= m[s];
    }
    if (out_total > ((int64_t)1 << 34)) return fail(CHEB_EINVAL, "grid too large");
    if (prec != CHEB_FP64) {
        for (int s = 0; s < d; ++s)
            if (m[s] > 256) return fail(CHEB_EUNSUPPORTED, "split forms support m[s] <= 256");
    }
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    const size_t esz = prec == CHEB_FP64 ? sizeof(double) : sizeof(float);
    // the largest intermediate of the chain (modes d-1..s evaluated)
    size_t cap = 0;
    {
        int64_t cur = total;
        for (int t = 0; t < d - 1; ++t) {
            const int mode = d - 1 - t;
            cur = cur / n[mode] * m[mode];
            cap = std::max(cap, (size_t)cur * esz);
        }
    }
    size_t toff = 0;
    for (int s = 0; s < d; ++s) toff += (size_t)m[s] * n[s];
    if ((st = ctx->tmats.reserve(sizeof(double) * toff))) return st;
    if (d > 1) {
        if ((st = ctx->ws[0].reserve(cap))) return st;
        if ((st = ctx->ws[1].reserve(cap))) return st;
    }
    double *T = static_cast<double *>(ctx->tmats.ptr);
    std::vector<double *> Ts(d);
    toff = 0;
    for (int s = 0; s < d; ++s) {
        Ts[s] = T + toff;
        toff += (size_t)m[s] * n[s];
    }
    if (prec == CHEB_FP64) {
        if ((st = cheb_matrices(d, x, m, n, a, b, Ts.data(), sm))) return st;
    }
    const void *src = coeffs;
    int64_t cur = total;
    for (int t = 0; t < d; ++t) {
        const int mode = d - 1 - t;
        void *dst = (t == d - 1) ? out : ctx->ws[t & 1].ptr;
        const int64_t R = cur / n[mode];
        if (prec == CHEB_FP64)
            st = modeprod_f64(static_cast<const double *>(src), Ts[mode], static_cast<double *>(dst), R,
                              n[mode], m[mode], sm);
        else
            st = modeprod_tc(ctx, src, t == 0, nullptr, static_cast<float *>(dst), R, n[mode], m[mode],
                             prec, sm, x[mode], a[mode], b[mode]);
        if (st) return st;
        cur = R * m[mode];
        src = dst;
    }
    return CHEB_OK;
}

cheb_status cheb_eval_grid_host(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                                const double *a, const double *b, const int32_t *m,
                                const double *const *x, void *out, cheb_precision prec, void *stream)
{
    NvtxRange nvtx_range("cheb_eval_grid_host");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    int64_t total = 0;
    if ((st = check_shape(d, n, 64, &total))) return st;
    if ((st = check_domain(d, a, b))) return st;
    if (!coeffs || !out || !m || !x) return fail(CHEB_EINVAL, "null argument");
    if (prec < CHEB_FP64 || prec > CHEB_BF16X6) return fail(CHEB_EINVAL, "bad precision");
    int64_t out_total = 1, npts = 0;
    for (int s = 0; s < d; ++s) {
        if (m[s] < 1 || m[s] > 4096) return fail(CHEB_EINVAL, "m[s] must be in [1, 4096]");
        if (!x[s]) return fail(CHEB_EINVAL, "null point array");
        out_total *= m[s];
        npts += m[s];
    }
    if (out_total > ((int64_t)1 << 34)) return fail(CHEB_EINVAL, "grid too large");
    const size_t cbytes = sizeof(double) * (size_t)total;
    const size_t xoff = (cbytes + 255) / 256 * 256;
    const size_t obytes = (prec == CHEB_FP64 ? sizeof(double) : sizeof(float)) * (size_t)out_total;
    if ((st = ctx->io_in.reserve(xoff + sizeof(double) * (size_t)npts))) return st;
    if ((st = ctx->io_out.reserve(obytes))) return st;
    const size_t xbytes = sizeof(double) * (size_t)npts;
    // the staging buffer is free once the previous call's copy out of it has
    // run (a call that failed after enqueuing it did not synchronise)
    if (!ctx->pts_done) CHEB_CUDA_TRY(cudaEventCreateWithFlags(&ctx->pts_done, cudaEventDisableTiming));
    CHEB_CUDA_TRY(cudaEventSynchronize(ctx->pts_done));
    if (ctx->pts_host_bytes < xbytes) {
        if (ctx->pts_host) cudaFreeHost(ctx->pts_host);
        ctx->pts_host = nullptr;
        ctx->pts_host_bytes = 0;
        if (cudaMallocHost(&ctx->pts_host, xbytes) != cudaSuccess) {
            ctx->pts_host = nullptr;
            cudaGetLastError();
            return fail(CHEB_ENOMEM, "cheb_eval_grid_host: page-locked staging of the points");
        }
        ctx->pts_host_bytes = xbytes;
    }
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    uint8_t *din = static_cast<uint8_t *>(ctx->io_in.ptr);
    std::vector<const double *> xd(d);
    size_t off = 0;
    for (int s = 0; s < d; ++s) {
        std::memcpy(static_cast<uint8_t *>(ctx->pts_host) + off, x[s], sizeof(double) * (size_t)m[s]);
        xd[s] = reinterpret_cast<const double *>(din + xoff + off);
        off += sizeof(double) * (size_t)m[s];
    }
    CHEB_CUDA_TRY(cudaMemcpyAsync(din + xoff, ctx->pts_host, xbytes, cudaMemcpyHostToDevice, sm));
    CHEB_CUDA_TRY(cudaEventRecord(ctx->pts_done, sm));
    CHEB_CUDA_TRY(cudaMemcpyAsync(din, coeffs, cbytes, cudaMemcpyHostToDevice, sm));
    // a page-locked, device-mapped `out` is written by the last mode product itself
    // (GPU stores over the host link, overlapped with the computation); any other
    // host memory gets a device result and a copy
    void *direct = nullptr;
    {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer != nullptr)
            direct = pa.devicePointer;
        else
            cudaGetLastError();
    }
    if ((st = cheb_eval_grid(ctx, d, n, reinterpret_cast<const double *>(din), a, b, m, xd.data(),
                             direct ? direct : ctx->io_out.ptr, prec, stream)))
        return st;
    tl_ctx = ctx;
    if (!direct) CHEB_CUDA_TRY(cudaMemcpyAsync(out, ctx->io_out.ptr, obytes, cudaMemcpyDeviceToHost, sm));
    CHEB_CUDA_TRY(cudaStreamSynchronize(sm));
    return CHEB_OK;
}

cheb_status cheb_eval_points(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                             const double *a, const double *b, int64_t P, const double *x,
                             void *out, cheb_precision prec, void *stream)
{
    NvtxRange nvtx_range("cheb_eval_points");
    cheb_status st = check_ctx(ctx);
    if (st) return st;
    int64_t total = 0;
    if ((st = check_shape(d, n, 64, &total))) return st;
    if ((st = check_domain(d, a, b))) return st;
    if (P < 0 || P > 0x7fffffffLL) return fail(CHEB_EINVAL, "P must be in [0, 2^31 - 1]");
    if (P == 0) return CHEB_OK;
    if (!coeffs || !x || !out) return fail(CHEB_EINVAL, "null argument");
    cudaStream_t sm = static_cast<cudaStream_t>(stream);
    if (prec == CHEB_FP64)
        return eval_points_f64(d, n, coeffs, a, b, P, x, static_cast<double *>(out), sm);
    if (prec < CHEB_FP64 || prec > CHEB_BF16X6) return fail(CHEB_EINVAL, "bad precision");
    return eval_points_tc(ctx, d, n, coeffs, a, b, P, x, static_cast<float *>(out), prec, sm);
}

}  // extern "C"
