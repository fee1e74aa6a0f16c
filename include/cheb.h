/*
 * cheb.h - C ABI of libcheb, a GB300 (sm_103a) implementation of the
 * tensorial Chebyshev method of de Castro, Gaton & Gomez, "A tensorial-
 * parallel Chebyshev method for a differential game theory problem"
 * (arXiv 2307.04688).
 *
 * Conventions shared by every call
 * ---------------------------------
 * - Tensors are dense and row-major: the LAST mode varies fastest. (The paper
 *   stores them column-major with the first mode fastest, Section 3.1.)
 * - Mode s of a coefficient or nodal tensor has n[s] = N_s + 1 entries. Node
 *   k of that mode is the Chebyshev-Lobatto point alpha^k = cos(pi k / N_s)
 *   of [-1, 1] (Section 3.1), so k = 0 is x = +1 and the nodes descend.
 * - "Device" pointers are CUDA device (or managed) memory on the context's
 *   device, owned by the caller; "host" pointers are ordinary host memory,
 *   read during the call only. The library never frees caller memory.
 * - Every call that takes a `stream` (a cudaStream_t passed as void*, NULL
 *   for the legacy default stream) is stream-ordered: it enqueues work and
 *   returns without waiting, unless stated otherwise.
 * - Argument errors are detected on the host before anything is enqueued
 *   and return CHEB_EINVAL (or CHEB_EUNSUPPORTED for valid shapes the
 *   library does not implement). There is no CPU fallback. The message of
 *   the last failure on the calling thread is returned by cheb_last_error().
 */
#ifndef CHEB_H
#define CHEB_H

#include <stdint.h>

#if defined(__GNUC__)
#define CHEB_API __attribute__((visibility("default")))
#else
#define CHEB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHEB_OK = 0,
    CHEB_EINVAL = 1,        /* bad argument (null pointer, bad size, bad domain) */
    CHEB_ENOMEM = 2,        /* device workspace allocation failed */
    CHEB_ECUDA = 3,         /* a CUDA runtime call failed */
    CHEB_ENOCONV = 4,       /* game: max_iter reached before the tolerance */
    CHEB_ESTALL = 5,        /* game: residual stopped decreasing above the tolerance */
    CHEB_ETIMEOUT = 6,      /* a bounded device-side wait ran out */
    CHEB_EUNSUPPORTED = 7,  /* valid request outside the implemented shapes */
    CHEB_EBOUNDS = 8        /* checked build only: a device bounds check failed */
} cheb_status;

/* Arithmetic of the mode products.
 *  CHEB_FP64    FP64 on the CUDA cores.
 *  CHEB_TF32X3  tensor cores, kind::tf32: each operand split x = hi + lo into
 *               two TF32 numbers, products hi*hi + hi*lo + lo*hi, FP32
 *               accumulation.
 *  CHEB_BF16X3  tensor cores, kind::f16 with BF16 inputs: two-way split, the
 *               same three products, FP32 accumulation.
 *  CHEB_BF16X6  three-way BF16 split x = x0 + x1 + x2, the six products with
 *               i + j <= 2, FP32 accumulation.
 *  CHEB_DF64    double-float: every value a pair of FP32 numbers (about 48
 *               significant bits), error-free products and compensated sums on
 *               the FP32 pipe (GB300's FP64 pipe is ~1.25 TFLOP/s); relative
 *               errors of a few 1e-14. game_solve only (its player update; the
 *               refit and the residual stay FP64); the other calls return
 *               CHEB_EINVAL for it.
 * The split forms return FP32 results. */
typedef enum {
    CHEB_FP64 = 0,
    CHEB_TF32X3 = 1,
    CHEB_BF16X3 = 2,
    CHEB_BF16X6 = 3,
    CHEB_DF64 = 4
} cheb_precision;

typedef struct cheb_ctx cheb_ctx;

/* Create a context on CUDA device `device`. The context owns device
 * workspaces, cached matrices and CUDA graphs; it is not thread-safe (use
 * one context per host thread). Returns CHEB_EINVAL for a null `ctx` or a
 * bad device ordinal, CHEB_ECUDA if the device cannot be used. */
CHEB_API cheb_status cheb_create(cheb_ctx **ctx, int device);

/* Synchronise the device, then free everything the context owns. */
CHEB_API cheb_status cheb_destroy(cheb_ctx *ctx);

/* Message of the last failed call on this host thread ("" if none). The
 * string stays valid until the next call on the same thread. */
CHEB_API const char *cheb_last_error(void);

/* Library version as "major.minor.patch"; the checked build (below) appends
 * "+check". */
CHEB_API const char *cheb_version(void);

/* Wait for all work on the context's device, then report and clear the
 * device error word that bounded device-side waits write when they run out
 * (CHEB_ETIMEOUT). In the checked build it then reads and clears the bounds
 * check words and returns CHEB_EBOUNDS, with the source file and line of the
 * first failed check in cheb_last_error(), if any check failed. Returns
 * CHEB_OK if no kernel reported a failure. */
CHEB_API cheb_status cheb_device_status(cheb_ctx *ctx);

/* The checked build. libcheb_check.so is the same library compiled with
 * -DCHEB_CHECK: its kernels test the indexes and shared-memory offsets they
 * compute against the extents of the buffers they address, record a failed
 * test (its source line) in a device word and skip that access instead of
 * trapping, and cheb_device_status reports it as CHEB_EBOUNDS. It exists to
 * find indexing faults while developing; the default build compiles no check.
 * cheb_check_selftest (checked build only; the default build does not export
 * it) launches one kernel on the context's device that fails one check
 * without touching memory, so that a caller can see the report path work. */
CHEB_API cheb_status cheb_check_selftest(cheb_ctx *ctx);

/* Bound of the device-side waits of the tensor-core grid evaluation
 * (cheb_eval_grid and cheb_eval_points in a split form): a CTA that has waited
 * `cycles` SM clock cycles for a bulk copy or an MMA gives up, records
 * CHEB_ETIMEOUT in the context's device error word (see cheb_device_status),
 * still waits with the default bound for the copies and MMAs it started, frees
 * its tensor memory and returns; the output of that call is then undefined.
 * cycles >= 0; 0 makes every such wait give up at once (for testing the
 * failure path). CHEB_WAIT_LIMIT_DEFAULT (2^32 cycles, about 2 s) is the
 * default. Not a paper concept: failure detection of the device code. */
#define CHEB_WAIT_LIMIT_DEFAULT 4294967296LL
CHEB_API cheb_status cheb_set_wait_limit(cheb_ctx *ctx, int64_t cycles);

/* Kernel timing. With profiling on, the library brackets every kernel it
 * launches with CUDA events on the launch stream (the stream the caller
 * passed) and accumulates, per kernel name, the launch count and the summed
 * device time. cheb_profile(ctx, 1) clears the totals and turns timing on;
 * cheb_profile(ctx, 0) clears and turns it off. cheb_profile_count waits for
 * the recorded events and returns the number of kernel names (-1 on a bad
 * context); cheb_profile_get copies entry `idx` (0-based, sorted by name):
 * its name into `name` (NUL-terminated, at most name_len bytes), its launch
 * count and its total time in milliseconds. Not for use inside stream
 * capture. */
CHEB_API cheb_status cheb_profile(cheb_ctx *ctx, int enable);
CHEB_API int cheb_profile_count(cheb_ctx *ctx);
CHEB_API cheb_status cheb_profile_get(cheb_ctx *ctx, int idx, char *name, int name_len,
                                      int64_t *launches, double *total_ms);

/* Tile-shape tuning of the split-precision game update. The paper has no
 * counterpart beyond its block-size sweep of the parallel evaluation (Section
 * 4, prior art for this): the library picks, per precision form, node count n
 * and batch-size class (1, then factors of 4), the MMA column chunk of the
 * player update (hence its N, shared memory and TMEM) and the CTAs per SM, by
 * timing every configuration on the caller's own first iteration of
 * game_solve before that solve's iterations are captured into a CUDA graph.
 * The timed runs are that iteration's own work and leave every result
 * unchanged; all configurations compute bit-identical iterates.
 * cheb_set_tuning: mode 0 tunes on first use (the default), 1 always uses the
 * default shape, 2 + k forces configuration k (k = 4 * chunk index + CTAs per
 * SM; game_solve returns CHEB_EINVAL if it does not exist for an n). Any
 * other mode is CHEB_EINVAL. Choices made so far are kept across modes.
 * cheb_tuning_report writes one line per tuned shape (its key, the chosen
 * configuration and the time of every configuration tried) into buf,
 * NUL-terminated and cut at buf_len bytes. Neither call launches work. */
CHEB_API cheb_status cheb_set_tuning(cheb_ctx *ctx, int mode);
CHEB_API cheb_status cheb_tuning_report(cheb_ctx *ctx, char *buf, int64_t buf_len);

/*
 * cheb_fit - coefficients of the d-dimensional Chebyshev interpolant.
 *
 * Section 3.1, Definition 3.2 with eq. (forcoef) and Algorithm Cnv: given the
 * values Gamma(k_1..k_d) = F(alpha^{k_1}_1, ..., alpha^{k_d}_d) at the tensor
 * grid of Chebyshev-Lobatto nodes, returns the coefficients p_l of
 * I_N F(x) = sum_l p_l T_{l_1}(x_1)...T_{l_d}(x_d). Each mode is one product
 * with the n_s x n_s matrix M[l,k] = (2/N) s_l s_k cos(pi l k / N),
 * s_0 = s_N = 1/2 and s = 1 otherwise (eq. (forcoef) in matrix form, which is
 * what Algorithm C1v computes with an FFT).
 *
 *  d       number of modes, 1 <= d <= 6
 *  n       host [d]; n[s] = N_s + 1 nodes of mode s, 2 <= n[s] <= 64
 *  values  device, prod(n) doubles, row-major, node k = 0 <-> x = +1
 *  coeffs  device, prod(n) doubles, row-major, coefficient index l_s per mode;
 *          may equal `values` (in place) but must not partially overlap it
 *  stream  CUDA stream
 * Arithmetic: FP64 on the CUDA cores.
 */
CHEB_API cheb_status cheb_fit(cheb_ctx *ctx, int d, const int32_t *n, const double *values,
                     double *coeffs, void *stream);

/*
 * cheb_filter - exponential spectral filter of a coefficient tensor, in place:
 * p_l *= prod_s exp(-alpha (l_s / N_s)^(2 order)). Not in the paper: the
 * standard filter of spectral methods (Vandeven 1991; Gottlieb & Hesthaven
 * 2001), used to smooth a predicted warm start before the iteration (the
 * iteration amplifies node-to-node noise in V^[0] near the clustered boundary
 * nodes). alpha = 36 makes the top mode vanish to double precision.
 *  d, n, coeffs  as in cheb_fit (device, modified in place)
 *  alpha >= 0, 1 <= order <= 32
 */
CHEB_API cheb_status cheb_filter(cheb_ctx *ctx, int d, const int32_t *n, double *coeffs, double alpha,
                                 int32_t order, void *stream);

/* cheb_smooth - nodal values -> fit (cheb_fit) -> cheb_filter -> values at the
 * same nodes, in place on `values` (device, prod(n) doubles). */
CHEB_API cheb_status cheb_smooth(cheb_ctx *ctx, int d, const int32_t *n, double *values, double alpha,
                                 int32_t order, void *stream);

/*
 * cheb_eval_grid - evaluate an interpolant on a tensor grid of points.
 *
 * Section 3.2: D(j_1..j_d) = I_N F(b^1_{j_1}, ..., b^d_{j_d}), computed as d
 * successive mode products of the coefficient tensor with the matrices
 * B_s(j, l) = T_l(b^s_j) (m_s x n_s).
 *
 *  d, n    as in cheb_fit
 *  coeffs  device, prod(n) doubles (output of cheb_fit)
 *  a, b    host [d]; the interpolant lives on prod_s [a_s, b_s], a_s < b_s;
 *          a point t of mode s is mapped to x = (2t - a_s - b_s) / (b_s - a_s)
 *  m       host [d]; points per mode, 1 <= m[s] <= 4096
 *  x       host array of d device pointers; x[s] holds m[s] doubles. Points
 *          outside [a_s, b_s] are allowed (the polynomial is continued by the
 *          three-term recurrence).
 *  out     device, prod(m) values, row-major in (j_1..j_d): doubles for
 *          CHEB_FP64, floats for the split forms
 *  prec    arithmetic of the mode products (see cheb_precision)
 * Intermediates live in a context-owned workspace that grows on demand
 * (CHEB_ENOMEM if that allocation fails).
 */
CHEB_API cheb_status cheb_eval_grid(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                           const double *a, const double *b, const int32_t *m,
                           const double *const *x, void *out, cheb_precision prec,
                           void *stream);

/*
 * cheb_eval_grid_host - cheb_eval_grid with host buffers.
 *
 * The same evaluation (Section 3.2) for callers whose data lives in host
 * memory: the call copies the coefficients and the points to the device,
 * evaluates as cheb_eval_grid does, copies the result back and returns once
 * it is in `out` (it synchronises `stream`, so it cannot be captured into a
 * CUDA graph). The point arrays are gathered into one page-locked context
 * buffer and copied together.
 *
 *  d, n, a, b, m, prec   as in cheb_eval_grid
 *  coeffs  host, prod(n) doubles
 *  x       host array of d host pointers; x[s] holds m[s] doubles
 *  out     host, prod(m) values, row-major in (j_1..j_d): doubles for
 *          CHEB_FP64, floats for the split forms
 * Page-locked (pinned) host memory gives asynchronous copies at the link's
 * rate; pageable memory works but is staged by the CUDA driver. A page-locked
 * `out` that the device can address is written directly by the last mode
 * product (no device copy of the result, no separate copy). The device
 * copies live in context-owned buffers that grow on demand (CHEB_ENOMEM if
 * that allocation fails). Errors of the arguments are reported before any
 * copy; a CUDA error of a copy or of the evaluation returns CHEB_ECUDA.
 */
CHEB_API cheb_status cheb_eval_grid_host(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                                const double *a, const double *b, const int32_t *m,
                                const double *const *x, void *out, cheb_precision prec,
                                void *stream);

/*
 * cheb_eval_points - evaluate an interpolant at P scattered points.
 *
 * Section 3.3 (one polynomial, a different point per evaluation):
 * f(x_j) = sum_l p_l prod_s T_{l_s}(x_{j,s}). The paper gathers a diagonal
 * out of a full pagemtimes product; here each point is contracted directly.
 *
 *  coeffs  device, prod(n) doubles
 *  a, b    host [d] domain as in cheb_eval_grid
 *  P       number of points, 0 <= P <= 2^31 - 1 (P = 0 is a no-op)
 *  x       device, P x d doubles, row-major (point j at x[j*d .. j*d+d-1])
 *  out     device, P values: doubles for CHEB_FP64, floats otherwise
 *  prec    CHEB_FP64 or a split form
 */
CHEB_API cheb_status cheb_eval_points(cheb_ctx *ctx, int d, const int32_t *n, const double *coeffs,
                             const double *a, const double *b, int64_t P, const double *x,
                             void *out, cheb_precision prec, void *stream);

/*
 * cheb_eval_grid_noalloc - cheb_eval_grid for the split forms, without any
 * allocation and without a context.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, for example inside a host framework that has
 * reserved all device memory in its own pool, or on a latency-bound path
 * where cudaMalloc/cudaFree would synchronise the device; a context
 * (cheb_create) allocates as well, so none is taken.
 *
 * Same arithmetic and arguments as cheb_eval_grid with prec in {CHEB_TF32X3,
 * CHEB_BF16X3, CHEB_BF16X6} and `out` a device float array of prod(m); works
 * on the current device. Limits: 2 <= n[s] <= 64, 1 <= m[s] <= 256, the
 * T matrices (8 * sum_s m[s] n[s] bytes) at most 1 MiB, and any two
 * consecutive intermediates of the mode-product chain together at most 64 MiB
 * of FP32; larger requests return CHEB_EINVAL with the size in the message.
 * coeffs must be 16-byte aligned.
 * Scratch: one fixed device array of 65 MiB inside the library (held by every
 * GPU that loads it until the process exits). Its address is looked up the
 * first time the call runs on a device; make that first call before any
 * stream capture. All calls share the array: calls that overlap on the GPU
 * race and must be serialised by the caller. A bounded device wait that runs
 * out (CHEB_ETIMEOUT) is recorded in the array's own error word, which every
 * call clears when it starts: read it with cheb_eval_grid_noalloc_status.
 */
CHEB_API cheb_status cheb_eval_grid_noalloc(int d, const int32_t *n, const double *coeffs,
                                            const double *a, const double *b, const int32_t *m,
                                            const double *const *x, float *out,
                                            cheb_precision prec, void *stream);

/* Device status of the last cheb_eval_grid_noalloc call on the current device:
 * waits for `stream` (the stream of that call), reads the error word of the
 * library's fixed array and returns CHEB_OK, or CHEB_ETIMEOUT if a bounded
 * device wait of that call ran out (its output is then undefined); the checked
 * build then reports failed bounds checks as cheb_device_status does. The word is
 * cleared by the next cheb_eval_grid_noalloc call, not by this one. Allocates
 * nothing; returns CHEB_EINVAL if cheb_eval_grid_noalloc never ran on the
 * current device. */
CHEB_API cheb_status cheb_eval_grid_noalloc_status(void *stream);

/* Bound, in SM cycles, of the device-side waits of cheb_eval_grid_noalloc
 * (process-wide, all devices; default CHEB_WAIT_LIMIT_DEFAULT). A wait that
 * runs out makes its kernel drain the copies and MMAs in flight and return;
 * cheb_eval_grid_noalloc_status then reports CHEB_ETIMEOUT. Takes effect for
 * calls made after it returns. Returns CHEB_EINVAL for a negative bound. */
CHEB_API cheb_status cheb_eval_grid_noalloc_set_wait_limit(int64_t cycles);

/* ------------------------------------------------------------------------
 * The J-player pollution game (Section 2, linear-quadratic specification,
 * time step h, Section 2.1):
 *   g_i(p, u) = (1/m) sum_{j != i} K[i][j] (p_j - p_i) - c_i p_i + beta_i u_i
 *               + u_i sum_{l != i} gamma[i][l] u_l,
 *   G_i(p, u_i) = u_i (A_i - u_i/2) - (phi_i/2) p_i^2,   delta_h = 1 - rho h,
 *   V_i(p) = max_{0 <= u_i <= U_M} h G_i + delta_h V_i(p + h g(p, [u_i, u*_{-i}])).
 * The printed coupling term k_ij (p_i - p_j) is anti-diffusive with k_ij >= 0;
 * the paper's matrices have zero row sums, and the term is taken as
 * K[i][j] (p_j - p_i), i.e. (K p)_i / m. Only the off-diagonal of K is used.
 * The coupling gamma (an emission-interaction term, zero in the paper's
 * examples) makes g non-separable in the controls: then the general method of
 * Section 2.1 runs - Step 0 interpolates g at every state node in all J
 * controls on n_u Lobatto control nodes per player (the g-interpolants),
 * Steps 1-2 evaluate them along each player's control line (per node, by
 * contraction with the other players' Chebyshev rows, Section 3.3) and
 * evaluate V_i at the resulting next states for the n_u control nodes, and
 * Step 3 maximises the C1v interpolant of those values in the control.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t J;          /* players, 1 <= J <= 4 */
    double K[16];       /* J x J row-major neighbour matrix (off-diagonal >= 0) */
    double m;           /* common region measure m_i > 0 */
    double A[4];        /* emission benefit A_i */
    double beta[4];     /* emission-to-pollution factor beta_i */
    double phi[4];      /* damage cost phi_i >= 0 */
    double c[4];        /* natural decay c_i */
    double rho;         /* discount rate, 0 < rho h < 1 */
    double gamma[16];   /* J x J row-major coupling, diagonal ignored; all zero for the
                           paper's linear-quadratic game */
} cheb_game_params;

typedef struct {
    double h;           /* time step h > 0 */
    double P_M;         /* state box [0, P_M]^J (Section 3.4, Step 0) */
    double U_M;         /* control interval [0, U_M] */
    double tol;         /* stop when max_{i,j} |V^[r+1]_i - V^[r]_i| < tol at the nodes */
    int32_t n;          /* state nodes per player N^p + 1, 3 <= n <= 33 */
    int32_t n_u;        /* control nodes N^u + 1; 0 means n. Without coupling it must
                           be 0 or >= n: then the control interpolant of Step 2 is exact
                           and the maximisation runs on the exact one-variable
                           polynomial. With coupling (or g_interp) 2 <= n_u <= 33: the
                           g-interpolants and the interpolant of Step 2 use n_u nodes */
    int64_t max_iter;   /* iteration cap (CHEB_ENOCONV when reached) */
    int32_t prec;       /* cheb_precision of the evaluation products */
    int32_t polish_fp64;/* split forms: once the split iteration stagnates, 1 =
                           continue with FP64-level accuracy in double-float
                           (the CHEB_DF64 update), 2 = continue on the FP64 pipe
                           (the CHEB_FP64 update); 0 = stop there (CHEB_ESTALL) */
    int32_t g_interp;   /* 1: run the general method (g-interpolants, Step 2 on the
                           control nodes) also without coupling; implied by a nonzero
                           gamma. The general method runs in CHEB_FP64 only
                           (CHEB_EUNSUPPORTED for the other forms) and needs
                           n^J J n_u^J doubles of workspace per instance */
} cheb_game_opts;

typedef struct {
    double *V;          /* device, J x n^J: coefficient tensors of V_1..V_J on
                           return (player-major, each tensor row-major) */
    double *u;          /* device, J x n^J: nodal controls u_i(pbar_j) on return */
    const double *V0;   /* device or NULL: initial NODAL values J x n^J (zero if NULL) */
    const double *u0;   /* device or NULL: initial nodal controls J x n^J (zero if NULL;
                           clamped to [0, U_M]) */
    int64_t iters;      /* out: iterations performed */
    int64_t iters_split;/* out: of which in split precision */
    double residual;    /* out: last residual */
    int32_t status;     /* out: cheb_status of this instance */
    double *Vn;         /* device or NULL: receives the nodal values V_i(pbar_j), J x n^J */
    int32_t restarts;   /* out: cold restarts after a diverging warm start (V0/u0 given):
                           a non-finite residual, or one 1000x above its best after 20
                           iterations, resets the instance to V = 0, u = 0 */
} cheb_game_result;

/*
 * game_solve - solve `batch` independent pollution games with the
 * Chebyshev collocation iteration (Section 2.1 Steps 0-4; Section 3.4).
 *
 * Step 0 fits V^[0] from the initial nodal values. Each iteration, for every
 * player i and state node pbar_j (all players at once from iterate r):
 * the next states pbar_j + h g(pbar_j, [u, u^[r]_{-i}(pbar_j)]) are affine in
 * u, so V^[r]_i along them is a one-variable Chebyshev series in u; its
 * maximiser over [0, U_M] (Newton with the derivative of Proposition 3.1,
 * projected, compared with the bounds) gives u^[r+1]_i(pbar_j) and
 * V^[r+1]_i(pbar_j); then V^[r+1]_i is refitted (cheb_fit) and the residual
 * max |V^[r+1] - V^[r]| over the nodes is tested against tol (Step 4).
 *
 *  batch   number of instances, >= 1
 *  params  host [batch]
 *  opts    host [batch]; instances may differ in n
 *  res     host [batch]; V and u must be distinct device buffers of
 *          J * n^J doubles each
 *  stream  CUDA stream
 * Synchronous: returns after every instance finished; per-instance status,
 * iteration count and residual are in res[]. The return value is CHEB_OK if
 * every instance converged, else the first non-OK instance status.
 */
CHEB_API cheb_status game_solve(cheb_ctx *ctx, int32_t batch, const cheb_game_params *params,
                       const cheb_game_opts *opts, cheb_game_result *res, void *stream);

/*
 * game_paths - equilibrium time paths (Section 4: the emission and
 * pollution-stock paths along the equilibrium strategy).
 *
 * The feedback policy of player i is the Chebyshev interpolant (Definition
 * 3.2) of its nodal controls u_i(pbar_j) on [0, P_M]^J - as game_solve returns
 * them in cheb_game_result.u - clamped to [0, U_M]. From each initial stock the
 * path takes T explicit steps of the dynamics of Section 2.1 with the
 * discretisation's time step: p_{t+1} = p_t + h g(p_t, u(p_t)). Stocks that
 * leave [0, P_M]^J are still evaluated (the polynomial extends), but the
 * policy is only an approximation inside the box.
 *
 *  params   host: the game (J <= 4)
 *  opts     host: n, h, P_M, U_M of the solve the controls come from
 *  u_nodal  device, J x n^J FP64 nodal controls (player-major, row-major)
 *  K        trajectories (>= 0); p0 device K x J FP64 initial stocks
 *  T        steps (>= 0)
 *  p_path   device, K x (T + 1) x J FP64: p_path[k][0] = p0[k]
 *  u_path   device, K x T x J FP64 controls applied at each step, or NULL
 *  stream   CUDA stream; asynchronous (no host synchronisation)
 * Errors: CHEB_EINVAL for J outside 1..4, n outside 2..64, negative K or T,
 * non-positive h, P_M or m, negative U_M, or a null array with K > 0;
 * CHEB_EUNSUPPORTED when n^(J-1) does not fit the per-CTA contraction
 * (J = 4 needs n <= 24). FP64 throughout; all arrays are caller-owned.
 */
CHEB_API cheb_status game_paths(cheb_ctx *ctx, const cheb_game_params *params, const cheb_game_opts *opts,
                                const double *u_nodal, int64_t K, const double *p0, int64_t T,
                                double *p_path, double *u_path, void *stream);

/* ------------------------------------------------------------------------
 * Learned warm start (surrogate). The paper starts the iteration from "some
 * given" V^[0] (Section 2.1, Step 0); here a multilayer perceptron
 * n_in -> width (x depth, GELU) -> n_out maps the game parameters to the
 * coefficient tensor of one player's value function. BF16 operands with FP32
 * accumulation on the tensor cores, FP32 master weights, Adam (b1 = 0.9,
 * b2 = 0.999, eps = 1e-8), mean-squared error on normalised targets.
 * ------------------------------------------------------------------------ */
typedef struct cheb_mlp cheb_mlp;

/* Create a network on the context's device. Weights He-uniform from
 * SplitMix64(seed), biases zero. 1 <= n_in, width <= 8192; 0 <= depth <= 16. */
CHEB_API cheb_status surrogate_create(cheb_ctx *ctx, int32_t n_in, int32_t width, int32_t depth,
                                      int32_t n_out, uint64_t seed, cheb_mlp **net);
CHEB_API cheb_status surrogate_destroy(cheb_mlp *net);

/* Copy the flat FP32 parameter vector out (get, host, *count floats) and/or in
 * (set, host; also resets the Adam state). Layout: for each layer W (out x in,
 * row-major) then b (out). *count receives the parameter count. */
CHEB_API cheb_status surrogate_params(cheb_mlp *net, float *get, const float *set, int64_t *count);

/* Loss and gradient of one batch without normalisation: X device B x n_in
 * FP32, T device B x n_out FP32; *loss (host) = mean squared error; grad
 * (device, parameter count floats, optional). Synchronous when loss != NULL. */
CHEB_API cheb_status surrogate_loss_grad(cheb_ctx *ctx, cheb_mlp *net, const float *X, const float *T,
                                         int32_t B, float *loss, float *grad, void *stream);

/* One Adam step (b1 = 0.9, b2 = 0.999, eps = 1e-8, bias-corrected with the
 * network's step count t, which this call increments) on the FP32 master
 * weights: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). grad: device,
 * parameter count floats in the surrogate_params layout, or NULL for the
 * gradient of the last surrogate_loss_grad call. Stream-ordered. */
CHEB_API cheb_status surrogate_adam_step(cheb_ctx *ctx, cheb_mlp *net, const float *grad, float lr, void *stream);

/* Train on S samples: X device FP64 (row i at X + i * x_stride, n_in values),
 * Y device FP64 targets (row stride y_stride, n_out values). Inputs and
 * targets are normalised by their training-set mean and standard deviation
 * (kept in the network). `epochs` passes of shuffled mini-batches of `batch`
 * samples (the shuffle is driven by SplitMix64(seed)); loss_per_epoch (host,
 * optional) receives the mean normalised loss of every epoch. Synchronous. */
CHEB_API cheb_status surrogate_train(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride,
                                     const double *Y, int64_t y_stride, int64_t S, int32_t epochs,
                                     int32_t batch, float lr, uint64_t seed, float *loss_per_epoch,
                                     void *stream);

/* Predict P outputs (device FP64, row stride y_stride) from device FP64 inputs. */
CHEB_API cheb_status surrogate_predict(cheb_ctx *ctx, cheb_mlp *net, const double *X, int64_t x_stride,
                                       int64_t P, double *Y, int64_t y_stride, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CHEB_H */
