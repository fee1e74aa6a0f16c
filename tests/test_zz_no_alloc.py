"""cheb_eval_grid_noalloc: the allocation-free entry point for callers that cannot
call cudaMalloc (a host framework owning all device memory in its own pool, or
a hot path where cudaMalloc/cudaFree would synchronise the device).

Its result must match the CPU oracle's FP64 evaluation within the split-form
bound of the other tests, and the ordinary cheb_eval_grid (which allocates
context workspaces) within the same bound, on two calls in a row (the scratch
array keeps the previous call's contents), with cheb_eval_grid_noalloc_status
reporting no timed-out device wait. This file is named to be collected last,
and passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(L, c, xs, prec, out):
    d = c.dim()
    n = (C.c_int32 * d)(*c.shape)
    m = (C.c_int32 * d)(*[x.numel() for x in xs])
    a = (C.c_double * d)(*([-1.0] * d))
    b = (C.c_double * d)(*([1.0] * d))
    ptrs = (C.c_void_p * d)(*[x.data_ptr() for x in xs])
    return L.cheb_eval_grid_noalloc(d, n, C.c_void_p(c.data_ptr()), a, b, m, ptrs,
                                    C.c_void_p(out.data_ptr()), prec,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_04688_gb300 import build as B
    B.build()
    import paper_2307_04688_gb300 as cb
    L = cb.load()
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)
    L.cheb_eval_grid_noalloc.argtypes = [C.c_int, ip, vp, dp, dp, ip, C.POINTER(vp), vp, C.c_int, vp]
    L.cheb_eval_grid_noalloc.restype = C.c_int
    L.cheb_eval_grid_noalloc_status.argtypes = [vp]
    L.cheb_eval_grid_noalloc_status.restype = C.c_int
    L.cheb_eval_grid_noalloc_set_wait_limit.argtypes = [C.c_int64]
    L.cheb_eval_grid_noalloc_set_wait_limit.restype = C.c_int
    import oracle as O
    O.build()
    return L


def _cases():
    """(coefficients, points per mode) on [-1, 1]^d: the d=4 n=33 64^4 workload, a ragged
    d=3 case, d=1, d=5 with odd n and m (odd m[s] n[s] offsets of the later T matrices and
    odd intermediate sizes), and points outside [-1, 1]."""
    from paper_2307_04688_gb300 import inputs as I
    w = I.tensor_grid_workload()
    out = [(w["coeffs"], list(w["grid"]))]
    rng = np.random.default_rng(5)
    out.append((rng.standard_normal((7, 17, 5)), [rng.uniform(-1, 1, k) for k in (4, 200, 45)]))
    out.append((rng.standard_normal(33), [rng.uniform(-1, 1, 129)]))
    out.append((rng.standard_normal((3, 5, 7, 9, 11)) * 0.5, [rng.uniform(-1, 1, k) for k in (5, 3, 7, 13, 9)]))
    out.append((rng.standard_normal((9, 17)), [rng.uniform(-1.3, 1.3, 31), rng.uniform(-1.2, 1.2, 33)]))
    return out


def _bound(prec_name, c, xs, ref):
    """Tolerance of the split-form tests, d * u * kappa, with kappa = max over the grid of
    sum_k |c_k| prod_s |T_{k_s}(x_s)| over max|f| (= sum|c| / max|f| on [-1, 1], where
    |T_k| <= 1; larger for points outside). u as in test_gpu_fit_eval.split_bound."""
    u = {"bf16x3": 3 * 2.0 ** -18, "bf16x6": 2.0 ** -24, "tf32x3": 3 * 2.0 ** -22}[prec_name] + 4 * 2.0 ** -24
    if max(np.abs(x).max() for x in xs) <= 1.0:
        mag = np.abs(c).sum()
    else:
        acc = np.abs(c)
        for s, x in enumerate(xs):
            V = np.abs(np.polynomial.chebyshev.chebvander(x, c.shape[s] - 1))    # |T_k(x_j)|
            acc = np.tensordot(V, acc, axes=([1], [s]))
            acc = np.moveaxis(acc, 0, s)
        mag = acc.max()
    return c.ndim * u * mag / np.abs(ref).max()


@pytest.mark.parametrize("prec_name", ["bf16x6", "tf32x3", "bf16x3"])
def test_noalloc_matches_oracle_and_cheb_eval_grid_twice(lib, prec_name):
    import oracle as O
    import paper_2307_04688_gb300 as cb
    prec = cb.precision(prec_name)
    ctx = cb.Context(0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for cn, xn in _cases():
        c = torch.from_numpy(np.ascontiguousarray(cn)).cuda()
        xs = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xn]
        orc = O.eval_grid(cn, xn)                      # FP64 oracle, nested mode products
        ours = cb.cheb_eval_grid(ctx, c, xs, prec=prec_name).double().cpu().numpy()
        tol = _bound(prec_name, cn, xn, orc)
        for call in range(2):
            out = torch.full(orc.shape, float("nan"), dtype=torch.float32, device="cuda")
            st = _noalloc(lib, c, xs, prec, out)
            assert st == 0, lib.cheb_last_error()
            assert lib.cheb_eval_grid_noalloc_status(stream) == 0, lib.cheb_last_error()
            got = out.double().cpu().numpy()
            scale = np.abs(orc).max()
            e_orc = float(np.abs(got - orc).max() / scale)
            e_sib = float(np.abs(got - ours).max() / scale)
            assert e_orc <= tol, (cn.shape, call, e_orc, tol)
            assert e_sib <= 2 * tol, (cn.shape, call, e_sib, tol)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    import paper_2307_04688_gb300 as cb
    c = torch.zeros((64, 64, 64, 64), dtype=torch.float64, device="cuda")
    xs = [torch.zeros(256, dtype=torch.float64, device="cuda") for _ in range(4)]
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    st = _noalloc(lib, c, xs, cb.precision("bf16x6"), out)
    assert st == 1
    assert b"maximum" in lib.cheb_last_error()
    st = _noalloc(lib, c[:2, :2, :2, :2].contiguous(), xs, cb.precision("fp64"), out)
    assert st == 1


def test_noalloc_reports_a_wait_that_ran_out(lib):
    """With a wait bound of 0 cycles every device-side wait gives up at once: the kernels
    drain their copies and MMAs with the full bound and return, and the status call reports
    CHEB_ETIMEOUT (6). With the default bound restored the next call is correct again. A
    negative bound is rejected."""
    import oracle as O
    import paper_2307_04688_gb300 as cb
    from paper_2307_04688_gb300 import _lib
    prec = cb.precision("bf16x6")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(9)
    cn = rng.standard_normal((17, 17, 9))
    xn = [rng.uniform(-1, 1, k) for k in (64, 40, 33)]
    c = torch.from_numpy(cn).cuda()
    xs = [torch.from_numpy(x).cuda() for x in xn]
    out = torch.zeros((64, 40, 33), dtype=torch.float32, device="cuda")
    assert lib.cheb_eval_grid_noalloc_set_wait_limit(-1) != 0
    try:
        assert lib.cheb_eval_grid_noalloc_set_wait_limit(0) == 0
        assert _noalloc(lib, c, xs, prec, out) == 0, lib.cheb_last_error()
        assert lib.cheb_eval_grid_noalloc_status(stream) == 6
    finally:
        assert lib.cheb_eval_grid_noalloc_set_wait_limit(_lib.CHEB_WAIT_LIMIT_DEFAULT) == 0
    assert _noalloc(lib, c, xs, prec, out) == 0, lib.cheb_last_error()
    assert lib.cheb_eval_grid_noalloc_status(stream) == 0, lib.cheb_last_error()
    orc = O.eval_grid(cn, xn)
    err = float(np.abs(out.double().cpu().numpy() - orc).max() / np.abs(orc).max())
    assert err <= _bound("bf16x6", cn, xn, orc), err
