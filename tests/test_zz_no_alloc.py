"""cheb_eval_grid_noalloc: the allocation-free entry point for callers that cannot
call cudaMalloc (a host framework owning all device memory in its own pool, or
a hot path where cudaMalloc/cudaFree would synchronise the device).

Its result must match the ordinary cheb_eval_grid (which allocates context
workspaces) within the split-form tolerance of the other tests, on two calls
in a row (the scratch array keeps the previous call's contents). This file is
named to be collected last, and passes alone in a fresh process as well.
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
    return L


@pytest.mark.parametrize("prec_name", ["bf16x6", "tf32x3", "bf16x3"])
def test_noalloc_matches_cheb_eval_grid_twice(lib, prec_name):
    import paper_2307_04688_gb300 as cb
    from paper_2307_04688_gb300 import inputs as I
    prec = cb.precision(prec_name)
    ctx = cb.Context(0)
    # the d=4, n=33 coefficient tensor on a 64^4 grid, and a ragged d=3 case
    w = I.tensor_grid_workload()
    cases = [(torch.from_numpy(w["coeffs"]).cuda(), [torch.from_numpy(g).cuda() for g in w["grid"]])]
    rng = np.random.default_rng(5)
    c3 = torch.from_numpy(rng.standard_normal((7, 17, 5))).cuda()
    cases.append((c3, [torch.from_numpy(rng.uniform(-1, 1, k)).cuda() for k in (130 % 129 + 3, 200, 45)]))
    for c, xs in cases:
        ref = cb.cheb_eval_grid(ctx, c, xs, prec=prec_name)
        cn = c.cpu().numpy()
        refn = ref.double().cpu().numpy()
        # tolerance of the split-form tests: d * u * kappa (see test_gpu_fit_eval.split_bound)
        u = {"bf16x3": 3 * 2.0 ** -18, "bf16x6": 2.0 ** -24, "tf32x3": 3 * 2.0 ** -22}[prec_name] + 4 * 2.0 ** -24
        tol = c.dim() * u * np.abs(cn).sum() / np.abs(refn).max()
        for call in range(2):
            out = torch.full(ref.shape, float("nan"), dtype=torch.float32, device="cuda")
            st = _noalloc(lib, c, xs, prec, out)
            assert st == 0, lib.cheb_last_error()
            torch.cuda.synchronize()
            e = float((out.double() - ref.double()).abs().max() / ref.double().abs().max())
            assert e <= tol, (call, e, tol)
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
