"""Parity of cheb_fit / cheb_eval_grid / cheb_eval_points (CUDA, through the C ABI)
against the FP64 CPU oracle, on seeded inputs.

Error measure: max |gpu - oracle| / max |oracle| (max-normalised).
Tolerances: FP64 1e-12 relative. Split forms: the bound derived for the form,
   d * u_form * kappa,  kappa = sum|c| / max|f|  (|T_l| <= 1 on [-1, 1]),
with u_form the per-product relative error of the split (see split_bound), and
at most 1e-6 for TF32x3 and BF16x6 on the d=4, n=33 tensor grid.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SPLITS = ["tf32x3", "bf16x3", "bf16x6"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def lobatto(n):
    return np.cos(np.pi * np.arange(n) / (n - 1))


def err(gpu, ref):
    g = gpu.double().cpu().numpy() if isinstance(gpu, torch.Tensor) else gpu
    return float(np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-300))


def split_bound(prec, d, c, ref):
    """d * u * kappa: u = per-product relative error of the split form.

    bf16x3: |x - x0 - x1| <= 2^-18 |x|, dropped x1*y1 <= 2^-18: u = 3 * 2^-18
    bf16x6: residual 2^-27, dropped terms i + j >= 3 about 2^-26: u = 2^-24
    tf32x3: |x - x0 - x1| <= 2^-22 |x|, dropped x1*y1 <= 2^-22: u = 3 * 2^-22
    plus FP32 accumulation and the FP32 intermediates, 4 * 2^-24 per mode.
    """
    u = {"bf16x3": 3 * 2.0 ** -18, "bf16x6": 2.0 ** -24, "tf32x3": 3 * 2.0 ** -22}[prec]
    u += 4 * 2.0 ** -24
    kappa = np.abs(c).sum() / np.abs(ref).max()
    return d * u * kappa


@pytest.fixture(scope="module")
def small():
    w = I.small_fit_workload()
    c = w["coeffs"]
    a = lobatto(17)
    G = O.eval_grid(c, [a, a])                      # nodal values (oracle)
    return w, c, G


def test_fit_small_workload(ctx, small):
    w, c, G = small
    coef = cb.cheb_fit(ctx, dev(G))
    ref = O.fit_nd(G)
    assert err(coef, ref) < 1e-13
    assert err(coef, c) < 1e-13
    # in place
    g2 = dev(G)
    cb.cheb_fit(ctx, g2, g2)
    assert err(g2, ref) < 1e-13


@pytest.mark.parametrize("prec", ["fp64"] + SPLITS)
def test_eval_grid_small_workload(ctx, small, prec):
    w, c, G = small
    coef = dev(O.fit_nd(G))
    g = w["grid"][0]
    ref = O.eval_grid(O.fit_nd(G), [g, g])
    out = cb.cheb_eval_grid(ctx, coef, [dev(g), dev(g)], prec=prec)
    e = err(out, ref)
    if prec == "fp64":
        assert e < 1e-13
    else:
        assert e < split_bound(prec, 2, c, ref), e


@pytest.mark.parametrize("prec", ["fp64"] + SPLITS)
def test_eval_points_small_workload(ctx, small, prec):
    w, c, G = small
    coefn = O.fit_nd(G)
    P = w["points"]
    ref = O.eval_points(coefn, P)
    out = cb.cheb_eval_points(ctx, dev(coefn), dev(P), prec=prec)
    e = err(out, ref)
    if prec == "fp64":
        assert e < 1e-13
    else:
        assert e < split_bound(prec, 2, c, ref), e


@pytest.fixture(scope="module")
def big():
    w = I.tensor_grid_workload()
    c = w["coeffs"]
    O.set_threads(max(1, min(16, __import__("os").cpu_count() or 1)))
    ref = O.eval_grid(c, w["grid"])                 # full 64^4 oracle grid
    return w, c, ref


@pytest.mark.parametrize("prec", ["fp64"] + SPLITS)
def test_tensor_grid_d4_n33(ctx, big, prec):
    w, c, ref = big
    xs = [dev(g) for g in w["grid"]]
    out = cb.cheb_eval_grid(ctx, dev(c), xs, prec=prec)
    torch.cuda.synchronize()
    e = err(out, ref)
    print(f"tensor grid d=4 n=33 64^4 {prec}: max-normalised error {e:.3e}")
    if prec == "fp64":
        assert e < 1e-12
    else:
        bound = split_bound(prec, 4, c, ref)
        assert e < bound, (e, bound)
        if prec in ("tf32x3", "bf16x6"):
            assert e < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
@pytest.mark.parametrize("pinned", [True, False])
def test_eval_grid_host_buffers(ctx, big, prec, pinned):
    """cheb_eval_grid_host (host coefficients, points and result; the library does the copies)
    returns exactly what cheb_eval_grid returns on device copies of the same inputs, for pinned
    and pageable host memory, on the full 64^4 grid."""
    w, c, ref = big
    ch = torch.from_numpy(np.ascontiguousarray(c))
    xh = [torch.from_numpy(np.ascontiguousarray(g)) for g in w["grid"]]
    if pinned:
        ch, xh = ch.pin_memory(), [x.pin_memory() for x in xh]
        out = None
    else:
        out = torch.empty((64,) * 4, dtype=torch.float64 if prec == "fp64" else torch.float32)
    got = cb.cheb_eval_grid_host(ctx, ch, xh, prec=prec, out=out)
    assert got.device.type == "cpu"
    want = cb.cheb_eval_grid(ctx, dev(c), [dev(g) for g in w["grid"]], prec=prec).cpu()
    assert torch.equal(got, want)
    assert err(got, ref) < (1e-12 if prec == "fp64" else 1e-6)


def test_eval_grid_host_small_and_invalid(ctx, small):
    """A small grid (points that fit the staging buffer of the earlier call; fewer modes), and
    argument errors reported before any copy."""
    w, c, G = small
    xs = [np.linspace(-1, 1, 5), np.linspace(-0.5, 1, 3)]
    got = cb.cheb_eval_grid_host(ctx, torch.from_numpy(np.ascontiguousarray(c)),
                                 [torch.from_numpy(x) for x in xs], prec="fp64")
    assert err(got.numpy(), O.eval_grid(c, xs)) < 1e-12
    with pytest.raises(cb.ChebError):
        cb.cheb_eval_grid_host(ctx, torch.from_numpy(np.ascontiguousarray(c)),
                               [torch.from_numpy(x) for x in xs], a=[1.0, 0.0], b=[0.0, 1.0])
    with pytest.raises(TypeError):
        cb.cheb_eval_grid_host(ctx, dev(c), [torch.from_numpy(x) for x in xs])
    ctx.device_status()


def test_fit_d4_n33(ctx, big):
    w, c, _ = big
    a = lobatto(33)
    G = O.eval_grid(c, [a] * 4)
    coef = cb.cheb_fit(ctx, dev(G))
    assert err(coef, O.fit_nd(G)) < 1e-12
    assert err(coef, c) < 1e-12


@pytest.mark.parametrize("shape,m", [((5, 7, 3), (1, 130, 17)), ((2,), (300,)), ((9, 4), (129, 3)),
                                     ((2, 3, 2, 3, 2, 3), (3, 2, 3, 2, 3, 2)), ((64, 2), (5, 64))])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x6"])
def test_ragged_and_degenerate_shapes(ctx, shape, m, prec):
    rng = np.random.default_rng(sum(shape))
    c = rng.standard_normal(shape)
    d = len(shape)
    a = rng.uniform(-2, 0, d)
    b = a + rng.uniform(0.5, 3, d)
    xs = [rng.uniform(a[s] - 0.1, b[s] + 0.1, m[s]) for s in range(d)]     # slightly outside too
    ref = O.eval_grid(c, xs, a, b)
    if prec != "fp64" and max(m) > 256:
        with pytest.raises(cb.ChebError) as ei:
            cb.cheb_eval_grid(ctx, dev(c), [dev(x) for x in xs], a, b, prec=prec)
        assert ei.value.status == 7
        return
    out = cb.cheb_eval_grid(ctx, dev(c), [dev(x) for x in xs], a, b, prec=prec)
    e = err(out, ref)
    tol = 1e-12 if prec == "fp64" else 8 * split_bound(prec, d, c, ref)
    assert e < tol, (e, tol)
    G = O.eval_grid(c, [lobatto(k) for k in shape])
    assert err(cb.cheb_fit(ctx, dev(G)), c) < 1e-12
    P = np.stack([rng.uniform(a[s], b[s], 257) for s in range(d)], axis=1)
    refp = O.eval_points(c, P, a, b)
    outp = cb.cheb_eval_points(ctx, dev(c), dev(P), a, b, prec="fp64")
    assert err(outp, refp) < 1e-12


def test_empty_and_invalid_arguments(ctx):
    c = dev(np.ones((3, 3)))
    out = cb.cheb_eval_points(ctx, c, torch.zeros((0, 2), dtype=torch.float64, device="cuda"))
    assert out.numel() == 0
    L = cb.load()
    import ctypes as C
    n = (C.c_int32 * 2)(3, 3)
    assert L.cheb_fit(ctx.handle, 0, n, C.c_void_p(c.data_ptr()), C.c_void_p(c.data_ptr()), None) == 1
    n_bad = (C.c_int32 * 2)(3, 65)
    assert L.cheb_fit(ctx.handle, 2, n_bad, C.c_void_p(c.data_ptr()), C.c_void_p(c.data_ptr()), None) == 1
    with pytest.raises(cb.ChebError):
        cb.cheb_eval_grid(ctx, c, [dev([0.0]), dev([0.0])], a=[1.0, 0.0], b=[0.0, 1.0])
    ctx.device_status()


@pytest.mark.parametrize("prec", SPLITS)
def test_fp64_inputs_round_like_cuda(ctx, prec):
    """The split kernels round FP64 inputs to FP32 (nearest, ties to even) before
    splitting them. Everything they do with an FP64 coefficient starts from that
    rounding, so evaluating FP64 coefficients must be bit-identical to evaluating
    the same coefficients rounded first by CUDA's own conversion (torch's
    .float() on the device): exact ties of both parities,
    exponents across a wide range (sums stay finite), and the trailing mode
    n = 33 (a tail column)."""
    rng = np.random.default_rng(11)
    shape = (5, 9, 33)
    c = rng.standard_normal(shape) * np.exp2(rng.integers(-40, 41, shape).astype(np.float64))
    flat = c.reshape(-1)
    f32 = flat[:400].astype(np.float32)
    half_ulp = 0.5 * np.spacing(np.abs(f32)).astype(np.float64)
    flat[:400] = f32.astype(np.float64) + np.sign(f32.astype(np.float64)) * half_ulp   # exact ties
    flat[400:420] = np.array([1.0, -1.0, 0.0, -0.0, 1.0e20, 1.0e-30, 2.0 ** -126, 1.5, 7.0, 0.1] * 2)
    cd = dev(c)
    cr = cd.float().double()
    assert not torch.equal(cd, cr)
    xs = [dev(rng.uniform(-1, 1, k)) for k in (3, 40, 70)]
    a = cb.cheb_eval_grid(ctx, cd, xs, prec=prec)
    b = cb.cheb_eval_grid(ctx, cr, xs, prec=prec)
    assert torch.equal(a, b)
    P = dev(rng.uniform(-1, 1, (300, 3)))
    assert torch.equal(cb.cheb_eval_points(ctx, cd, P, prec=prec), cb.cheb_eval_points(ctx, cr, P, prec=prec))


@pytest.mark.parametrize("prec", SPLITS)
def test_k_tail_shapes(ctx, prec):
    """n = 16q + 1 and 16q + 2 (BF16) or 8q + 1 and 8q + 2 (TF32) leave one or two K columns
    beyond the tensor cores' K, added in FP32 in the epilogue: grid evaluation (T rows formed
    in the kernel) and point evaluation (the FP64 T matrix passed as B) on such shapes."""
    rng = np.random.default_rng(23)
    shape = (17, 18, 34)
    c = rng.standard_normal(shape) * 0.8 ** np.add.outer(np.add.outer(np.arange(17), np.arange(18)),
                                                           np.arange(34))
    d = 3
    a, b = np.array([-1.0, 0.0, -2.0]), np.array([1.0, 2.0, 1.0])
    xs = [rng.uniform(a[s], b[s], k) for s, k in enumerate((40, 17, 33))]
    ref = O.eval_grid(c, xs, a, b)
    out = cb.cheb_eval_grid(ctx, dev(c), [dev(x) for x in xs], a, b, prec=prec)
    assert err(out, ref) < 8 * split_bound(prec, d, c, ref)
    # point evaluation puts the trailing mode on the tensor cores (its leading modes'
    # product must stay <= 256): trailing n = 34 (tail 2) and 17 (tail 1)
    for pshape in ((9, 17, 34), (9, 18, 17)):
        cp = rng.standard_normal(pshape)
        P = np.stack([rng.uniform(a[s], b[s], 1000) for s in range(d)], axis=1)
        refp = O.eval_points(cp, P, a, b)
        outp = cb.cheb_eval_points(ctx, dev(cp), dev(P), a, b, prec=prec)
        assert err(outp, refp) < 8 * split_bound(prec, d, cp, refp)


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x3"])
def test_bounded_wait_timeout_reports_and_recovers(ctx, small, prec):
    """Failure detection without a GPU fault: with the wait limit at 0 every bounded wait of
    the split mode products gives up at once, records CHEB_ETIMEOUT in the context's error
    word, drains its copies and MMAs with the default bound and returns; device_status()
    reports it and clears it, and with the default limit back the same call is correct."""
    w, c, _ = small
    g = w["grid"][0]
    ref = O.eval_grid(c, [g, g])
    ctx.device_status()                                   # start from a clean error word
    try:
        ctx.set_wait_limit(0)
        out = cb.cheb_eval_grid(ctx, dev(c), [dev(g), dev(g)], prec=prec)
        torch.cuda.synchronize()
        with pytest.raises(cb.ChebError) as ei:
            ctx.device_status()
        assert ei.value.status == cb._lib.CHEB_ETIMEOUT
    finally:
        ctx.set_wait_limit()
    ctx.device_status()                                   # cleared by the read above
    out = cb.cheb_eval_grid(ctx, dev(c), [dev(g), dev(g)], prec=prec).double().cpu().numpy()
    ctx.device_status()
    assert err(out, ref) <= split_bound(prec, 2, c, ref)


def test_wait_limit_rejects_negative(ctx):
    with pytest.raises(cb.ChebError):
        ctx.set_wait_limit(-1)


def abs_kappa(c, xs, a=None, b=None):
    """max over the grid of sum_k |c_k| prod_s |T_{k_s}(x~_s)| (= sum|c| on [-1, 1]^d)."""
    acc = np.abs(c)
    for s, x in enumerate(xs):
        xr = x if a is None else (2 * x - a[s] - b[s]) / (b[s] - a[s])
        V = np.abs(np.polynomial.chebyshev.chebvander(xr, c.shape[s] - 1))
        acc = np.moveaxis(np.tensordot(V, acc, axes=([1], [s])), 0, s)
    return float(acc.max())


@pytest.mark.parametrize("prec", SPLITS)
@pytest.mark.parametrize("shape,m", [
    ((17, 18, 34, 9), (40, 17, 33, 5)),       # K tails of one and two columns; ragged tiles
    ((33, 33, 33, 33), (130, 64, 100, 3)),    # 130 points on one mode, 3 on another
    ((5, 64, 64, 2), (3, 128, 1, 9)),         # n = 64 and n = 2, one point on a mode
    ((9, 2, 3, 4, 33, 17), (11, 3, 2, 5, 7, 64)),   # d = 6
])
def test_four_and_six_mode_shapes(ctx, shape, m, prec):
    """d = 4 and d = 6 split-form chains on shapes that exercise the K tails of one and two
    columns, ragged row tiles, padded rows and columns of the MMAs, point counts from 1 to
    130, and points outside the domain, against the oracle within d u_form kappa (kappa from
    |T| on the actual points)."""
    rng = np.random.default_rng(sum(shape) + sum(m))
    d = len(shape)
    c = rng.standard_normal(shape)
    a = rng.uniform(-2, 0, d)
    b = a + rng.uniform(0.5, 3, d)
    xs = [rng.uniform(a[s] - 0.05 * (b[s] - a[s]), b[s] + 0.05 * (b[s] - a[s]), m[s]) for s in range(d)]
    ref = O.eval_grid(c, xs, a, b)
    out = cb.cheb_eval_grid(ctx, dev(c), [dev(x) for x in xs], a, b, prec=prec)
    e = err(out, ref)
    u = {"bf16x3": 3 * 2.0 ** -18, "bf16x6": 2.0 ** -24, "tf32x3": 3 * 2.0 ** -22}[prec] + 4 * 2.0 ** -24
    tol = d * u * abs_kappa(c, xs, a, b) / np.abs(ref).max()
    assert e < tol, (e, tol)
