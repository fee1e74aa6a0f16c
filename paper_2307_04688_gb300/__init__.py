"""GB300 implementation of the tensorial Chebyshev method (arXiv 2307.04688).

The computation lives in libcheb.so (C ABI, include/cheb.h). This package
only marshals torch CUDA tensors into those calls; the functions keep the
C names: cheb_fit, cheb_eval_grid, cheb_eval_points, game_solve.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (CHEB_BF16X3, CHEB_BF16X6, CHEB_FP64, CHEB_TF32X3, PRECISIONS, ChebError,
                   GameOpts, GameParams, GameResult, check, load)

__all__ = ["Context", "Surrogate", "cheb_filter", "cheb_smooth", "cheb_fit", "cheb_eval_grid", "cheb_eval_grid_host", "cheb_eval_points", "game_solve",
           "CHEB_FP64", "CHEB_TF32X3", "CHEB_BF16X3", "CHEB_BF16X6", "ChebError", "precision"]


def precision(p) -> int:
    if isinstance(p, str):
        return PRECISIONS[p.lower()]
    return int(p)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _i32(v):
    arr = (C.c_int32 * len(v))(*[int(t) for t in v])
    return arr


def _f64(v):
    return (C.c_double * len(v))(*[float(t) for t in v])


class Context:
    """A libcheb context on one CUDA device (owns workspaces and caches)."""

    def __init__(self, device: int = 0):
        L = load()
        self._h = C.c_void_p()
        check(L.cheb_create(C.byref(self._h), int(device)))
        self.device = int(device)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().cheb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self) -> None:
        check(load().cheb_device_status(self._h))

    def check_selftest(self) -> None:
        """Checked build only (CHEB_LIBRARY=check): launch one kernel that fails a
        bounds check without touching memory; device_status() then raises CHEB_EBOUNDS."""
        L = load()
        if not hasattr(L, "cheb_check_selftest"):
            raise RuntimeError("cheb_check_selftest needs the checked build (CHEB_LIBRARY=check)")
        check(L.cheb_check_selftest(self._h))

    def profile(self, enable: bool) -> None:
        """Turn per-kernel CUDA-event timing on or off (clears the totals)."""
        check(load().cheb_profile(self._h, int(bool(enable))))

    def set_tuning(self, mode: int) -> None:
        """Tile-shape tuning of the split game update: 0 tune on first use (default),
        1 default shapes, 2 + k force configuration k (4 * chunk index + CTAs per SM)."""
        check(load().cheb_set_tuning(self._h, int(mode)))

    def set_wait_limit(self, cycles: int = _lib.CHEB_WAIT_LIMIT_DEFAULT) -> None:
        """Bound, in SM cycles, of the device-side waits of the split-form grid and point
        evaluation (default 2^32); a wait that runs out reports CHEB_ETIMEOUT through
        device_status(). 0 makes every such wait give up at once."""
        check(load().cheb_set_wait_limit(self._h, int(cycles)))

    def tuning_report(self) -> str:
        """One line per tuned shape: key, chosen configuration, time of each one tried."""
        buf = C.create_string_buffer(1 << 16)
        check(load().cheb_tuning_report(self._h, buf, len(buf)))
        return buf.value.decode()

    def profile_read(self) -> dict:
        """{kernel name: (launches, total milliseconds)} since profiling was turned on."""
        L = load()
        cnt = L.cheb_profile_count(self._h)
        if cnt < 0:
            check(_lib.CHEB_EINVAL)
        out = {}
        for i in range(cnt):
            buf = C.create_string_buffer(128)
            nl, ms = C.c_int64(), C.c_double()
            check(L.cheb_profile_get(self._h, i, buf, 128, C.byref(nl), C.byref(ms)))
            out[buf.value.decode()] = (int(nl.value), float(ms.value))
        return out


def _need_cuda(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def cheb_fit(ctx: Context, values, coeffs=None, stream=None):
    """Coefficients of the interpolant of nodal values (float64 tensor, any d <= 6)."""
    import torch
    _need_cuda(values, torch.float64, "values")
    if coeffs is None:
        coeffs = torch.empty_like(values)
    _need_cuda(coeffs, torch.float64, "coeffs")
    n = _i32(values.shape)
    check(load().cheb_fit(ctx.handle, values.dim(), n, C.c_void_p(values.data_ptr()),
                          C.c_void_p(coeffs.data_ptr()), _stream_ptr(stream)))
    return coeffs


def cheb_filter(ctx: Context, coeffs, alpha: float = 36.0, order: int = 4, stream=None):
    """Exponential spectral filter of a float64 coefficient tensor, in place."""
    import torch
    _need_cuda(coeffs, torch.float64, "coeffs")
    check(load().cheb_filter(ctx.handle, coeffs.dim(), _i32(coeffs.shape), C.c_void_p(coeffs.data_ptr()),
                             float(alpha), int(order), _stream_ptr(stream)))
    return coeffs


def cheb_smooth(ctx: Context, values, alpha: float = 36.0, order: int = 4, stream=None):
    """Nodal values -> fit -> spectral filter -> values at the same nodes, in place."""
    import torch
    _need_cuda(values, torch.float64, "values")
    check(load().cheb_smooth(ctx.handle, values.dim(), _i32(values.shape), C.c_void_p(values.data_ptr()),
                             float(alpha), int(order), _stream_ptr(stream)))
    return values


def cheb_eval_grid(ctx: Context, coeffs, xs, a=None, b=None, prec="fp64", out=None, stream=None):
    """Values of the interpolant on the tensor grid xs[0] x ... x xs[d-1]."""
    import torch
    _need_cuda(coeffs, torch.float64, "coeffs")
    d = coeffs.dim()
    if len(xs) != d:
        raise ValueError("need one point array per mode")
    for i, x in enumerate(xs):
        _need_cuda(x, torch.float64, f"xs[{i}]")
    a = [-1.0] * d if a is None else list(a)
    b = [1.0] * d if b is None else list(b)
    p = precision(prec)
    shape = tuple(int(x.numel()) for x in xs)
    if out is None:
        out = torch.empty(shape, dtype=torch.float64 if p == CHEB_FP64 else torch.float32,
                          device=coeffs.device)
    _need_cuda(out, torch.float64 if p == CHEB_FP64 else torch.float32, "out")
    ptrs = (C.c_void_p * d)(*[x.data_ptr() for x in xs])
    check(load().cheb_eval_grid(ctx.handle, d, _i32(coeffs.shape), C.c_void_p(coeffs.data_ptr()),
                                _f64(a), _f64(b), _i32(shape), ptrs, C.c_void_p(out.data_ptr()), p,
                                _stream_ptr(stream)))
    return out


def _need_host(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError(f"{name} must be a CPU tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def cheb_eval_grid_host(ctx: Context, coeffs, xs, a=None, b=None, prec="fp64", out=None, stream=None):
    """cheb_eval_grid with host (CPU) tensors in and out: the library copies the coefficients and
    points to the device, evaluates, and copies the grid back before returning. Pinned tensors
    (`pin_memory()`) give the fastest copies; `out` defaults to a new pinned tensor."""
    import torch
    _need_host(coeffs, torch.float64, "coeffs")
    d = coeffs.dim()
    if len(xs) != d:
        raise ValueError("need one point array per mode")
    for i, x in enumerate(xs):
        _need_host(x, torch.float64, f"xs[{i}]")
    a = [-1.0] * d if a is None else list(a)
    b = [1.0] * d if b is None else list(b)
    p = precision(prec)
    shape = tuple(int(x.numel()) for x in xs)
    dt = torch.float64 if p == CHEB_FP64 else torch.float32
    if out is None:
        out = torch.empty(shape, dtype=dt, pin_memory=True)
    _need_host(out, dt, "out")
    ptrs = (C.c_void_p * d)(*[x.data_ptr() for x in xs])
    check(load().cheb_eval_grid_host(ctx.handle, d, _i32(coeffs.shape), C.c_void_p(coeffs.data_ptr()),
                                     _f64(a), _f64(b), _i32(shape), ptrs, C.c_void_p(out.data_ptr()), p,
                                     _stream_ptr(stream)))
    return out


def cheb_eval_points(ctx: Context, coeffs, x, a=None, b=None, prec="fp64", out=None, stream=None):
    """Values of the interpolant at the rows of x (P x d, float64)."""
    import torch
    _need_cuda(coeffs, torch.float64, "coeffs")
    _need_cuda(x, torch.float64, "x")
    d = coeffs.dim()
    if x.dim() != 2 or x.shape[1] != d:
        raise ValueError("x must be P x d")
    a = [-1.0] * d if a is None else list(a)
    b = [1.0] * d if b is None else list(b)
    p = precision(prec)
    P = int(x.shape[0])
    if out is None:
        out = torch.empty(P, dtype=torch.float64 if p == CHEB_FP64 else torch.float32,
                          device=coeffs.device)
    _need_cuda(out, torch.float64 if p == CHEB_FP64 else torch.float32, "out")
    check(load().cheb_eval_points(ctx.handle, d, _i32(coeffs.shape), C.c_void_p(coeffs.data_ptr()),
                                  _f64(a), _f64(b), P, C.c_void_p(x.data_ptr()),
                                  C.c_void_p(out.data_ptr()), p, _stream_ptr(stream)))
    return out


def game_params(p) -> GameParams:
    g = GameParams()
    J = int(p["J"])
    g.J = J
    K = np.asarray(p["K"], dtype=np.float64).reshape(J, J)
    for t in range(J * J):
        g.K[t] = float(K.flat[t])
    g.m = float(p["m"])
    for s in range(J):
        g.A[s] = float(p["A"][s])
        g.beta[s] = float(p["beta"][s])
        g.phi[s] = float(p["phi"][s])
        g.c[s] = float(p["c"][s])
    g.rho = float(p["rho"])
    G = np.asarray(p.get("gamma", np.zeros((J, J))), dtype=np.float64).reshape(J, J)
    for t in range(J * J):
        g.gamma[t] = float(G.flat[t])
    return g


def game_opts(n: int, h: float = 1e-2, P_M: float = 1.0, U_M: float = 1.0, tol: float = 1e-10,
              max_iter: int = 100000, prec="fp64", polish_fp64=True, n_u: int = 0,
              g_interp: bool = False) -> GameOpts:
    """polish_fp64 (split forms, once the split iteration stagnates): True or 1 continue in
    double-float (FP64-level accuracy on the FP32 pipe), 2 on the FP64 pipe, False stop.
    g_interp: the general method (g-interpolants in the controls, Step 2 on n_u control
    nodes), implied by a nonzero coupling gamma in the parameters."""
    o = GameOpts()
    o.h, o.P_M, o.U_M, o.tol = float(h), float(P_M), float(U_M), float(tol)
    o.n, o.n_u, o.max_iter = int(n), int(n_u), int(max_iter)
    o.prec = precision(prec)
    o.polish_fp64 = 2 if polish_fp64 == 2 else int(bool(polish_fp64))
    o.g_interp = int(bool(g_interp))
    return o


def game_solve(ctx: Context, params, opts, V=None, u=None, V0=None, u0=None, stream=None,
               raise_on_error: bool = True, Vn=None):
    """Solve len(params) games; returns (V list, u list, result structs). V: coefficient
    tensors, u: nodal controls; Vn (optional list of J x n^J tensors) receives nodal values."""
    import torch
    if isinstance(params, dict):
        params = [params]
    if isinstance(opts, GameOpts):
        opts = [opts] * len(params)
    B = len(params)
    P = (GameParams * B)(*[game_params(p) for p in params])
    O = (GameOpts * B)(*opts)
    R = (GameResult * B)()
    Vs, us = [], []
    dev = torch.device("cuda", ctx.device)
    for i in range(B):
        J = int(params[i]["J"])
        NP = int(opts[i].n) ** J
        Vi = torch.empty((J, NP), dtype=torch.float64, device=dev) if V is None else V[i]
        ui = torch.empty((J, NP), dtype=torch.float64, device=dev) if u is None else u[i]
        Vs.append(Vi)
        us.append(ui)
        R[i].V = Vi.data_ptr()
        R[i].u = ui.data_ptr()
        R[i].V0 = None if V0 is None or V0[i] is None else V0[i].data_ptr()
        R[i].u0 = None if u0 is None or u0[i] is None else u0[i].data_ptr()
        R[i].Vn = None if Vn is None or Vn[i] is None else Vn[i].data_ptr()
    st = load().game_solve(ctx.handle, B, P, O, R, _stream_ptr(stream))
    if raise_on_error and st not in (_lib.CHEB_OK,):
        check(st)
    return Vs, us, [R[i] for i in range(B)]


def game_paths(ctx: Context, params, opts, u_nodal, p0, T: int, stream=None, with_controls: bool = True):
    """Equilibrium time paths: from each row of p0 (K x J, device FP64), T explicit steps
    along the clamped interpolant of the nodal controls u_nodal (J x n^J, device FP64, as
    game_solve returns them). Returns (p_path [K, T+1, J], u_path [K, T, J] or None)."""
    import torch
    P = game_params(params)
    J = int(params["J"])
    _need_cuda(u_nodal, torch.float64, "u_nodal")
    _need_cuda(p0, torch.float64, "p0")
    K = int(p0.shape[0]) if p0.dim() == 2 else 0
    if p0.dim() != 2 or p0.shape[1] != J:
        raise ValueError("p0 must be K x J")
    dev = p0.device
    pp = torch.empty((K, T + 1, J), dtype=torch.float64, device=dev)
    up = torch.empty((K, T, J), dtype=torch.float64, device=dev) if with_controls else None
    check(load().game_paths(ctx.handle, C.byref(P), C.byref(opts), C.c_void_p(u_nodal.data_ptr()), K,
                            C.c_void_p(p0.data_ptr()), int(T), C.c_void_p(pp.data_ptr()),
                            None if up is None else C.c_void_p(up.data_ptr()), _stream_ptr(stream)))
    return pp, up


class Surrogate:
    """The warm-start network (surrogate_* entry points of include/cheb.h)."""

    def __init__(self, ctx: Context, n_in: int, width: int, depth: int, n_out: int, seed: int = 0):
        self.ctx = ctx
        self._h = C.c_void_p()
        check(load().surrogate_create(ctx.handle, n_in, width, depth, n_out, C.c_uint64(seed), C.byref(self._h)))
        self.n_in, self.n_out = n_in, n_out

    def close(self):
        if self._h:
            load().surrogate_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def param_count(self) -> int:
        n = C.c_int64()
        check(load().surrogate_params(self._h, None, None, C.byref(n)))
        return int(n.value)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.param_count(), dtype=np.float32)
        check(load().surrogate_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), None, None))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.param_count():
            raise ValueError("wrong parameter count")
        check(load().surrogate_params(self._h, None, p.ctypes.data_as(C.POINTER(C.c_float)), None))

    def loss_grad(self, X, T, stream=None):
        """Unnormalised MSE loss and gradient of a batch (X, T float32 CUDA tensors)."""
        import torch
        _need_cuda(X, torch.float32, "X")
        _need_cuda(T, torch.float32, "T")
        g = torch.empty(self.param_count(), dtype=torch.float32, device=X.device)
        loss = C.c_float()
        check(load().surrogate_loss_grad(self.ctx.handle, self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                         int(X.shape[0]), C.byref(loss), C.c_void_p(g.data_ptr()),
                                         _stream_ptr(stream)))
        return float(loss.value), g

    def adam_step(self, grad=None, lr: float = 1e-3, stream=None) -> None:
        """One Adam step on the FP32 master weights with `grad` (float32 CUDA tensor of
        param_count() entries) or, if None, the gradient of the last loss_grad call."""
        import torch
        if grad is not None:
            _need_cuda(grad, torch.float32, "grad")
            if grad.numel() != self.param_count():
                raise ValueError("wrong gradient size")
        check(load().surrogate_adam_step(self.ctx.handle, self._h,
                                         None if grad is None else C.c_void_p(grad.data_ptr()), float(lr),
                                         _stream_ptr(stream)))

    def train(self, X, Y, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, stream=None):
        """X (S x n_in) and Y (S x n_out, any row stride) float64 CUDA tensors; returns the loss per epoch."""
        import torch
        if X.dtype != torch.float64 or Y.dtype != torch.float64 or not X.is_cuda or not Y.is_cuda:
            raise TypeError("X and Y must be float64 CUDA tensors")
        if X.stride(1) != 1 or Y.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        losses = (C.c_float * max(epochs, 1))()
        check(load().surrogate_train(self.ctx.handle, self._h, C.c_void_p(X.data_ptr()), X.stride(0),
                                     C.c_void_p(Y.data_ptr()), Y.stride(0), int(X.shape[0]), int(epochs), int(batch),
                                     float(lr), C.c_uint64(seed), losses, _stream_ptr(stream)))
        return [float(v) for v in losses[:epochs]]

    def predict(self, X, out=None, stream=None):
        import torch
        if X.dtype != torch.float64 or not X.is_cuda or X.stride(1) != 1:
            raise TypeError("X must be a float64 CUDA tensor with contiguous rows")
        P = int(X.shape[0])
        if out is None:
            out = torch.empty((P, self.n_out), dtype=torch.float64, device=X.device)
        check(load().surrogate_predict(self.ctx.handle, self._h, C.c_void_p(X.data_ptr()), X.stride(0), P,
                                       C.c_void_p(out.data_ptr()), out.stride(0), _stream_ptr(stream)))
        return out
