"""ctypes binding of the plain FP64 CPU oracle (``liboracle.so``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use it to produce expected values. The product library
shares no code with it.

Every function takes and returns numpy float64 arrays in row-major layout
(last mode fastest), with node k of a mode at cos(pi k / N).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = ["cheb_oracle.c", "game_oracle.c", "mlp_oracle.c"]
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, OpenMP)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", _SO] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_SO)
        _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class GameParams(C.Structure):
    _fields_ = [("J", C.c_int), ("K", C.c_double * 16), ("m", C.c_double),
                ("A", C.c_double * 4), ("beta", C.c_double * 4), ("phi", C.c_double * 4),
                ("c", C.c_double * 4), ("rho", C.c_double), ("gamma", C.c_double * 16)]


class GameOpts(C.Structure):
    _fields_ = [("h", C.c_double), ("P_M", C.c_double), ("U_M", C.c_double), ("tol", C.c_double),
                ("n", C.c_int), ("n_u", C.c_int), ("max_iter", C.c_long), ("g_interp", C.c_int)]


def _declare(L):
    L.orc_nodes.argtypes = [C.c_int, _dp]
    L.orc_cheb_T.argtypes = [C.c_int, C.c_double, _dp]
    L.orc_fit_1d.argtypes = [C.c_int, _dp, _dp]
    L.orc_c1v.argtypes = [C.c_int, _dp, _dp]
    L.orc_deriv_coeffs.argtypes = [C.c_int, _dp, _dp]
    L.orc_series.argtypes = [C.c_int, _dp, C.c_double]
    L.orc_series.restype = C.c_double
    L.orc_fit_nd.argtypes = [C.c_int, _ip, _dp, _dp]
    L.orc_cnv.argtypes = [C.c_int, _ip, _dp, _dp]
    L.orc_eval_grid.argtypes = [C.c_int, _ip, _dp, _dp, _dp, _ip, C.POINTER(_dp), _dp]
    L.orc_eval_direct.argtypes = [C.c_int, _ip, _dp, _dp]
    L.orc_eval_direct.restype = C.c_double
    L.orc_eval_points.argtypes = [C.c_int, _ip, _dp, _dp, _dp, C.c_long, _dp, _dp]
    L.orc_eval_nested.argtypes = [C.c_int, _ip, _dp, _dp, _dp]
    L.orc_eval_nested.restype = C.c_double
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_get_threads.restype = C.c_int
    L.orc_game_dynamics.argtypes = [C.POINTER(GameParams), _dp, _dp, _dp]
    L.orc_game_node.argtypes = [C.POINTER(GameOpts), C.c_int, C.c_long, _dp, _dp]
    L.orc_game_g_interp.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), _dp, _dp]
    L.orc_game_g_eval.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), _dp, _dp, _dp]
    L.orc_game_node_update.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), C.c_int, _dp,
                                       _dp, _dp, _dp, _dp, _ip]
    L.orc_game_node_update.restype = C.c_int
    L.orc_game_iterate.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), _dp, _dp, _dp,
                                   _dp, _dp, _dp, C.POINTER(C.c_long), C.POINTER(C.c_long)]
    L.orc_game_iterate.restype = C.c_double
    L.orc_game_solve.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), _dp, _dp, _dp, _dp,
                                 _dp, C.POINTER(C.c_long), _dp, _dp]
    L.orc_game_solve.restype = C.c_int
    L.orc_game_lq.argtypes = [C.POINTER(GameParams), C.c_double, C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_game_paths.argtypes = [C.POINTER(GameParams), C.POINTER(GameOpts), _dp, C.c_long, _dp, C.c_long, _dp,
                                 _dp]
    if hasattr(L, "orc_mlp_forward"):
        _declare_mlp(L)


def _declare_mlp(L):
    L.orc_mlp_forward.argtypes = [C.c_int, _ip, _dp, C.c_int, _dp, _dp, _dp]
    L.orc_mlp_loss_grad.argtypes = [C.c_int, _ip, _dp, C.c_int, _dp, _dp, _dp, _dp]
    L.orc_mlp_loss_grad.restype = C.c_double
    L.orc_gelu.argtypes = [C.c_double]
    L.orc_gelu.restype = C.c_double
    L.orc_gelu_grad.argtypes = [C.c_double]
    L.orc_gelu_grad.restype = C.c_double
    L.orc_adam_step.argtypes = [C.c_long, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_long]


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ivec(v) -> np.ndarray:
    return np.ascontiguousarray(v, dtype=np.int32)


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ---- Section 3.1 -----------------------------------------------------------

def nodes(n: int) -> np.ndarray:
    out = np.empty(n)
    lib().orc_nodes(n, _p(out))
    return out


def cheb_T(n: int, x: float) -> np.ndarray:
    out = np.empty(n)
    lib().orc_cheb_T(n, float(x), _p(out))
    return out


def fit_1d(F) -> np.ndarray:
    F = _f64(F)
    out = np.empty_like(F)
    lib().orc_fit_1d(F.size, _p(F), _p(out))
    return out


def c1v(F) -> np.ndarray:
    F = _f64(F)
    out = np.empty_like(F)
    lib().orc_c1v(F.size, _p(F), _p(out))
    return out


def deriv_coeffs(p) -> np.ndarray:
    p = _f64(p)
    out = np.empty_like(p)
    lib().orc_deriv_coeffs(p.size, _p(p), _p(out))
    return out


def series(p, x: float) -> float:
    p = _f64(p)
    return float(lib().orc_series(p.size, _p(p), float(x)))


def fit_nd(Gamma) -> np.ndarray:
    G = _f64(Gamma)
    n = _ivec(G.shape)
    out = np.empty_like(G)
    lib().orc_fit_nd(G.ndim, n.ctypes.data_as(_ip), _p(G), _p(out))
    return out


def cnv(Gamma) -> np.ndarray:
    G = _f64(Gamma)
    n = _ivec(G.shape)
    out = np.empty_like(G)
    lib().orc_cnv(G.ndim, n.ctypes.data_as(_ip), _p(G), _p(out))
    return out


def eval_grid(coef, xs, a=None, b=None) -> np.ndarray:
    c = _f64(coef)
    d = c.ndim
    a = _f64(np.full(d, -1.0) if a is None else a)
    b = _f64(np.full(d, 1.0) if b is None else b)
    xs = [_f64(x) for x in xs]
    m = _ivec([x.size for x in xs])
    arr = (_dp * d)(*[_p(x) for x in xs])
    out = np.empty(tuple(int(v) for v in m))
    n = _ivec(c.shape)
    lib().orc_eval_grid(d, n.ctypes.data_as(_ip), _p(c), _p(a), _p(b), m.ctypes.data_as(_ip),
                        arr, _p(out))
    return out


def eval_direct(coef, xref) -> float:
    c = _f64(coef)
    x = _f64(xref)
    n = _ivec(c.shape)
    return float(lib().orc_eval_direct(c.ndim, n.ctypes.data_as(_ip), _p(c), _p(x)))


def eval_nested(coef, xref) -> float:
    c = _f64(coef)
    x = _f64(xref)
    n = _ivec(c.shape)
    work = np.empty(c.size)
    return float(lib().orc_eval_nested(c.ndim, n.ctypes.data_as(_ip), _p(c), _p(x), _p(work)))


def eval_points(coef, x, a=None, b=None) -> np.ndarray:
    c = _f64(coef)
    d = c.ndim
    x = _f64(x).reshape(-1, d)
    a = _f64(np.full(d, -1.0) if a is None else a)
    b = _f64(np.full(d, 1.0) if b is None else b)
    out = np.empty(x.shape[0])
    n = _ivec(c.shape)
    lib().orc_eval_points(d, n.ctypes.data_as(_ip), _p(c), _p(a), _p(b), x.shape[0], _p(x), _p(out))
    return out


# ---- Section 2.1 / 3.4: the game ------------------------------------------

def make_params(p) -> GameParams:
    g = GameParams()
    J = int(p["J"])
    g.J = J
    K = np.asarray(p["K"], dtype=np.float64).reshape(J, J)
    for t in range(J * J):
        g.K[t] = K.flat[t]
    g.m = float(p["m"])
    for s in range(J):
        g.A[s] = float(p["A"][s])
        g.beta[s] = float(p["beta"][s])
        g.phi[s] = float(p["phi"][s])
        g.c[s] = float(p["c"][s])
    g.rho = float(p["rho"])
    G = np.asarray(p.get("gamma", np.zeros((J, J))), dtype=np.float64).reshape(J, J)
    for t in range(J * J):
        g.gamma[t] = G.flat[t]
    return g


def make_opts(n: int, h: float = 1e-2, P_M: float = 1.0, U_M: float = 1.0, tol: float = 1e-10,
              n_u: int | None = None, max_iter: int = 100000, g_interp: bool = False) -> GameOpts:
    """g_interp: evaluate g in Steps 1-2 through the Step 0 interpolants in the controls
    (the general method; required when the coupling gamma is nonzero)."""
    o = GameOpts()
    o.h, o.P_M, o.U_M, o.tol = float(h), float(P_M), float(U_M), float(tol)
    o.n = int(n)
    o.n_u = int(n if n_u is None else n_u)
    o.max_iter = int(max_iter)
    o.g_interp = int(bool(g_interp))
    return o


def game_dynamics(p, pvec, uvec) -> np.ndarray:
    P = make_params(p)
    pv, uv = _f64(pvec), _f64(uvec)
    g = np.empty(P.J)
    lib().orc_game_dynamics(C.byref(P), _p(pv), _p(uv), _p(g))
    return g


def game_nodes(opts: GameOpts, J: int):
    """All state nodes (N_P x J) in physical and reference coordinates."""
    NP = opts.n ** J
    pb = np.empty((NP, J))
    xr = np.empty((NP, J))
    for j in range(NP):
        lib().orc_game_node(C.byref(opts), J, j, _p(pb[j]), _p(xr[j]))
    return pb, xr


def game_g_interp(p, opts: GameOpts, pbar) -> np.ndarray:
    """Step 0: the J interpolants of g(pbar, .) in the controls (J x n_u^J coefficients)."""
    P = make_params(p)
    J = P.J
    gc = np.empty(J * opts.n_u ** J)
    lib().orc_game_g_interp(C.byref(P), C.byref(opts), _p(_f64(pbar)), _p(gc))
    return gc.reshape(J, -1)


def game_g_eval(p, opts: GameOpts, gc, u) -> np.ndarray:
    """g at controls u through the Step 0 interpolants gc."""
    P = make_params(p)
    g = np.empty(P.J)
    lib().orc_game_g_eval(C.byref(P), C.byref(opts), _p(_f64(gc)), _p(_f64(u)), _p(g))
    return g


def game_node_update(p, opts: GameOpts, i: int, pbar, u_old, Vcoef_i):
    P = make_params(p)
    pb, uo, vc = _f64(pbar), _f64(u_old), _f64(Vcoef_i)
    us, vs = C.c_double(), C.c_double()
    cc = C.c_int(1)
    inside = lib().orc_game_node_update(C.byref(P), C.byref(opts), int(i), _p(pb), _p(uo), _p(vc),
                                        C.byref(us), C.byref(vs), C.byref(cc))
    return us.value, vs.value, bool(inside), bool(cc.value)


def game_iterate(p, opts: GameOpts, Vcoef, Vnod, u):
    P = make_params(p)
    Vc, Vn, uu = _f64(Vcoef), _f64(Vnod), _f64(u)
    Vc2, Vn2, u2 = np.empty_like(Vc), np.empty_like(Vn), np.empty_like(uu)
    n_in, n_nc = C.c_long(), C.c_long()
    res = lib().orc_game_iterate(C.byref(P), C.byref(opts), _p(Vc), _p(Vn), _p(uu), _p(Vc2),
                                 _p(Vn2), _p(u2), C.byref(n_in), C.byref(n_nc))
    return {"Vcoef": Vc2, "Vnod": Vn2, "u": u2, "residual": float(res),
            "interior": int(n_in.value), "nonconcave": int(n_nc.value)}


def game_solve(p, opts: GameOpts, V0=None, u0=None, history: bool = False):
    P = make_params(p)
    J = P.J
    NP = opts.n ** J
    Vc = np.empty((J, NP))
    Vn = np.empty((J, NP))
    u = np.empty((J, NP))
    iters = C.c_long()
    res = C.c_double()
    hist = np.empty(opts.max_iter) if history else None
    v0 = None if V0 is None else _f64(V0)
    uu0 = None if u0 is None else _f64(u0)
    st = lib().orc_game_solve(C.byref(P), C.byref(opts), None if v0 is None else _p(v0),
                              None if uu0 is None else _p(uu0), _p(Vc), _p(Vn), _p(u),
                              C.byref(iters), C.byref(res), None if hist is None else _p(hist))
    out = {"status": int(st), "iters": int(iters.value), "residual": float(res.value),
           "Vcoef": Vc, "Vnod": Vn, "u": u}
    if history:
        out["history"] = hist[: iters.value].copy()
    return out


def game_lq(p, h: float, R: int):
    P = make_params(p)
    J = P.J
    Q = np.empty((R, J, J, J))
    b = np.empty((R, J, J))
    a = np.empty((R, J))
    F = np.empty((R, J, J))
    f = np.empty((R, J))
    lib().orc_game_lq(C.byref(P), float(h), int(R), _p(Q), _p(b), _p(a), _p(F), _p(f))
    return {"Q": Q, "b": b, "a": a, "F": F, "f": f}


def game_paths(p, opts: GameOpts, u_nodal, p0, T: int):
    """Time paths along the policy interpolated from the nodal controls: returns
    (p_path [K, T+1, J], u_path [K, T, J])."""
    P = make_params(p)
    J = P.J
    un = _f64(u_nodal).reshape(-1)
    q0 = _f64(p0).reshape(-1, J)
    K = q0.shape[0]
    pp = np.empty((K, T + 1, J))
    up = np.empty((K, T, J))
    lib().orc_game_paths(C.byref(P), C.byref(opts), _p(un), int(K), _p(q0), int(T), _p(pp), _p(up))
    return pp, up


# ---- surrogate network (FP64) ----------------------------------------------

def mlp_param_count(dims) -> int:
    return int(sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1)))


def mlp_forward(dims, params, X) -> np.ndarray:
    d = _ivec(dims)
    p, x = _f64(params), _f64(X)
    B = x.shape[0]
    out = np.empty((B, dims[-1]))
    lib().orc_mlp_forward(len(dims) - 1, d.ctypes.data_as(_ip), _p(p), B, _p(x), _p(out), None)
    return out


def mlp_loss_grad(dims, params, X, T):
    d = _ivec(dims)
    p, x, t = _f64(params), _f64(X), _f64(T)
    g = np.empty_like(p)
    loss = lib().orc_mlp_loss_grad(len(dims) - 1, d.ctypes.data_as(_ip), _p(p), x.shape[0], _p(x), _p(t),
                                   _p(g), None)
    return float(loss), g


def gelu(z: float) -> float:
    return float(lib().orc_gelu(float(z)))


def gelu_grad(z: float) -> float:
    return float(lib().orc_gelu_grad(float(z)))


def adam_step(w, g, m, v, lr, b1, b2, eps, t):
    """In place on w, m, v (float64 arrays)."""
    lib().orc_adam_step(w.size, _p(w), _p(_f64(g)), _p(m), _p(v), lr, b1, b2, eps, t)
