"""The checked build (libcheb_check.so, -DCHEB_CHECK) on the GPU.

Its kernels test the indexes and shared-memory offsets they compute against
the extents of what they address and report a failure as CHEB_EBOUNDS from
cheb_device_status instead of trapping. A child process loads it
(CHEB_LIBRARY=check) and runs every entry point on small ragged shapes:
fit, grid evaluation in every form (device and host buffers), the
allocation-free evaluation, point evaluation, FP64 / double-float / split game
solves for J = 2, 3, 4, the general (coupled) method, equilibrium paths and the
warm-start network. Each result is checked against the CPU oracle, and no check
may fire. cheb_check_selftest then fails one check without touching memory,
and the next cheb_device_status must name its file and line.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import ctypes as C
import numpy as np
import torch
import oracle as O
import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import _lib, inputs as I

L = cb.load()
assert L.cheb_version().decode().endswith("+check"), L.cheb_version()
O.build()
ctx = cb.Context(0)
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
rng = np.random.default_rng(11)


def rel(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / np.abs(b).max())


# grid evaluation, every form, ragged shapes d = 1..4 (one point set outside [-1, 1])
TOL = {"fp64": 1e-12, "bf16x3": 2e-3, "tf32x3": 2e-4, "bf16x6": 2e-5}
for shape, ms, lim in [((17,), (130,), 1.0), ((9, 33), (64, 77), 1.0), ((17, 5, 33), (40, 64, 3), 1.2),
                       ((9, 9, 9, 17), (20, 33, 8, 64), 1.0)]:
    c = rng.standard_normal(shape) / np.prod(np.meshgrid(*[1.0 + np.arange(k) for k in shape], indexing="ij"), axis=0)
    xs = [rng.uniform(-lim, lim, k) for k in ms]
    ref = O.eval_grid(c, xs)
    for prec, tol in TOL.items():
        out = cb.cheb_eval_grid(ctx, dev(c), [dev(x) for x in xs], prec=prec)
        assert rel(out.double().cpu().numpy(), ref) < tol, (shape, prec)
    host = cb.cheb_eval_grid_host(ctx, torch.from_numpy(c), [torch.from_numpy(x) for x in xs], prec="bf16x6")
    assert rel(host.double().numpy(), ref) < TOL["bf16x6"], shape
    # allocation-free evaluation of the same grid
    d = c.ndim
    L.cheb_eval_grid_noalloc.argtypes = [C.c_int, C.POINTER(C.c_int32), C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_void_p),
                                         C.c_void_p, C.c_int, C.c_void_p]
    L.cheb_eval_grid_noalloc_status.argtypes = [C.c_void_p]
    cd, xd = dev(c), [dev(x) for x in xs]
    out = torch.empty(ref.shape, dtype=torch.float32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.cheb_eval_grid_noalloc(d, (C.c_int32 * d)(*shape), C.c_void_p(cd.data_ptr()),
                                  (C.c_double * d)(*([-1.0] * d)), (C.c_double * d)(*([1.0] * d)),
                                  (C.c_int32 * d)(*ms), (C.c_void_p * d)(*[x.data_ptr() for x in xd]),
                                  C.c_void_p(out.data_ptr()), cb.precision("bf16x6"), s)
    assert st == 0 and L.cheb_eval_grid_noalloc_status(s) == 0, L.cheb_last_error()
    assert rel(out.double().cpu().numpy(), ref) < TOL["bf16x6"], shape
    # points
    P = rng.uniform(-1, 1, (777, d))
    refp = O.eval_points(c, P)
    for prec, tol in (("fp64", 1e-12), ("bf16x6", 2e-5)):
        if prec != "fp64" and np.prod(shape[:-1]) > 256:
            continue                  # the split point form takes prod(n[0..d-2]) <= 256
        outp = cb.cheb_eval_points(ctx, dev(c), dev(P), prec=prec)
        assert rel(outp.double().cpu().numpy(), refp) < tol, (shape, prec)
    # fit at the Lobatto nodes
    nodes = [np.cos(np.pi * np.arange(k) / (k - 1)) for k in shape]
    G = O.eval_grid(c, nodes)
    assert rel(cb.cheb_fit(ctx, dev(G)).cpu().numpy(), O.fit_nd(G)) < 1e-12, shape

# games: three iterations of each path against the oracle's
for J, n, prec, tol in [(3, 9, "fp64", 1e-12), (3, 9, "df64", 1e-10), (3, 17, "bf16x6", 1e-5),
                        (2, 17, "bf16x6", 1e-5), (4, 9, "bf16x6", 1e-5), (4, 5, "fp64", 1e-12)]:
    p = I.single_game_workload(J=J)
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=3))
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=3, prec=prec, polish_fp64=False),
                              raise_on_error=False)
    assert res[0].iters == 3 and rel(V[0].cpu().numpy(), ref["Vcoef"]) < tol, (J, n, prec)
# the general method (controls coupled in the dynamics)
p = I.game_params(2, gamma=[[0.0, 0.5], [-0.3, 0.0]])
ref = O.game_solve(p, O.make_opts(9, tol=0.0, max_iter=3, n_u=9, g_interp=True))
V, u, res = cb.game_solve(ctx, p, cb.game_opts(9, tol=0.0, max_iter=3, prec="fp64", n_u=9, g_interp=True),
                          raise_on_error=False)
assert rel(V[0].cpu().numpy(), ref["Vcoef"]) < 1e-12
# equilibrium paths along an FP64 policy
p = I.single_game_workload()
V, u, res = cb.game_solve(ctx, p, cb.game_opts(9, tol=0.0, max_iter=5, prec="fp64"), raise_on_error=False)
p0 = np.array([[0.0, 0.5, 1.0], [0.2, 0.2, 0.2]])
pp, up = cb.game_paths(ctx, p, cb.game_opts(9), u[0], dev(p0), 40)
ppo, upo = O.game_paths(p, O.make_opts(9), u[0].cpu().numpy(), p0, 40)
assert np.abs(pp.cpu().numpy() - ppo).max() < 1e-12
# the warm-start network: a few epochs on ragged batches, then a prediction
net = cb.Surrogate(ctx, 8, 256, 3, 1300, seed=1)
X = dev(rng.uniform(-1, 1, (700, 8)))
Y = dev(rng.standard_normal((700, 1300)) * 0.1)
losses = net.train(X, Y, epochs=3, batch=200, lr=1e-3)
assert all(np.isfinite(losses)), losses
pred = net.predict(X[:333])
assert bool(torch.isfinite(pred).all())
net.close()
torch.cuda.synchronize()
ctx.device_status()          # raises ChebError(CHEB_EBOUNDS) if any check fired

# the report path: one failed check, named by file and line, then cleared
ctx.check_selftest()
try:
    ctx.device_status()
    raise AssertionError("the failed check was not reported")
except cb.ChebError as e:
    assert e.status == _lib.CHEB_EBOUNDS and "abi.cu:" in str(e), str(e)
ctx.device_status()
ctx.close()
print("checked build ok")
'''


def test_checked_build_runs_every_entry_point_without_a_failed_check():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_04688_gb300 import build as B
    B.build()
    env = dict(os.environ, CHEB_LIBRARY="check", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked build ok" in r.stdout
