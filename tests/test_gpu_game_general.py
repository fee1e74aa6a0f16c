"""The general method (Section 2.1 Steps 0-3 with the g-interpolants in the controls,
Section 3.3) on the GPU, through the C ABI: dynamics with the emission-interaction
coupling gamma, which makes g non-separable in the controls.

- iteration by iteration against the oracle's literal Steps 0-4 (oracle/game_oracle.c
  with g_interp), J = 2, 3, 4, coupled, with and without an active control bound:
  coefficients 1e-12 relative, controls 1e-11 (both FP64; they differ in summation order
  and in the maximiser's search, which converges to the same point);
- without coupling the general method reproduces the separable path's iterates (its
  control interpolant is exact there);
- a coupled 2-player game solved to 1e-10 against the oracle's full solve;
- symmetric players stay symmetric; equilibrium paths of the coupled game match the
  oracle's; argument errors.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def coupling(J, scale=0.4, seed=7):
    rng = np.random.default_rng(seed)
    G = rng.uniform(-scale, scale, (J, J))
    np.fill_diagonal(G, 0.0)
    return G


@pytest.mark.parametrize("J,n,n_u,R,U_M", [(2, 5, 5, 6, 1.0), (3, 5, 6, 3, 1.0), (3, 4, 9, 4, 0.35),
                                           (4, 3, 4, 3, 1.0), (2, 7, 16, 5, 1.0)])
def test_general_iterations_match_oracle(ctx, J, n, n_u, R, U_M):
    p = I.draw_game_params(I.SplitMix64(40 + J * 7 + n), J)
    p["gamma"] = coupling(J, seed=J + n)
    o = cb.game_opts(n, tol=0.0, max_iter=R, prec="fp64", n_u=n_u, U_M=U_M)
    V, u, res = cb.game_solve(ctx, p, o, raise_on_error=False)
    assert res[0].iters == R
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R, n_u=n_u, U_M=U_M, g_interp=True))
    if U_M < 1.0:
        assert ((ref["u"] == 0.0) | (ref["u"] == U_M)).any()      # a bound is active somewhere
    assert rel(V[0].cpu().numpy(), ref["Vcoef"]) < 1e-12
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-11
    assert abs(res[0].residual - ref["residual"]) <= 1e-12 * max(ref["residual"], 1e-300) + 1e-17


@pytest.mark.parametrize("J,n", [(2, 6), (3, 5)])
def test_general_method_without_coupling_is_the_separable_path(ctx, J, n):
    p = I.draw_game_params(I.SplitMix64(3 + J), J)
    R = 5
    V1, u1, _ = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R, prec="fp64"), raise_on_error=False)
    V2, u2, _ = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R, prec="fp64", g_interp=True),
                              raise_on_error=False)
    assert rel(V2[0].cpu().numpy(), V1[0].cpu().numpy()) < 1e-12
    assert np.abs(u2[0].cpu().numpy() - u1[0].cpu().numpy()).max() < 1e-11


def test_coupled_game_full_solve_matches_oracle(ctx):
    J, n, n_u = 2, 7, 14
    p = I.game_params(J, gamma=[[0.0, 0.5], [-0.3, 0.0]])
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=1e-10, max_iter=20000, prec="fp64", n_u=n_u),
                              raise_on_error=False)
    assert res[0].status == 0 and res[0].residual < 1e-10
    ref = O.game_solve(p, O.make_opts(n, tol=1e-10, max_iter=20000, n_u=n_u, g_interp=True))
    assert ref["status"] == 0
    assert abs(res[0].iters - ref["iters"]) <= 1
    # both stop within tol / (1 - delta_h) = 2e-8 of the fixed point
    assert np.abs(V[0].cpu().numpy() - ref["Vcoef"]).max() < 4e-8
    # the coupling changes the equilibrium
    Vlq, _, _ = cb.game_solve(ctx, I.game_params(J), cb.game_opts(n, tol=1e-10, max_iter=20000, prec="fp64"))
    assert np.abs(Vlq[0].cpu().numpy() - V[0].cpu().numpy()).max() > 1e-4


def test_coupled_symmetric_players_on_gpu(ctx):
    G = np.array([[0.0, 0.3, -0.2], [0.1, 0.0, 0.1], [-0.2, 0.3, 0.0]])
    p = I.game_params(3, gamma=G)
    n = 5
    _, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=6, prec="fp64", n_u=8),
                              raise_on_error=False)
    Vn = torch.empty((3, n ** 3), dtype=torch.float64, device="cuda")
    cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=6, prec="fp64", n_u=8), Vn=[Vn], raise_on_error=False)
    V = Vn.cpu().numpy().reshape(3, n, n, n)
    U = u[0].cpu().numpy().reshape(3, n, n, n)
    assert np.abs(V[0] - np.transpose(V[2], (2, 1, 0))).max() <= 1e-12 * np.abs(V).max()
    assert np.abs(U[0] - np.transpose(U[2], (2, 1, 0))).max() <= 1e-12


def test_coupled_game_paths_match_oracle(ctx):
    J, n = 3, 5
    p = I.game_params(J, gamma=coupling(J, 0.5, seed=3))
    o = cb.game_opts(n, tol=1e-9, max_iter=20000, prec="fp64", n_u=9)
    _, u, res = cb.game_solve(ctx, p, o, raise_on_error=False)
    assert res[0].status == 0
    rng = np.random.default_rng(5)
    p0 = rng.uniform(0, 1, (6, J))
    pp, _ = cb.game_paths(ctx, p, o, u[0], torch.from_numpy(p0).cuda(), 200)
    ppo, _ = O.game_paths(p, O.make_opts(n), u[0].cpu().numpy(), p0, 200)
    assert np.abs(pp.cpu().numpy() - ppo).max() < 1e-12


def test_general_method_arguments(ctx):
    p = I.game_params(3, gamma=coupling(3))
    for kw in ({"prec": "bf16x6"}, {"prec": "df64"}):
        with pytest.raises(cb.ChebError) as ei:
            cb.game_solve(ctx, p, cb.game_opts(9, max_iter=2, **kw))
        assert ei.value.status == 7
    with pytest.raises(cb.ChebError) as ei:
        cb.game_solve(ctx, p, cb.game_opts(5, max_iter=2, prec="fp64", n_u=1))
    assert ei.value.status == 1
    bad = dict(p)
    bad["gamma"] = np.full((3, 3), np.nan)
    with pytest.raises(cb.ChebError):
        cb.game_solve(ctx, bad, cb.game_opts(5, max_iter=2, prec="fp64"))
