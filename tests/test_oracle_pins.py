"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the Chebyshev polynomials, numpy's independent Chebyshev routines,
brute-force sums on tiny tensors, the aliasing identity at Lobatto nodes,
spectral decay on analytic functions, and (for the game) the closed-form
linear-quadratic recursion plus a brute-force Bellman check of its fixed point.
"""
import math

import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest

import oracle as O
from paper_2307_04688_gb300 import inputs as I


def lobatto(n):
    N = n - 1
    return np.cos(np.pi * np.arange(n) / N)


# ---- Section 3.1: T_n, nodes --------------------------------------------------

def test_nodes_are_cos_pi_k_over_N_and_extrema_of_T_N():
    for n in (2, 3, 9, 17, 33, 64):
        a = O.nodes(n)
        N = n - 1
        assert np.allclose(a, np.cos(np.pi * np.arange(n) / N), atol=0, rtol=0)
        T = np.array([O.cheb_T(n, x)[N] for x in a])
        assert np.allclose(T, (-1.0) ** np.arange(n), atol=1e-12)


def test_T_closed_form_on_and_off_the_interval():
    rng = np.random.default_rng(1)
    for theta in rng.uniform(0, np.pi, 20):
        T = O.cheb_T(65, math.cos(theta))
        assert np.allclose(T, np.cos(np.arange(65) * theta), atol=2e-13)
    for x in (1.01, 1.3, -1.2):
        T = O.cheb_T(20, x)
        k = np.arange(20)
        ref = np.sign(x) ** k * np.cosh(k * np.arccosh(abs(x)))
        assert np.allclose(T, ref, rtol=1e-12)


# ---- Section 3.1: one-dimensional fit -----------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 9, 17, 33, 64])
def test_fit_1d_reproduces_polynomials_and_matches_c1v(n):
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n)
    F = npc.chebval(lobatto(n), c)          # numpy's evaluation at the nodes
    assert np.abs(O.fit_1d(F) - c).max() < 1e-13 * max(1.0, np.abs(c).max()) * n
    assert np.abs(O.c1v(F) - c).max() < 1e-13 * max(1.0, np.abs(c).max()) * n


def test_fit_1d_equals_numpy_interpolation_at_lobatto_nodes():
    rng = np.random.default_rng(7)
    for n in (4, 9, 17):
        F = rng.standard_normal(n)          # arbitrary data, not a polynomial of low degree
        ref = npc.chebfit(lobatto(n), F, n - 1)
        assert np.allclose(O.fit_1d(F), ref, atol=1e-11)
        assert np.allclose(O.c1v(F), O.fit_1d(F), atol=1e-14)


@pytest.mark.parametrize("n", [5, 9, 17])
def test_fit_aliasing_closed_form(n):
    """T_j at the Lobatto nodes equals T_alias(j), alias(j) = j mod 2N folded into [0, N]."""
    N = n - 1
    x = lobatto(n)
    for j in range(N + 1, 4 * N + 1):
        F = np.cos(j * np.arccos(np.clip(x, -1, 1)))
        t = j % (2 * N)
        alias = t if t <= N else 2 * N - t
        e = np.zeros(n)
        e[alias] = 1.0
        assert np.abs(O.fit_1d(F) - e).max() < 1e-13, (j, alias)


def test_spectral_decay_on_analytic_function():
    """|f - I_N f| ~ C rho^-N for f = 1/(2 - x), analytic inside the Bernstein ellipse rho = 2 + sqrt 3."""
    xs = np.linspace(-1, 1, 2001)
    f = lambda x: 1.0 / (2.0 - x)
    Ns, errs = [], []
    for N in range(4, 25, 2):
        n = N + 1
        p = O.fit_1d(f(lobatto(n)))
        err = np.abs(npc.chebval(xs, p) - f(xs)).max()
        Ns.append(N)
        errs.append(err)
    slope = np.polyfit(Ns, np.log(errs), 1)[0]
    assert abs(slope + math.log(2 + math.sqrt(3))) < 0.1 * math.log(2 + math.sqrt(3))
    # two-dimensional product of two such functions, through fit_nd / eval_grid
    n = 17
    a = lobatto(n)
    G = np.outer(f(a), f(0.5 * a))
    c = O.fit_nd(G)
    g = np.linspace(-1, 1, 41)
    D = O.eval_grid(c, [g, g])
    assert np.abs(D - np.outer(f(g), f(0.5 * g))).max() < 5e-8


# ---- Section 3.1: derivative (Proposition 3.1) -------------------------------

def test_derivative_coefficients():
    rng = np.random.default_rng(3)
    for n in (2, 3, 8, 17):
        p = rng.standard_normal(n)
        q = O.deriv_coeffs(p)
        ref = npc.chebder(p) if n > 1 else np.zeros(0)
        assert np.allclose(q[: n - 1], ref, atol=1e-12)
        assert q[n - 1] == 0.0
    # closed form T_k'(cos t) = k sin(k t) / sin(t)
    for k in range(1, 12):
        e = np.zeros(12)
        e[k] = 1.0
        q = O.deriv_coeffs(e)
        for t in (0.3, 1.1, 2.5):
            assert abs(O.series(q, math.cos(t)) - k * math.sin(k * t) / math.sin(t)) < 1e-11


# ---- Sections 3.1-3.3: n-dimensional fit and evaluation -----------------------

@pytest.mark.parametrize("shape", [(3,), (5, 4), (3, 4, 5), (2, 3, 2, 3)])
def test_fit_nd_and_cnv_reproduce_tensor_polynomials(shape):
    rng = np.random.default_rng(len(shape))
    c = rng.standard_normal(shape)
    # nodal values by brute-force direct summation over every multi-index
    G = np.zeros(shape)
    for idx in np.ndindex(*shape):
        x = [lobatto(shape[s])[idx[s]] for s in range(len(shape))]
        tot = 0.0
        for l in np.ndindex(*shape):
            t = c[l]
            for s in range(len(shape)):
                t *= math.cos(l[s] * math.acos(max(-1.0, min(1.0, x[s]))))
            tot += t
        G[idx] = tot
    assert np.abs(O.fit_nd(G) - c).max() < 1e-13
    assert np.abs(O.cnv(G) - c).max() < 1e-13


def test_eval_matches_numpy_and_brute_force():
    rng = np.random.default_rng(11)
    c = rng.standard_normal((4, 5, 3))
    xs = [rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 7), rng.uniform(-1, 1, 5)]
    D = O.eval_grid(c, xs)
    assert np.allclose(D, npc.chebgrid3d(xs[0], xs[1], xs[2], c), atol=1e-13)
    P = rng.uniform(-1, 1, (50, 3))
    v = O.eval_points(c, P)
    assert np.allclose(v, npc.chebval3d(P[:, 0], P[:, 1], P[:, 2], c), atol=1e-13)
    for j in range(5):
        assert abs(O.eval_direct(c, P[j]) - v[j]) < 1e-14
        assert abs(O.eval_nested(c, P[j]) - v[j]) < 1e-13
    # a physical box [a, b] maps affinely to [-1, 1]
    a, b = np.array([0.0, 2.0, -3.0]), np.array([1.0, 5.0, -1.0])
    Pt = a + (b - a) * (P + 1) / 2
    assert np.allclose(O.eval_points(c, Pt, a, b), v, atol=1e-12)


def test_small_fit_workload_full_oracle_path():
    """d=2, n=17 coefficients 0.5^(k1+k2) N(0,1): nodal values, refit, grid and points."""
    w = I.small_fit_workload()
    c = w["coeffs"]
    a = lobatto(17)
    G = npc.chebgrid2d(a, a, c)
    fit = O.fit_nd(G)
    assert np.abs(fit - c).max() / np.abs(c).max() < 1e-13
    g = w["grid"][0]
    D = O.eval_grid(fit, [g, g])
    assert np.abs(D - npc.chebgrid2d(g, g, c)).max() / np.abs(D).max() < 1e-13
    P = w["points"]
    v = O.eval_points(fit, P)
    assert np.abs(v - npc.chebval2d(P[:, 0], P[:, 1], c)).max() / np.abs(v).max() < 1e-13


# ---- Section 2.1 / 3.4: the game ----------------------------------------------

def lq_values(lq, r, pb):
    J = pb.shape[1]
    V = np.empty((J, pb.shape[0]))
    U = np.empty((J, pb.shape[0]))
    for i in range(J):
        Q, b, a = lq["Q"][r, i], lq["b"][r, i], lq["a"][r, i]
        V[i] = 0.5 * np.einsum("nj,jk,nk->n", pb, Q, pb) + pb @ b + a
        U[i] = pb @ lq["F"][r, i] + lq["f"][r, i]
    return V, U


@pytest.mark.parametrize("J", [2, 3, 4])
def test_game_iteration_equals_lq_recursion(J):
    """While the bounds are inactive every iterate is the J x J LQ recursion's quadratic."""
    p = I.draw_game_params(I.SplitMix64(100 + J), J)
    n = 4 if J == 4 else 5
    R = 6
    opts = O.make_opts(n, h=1e-2, P_M=0.25, U_M=1.0, tol=0.0, max_iter=R)
    res = O.game_solve(p, opts)
    assert res["iters"] == R
    lq = O.game_lq(p, 1e-2, R)
    pb, _ = O.game_nodes(opts, J)
    V, U = lq_values(lq, R - 1, pb)
    assert (U > 0).all() and (U < 1).all()        # bounds inactive: the pin applies
    assert np.abs(res["Vnod"] - V).max() <= 1e-12 * np.abs(V).max()
    assert np.abs(res["u"] - U).max() <= 1e-12
    # and the coefficients: refit of a quadratic has nothing beyond degree 2
    Vc = res["Vcoef"].reshape((J,) + (n,) * J)
    for i in range(J):
        hi = np.indices((n,) * J).sum(axis=0) > 2
        assert np.abs(Vc[i][hi]).max() < 1e-14


def test_lq_recursion_first_step_and_fixed_point_bellman():
    """r=1 from V=0: u=A, V = h(A^2/2 - phi p_i^2 / 2); the fixed point satisfies Bellman's equation."""
    p = I.game_params(2)
    h = 1e-2
    lq = O.game_lq(p, h, 1)
    for i in range(2):
        Q = np.zeros((2, 2))
        Q[i, i] = -h * p["phi"][i]
        assert np.allclose(lq["Q"][0, i], Q, atol=1e-15)
        assert np.allclose(lq["b"][0, i], 0, atol=1e-15)
        assert abs(lq["a"][0, i] - h * p["A"][i] ** 2 / 2) < 1e-15
        assert np.allclose(lq["F"][0, i], 0) and abs(lq["f"][0, i] - p["A"][i]) < 1e-15
    R = 6000
    lq = O.game_lq(p, h, R)
    delta = 1 - p["rho"] * h
    rng = np.random.default_rng(5)
    ug = np.linspace(0, 1, 200001)
    for _ in range(5):
        x = rng.uniform(0, 0.5, 2)
        for i in range(2):
            Q, b, a = lq["Q"][-1, i], lq["b"][-1, i], lq["a"][-1, i]
            Vf = lambda q: 0.5 * q @ Q @ q + b @ q + a
            j = 1 - i
            uj = lq["F"][-1, j] @ x + lq["f"][-1, j]
            best = -np.inf
            g0 = I.neighbour_matrix(2) @ x - p["c"] * x
            for ui in (ug,):
                u = np.zeros((ui.size, 2))
                u[:, i] = ui
                u[:, j] = uj
                q = x + h * (g0 + p["beta"] * u)
                vals = h * (ui * (p["A"][i] - ui / 2) - p["phi"][i] / 2 * x[i] ** 2) + \
                    delta * (0.5 * np.einsum("nj,jk,nk->n", q, Q, q) + q @ b + a)
                best = vals.max()
            assert abs(best - Vf(x)) < 1e-9


def test_game_symmetric_players_coincide():
    """Paper Section 4.2: players 1 and 3 of the 3-region chain are symmetric."""
    p = I.game_params(3, A=[0.45, 0.55, 0.45], phi=[0.9, 1.2, 0.9])
    n = 5
    opts = O.make_opts(n, h=1e-2, P_M=1.0, U_M=1.0, tol=0.0, max_iter=40)
    res = O.game_solve(p, opts)
    V = res["Vnod"].reshape(3, n, n, n)
    U = res["u"].reshape(3, n, n, n)
    assert np.abs(V[0] - V[2].transpose(2, 1, 0)).max() < 1e-13
    assert np.abs(U[0] - U[2].transpose(2, 1, 0)).max() < 1e-12


def test_game_contraction_rate_is_delta():
    p = I.single_game_workload()
    opts = O.make_opts(5, h=1e-2, P_M=1.0, U_M=1.0, tol=0.0, max_iter=1200)
    res = O.game_solve(p, opts, history=True)
    h = res["history"]
    ratio = h[-1] / h[-2]
    assert abs(ratio - (1 - p["rho"] * 1e-2)) < 1e-5
    assert (np.diff(h[200:]) < 0).all()


def test_game_dynamics_reading():
    """g_i = (1/m) sum_{j != i} k_ij (p_j - p_i) - c_i p_i + beta_i u_i; uniform p has no diffusion."""
    p = I.game_params(3)
    g = O.game_dynamics(p, [0.3, 0.3, 0.3], [0.1, 0.2, 0.0])
    assert np.allclose(g, -0.5 * 0.3 + np.array([0.1, 0.2, 0.0]))
    g = O.game_dynamics(p, [1.0, 0.0, 0.0], [0, 0, 0])
    assert np.allclose(g, [-1.0 - 0.5, 1.0, 0.0])      # pollution flows from 1 to its neighbour 2


def test_game_node_update_matches_direct_maximisation():
    """Steps 1-3 at one node: the C1v interpolant's maximiser vs a brute-force search of W(u)."""
    p = I.single_game_workload()
    n = 5
    J = 3
    opts = O.make_opts(n, h=1e-2, P_M=1.0, U_M=1.0, tol=0.0, max_iter=30)
    res = O.game_solve(p, opts)
    pb, _ = O.game_nodes(opts, J)
    delta = 1 - p["rho"] * 1e-2
    ug = np.linspace(0, 1, 100001)
    for j in (0, 17, 62, 124):
        for i in range(J):
            uo = res["u"][:, j]
            us, vs, inside, conc = O.game_node_update(p, opts, i, pb[j], uo, res["Vcoef"][i])
            vals = []
            for u in ug[::100]:
                uu = uo.copy()
                uu[i] = u
                q = pb[j] + 1e-2 * O.game_dynamics(p, pb[j], uu)
                xr = 2 * q - 1
                Vq = O.eval_direct(res["Vcoef"][i].reshape(n, n, n), xr)
                vals.append(1e-2 * (u * (p["A"][i] - u / 2) - p["phi"][i] / 2 * pb[j][i] ** 2) + delta * Vq)
            vals = np.array(vals)
            assert vs >= vals.max() - 1e-15
            assert abs(vs - vals.max()) < 2e-9      # grid step 1e-3: h (1e-3)^2 / 8 bound


@pytest.mark.parametrize("J,n,pair,perm", [(2, 5, (0, 1), (1, 0)), (3, 5, (0, 2), (2, 1, 0)),
                                           (4, 4, (2, 3), (0, 1, 3, 2))])
def test_game_symmetric_players(J, n, pair, perm):
    """Section 4's examples with identical player parameters: the two players of
    the 2-player game, players 1 and 3 of the 3-player chain and players 3 and 4
    of the 4-player configuration are symmetric, so V_i(p) = V_k(sigma p) and
    u_i(p) = u_k(sigma p) with sigma the swap of coordinates i and k, iterate by
    iterate (a wrong neighbour entry or a contraction over the wrong mode breaks
    it)."""
    p = I.game_params(J)
    res = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=6))
    shape = (J,) + (n,) * J
    V, u = res["Vnod"].reshape(shape), res["u"].reshape(shape)
    i, k = pair
    assert np.abs(V[i] - np.transpose(V[k], perm)).max() <= 1e-12 * np.abs(V).max()
    assert np.abs(u[i] - np.transpose(u[k], perm)).max() <= 1e-12
    # and the pair is not trivially equal to a non-symmetric player
    others = [q for q in range(J) if q not in pair]
    if others:
        assert np.abs(V[others[0]] - V[i]).max() > 1e-6 * np.abs(V).max()


def test_game_paths_follow_affine_lq_policy():
    """With no control bound active the equilibrium policy of the discrete game is
    affine, u = F p + f (the closed-form LQ recursion). Its nodal values are
    reproduced exactly by the interpolant, so the oracle's time path must equal
    the affine recursion p_{t+1} = p_t + h ((K/m - diag c) p_t + beta (F p_t + f))
    computed here with numpy. Domain P_M = 0.8: the steady state (about 0.5) is
    inside it and the controls stay in (0.09, 0.45) on the whole box, and the
    paths are checked to stay in it (outside, polynomial extrapolation multiplies
    rounding-level coefficients by large T_k). Bound: the interpolant's rounding,
    about J n^J ulp (<= 3e-13) per step, damped by the recursion (eigenvalues of
    K/m - diag c + diag(beta) F at or below -0.8): <= 4e-11; 1e-10 asserted."""
    for J in (2, 3, 4):
        p = I.game_params(J)
        h, P_M, n = 1e-2, 0.8, 5
        lq = O.game_lq(p, h, 6000)
        F, f = lq["F"][-1], lq["f"][-1]
        opts = O.make_opts(n, h=h, P_M=P_M, U_M=1.0)
        pb, _ = O.game_nodes(opts, J)
        U = (pb @ F.T + f).T                       # J x n^J nodal controls
        assert (U > 0).all() and (U < 1).all()
        rng = np.random.default_rng(J)
        p0 = rng.uniform(0, P_M, (3, J))
        T = 600
        pp, up = O.game_paths(p, opts, U, p0, T)
        assert (pp >= 0).all() and (pp <= P_M).all()
        M = p["K"] / p["m"] - np.diag(p["c"]) + np.diag(p["beta"]) @ F
        q = p0.copy()
        for t in range(T):
            u = q @ F.T + f
            assert np.abs(up[:, t] - u).max() < 1e-10
            q = q + h * (q @ M.T + p["beta"] * f)
            assert np.abs(pp[:, t + 1] - q).max() < 1e-10
        # the path approaches the steady state -M^{-1} beta f
        ps = -np.linalg.solve(M, p["beta"] * f)
        assert np.abs(pp[:, -1] - ps).max() < np.abs(p0 - ps).max()


def test_game_paths_of_symmetric_players_coincide():
    """Players 1 and 3 of the 3-player chain are symmetric: from stocks with
    p_1 = p_3 their emission and stock paths coincide (solved policy, bounds
    active on part of the box)."""
    p = I.game_params(3)
    opts = O.make_opts(5, tol=0.0, max_iter=200)
    r = O.game_solve(p, opts)
    p0 = np.array([[0.1, 0.4, 0.1], [0.8, 0.2, 0.8], [0.0, 0.0, 0.0]])
    pp, up = O.game_paths(p, opts, r["u"], p0, 400)
    assert np.abs(pp[:, :, 0] - pp[:, :, 2]).max() < 1e-13
    assert np.abs(up[:, :, 0] - up[:, :, 2]).max() < 1e-13
    assert np.abs(pp[:, :, 0] - pp[:, :, 1]).max() > 1e-3


# ---- the MLP oracle (learned warm start) -------------------------------------------------------

def test_mlp_oracle_gelu_identities():
    """GELU(z) = z Phi(z): GELU(z) - GELU(-z) = z (Phi(z) + Phi(-z) = 1), GELU(0) = 0, GELU'(0) =
    1/2, GELU(z) -> z for large z and -> 0 for very negative z; GELU' against central
    differences of GELU."""
    assert O.gelu(0.0) == 0.0
    assert abs(O.gelu_grad(0.0) - 0.5) < 1e-15
    for z in (-3.0, -1.2, -0.3, 0.25, 0.9, 2.7):
        assert abs(O.gelu(z) - O.gelu(-z) - z) < 1e-15
        h = 1e-5
        num = (O.gelu(z + h) - O.gelu(z - h)) / (2 * h)
        assert abs(num - O.gelu_grad(z)) < 1e-9
    assert abs(O.gelu(12.0) - 12.0) < 1e-12 and abs(O.gelu(-12.0)) < 1e-12


def test_mlp_oracle_single_layer_is_affine_least_squares():
    """One layer (no activation): forward = X W^T + b, and the mean-squared-error gradient is the
    linear least-squares one, dW = 2/(B m) (Y - T)^T X, db = 2/(B m) sum_b (Y - T)."""
    rng = np.random.default_rng(4)
    n_in, n_out, B = 5, 3, 7
    W = rng.standard_normal((n_out, n_in))
    b = rng.standard_normal(n_out)
    p = np.concatenate([W.ravel(), b])
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, n_out))
    Y = X @ W.T + b
    assert np.abs(O.mlp_forward([n_in, n_out], p, X) - Y).max() < 1e-13
    loss, g = O.mlp_loss_grad([n_in, n_out], p, X, T)
    R = Y - T
    assert abs(loss - np.mean(R ** 2)) < 1e-13
    s = 2.0 / (B * n_out)
    assert np.abs(g[:W.size].reshape(n_out, n_in) - s * R.T @ X).max() < 1e-13
    assert np.abs(g[W.size:] - s * R.sum(axis=0)).max() < 1e-13


def test_mlp_oracle_gradient_against_finite_differences():
    """The full back-propagated gradient (GELU hidden layers) against central differences of the
    loss."""
    dims = [3, 6, 4, 2]
    rng = np.random.default_rng(2)
    p = rng.standard_normal(O.mlp_param_count(dims)) * 0.5
    X = rng.standard_normal((5, 3))
    T = rng.standard_normal((5, 2))
    _, g = O.mlp_loss_grad(dims, p, X, T)
    h = 1e-6
    for i in range(0, p.size, 7):
        e = np.zeros_like(p)
        e[i] = h
        num = (O.mlp_loss_grad(dims, p + e, X, T)[0] - O.mlp_loss_grad(dims, p - e, X, T)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-8 * max(1.0, abs(g[i]))


def test_mlp_oracle_first_adam_step_is_a_signed_step():
    """At t = 1 the bias-corrected moments are g and g^2, so Adam moves every weight by
    lr g / (|g| + eps): lr sign(g) up to eps."""
    rng = np.random.default_rng(6)
    w0 = rng.standard_normal(11)
    g = rng.standard_normal(11)
    w, m, v = w0.copy(), np.zeros(11), np.zeros(11)
    lr, eps = 1e-3, 1e-12
    O.adam_step(w, g, m, v, lr, 0.9, 0.999, eps, 1)
    assert np.abs(w - (w0 - lr * g / (np.abs(g) + eps))).max() < 1e-15
    assert np.abs(m - 0.1 * g).max() < 1e-15 and np.abs(v - 0.001 * g * g).max() < 1e-15


# ---- non-separable dynamics: Step 0 g-interpolants (Section 2.1, Section 3.3) --------

def _coupling(J, scale=0.4, seed=7):
    rng = np.random.default_rng(seed)
    G = rng.uniform(-scale, scale, (J, J))
    np.fill_diagonal(G, 0.0)
    return G


@pytest.mark.parametrize("J,n_u", [(2, 2), (3, 3), (3, 6), (4, 2)])
def test_g_interpolants_reproduce_the_dynamics(J, n_u):
    """The dynamics are affine in each control separately (bilinear in pairs of controls), so
    their interpolant on n_u >= 2 Lobatto control nodes per player reproduces them exactly at
    any control, also off the nodes; with the coupling, g_i moves with the other players'
    controls (it is not separable)."""
    p = I.game_params(J, gamma=_coupling(J))
    opts = O.make_opts(5, n_u=n_u, U_M=1.0, g_interp=True)
    rng = np.random.default_rng(J * 10 + n_u)
    for _ in range(4):
        pb = rng.uniform(0, 1, J)
        gc = O.game_g_interp(p, opts, pb)
        for _ in range(6):
            u = rng.uniform(0, 1, J)
            assert np.allclose(O.game_g_eval(p, opts, gc, u), O.game_dynamics(p, pb, u), rtol=0, atol=1e-14)
    pb, u = rng.uniform(0, 1, J), rng.uniform(0, 1, J)
    u2 = u.copy()
    u2[1] += 0.3
    assert abs(O.game_dynamics(p, pb, u2)[0] - O.game_dynamics(p, pb, u)[0]) > 1e-3


@pytest.mark.parametrize("J", [2, 3])
def test_g_interpolant_path_without_coupling_is_the_lq_iteration(J):
    """With gamma = 0 the Steps 1-2 through the Step 0 interpolants give the same iterates as
    the direct evaluation of g (and so the same as the closed-form LQ recursion pinned above)."""
    p = I.game_params(J)
    a = O.game_solve(p, O.make_opts(5, tol=0.0, max_iter=4, P_M=0.25))
    b = O.game_solve(p, O.make_opts(5, tol=0.0, max_iter=4, P_M=0.25, g_interp=True))
    assert np.abs(a["Vcoef"] - b["Vcoef"]).max() <= 1e-13 * np.abs(a["Vcoef"]).max()
    assert np.abs(a["u"] - b["u"]).max() <= 1e-13


@pytest.mark.parametrize("J", [2, 3])
def test_coupled_node_update_matches_direct_maximisation(J):
    """With the coupling every next-state coordinate moves with the player's own control, so
    W(u) = h G_i + delta V_i(pbar + h g(pbar, [u, u_-i])) is a polynomial of degree at most
    J (n - 1) + 2 in u; with that many control nodes the C1v interpolant of Step 2 is exact and
    the node update must equal a brute-force maximisation of W on a fine grid."""
    n = 4
    n_u = J * (n - 1) + 3
    p = I.game_params(J, gamma=_coupling(J, 0.5))
    opts = O.make_opts(n, n_u=n_u, tol=0.0, max_iter=8, g_interp=True)
    res = O.game_solve(p, opts)
    pb, _ = O.game_nodes(opts, J)
    delta = 1 - p["rho"] * 1e-2
    ug = np.linspace(0, 1, 1001)
    for j in (0, 5, n ** J - 1):
        for i in range(J):
            uo = res["u"][:, j]
            us, vs, inside, conc = O.game_node_update(p, opts, i, pb[j], uo, res["Vcoef"][i])
            vals = []
            for u in ug:
                uu = uo.copy()
                uu[i] = u
                q = pb[j] + 1e-2 * O.game_dynamics(p, pb[j], uu)
                Vq = O.eval_direct(res["Vcoef"][i].reshape((n,) * J), 2 * q - 1)
                vals.append(1e-2 * (u * (p["A"][i] - u / 2) - p["phi"][i] / 2 * pb[j][i] ** 2) + delta * Vq)
            vals = np.array(vals)
            assert vs >= vals.max() - 1e-14
            assert abs(vs - vals.max()) < 2e-9      # grid step 1e-3
            assert abs(us - ug[int(np.argmax(vals))]) < 2e-3


def test_coupled_symmetric_players_coincide():
    """Players 1 and 3 of the 3-player chain with identical parameters and a coupling that is
    symmetric under the swap of players 1 and 3 stay symmetric iterate by iterate."""
    G = np.array([[0.0, 0.3, -0.2], [0.1, 0.0, 0.1], [-0.2, 0.3, 0.0]])
    p = I.game_params(3, gamma=G)
    n = 4
    res = O.game_solve(p, O.make_opts(n, n_u=8, tol=0.0, max_iter=5, g_interp=True))
    V, u = res["Vnod"].reshape((3, n, n, n)), res["u"].reshape((3, n, n, n))
    assert np.abs(V[0] - np.transpose(V[2], (2, 1, 0))).max() <= 1e-12 * np.abs(V).max()
    assert np.abs(u[0] - np.transpose(u[2], (2, 1, 0))).max() <= 1e-12
    base = O.game_solve(I.game_params(3), O.make_opts(n, n_u=8, tol=0.0, max_iter=5))
    assert np.abs(base["Vnod"] - res["Vnod"]).max() > 1e-6      # the coupling changes the game
