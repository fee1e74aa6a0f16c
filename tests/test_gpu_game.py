"""Parity of game_solve (CUDA, through the C ABI) with the FP64 CPU oracle.

- iteration by iteration on small instances (J = 2, 3, 4; tol = 0, fixed
  number of passes): coefficient tensors and nodal controls, 1e-12 relative;
- full size n = 17, J = 3 (the +-30 % parameter draw, seed 2): the converged
  FP64 solve against the closed-form LQ recursion run for the same number of
  passes (valid while the control bounds stay inactive, which is checked),
  and single node updates at sampled nodes against the oracle's Steps 1-3;
- batches mixing instances and sizes;
- the split forms: solve to the split form's own residual floor, then state
  the error against the FP64 solve.
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


@pytest.mark.parametrize("J,n,R", [(3, 5, 1), (3, 5, 2), (3, 5, 7), (2, 5, 40), (4, 4, 5), (3, 9, 3),
                                   (1, 6, 10)])
def test_iterations_match_oracle(ctx, J, n, R):
    p = I.draw_game_params(I.SplitMix64(10 + J * 7 + n), J)
    o = cb.game_opts(n, tol=0.0, max_iter=R, prec="fp64")
    V, u, res = cb.game_solve(ctx, p, o, raise_on_error=False)
    assert res[0].iters == R
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R))
    assert rel(V[0].cpu().numpy(), ref["Vcoef"]) < 1e-12
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-11
    assert abs(res[0].residual - ref["residual"]) <= 1e-12 * max(ref["residual"], 1e-300) + 1e-17


def test_kinked_domain_with_active_bound_matches_oracle(ctx):
    """High damage, low benefit: u >= 0 binds at high pollution; V is only C^1 there."""
    p = I.game_params(3, A=[0.2, 0.25, 0.2], phi=[3.0, 3.0, 3.0])
    n, R = 7, 25
    o = cb.game_opts(n, tol=0.0, max_iter=R, prec="fp64")
    V, u, res = cb.game_solve(ctx, p, o, raise_on_error=False)
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R))
    assert (ref["u"] == 0.0).any()                      # the bound is active somewhere
    assert rel(V[0].cpu().numpy(), ref["Vcoef"]) < 1e-11
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-10


def lq_nodal(p, h, R, pb):
    lq = O.game_lq(p, h, R)
    J = pb.shape[1]
    V = np.empty((J, pb.shape[0]))
    U = np.empty((J, pb.shape[0]))
    for i in range(J):
        Q, b, a = lq["Q"][R - 1, i], lq["b"][R - 1, i], lq["a"][R - 1, i]
        V[i] = 0.5 * np.einsum("nj,jk,nk->n", pb, Q, pb) + pb @ b + a
        U[i] = pb @ lq["F"][R - 1, i] + lq["f"][R - 1, i]
    return V, U


@pytest.fixture(scope="module")
def full_fp64(ctx):
    p = I.single_game_workload()
    o = cb.game_opts(17, tol=1e-10, max_iter=20000, prec="fp64")
    V, u, res = cb.game_solve(ctx, p, o)
    return p, V[0].cpu().numpy(), u[0].cpu().numpy(), res[0]


def test_full_size_fp64_converges_to_lq_solution(full_fp64):
    p, V, u, r = full_fp64
    assert r.status == 0 and r.residual < 1e-10
    opts = O.make_opts(17)
    pb, xr = O.game_nodes(opts, 3)
    Vlq, Ulq = lq_nodal(p, 1e-2, int(r.iters), pb)
    assert (Ulq > 0).all() and (Ulq < 1).all()          # bounds inactive: the pin applies
    # nodal values of the GPU coefficients, evaluated by the oracle at the nodes
    a = np.cos(np.pi * np.arange(17) / 16)
    Vn = np.stack([O.eval_grid(V[i].reshape(17, 17, 17), [a, a, a]).reshape(-1) for i in range(3)])
    assert rel(Vn, Vlq) < 1e-11
    assert np.abs(u - Ulq).max() < 1e-10


def test_full_size_sampled_node_updates(ctx):
    p = I.single_game_workload()
    n, R = 17, 12
    V1, u1, _ = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R - 1), raise_on_error=False)
    V2, u2, _ = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R), raise_on_error=False)
    C1, U1 = V1[0].cpu().numpy(), u1[0].cpu().numpy()
    C2, U2 = V2[0].cpu().numpy(), u2[0].cpu().numpy()
    opts = O.make_opts(n, tol=0.0, max_iter=R)
    pb, xr = O.game_nodes(opts, 3)
    rng = np.random.default_rng(0)
    for j in rng.choice(n ** 3, 12, replace=False):
        for i in range(3):
            us, vs, inside, conc = O.game_node_update(p, opts, i, pb[j], U1[:, j], C1[i])
            assert abs(us - U2[i, j]) < 1e-10
            v_gpu = O.eval_direct(C2[i].reshape(n, n, n), xr[j])
            assert abs(vs - v_gpu) < 1e-12 * max(1.0, abs(vs))


def test_batch_of_mixed_instances(ctx):
    rng = I.SplitMix64(77)
    ps = [I.draw_game_params(rng, 3) for _ in range(4)]
    ns = [5, 7, 5, 6]
    R = 6
    opts = [cb.game_opts(k, tol=0.0, max_iter=R) for k in ns]
    V, u, res = cb.game_solve(ctx, ps, opts, raise_on_error=False)
    for q in range(4):
        ref = O.game_solve(ps[q], O.make_opts(ns[q], tol=0.0, max_iter=R))
        assert res[q].iters == R
        assert rel(V[q].cpu().numpy(), ref["Vcoef"]) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_batch_instances_finishing_at_different_iterations(ctx, prec):
    """Instances of one size class that stop at different iterations: the refit skips the
    finished ones, so each must keep exactly the coefficients of its own last iteration, as
    when solved alone (FP64: and as the oracle's solve)."""
    rng = I.SplitMix64(91)
    ps = [I.draw_game_params(rng, 3) for _ in range(5)]
    n = 9
    iters = [3, 40, 7, 1, 20]
    opts = [cb.game_opts(n, tol=0.0, max_iter=k, prec=prec, polish_fp64=False) for k in iters]
    V, u, res = cb.game_solve(ctx, ps, opts, raise_on_error=False)
    for q in range(5):
        assert res[q].iters == iters[q]
        Vq, uq, rq = cb.game_solve(ctx, ps[q], opts[q], raise_on_error=False)
        assert torch.equal(V[q], Vq[0]) and torch.equal(u[q], uq[0])
        assert res[q].residual == rq[0].residual
    if prec == "fp64":
        for q in (0, 1):
            ref = O.game_solve(ps[q], O.make_opts(n, tol=0.0, max_iter=iters[q]))
            assert rel(V[q].cpu().numpy(), ref["Vcoef"]) < 1e-12


@pytest.mark.parametrize("n,count", [(33, 8), (17, 24), (9, 81), (17, 1)])
def test_split_refit_is_the_fp64_fit_of_the_nodal_values(ctx, n, count):
    """The coefficients a split-precision solve returns are the fit (eq. (forcoef) along every
    mode, the oracle's FP64 DCT-I) of the nodal values it returns, to 1e-13. Split-precision
    groups refit in double-float on the FP32 pipe: 24 n = 17 or 81 n = 9 instances one launch
    per mode, 8 n = 33 instances and a single instance all modes in one launch."""
    rng = I.SplitMix64(5 + n + count)
    ps = [I.draw_game_params(rng, 3) for _ in range(count)]
    o = cb.game_opts(n, tol=0.0, max_iter=3, prec="bf16x6", polish_fp64=False)
    Vn = [torch.empty((3, n ** 3), dtype=torch.float64, device="cuda") for _ in range(count)]
    V, u, res = cb.game_solve(ctx, ps, [o] * count, Vn=Vn, raise_on_error=False)
    for q in sorted({0, count - 1}):
        assert res[q].iters == 3
        for i in range(3):
            ref = O.fit_nd(Vn[q][i].cpu().numpy().reshape(n, n, n))
            assert rel(V[q][i].cpu().numpy().reshape(n, n, n), ref) < 1e-13


def test_invalid_arguments(ctx):
    p = I.single_game_workload()
    with pytest.raises(cb.ChebError) as e:
        cb.game_solve(ctx, p, cb.game_opts(2))
    assert e.value.status == 1
    with pytest.raises(cb.ChebError) as e:
        cb.game_solve(ctx, p, cb.game_opts(5, n_u=3))
    assert e.value.status == 7
    bad = dict(p)
    bad["rho"] = -1.0
    with pytest.raises(cb.ChebError):
        cb.game_solve(ctx, bad, cb.game_opts(5))


SPLIT_FORMS = ["bf16x6", "tf32x3", "bf16x3"]
# relative error of one split evaluation, as in the grid tests (u_form + FP32 terms)
U_FORM = {"bf16x3": 3 * 2.0 ** -18, "bf16x6": 2.0 ** -24, "tf32x3": 3 * 2.0 ** -22}


@pytest.mark.parametrize("prec", SPLIT_FORMS)
@pytest.mark.parametrize("n", [5, 9])
def test_split_iterations_close_to_oracle(ctx, prec, n):
    """A few passes in split precision: each evaluation carries the form's relative error
    (bound: passes * (u_form + 2^-20) * kappa, kappa = sum |w| / |V| <= 10 for these smooth V)."""
    p = I.single_game_workload()
    R = 6
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R, prec=prec, polish_fp64=False),
                              raise_on_error=False)
    assert res[0].iters == R and res[0].iters_split == R
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R))
    bound = R * (U_FORM[prec] + 2.0 ** -20) * 10
    e = rel(V[0].cpu().numpy(), ref["Vcoef"])
    print(f"split {prec} n={n} after {R} passes: coefficient error {e:.2e} (bound {bound:.1e})")
    assert e < bound
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-5


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x3"])
def test_split_sampled_node_updates_n33(ctx, prec):
    """n = 33 (35,937 nodes): one split pass from a given state against the oracle's Steps 1-3
    at sampled nodes (the oracle computes one node at a time)."""
    p = I.single_game_workload()
    n, R = 33, 4
    o1 = cb.game_opts(n, tol=0.0, max_iter=R - 1, prec=prec, polish_fp64=False)
    o2 = cb.game_opts(n, tol=0.0, max_iter=R, prec=prec, polish_fp64=False)
    V1, u1, _ = cb.game_solve(ctx, p, o1, raise_on_error=False)
    V2, u2, _ = cb.game_solve(ctx, p, o2, raise_on_error=False)
    C1, U1 = V1[0].cpu().numpy(), u1[0].cpu().numpy()
    C2, U2 = V2[0].cpu().numpy(), u2[0].cpu().numpy()
    opts = O.make_opts(n, tol=0.0, max_iter=R)
    rng = np.random.default_rng(1)
    js = rng.choice(n ** 3, 6, replace=False)
    for j in js:
        pb = np.empty(3)
        xr = np.empty(3)
        import ctypes
        O.lib().orc_game_node(ctypes.byref(opts), 3, int(j), pb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              xr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        for i in range(3):
            us, vs, inside, conc = O.game_node_update(p, opts, i, pb, U1[:, j], C1[i])
            v_gpu = O.eval_direct(C2[i].reshape(n, n, n), xr)
            assert abs(us - U2[i, j]) < 1e-5
            assert abs(vs - v_gpu) < 50 * (U_FORM[prec] + 2.0 ** -20) * max(1.0, abs(vs))


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x3"])
def test_split_full_solve_error_vs_fp64(ctx, full_fp64, prec):
    """n = 17 to the split form's residual floor, then with FP64 polish to 1e-10."""
    p, Vf, uf, rf = full_fp64
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(17, tol=1e-10, max_iter=20000, prec=prec,
                                                    polish_fp64=False), raise_on_error=False)
    r = res[0]
    e = rel(V[0].cpu().numpy(), Vf)
    print(f"split {prec} n=17: status {r.status} iters {r.iters} residual {r.residual:.2e} "
          f"coefficient error vs FP64 solve {e:.2e}")
    assert r.status in (0, 5)
    # floor of the split iteration: a few times the per-pass FP32-operand error (~4e-8)
    assert r.residual < 1e-6
    assert e < 1e-5
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(17, tol=1e-10, max_iter=20000, prec=prec,
                                                    polish_fp64=True), raise_on_error=False)
    r = res[0]
    e = rel(V[0].cpu().numpy(), Vf)
    print(f"split {prec} + FP64 polish n=17: status {r.status} iters {r.iters} (split {r.iters_split}) "
          f"residual {r.residual:.2e} error {e:.2e}")
    assert r.status == 0 and r.residual < 1e-10
    # both solves stop within tol / (1 - delta_h) ~ 2e-8 of the fixed point, from either side
    assert e < 1e-6


def test_diverging_warm_start_falls_back_to_cold(ctx):
    """A warm start with large node-to-node noise diverges (the iteration amplifies it near the
    clustered boundary nodes); the solver detects it, restarts cold and still converges."""
    p = I.single_game_workload()
    n, J = 17, 3
    o = cb.game_opts(n, tol=1e-10, max_iter=20000, prec="fp64")
    Vc, uc, rc = cb.game_solve(ctx, p, o)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    V0 = 0.05 * torch.randn((J, n ** J), generator=g, device="cuda", dtype=torch.float64)
    Vw, uw, rw = cb.game_solve(ctx, p, o, V0=[V0], raise_on_error=False)
    assert rw[0].restarts >= 1 and rw[0].status == 0
    assert rel(Vw[0].cpu().numpy(), Vc[0].cpu().numpy()) < 1e-6
    # a good warm start (the converged values) needs no restart and a single pass
    Vn = torch.empty((J, n ** J), dtype=torch.float64, device="cuda")
    cb.game_solve(ctx, p, o, Vn=[Vn])
    Vg, ug, rg = cb.game_solve(ctx, p, o, V0=[Vn], u0=[uc[0]])
    assert rg[0].restarts == 0 and rg[0].iters <= 2


@pytest.mark.parametrize("J,n,prec,pair,perm,tol", [
    (2, 9, "fp64", (0, 1), (1, 0), 1e-12),
    (3, 9, "fp64", (0, 2), (2, 1, 0), 1e-12),
    (4, 5, "fp64", (2, 3), (0, 1, 3, 2), 1e-12),
    (3, 17, "bf16x6", (0, 2), (2, 1, 0), 2e-5),
    (3, 33, "tf32x3", (0, 2), (2, 1, 0), 2e-5),
    (2, 17, "bf16x6", (0, 1), (1, 0), 2e-5),
    (4, 9, "fp64", (2, 3), (0, 1, 3, 2), 1e-12),
    (4, 9, "bf16x6", (2, 3), (0, 1, 3, 2), 2e-5)])
def test_symmetric_players_on_gpu(ctx, J, n, prec, pair, perm, tol):
    """The symmetry invariants of Section 4's J = 2, 3, 4 examples on the converged
    GPU solves: V_i(p) = V_k(sigma p), u_i(p) = u_k(sigma p) for the symmetric pair
    (FP64 to rounding; each split player's solution is within ~1e-5 of the FP64 one
    (the split form's floor), so a symmetric pair may differ by twice that; a
    control is the maximiser of W, its error that of W' over |W''|, which is of the
    order of h = 1e-2 here, so controls get ten times the value bound)."""
    p = I.game_params(J)
    Vn = [torch.empty((J, n ** J), dtype=torch.float64, device="cuda")]
    _, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=1e-10, max_iter=20000, prec=prec, polish_fp64=False),
                              Vn=Vn, raise_on_error=False)
    assert res[0].status in (0, 5)        # converged, or (split) stopped at its floor
    shape = (J,) + (n,) * J
    V = Vn[0].cpu().numpy().reshape(shape)
    U = u[0].cpu().numpy().reshape(shape)
    i, k = pair
    assert np.abs(V[i] - np.transpose(V[k], perm)).max() <= tol * np.abs(V).max()
    assert np.abs(U[i] - np.transpose(U[k], perm)).max() <= (tol if prec == "fp64" else 10 * tol)


@pytest.mark.parametrize("J,n,R", [(3, 5, 7), (2, 5, 40), (4, 4, 5), (3, 9, 3), (1, 6, 10)])
def test_df64_iterations_match_oracle(ctx, J, n, R):
    """CHEB_DF64: the player update in double-float (FP32 pairs, error-free products,
    compensated sums). Per value a relative error of about n^2 2^-48 (< 1e-13 here),
    carried through R contracting iterations: 1e-10 on coefficients and controls."""
    p = I.draw_game_params(I.SplitMix64(10 + J * 7 + n), J)
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R, prec="df64"), raise_on_error=False)
    assert res[0].iters == R
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R))
    assert rel(V[0].cpu().numpy(), ref["Vcoef"]) < 1e-10
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-10
    assert abs(res[0].residual - ref["residual"]) <= 1e-10 * ref["residual"] + 1e-14


def test_df64_full_size_tracks_fp64(ctx):
    """n = 17, the +-30 % draw: 300 iterations in double-float and in FP64 from the same
    cold start stay within 300 x ~1e-13 of each other; then the double-float solve
    converges to 1e-10 like the FP64 one."""
    p = I.single_game_workload()
    R = 300
    Vd, ud, rd = cb.game_solve(ctx, p, cb.game_opts(17, tol=0.0, max_iter=R, prec="df64"), raise_on_error=False)
    Vf, uf, rf = cb.game_solve(ctx, p, cb.game_opts(17, tol=0.0, max_iter=R, prec="fp64"), raise_on_error=False)
    assert rel(Vd[0].cpu().numpy(), Vf[0].cpu().numpy()) < 1e-9
    assert (ud[0] - uf[0]).abs().max().item() < 1e-9
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(17, tol=1e-10, max_iter=20000, prec="df64"), raise_on_error=False)
    assert res[0].status == 0 and res[0].residual < 1e-10


@pytest.mark.parametrize("polish", [1, 2])
def test_split_polish_modes_reach_tol(ctx, polish):
    """A stalled split iteration continues in double-float (polish 1) or on the FP64 pipe
    (polish 2); both reach tol = 1e-10 and the same solution (both within tol / (1 - delta)
    of the fixed point)."""
    p = I.single_game_workload()
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(9, tol=1e-10, max_iter=20000, prec="bf16x6", polish_fp64=polish),
                              raise_on_error=False)
    r = res[0]
    assert r.status == 0 and r.residual < 1e-10 and r.iters > r.iters_split > 0
    Vf, _, _ = cb.game_solve(ctx, p, cb.game_opts(9, tol=1e-10, max_iter=20000, prec="fp64"))
    assert rel(V[0].cpu().numpy(), Vf[0].cpu().numpy()) < 1e-6


def _node(opts, J, j):
    import ctypes
    pb, xr = np.empty(J), np.empty(J)
    O.lib().orc_game_node(ctypes.byref(opts), J, int(j), pb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          xr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return pb, xr


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x3"])
def test_mixed_size_split_batch_sampled_nodes_match_oracle(ctx, prec):
    """The batched split path at its real shape: one game_solve over 4 n = 9, 4 n = 17 and
    6 n = 33 instances (interleaved in the batch; the n = 33 group is large enough for the
    double-float refit and its own tuned tile shape). Two solves, R - 1 and R passes, give
    the GPU's iterate r = R - 1 and the pass from it; at sampled nodes of every instance and
    every player, the oracle's Steps 1-3 from the GPU's iterate R - 1 (its coefficients and
    controls) must give the GPU's control and value of iterate R (same bounds as the
    single-instance sampled test)."""
    sizes = [9, 17, 33, 9, 33, 17, 33, 9, 33, 17, 33, 9, 33, 17]
    rng_p = I.SplitMix64(77)
    ps = [I.draw_game_params(rng_p, 3) for _ in sizes]
    R = 3
    o1 = [cb.game_opts(n, tol=0.0, max_iter=R - 1, prec=prec, polish_fp64=False) for n in sizes]
    o2 = [cb.game_opts(n, tol=0.0, max_iter=R, prec=prec, polish_fp64=False) for n in sizes]
    V1, u1, r1 = cb.game_solve(ctx, ps, o1, raise_on_error=False)
    V2, u2, r2 = cb.game_solve(ctx, ps, o2, raise_on_error=False)
    assert all(r.iters == R - 1 for r in r1) and all(r.iters == R for r in r2)
    assert all(r.iters_split == R for r in r2)
    rng = np.random.default_rng(3)
    tol_v = 50 * (U_FORM[prec] + 2.0 ** -20)
    for q, n in enumerate(sizes):
        C1, U1 = V1[q].cpu().numpy(), u1[q].cpu().numpy()
        C2, U2 = V2[q].cpu().numpy(), u2[q].cpu().numpy()
        opts = O.make_opts(n, tol=0.0, max_iter=R)
        for j in rng.choice(n ** 3, 3, replace=False):
            pb, xr = _node(opts, 3, j)
            for i in range(3):
                us, vs, inside, conc = O.game_node_update(ps[q], opts, i, pb, U1[:, j], C1[i])
                v_gpu = O.eval_direct(C2[i].reshape(n, n, n), xr)
                assert abs(us - U2[i, j]) < 1e-5, (q, n, int(j), i, us, U2[i, j])
                assert abs(vs - v_gpu) < tol_v * max(1.0, abs(vs)), (q, n, int(j), i, vs, v_gpu)


@pytest.mark.parametrize("prec", ["bf16x6", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("J,n", [(2, 5), (2, 9), (2, 17), (4, 5), (4, 9)])
def test_split_iterations_close_to_oracle_two_and_four_players(ctx, J, n, prec):
    """The split player update for J = 2 (the GEMM is the series itself) and J = 4 (two
    rest modes reduced with T_{k_b} T_{k_c}): a few passes against the oracle's FP64
    passes, with the bound of the J = 3 test."""
    p = I.draw_game_params(I.SplitMix64(60 + J * 5 + n), J)
    R = 3 if J == 4 and n == 9 else 6
    V, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=0.0, max_iter=R, prec=prec, polish_fp64=False),
                              raise_on_error=False)
    assert res[0].iters == R and res[0].iters_split == R
    ref = O.game_solve(p, O.make_opts(n, tol=0.0, max_iter=R))
    bound = R * (U_FORM[prec] + 2.0 ** -20) * 10
    e = rel(V[0].cpu().numpy(), ref["Vcoef"])
    print(f"split {prec} J={J} n={n} after {R} passes: coefficient error {e:.2e} (bound {bound:.1e})")
    assert e < bound
    assert np.abs(u[0].cpu().numpy() - ref["u"]).max() < 1e-5


@pytest.mark.parametrize("J,n", [(2, 17), (4, 9)])
def test_split_sampled_node_updates_two_and_four_players(ctx, J, n):
    """One split pass (BF16x6) from the GPU's own iterate against the oracle's Steps 1-3 at
    sampled nodes: J = 2 at n = 17, J = 4 at n = 9 (N_P = 6,561, GEMM N = n^3 = 729)."""
    p = I.draw_game_params(I.SplitMix64(70 + J), J)
    R = 4
    o1 = cb.game_opts(n, tol=0.0, max_iter=R - 1, prec="bf16x6", polish_fp64=False)
    o2 = cb.game_opts(n, tol=0.0, max_iter=R, prec="bf16x6", polish_fp64=False)
    V1, u1, _ = cb.game_solve(ctx, p, o1, raise_on_error=False)
    V2, u2, _ = cb.game_solve(ctx, p, o2, raise_on_error=False)
    C1, U1 = V1[0].cpu().numpy(), u1[0].cpu().numpy()
    C2, U2 = V2[0].cpu().numpy(), u2[0].cpu().numpy()
    opts = O.make_opts(n, tol=0.0, max_iter=R)
    rng = np.random.default_rng(J)
    for j in rng.choice(n ** J, 8, replace=False):
        pb, xr = _node(opts, J, j)
        for i in range(J):
            us, vs, inside, conc = O.game_node_update(p, opts, i, pb, U1[:, j], C1[i])
            v_gpu = O.eval_direct(C2[i].reshape((n,) * J), xr)
            assert abs(us - U2[i, j]) < 1e-5, (int(j), i, us, U2[i, j])
            assert abs(vs - v_gpu) < 50 * (U_FORM["bf16x6"] + 2.0 ** -20) * max(1.0, abs(vs)), (int(j), i)


def test_split_two_players_full_solve_with_polish(ctx):
    """J = 2, n = 17 in BF16x6 to its floor, then polished in double-float to 1e-10, against
    the FP64 solve (both within tol / (1 - delta_h) of the fixed point)."""
    p = I.game_params(2)
    Vf, _, rf = cb.game_solve(ctx, p, cb.game_opts(17, tol=1e-10, max_iter=20000, prec="fp64"))
    V, _, r = cb.game_solve(ctx, p, cb.game_opts(17, tol=1e-10, max_iter=20000, prec="bf16x6", polish_fp64=True),
                            raise_on_error=False)
    assert r[0].status == 0 and r[0].residual < 1e-10 and r[0].iters_split > 0
    assert rel(V[0].cpu().numpy(), Vf[0].cpu().numpy()) < 1e-6


@pytest.mark.parametrize("prec,polish", [("bf16x6", 1), ("bf16x6", 2), ("df64", 0), ("fp64", 0)])
def test_solves_are_bit_reproducible(ctx, prec, polish):
    """Every reduction of the iteration has a fixed order (the residual is an integer max of
    FP64 bit patterns), so a solve is deterministic: two solves of the same mixed batch (two
    size classes, instances that stop at different iterations, the split phase, the switch to
    the polish and the polish phase) give bit-identical coefficients, controls, iteration
    counts and residuals."""
    rng = I.SplitMix64(123)
    ps = [I.draw_game_params(rng, 3) for _ in range(5)]
    ns = [9, 17, 9, 17, 9]
    its = [400, 100000, 37, 250, 100000]
    opts = [cb.game_opts(k, tol=1e-10, max_iter=m, prec=prec, polish_fp64=polish) for k, m in zip(ns, its)]
    V1, u1, r1 = cb.game_solve(ctx, ps, opts, raise_on_error=False)
    V2, u2, r2 = cb.game_solve(ctx, ps, opts, raise_on_error=False)
    for q in range(5):
        assert torch.equal(V1[q], V2[q]) and torch.equal(u1[q], u2[q]), q
        assert (r1[q].iters, r1[q].iters_split, r1[q].status) == (r2[q].iters, r2[q].iters_split, r2[q].status)
        assert r1[q].residual == r2[q].residual
        assert r1[q].iters <= its[q]
    ctx.device_status()


def test_one_launch_refit_matches_the_per_mode_refit(ctx):
    """The small-group refit (all modes in one launch per slab and last index) forms the same
    compensated sums in the same order as the per-mode refit of large groups: an instance solved
    alone and the same instance inside a 24-instance n = 17 group (per-mode refit) give
    bit-identical coefficients, controls and nodal values (default tile shape in both)."""
    rng = I.SplitMix64(321)
    ps = [I.draw_game_params(rng, 3) for _ in range(24)]
    o = cb.game_opts(17, tol=0.0, max_iter=4, prec="bf16x6", polish_fp64=False)
    ctx.set_tuning(1)
    try:
        Vn_b = [torch.empty((3, 17 ** 3), dtype=torch.float64, device="cuda") for _ in range(24)]
        Vb, ub, rb = cb.game_solve(ctx, ps, [o] * 24, Vn=Vn_b, raise_on_error=False)
        Vn_1 = [torch.empty((3, 17 ** 3), dtype=torch.float64, device="cuda")]
        V1, u1, r1 = cb.game_solve(ctx, ps[5], o, Vn=Vn_1, raise_on_error=False)
    finally:
        ctx.set_tuning(0)
    assert rb[5].iters == r1[0].iters == 4
    assert torch.equal(Vn_b[5], Vn_1[0]) and torch.equal(ub[5], u1[0])
    assert torch.equal(Vb[5], V1[0])
