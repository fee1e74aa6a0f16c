"""game_paths: equilibrium time paths (Section 4) on the GPU, through the C ABI.

- parity with the FP64 oracle (oracle/game_oracle.c orc_game_paths) on the same
  nodal controls, J = 1..4, bound-active policies (the clamp is exercised);
  both are FP64 and differ only in summation order: 1e-12 relative;
- the affine LQ policy (no bound active on [0, 0.8]^J): the path equals the
  affine recursion computed with numpy (independent of both interpolants);
- edge cases: no trajectory, no step, controls not requested, bad arguments.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("J,n,K,T", [(1, 9, 3, 50), (2, 9, 5, 300), (3, 9, 7, 300), (3, 17, 4, 200), (4, 5, 3, 150)])
def test_paths_match_oracle(ctx, J, n, K, T):
    # U_M = 0.35 is below the unconstrained policy's maximum, so a bound binds
    # on part of the box and the clamp is exercised along the paths
    p = I.game_params(J)
    U_M = 0.35
    _, u, res = cb.game_solve(ctx, p, cb.game_opts(n, U_M=U_M, tol=1e-9, max_iter=20000), raise_on_error=False)
    assert res[0].status == 0
    un = u[0].cpu().numpy()
    assert ((un == 0.0) | (un == U_M)).any()          # a bound binds somewhere
    rng = np.random.default_rng(J * 100 + n)
    p0 = rng.uniform(0, 1, (K, J))
    p0[0], p0[1] = 0.0, 1.0          # clean and saturated corners: the policy is clamped there
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n, U_M=U_M), u[0], dev(p0), T)
    ppo, upo = O.game_paths(p, O.make_opts(n, U_M=U_M), un, p0, T)
    assert ((upo == 0.0) | (upo == U_M)).any()
    assert np.abs(pp.cpu().numpy() - ppo).max() <= 1e-12 * np.abs(ppo).max()
    assert np.abs(up.cpu().numpy() - upo).max() <= 1e-12


def test_paths_follow_affine_lq_policy(ctx):
    for J in (2, 3, 4):
        p = I.game_params(J)
        h, P_M, n = 1e-2, 0.8, 5
        lq = O.game_lq(p, h, 6000)
        F, f = lq["F"][-1], lq["f"][-1]
        pb, _ = O.game_nodes(O.make_opts(n, h=h, P_M=P_M), J)
        U = (pb @ F.T + f).T
        rng = np.random.default_rng(J)
        p0 = rng.uniform(0, P_M, (6, J))
        T = 600
        pp, up = cb.game_paths(ctx, p, cb.game_opts(n, h=h, P_M=P_M), dev(U), dev(p0), T)
        pp, up = pp.cpu().numpy(), up.cpu().numpy()
        M = p["K"] / p["m"] - np.diag(p["c"]) + np.diag(p["beta"]) @ F
        q = p0.copy()
        for t in range(T):
            assert np.abs(up[:, t] - (q @ F.T + f)).max() < 1e-10
            q = q + h * (q @ M.T + p["beta"] * f)
            assert np.abs(pp[:, t + 1] - q).max() < 1e-10


def test_paths_edge_cases(ctx):
    p = I.game_params(3)
    n = 5
    U = dev(np.full((3, n ** 3), 0.3))
    p0 = dev(np.array([[0.1, 0.2, 0.3]]))
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n), U, p0, 0)
    assert pp.shape == (1, 1, 3) and torch.equal(pp[0, 0], p0[0]) and up.shape == (1, 0, 3)
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n), U, torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 10)
    assert pp.shape == (0, 11, 3)
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n), U, p0, 7, with_controls=False)
    assert up is None
    # a constant policy u = 0.3: every control along the path is 0.3
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n), U, p0, 7)
    assert torch.allclose(up, torch.full_like(up, 0.3), rtol=0, atol=1e-14)
    with pytest.raises(cb.ChebError):
        cb.game_paths(ctx, p, cb.game_opts(1), U, p0, 3)
    with pytest.raises(cb.ChebError):
        cb.game_paths(ctx, p, cb.game_opts(n, h=0.0), U, p0, 3)
    with pytest.raises(cb.ChebError):                 # J = 4 with n = 33: too large per CTA
        q4 = I.game_params(4)
        cb.game_paths(ctx, q4, cb.game_opts(33), dev(np.zeros((4, 33 ** 4))), dev(np.zeros((1, 4))), 3)
    ctx.device_status()


def test_paths_full_size_sample(ctx):
    """The config-3 game (n = 17, parameters drawn +-30 %): FP64 solve, then 8 paths of
    2,000 steps against the oracle."""
    p = I.single_game_workload(2)
    n = 17
    _, u, res = cb.game_solve(ctx, p, cb.game_opts(n, tol=1e-10, max_iter=20000), raise_on_error=False)
    assert res[0].status == 0
    rng = np.random.default_rng(7)
    p0 = rng.uniform(0, 1, (8, 3))
    T = 2000
    pp, up = cb.game_paths(ctx, p, cb.game_opts(n), u[0], dev(p0), T)
    ppo, upo = O.game_paths(p, O.make_opts(n), u[0].cpu().numpy(), p0, T)
    assert np.abs(pp.cpu().numpy() - ppo).max() <= 1e-12 * np.abs(ppo).max()
    assert np.abs(up.cpu().numpy() - upo).max() <= 1e-12
    # the stocks settle: the last steps move by less than 1e-6 per step
    last = pp.cpu().numpy()[:, -2:]
    assert np.abs(last[:, 1] - last[:, 0]).max() < 1e-6
