"""Tile-shape tuning of the split-precision game update (cheb_set_tuning,
cheb_tuning_report of include/cheb.h).

Every tile configuration (MMA column chunk x CTAs per SM) computes the same
per-node contractions in the same order, so forcing any of them, or letting
the tuner time them all on the first iteration, must leave the iterates
bit-identical to the default shape's.
"""
import pytest
import torch

import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ITERS = 40


def solve(ctx, params, ns, prec="bf16x6"):
    opts = [cb.game_opts(n, tol=0.0, max_iter=ITERS, prec=prec, polish_fp64=False) for n in ns]
    return cb.game_solve(ctx, params, opts, raise_on_error=False)


@pytest.mark.parametrize("n", [9, 17, 33])
def test_every_configuration_gives_identical_iterates(ctx, n):
    p = [I.single_game_workload(2)]
    try:
        ctx.set_tuning(1)
        V0, u0, r0 = solve(ctx, p, [n])
        assert r0[0].iters == ITERS
        ran = 0
        for c in range(3):
            for k in (1, 2, 3):
                ctx.set_tuning(2 + 4 * c + k)
                V, u, r = solve(ctx, p, [n])
                if r[0].iters == 0:        # that configuration does not exist for n (CHEB_EINVAL)
                    continue
                ran += 1
                assert r[0].iters == ITERS
                assert torch.equal(V[0], V0[0]) and torch.equal(u[0], u0[0]), (c, k)
        assert ran >= 2
        ctx.set_tuning(0)
        V, u, r = solve(ctx, p, [n])
        assert torch.equal(V[0], V0[0]) and torch.equal(u[0], u0[0])
        rep = ctx.tuning_report()
        assert f"bf16x6 J=3 n={n} batch class 0" in rep and "tried" in rep
    finally:
        ctx.set_tuning(0)


def test_tuned_batch_matches_default(ctx):
    inst = I.batched_game_workload(seed=2, count=12, sizes=(9, 17))
    params = [q for _, q in inst]
    ns = [n for n, _ in inst]
    try:
        ctx.set_tuning(1)
        V0, u0, _ = solve(ctx, params, ns, prec="tf32x3")
        ctx.set_tuning(0)
        V, u, _ = solve(ctx, params, ns, prec="tf32x3")
        for q in range(len(params)):
            assert torch.equal(V[q], V0[q]) and torch.equal(u[q], u0[q])
        rep = ctx.tuning_report()
        assert "tf32x3 J=3 n=9" in rep and "tf32x3 J=3 n=17" in rep
    finally:
        ctx.set_tuning(0)


def test_invalid_tuning_mode(ctx):
    with pytest.raises(cb.ChebError):
        ctx.set_tuning(-1)
    with pytest.raises(cb.ChebError):
        ctx.set_tuning(99)
