"""The warm-start network on the GPU (surrogate_* of include/cheb.h).

- forward pass and gradients against the FP64 oracle (oracle/mlp_oracle.c) at
  the same FP32 parameters; the GPU rounds every GEMM operand to BF16
  (relative 2^-9), accumulates in FP32, so the bound used is a relative L2
  error of 3e-2 per parameter tensor and a cosine similarity above 0.999;
- training lowers the loss on a smooth regression;
- a warm start learned from method-generated solves (n = 5) needs fewer
  iterations than the cold start and reaches the same fixed point.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_04688_gb300 as cb
from paper_2307_04688_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def split_params(dims, flat):
    out, off = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        out.append(flat[off:off + nw])
        off += nw
        out.append(flat[off:off + dims[l + 1]])
        off += dims[l + 1]
    return out


@pytest.mark.parametrize("dims", [[8, 32, 32, 20], [8, 256, 256, 300], [3, 16, 5]])
def test_gradients_match_oracle(ctx, dims):
    rng = np.random.default_rng(sum(dims))
    net = cb.Surrogate(ctx, dims[0], dims[1], len(dims) - 2, dims[-1], seed=1)
    p = (rng.standard_normal(net.param_count()) * 0.2).astype(np.float32)
    net.set_params(p)
    B = 64
    X = rng.standard_normal((B, dims[0])).astype(np.float32)
    T = rng.standard_normal((B, dims[-1])).astype(np.float32)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lref, gref = O.mlp_loss_grad(dims, p.astype(np.float64), X, T)
    assert abs(loss - lref) / lref < 1e-2
    g = g.cpu().numpy().astype(np.float64)
    for a, b in zip(split_params(dims, g), split_params(dims, gref)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel < 3e-2 and cos > 0.999, (rel, cos)
    # forward through predict (normalisation is the identity before training)
    Y = net.predict(torch.from_numpy(X.astype(np.float64)).cuda()).cpu().numpy()
    Yref = O.mlp_forward(dims, p.astype(np.float64), X)
    assert np.linalg.norm(Y - Yref) / np.linalg.norm(Yref) < 2e-2
    net.close()


def test_oracle_gradient_against_finite_differences():
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


def test_training_reduces_loss(ctx):
    rng = np.random.default_rng(4)
    S, F, Ov = 4096, 8, 64
    X = rng.uniform(-1, 1, (S, F))
    Wt = rng.standard_normal((F, Ov))
    Y = np.sin(X @ Wt) + 0.1 * (X @ Wt) ** 2
    net = cb.Surrogate(ctx, F, 128, 3, Ov, seed=3)
    losses = net.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=40, batch=256, lr=2e-3)
    assert losses[-1] < 0.1 * losses[0], losses[::8]
    pred = net.predict(torch.from_numpy(X[:512]).cuda()).cpu().numpy()
    rel = np.linalg.norm(pred - Y[:512]) / np.linalg.norm(Y[:512] - Y[:512].mean(0))
    assert rel < 0.3
    net.close()


def test_warm_start_saves_iterations_small_games(ctx):
    """Train on method-generated solves (n = 5, FP64), warm-start held-out games."""
    n, J = 5, 3
    NP = n ** J
    rng = I.SplitMix64(31)
    ps = [I.draw_game_params(rng, J) for _ in range(600)]
    X = np.stack([I.game_param_vector(p) for p in ps])
    Vbig = torch.empty((len(ps), J, NP), dtype=torch.float64, device="cuda")
    opts = [cb.game_opts(n, tol=1e-10, max_iter=20000, prec="fp64")] * len(ps)
    _, _, res = cb.game_solve(ctx, ps, opts, V=[Vbig[q] for q in range(len(ps))], raise_on_error=False)
    cold_iters = np.array([r.iters for r in res])
    assert all(r.status == 0 for r in res)
    train, test = slice(0, 512), slice(512, 600)
    Xd = torch.from_numpy(X).cuda()
    nets, V0 = [], []
    a = torch.cos(torch.pi * torch.arange(n, dtype=torch.float64) / (n - 1)).cuda()
    pred = torch.empty((600 - 512, J, NP), dtype=torch.float64, device="cuda")
    for i in range(J):
        net = cb.Surrogate(ctx, X.shape[1], 128, 3, NP, seed=10 + i)
        net.train(Xd[train], Vbig[train, i, :], epochs=150, batch=64, lr=2e-3, seed=i)
        net.predict(Xd[test].contiguous(), out=pred[:, i, :])
        nets.append(net)
    # predicted coefficients -> nodal values (the iteration starts from nodal values)
    V0 = []
    for q in range(pred.shape[0]):
        V0.append(torch.stack([cb.cheb_eval_grid(ctx, pred[q, i].reshape(n, n, n).contiguous(), [a, a, a]).reshape(-1)
                               for i in range(J)]).contiguous())
    tps = ps[512:]
    Vw, uw, resw = cb.game_solve(ctx, tps, [opts[0]] * len(tps), V0=V0, raise_on_error=False)
    warm_iters = np.array([r.iters for r in resw])
    assert all(r.status == 0 for r in resw)
    print(f"warm start n=5: cold {cold_iters[test].mean():.0f} iterations, warm {warm_iters.mean():.0f}")
    assert warm_iters.mean() < 0.9 * cold_iters[test].mean()
    # same fixed point (both within tol / (1 - delta) of it)
    for q in range(len(tps)):
        d = float((Vw[q] - Vbig[512 + q]).abs().max() / Vbig[512 + q].abs().max())
        assert d < 1e-6
    for net in nets:
        net.close()
