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


def test_training_reduces_loss(ctx):
    rng = np.random.default_rng(4)
    S, F, Ov = 4096, 8, 64
    X = rng.uniform(-1, 1, (S, F))
    Wt = rng.standard_normal((F, Ov))
    Y = np.sin(X @ Wt) + 0.1 * (X @ Wt) ** 2
    net = cb.Surrogate(ctx, F, 128, 3, Ov, seed=3)
    losses = net.train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=80, batch=256, lr=2e-3)
    assert losses[-1] < 0.1 * losses[0], losses[::8]
    pred = net.predict(torch.from_numpy(X[:512]).cuda()).cpu().numpy()
    rel = np.linalg.norm(pred - Y[:512]) / np.linalg.norm(Y[:512] - Y[:512].mean(0))
    assert rel < 0.35
    net.close()


def test_warm_start_saves_iterations_small_games(ctx):
    """Train on method-generated solves (n = 5, FP64): nodal values and controls of one
    player per network; warm-start held-out games from the predictions."""
    n, J = 5, 3
    NP = n ** J
    rng = I.SplitMix64(31)
    ps = [I.draw_game_params(rng, J) for _ in range(600)]
    X = torch.from_numpy(np.stack([I.game_param_vector(p) for p in ps])).cuda()
    V = torch.empty((len(ps), J, NP), dtype=torch.float64, device="cuda")
    Vn = torch.empty_like(V)
    U = torch.empty_like(V)
    opts = [cb.game_opts(n, tol=1e-10, max_iter=20000, prec="fp64")] * len(ps)
    _, _, res = cb.game_solve(ctx, ps, opts, V=[V[q] for q in range(len(ps))], u=[U[q] for q in range(len(ps))],
                              Vn=[Vn[q] for q in range(len(ps))], raise_on_error=False)
    cold_iters = np.array([r.iters for r in res])
    assert all(r.status == 0 for r in res)
    # nodal values returned by the solver are the values of its coefficient tensors at the nodes
    a = np.cos(np.pi * np.arange(n) / (n - 1))
    for q in (0, 7):
        ref = np.stack([O.eval_grid(V[q, i].cpu().numpy().reshape(n, n, n), [a, a, a]).reshape(-1) for i in range(J)])
        assert np.abs(Vn[q].cpu().numpy() - ref).max() < 1e-13
    Y = torch.empty((len(ps), J, 2, NP), dtype=torch.float64, device="cuda")
    Y[:, :, 0] = Vn
    Y[:, :, 1] = U
    ntr = 512
    pred = torch.empty((len(ps) - ntr, J, 2, NP), dtype=torch.float64, device="cuda")
    nets = []
    for i in range(J):
        net = cb.Surrogate(ctx, X.shape[1], 128, 3, 2 * NP, seed=10 + i)
        net.train(X[:ntr], Y[:ntr, i].reshape(ntr, 2 * NP), epochs=200, batch=64, lr=2e-3, seed=i)
        net.predict(X[ntr:].contiguous(), out=pred[:, i].reshape(-1, 2 * NP))
        nets.append(net)
    tps = ps[ntr:]
    V0 = [pred[q, :, 0].contiguous() for q in range(len(tps))]
    for v in V0:
        for i in range(J):
            cb.cheb_smooth(ctx, v[i].view(n, n, n))
    u0 = [pred[q, :, 1].contiguous() for q in range(len(tps))]
    Vw, uw, resw = cb.game_solve(ctx, tps, [opts[0]] * len(tps), V0=V0, u0=u0, raise_on_error=False)
    warm_iters = np.array([r.iters for r in resw])
    assert all(r.status == 0 for r in resw)
    print(f"warm start n=5: cold {cold_iters[ntr:].mean():.0f} iterations, warm {warm_iters.mean():.0f}")
    assert warm_iters.mean() < 0.85 * cold_iters[ntr:].mean()
    # same fixed point (both within tol / (1 - delta) of it)
    for q in range(len(tps)):
        d = float((Vw[q] - V[ntr + q]).abs().max() / V[ntr + q].abs().max())
        assert d < 1e-6
    for net in nets:
        net.close()


def test_spectral_filter_and_smoothing(ctx):
    """cheb_filter multiplies coefficient l by prod_s exp(-alpha (l_s/N_s)^(2 order)); cheb_smooth
    (fit -> filter -> nodes) leaves a low-degree polynomial's nodal values nearly unchanged."""
    rng = np.random.default_rng(9)
    shape = (5, 9, 17)
    c = rng.standard_normal(shape)
    cd = torch.from_numpy(c).cuda()
    cb.cheb_filter(ctx, cd, alpha=36.0, order=4)
    eta = [np.arange(k) / (k - 1) for k in shape]
    f = np.exp(-36.0 * (eta[0][:, None, None] ** 8 + eta[1][None, :, None] ** 8 + eta[2][None, None, :] ** 8))
    assert np.abs(cd.cpu().numpy() - c * f).max() < 1e-14
    # degree <= 2 polynomial at the nodes: smoothing changes it by at most ~1e-5 relative
    p2 = np.zeros((17, 17, 17))
    p2[0, 0, 0], p2[1, 0, 0], p2[0, 2, 0], p2[1, 1, 0], p2[0, 0, 2] = 0.3, -0.1, 0.05, 0.02, -0.04
    a = np.cos(np.pi * np.arange(17) / 16)
    nod = O.eval_grid(p2, [a, a, a])
    v = torch.from_numpy(nod).cuda()
    cb.cheb_smooth(ctx, v)
    assert np.abs(v.cpu().numpy() - nod).max() < 1e-5 * np.abs(nod).max()
