"""The warm-start network on the GPU (surrogate_* of include/cheb.h).

- forward output, loss, every gradient entry and the weights after 1, 2 and 10
  Adam steps against the FP64 oracle (oracle/mlp_oracle.c) at the same FP32
  parameters, element by element, under first-order error bounds derived from
  the GPU arithmetic (see first_order_bounds);
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

U_BF16 = 2.0 ** -8      # unit roundoff of BF16 (8 significant bits), operands rounded to nearest
U_F32 = 2.0 ** -24


def split_params(dims, flat):
    out, off = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        out.append(flat[off:off + nw].reshape(dims[l + 1], dims[l]))
        off += nw
        out.append(flat[off:off + dims[l + 1]])
        off += dims[l + 1]
    return out


def _phi(z):
    return np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def first_order_bounds(dims, p, X, T):
    """Per-entry bounds on |GPU - exact| of the forward output and of the gradient.

    The GPU rounds both operands of every GEMM to BF16 (relative error <= U_BF16 each, so
    <= 2 U_BF16 per product) and accumulates K products in FP32 (<= K U_F32); biases, GELU,
    GELU' and the loss gradient are FP32. Propagating absolute errors to first order through
    the network, with magnitudes |.| of the exact intermediates (computed here in FP64 only
    for this bound; the expected values themselves come from the oracle):
      dZ  <= (2 U_BF16 + K U_F32) |H| |W|^T + dH |W|^T + 4 U_F32 |Z|
      dH  <= |GELU'(Z)| dZ + 4 U_F32 |H|
      d(dY) = 2 dY / (B out)
      d(gW) <= (2 U_BF16 + B U_F32) |dZ|^T |H| + d(dZ)^T |H| + |dZ|^T dH
      d(gb) <= sum_b d(dZ) + B U_F32 sum_b |dZ|
      d(dH) <= (2 U_BF16 + K U_F32) |dZ| |W| + d(dZ) |W|
      d(dZ) <= |GELU'(Z)| d(dH) + |dH| |GELU''(Z)| dZ + 4 U_F32 |dZ|
    with GELU''(z) = phi(z) (2 - z^2)."""
    Ws = split_params(dims, p)
    L = len(dims) - 1
    H, dHe, Zs = [X], [np.zeros_like(X)], []
    for l in range(L):
        W, b = Ws[2 * l], Ws[2 * l + 1]
        Z = H[-1] @ W.T + b
        eZ = (2 * U_BF16 + dims[l] * U_F32) * (np.abs(H[-1]) @ np.abs(W).T) + dHe[-1] @ np.abs(W).T \
            + 4 * U_F32 * np.abs(Z)
        Zs.append((Z, eZ))
        if l < L - 1:
            Hn = Z * 0.5 * (1.0 + np.vectorize(__import__("math").erf)(Z / np.sqrt(2.0)))
            gp = 0.5 * (1.0 + np.vectorize(__import__("math").erf)(Z / np.sqrt(2.0))) + Z * _phi(Z)
            H.append(Hn)
            dHe.append(np.abs(gp) * eZ + 4 * U_F32 * np.abs(Hn))
    Y, eY = Zs[-1]
    B, nout = X.shape[0], dims[-1]
    dZ = 2.0 * (Y - T) / (B * nout)
    edZ = 2.0 * eY / (B * nout) + 4 * U_F32 * np.abs(dZ)
    gW_b, gb_b = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        W = Ws[2 * l]
        Hl, eHl = H[l], dHe[l]
        gW_b[l] = (2 * U_BF16 + B * U_F32) * (np.abs(dZ).T @ np.abs(Hl)) + edZ.T @ np.abs(Hl) + np.abs(dZ).T @ eHl
        gb_b[l] = edZ.sum(0) + B * U_F32 * np.abs(dZ).sum(0)
        if l > 0:
            dH = dZ @ W
            edH = (2 * U_BF16 + dims[l + 1] * U_F32) * (np.abs(dZ) @ np.abs(W)) + edZ @ np.abs(W)
            Zp, eZp = Zs[l - 1]
            gp = 0.5 * (1.0 + np.vectorize(__import__("math").erf)(Zp / np.sqrt(2.0))) + Zp * _phi(Zp)
            gpp = _phi(Zp) * (2.0 - Zp * Zp)
            dZn = dH * gp
            edZ = np.abs(gp) * edH + np.abs(dH) * np.abs(gpp) * eZp + 4 * U_F32 * np.abs(dZn)
            dZ = dZn
    gbound = np.concatenate([np.concatenate([gW_b[l].reshape(-1), gb_b[l]]) for l in range(L)])
    return eY, gbound


def _inputs(dims, regime, seed, count, B=64):
    """Parameters, inputs and targets (FP32 values). 'mixed': N(0, 0.2^2) parameters, N(0, 1)
    inputs and targets (signs cancel in every sum, so the worst-case bounds are loose).
    'positive': weights in [0, 2/fan_in), biases in [-0.3, 0.3), inputs in [0.1, 1) and targets
    in [-3, -2) so that Y - T > 0: almost every term of every sum has one sign, the bounds are
    within ~10 % of each entry, and any wrong entry exceeds them."""
    rng = np.random.default_rng(seed)
    if regime == "mixed":
        p = rng.standard_normal(count) * 0.2
        X = rng.standard_normal((B, dims[0]))
        T = rng.standard_normal((B, dims[-1]))
    else:
        parts = []
        for l in range(len(dims) - 1):
            parts.append(rng.uniform(0.0, 2.0 / dims[l], dims[l + 1] * dims[l]))
            parts.append(rng.uniform(-0.3, 0.3, dims[l + 1]))
        p = np.concatenate(parts)
        X = rng.uniform(0.1, 1.0, (B, dims[0]))
        T = rng.uniform(-3.0, -2.0, (B, dims[-1]))
    return p.astype(np.float32), X.astype(np.float32), T.astype(np.float32)


@pytest.mark.parametrize("regime", ["positive", "mixed"])
@pytest.mark.parametrize("dims,batch", [([8, 32, 32, 20], 64), ([8, 256, 256, 300], 64), ([3, 16, 5], 64),
                                        ([8, 130, 130, 33], 64), ([8, 256, 1300], 200), ([5, 200, 200, 2100], 130),
                                        ([8, 4992, 16], 256), ([8, 256, 4992], 256)])
def test_forward_and_gradient_entries_match_oracle(ctx, dims, batch, regime):
    """Every output and every gradient entry within twice its first-order bound (the factor
    covers second-order terms). Batches of 200 and 130 leave a ragged K tile in the weight
    gradients (K = batch) and a ragged row tile everywhere; outputs of 1,300 and 2,100 make the
    hidden-layer gradient a long-K product with four or fewer output tiles, which is split
    across CTAs and summed in a fixed order. A 4,992-wide hidden layer and a 4,992-wide
    output layer at batch 256 give products with 78 output tiles, finished inside the GEMM
    (GELU with both packed copies, the GELU derivative, the bias-only output and the wide
    weight gradient)."""
    net = cb.Surrogate(ctx, dims[0], dims[1], len(dims) - 2, dims[-1], seed=1)
    p, X, T = _inputs(dims, regime, sum(dims), net.param_count(), B=batch)
    net.set_params(p)
    B = X.shape[0]
    p64, X64, T64 = p.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    loss, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lref, gref = O.mlp_loss_grad(dims, p64, X64, T64)
    Yref = O.mlp_forward(dims, p64, X64)
    eY, gb = first_order_bounds(dims, p64, X64, T64)
    if regime == "positive":
        assert np.median(gb / np.abs(gref)) < 0.1      # the bounds are sharp here
    # forward (predict applies the identity normalisation of an untrained network)
    Y = net.predict(torch.from_numpy(X64).cuda()).cpu().numpy()
    assert np.all(np.abs(Y - Yref) <= 2 * eY + 1e-30), float((np.abs(Y - Yref) / eY).max())
    # loss: |sum d^2 - sum d_ref^2| <= sum 2 |d| eY / (B out) + FP32 summation
    lb = float(2 * (np.abs(Yref - T64) * eY).sum() / (B * dims[-1]) + 2 * B * dims[-1] * U_F32 * lref)
    assert abs(loss - lref) <= 2 * lb, (loss, lref, lb)
    g = g.cpu().numpy().astype(np.float64)
    ratio = np.abs(g - gref) / (2 * gb + 1e-30)
    worst = int(np.argmax(ratio))
    assert ratio.max() <= 1.0, (worst, g[worst], gref[worst], gb[worst])
    net.close()


def test_adam_steps_match_oracle(ctx):
    """Weights after t = 1, 2 and 10 Adam steps with given gradients, element by element
    against orc_adam_step. The GPU state (w, m, v) is FP32: each step rounds m, v and the
    update to FP32 (a few ulp each) and w - update to FP32, so after t steps
    |w_gpu - w_ref| <= sum over steps of (2 ulp(|w|) + 16 U_F32 |update|) plus the
    propagated differences of m and v, bounded here by a factor 2."""
    dims = [8, 32, 16]
    rng = np.random.default_rng(12)
    net = cb.Surrogate(ctx, dims[0], dims[1], len(dims) - 2, dims[-1], seed=2)
    n = net.param_count()
    w0 = (rng.standard_normal(n) * 0.3).astype(np.float32)
    net.set_params(w0)                   # also resets m, v and the step count
    w = w0.astype(np.float64)
    m = np.zeros(n)
    v = np.zeros(n)
    lr = 1e-2
    tol = np.zeros(n)
    for t in range(1, 11):
        g = (rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 1, n)).astype(np.float32)
        net.adam_step(torch.from_numpy(g).cuda(), lr=lr)
        w_before = w.copy()
        O.adam_step(w, g.astype(np.float64), m, v, lr, 0.9, 0.999, 1e-8, t)
        tol += 2 * U_F32 * 2 * np.abs(w) + 16 * U_F32 * np.abs(w - w_before)
        if t in (1, 2, 10):
            got = net.get_params().astype(np.float64)
            ratio = np.abs(got - w) / (2 * tol + 1e-30)
            assert ratio.max() <= 1.0, (t, float(ratio.max()))
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


def test_training_is_deterministic_and_timed_inside_the_graph(ctx):
    """Training runs as CUDA graphs with the weight and bias gradients on a second stream; the
    split-K partials and the loss are summed in a fixed order, so two runs from the same
    parameters and seed give bit-identical weights and losses. With kernel timing on, the
    timing events are captured into the graph and every kernel reports a positive time."""
    rng = np.random.default_rng(6)
    S, F, Ov = 2048, 8, 300
    X = torch.from_numpy(rng.uniform(-1, 1, (S, F))).cuda()
    Y = torch.from_numpy(rng.standard_normal((S, Ov))).cuda()
    runs = []
    for timed in (False, True):
        net = cb.Surrogate(ctx, F, 256, 2, Ov, seed=11)
        ctx.profile(timed)
        losses = net.train(X, Y, epochs=3, batch=256, lr=1e-3, seed=5)
        torch.cuda.synchronize()
        if timed:
            prof = ctx.profile_read()
            ctx.profile(False)
            gemms = {k: v for k, v in prof.items() if k.startswith("mlp_gemm")}
            assert gemms and all(n > 0 and ms > 0 for n, ms in gemms.values()), prof
        runs.append((net.get_params(), losses))
        net.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]


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
