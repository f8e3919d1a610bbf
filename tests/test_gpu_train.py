"""GPU parity of the learned part (a6): drag targets, MSE gradient and the Adam
training trajectory against the FP64 oracle, and the closed-loop benefit of
the trained residual over the nominal model on the drag plant."""
import numpy as np
import pytest

import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
QUAD = W.QUAD


@pytest.fixture(scope="module")
def rtn():
    import paper_2203_07747_b300 as rtn
    rtn.load(build_if_missing=True)
    return rtn


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def ctl_for(rtn, layers, B=2, precision="fp32", train_bf16=False):
    return rtn.Controller(np.full(B, 5, np.int32), np.full(B, 0.05), W.Q_DIAG, W.R_DIAG, quad=QUAD,
                          layers=layers, precision=precision, train_bf16=train_bf16)


def test_drag_targets_match_oracle(rtn, orc):
    X, _ = W.training_samples(4096, 3)
    X = f32(X)
    ctl = ctl_for(rtn, [(f32(w), f32(b)) for w, b in W.xavier_mlp([17, 8, 3], 0)])
    Y = ctl.drag_targets(dev(X)).double().cpu().numpy()
    Yr = orc.drag_targets(X)
    err = np.linalg.norm(Y - Yr, axis=1) / np.maximum(np.linalg.norm(Yr, axis=1), 1e-3)
    assert err.max() < 1e-5


@pytest.mark.parametrize("widths,n", [([17, 32, 32, 3], 256), ([17, 100, 60, 70, 3], 333)])
def test_mse_gradient_matches_oracle(rtn, orc, widths, n):
    layers = [(f32(w), f32(np.random.default_rng(i).normal(0, 0.1, b.shape))) for i, (w, b) in
              enumerate(W.xavier_mlp(widths, 1))]
    X, U = W.training_samples(n, 4)
    X, U = f32(X), f32(U)
    Y = orc.drag_targets(X)
    Z = np.concatenate([X, U], 1)
    loss_r, G_r = orc.mse_grad(layers, Z, Y)
    ctl = ctl_for(rtn, layers)
    loss, g = ctl.mse_grad(dev(X), dev(U), dev(Y))
    g = g.double().cpu().numpy()
    assert abs(loss - loss_r) / loss_r < 1e-5
    nw = sum(w.size for w, _ in layers)
    ow, ob = 0, nw
    for (Wr, br) in G_r:
        gw = g[ow:ow + Wr.size].reshape(Wr.shape)
        gb = g[ob:ob + br.size]
        assert np.linalg.norm(gw - Wr) / np.linalg.norm(Wr) < 1e-5
        assert np.linalg.norm(gb - br) / np.linalg.norm(br) < 1e-5
        ow += Wr.size
        ob += br.size


@pytest.mark.parametrize("widths,n", [([17, 32, 32, 3], 256), ([17, 100, 60, 70, 3], 333),
                                      ([17, 512, 512, 512, 3], 1024)])
def test_mse_gradient_bf16_operands(rtn, orc, widths, n):
    # train_bf16: every GEMM operand rounded to BF16 (one MMA per product),
    # FP32 accumulation.  Each rounding moves an operand by <= 2^-9 relative;
    # a gradient passes through ~2 L of them (activations forward, gradients
    # backward), so its norm-relative error stays near 2^-9 sqrt(2 L) < 1e-2:
    # gate 2e-2 per layer, and the loss (one forward pass) 5e-3
    layers = [(f32(w), f32(np.random.default_rng(i).normal(0, 0.1, b.shape))) for i, (w, b) in
              enumerate(W.xavier_mlp(widths, 1))]
    X, U = W.training_samples(n, 4)
    X, U = f32(X), f32(U)
    Y = orc.drag_targets(X)
    Z = np.concatenate([X, U], 1)
    loss_r, G_r = orc.mse_grad(layers, Z, Y)
    ctl = ctl_for(rtn, layers, train_bf16=True)
    loss, g = ctl.mse_grad(dev(X), dev(U), dev(Y))
    g = g.double().cpu().numpy()
    assert abs(loss - loss_r) / loss_r < 5e-3
    nw = sum(w.size for w, _ in layers)
    ow, ob = 0, nw
    errs = []
    for (Wr, br) in G_r:
        gw = g[ow:ow + Wr.size].reshape(Wr.shape)
        gb = g[ob:ob + br.size]
        errs.append((np.linalg.norm(gw - Wr) / np.linalg.norm(Wr), np.linalg.norm(gb - br) / np.linalg.norm(br)))
        ow += Wr.size
        ob += br.size
    assert max(max(e) for e in errs) < 2e-2, errs
    # and it is a BF16 result, not the split one: some layer is off by > 1e-5
    assert max(max(e) for e in errs) > 1e-5, errs


def test_bf16_training_follows_split_training(rtn, orc):
    # the same 64 Adam steps with BF16 and with split operands: the BF16
    # losses stay within 2% of the split ones and both fall
    widths = [17, 128, 128, 128, 3]
    layers = [(f32(w), f32(b)) for w, b in W.xavier_mlp(widths, 6)]
    n, bs = 8192, 256
    X, U = W.training_samples(n, 9)
    X, U = f32(X), f32(U)
    Y = f32(orc.drag_targets(X))
    out = {}
    for mode in (False, True):
        ctl = ctl_for(rtn, layers, train_bf16=mode)
        out[mode] = ctl.train(dev(X), dev(U), dev(Y), epochs=2, batch=bs, lr=1e-3)
        ctl.close()
    a, b = out[False], out[True]
    assert len(a) == len(b) == 2 * (n // bs)
    assert a[-8:].mean() < 0.5 * a[:8].mean() and b[-8:].mean() < 0.5 * b[:8].mean()
    assert np.max(np.abs(b - a) / a) < 2e-2, np.max(np.abs(b - a) / a)


def test_adam_training_trajectory_matches_oracle(rtn, orc):
    widths = [17, 32, 32, 3]
    layers = [(f32(w), f32(b)) for w, b in W.xavier_mlp(widths, 2)]
    n, bs, steps, lr = 1024, 128, 16, 1e-3
    X, U = W.training_samples(n, 5)
    X, U = f32(X), f32(U)
    Y = f32(orc.drag_targets(X))
    ctl = ctl_for(rtn, layers)
    losses = ctl.train(dev(X), dev(U), dev(Y), epochs=2, batch=bs, lr=lr)
    assert len(losses) == steps
    # oracle: same minibatch order, FP64 gradients, Adam
    Z = np.concatenate([X, U], 1)
    P = np.concatenate([np.concatenate([w.ravel() for w, _ in layers]),
                        np.concatenate([b.ravel() for _, b in layers])])
    P0 = P.copy()
    m, v = np.zeros_like(P), np.zeros_like(P)
    nw = sum(w.size for w, _ in layers)
    ref_losses = []
    for k in range(steps):
        s = (k % (n // bs)) * bs
        cur, ow, ob = [], 0, nw
        for w, b in layers:
            cur.append((P[ow:ow + w.size].reshape(w.shape), P[ob:ob + b.size]))
            ow += w.size
            ob += b.size
        loss, G = orc.mse_grad(cur, Z[s:s + bs], Y[s:s + bs])
        ref_losses.append(loss)
        g = np.concatenate([np.concatenate([gw.ravel() for gw, _ in G]),
                            np.concatenate([gb.ravel() for _, gb in G])])
        orc.adam(P, g, m, v, k + 1, lr)
    assert np.max(np.abs(losses - ref_losses) / np.array(ref_losses)) < 1e-4
    got = ctl.get_params()
    Pg = np.concatenate([np.concatenate([w.ravel() for w, _ in got]),
                         np.concatenate([b.ravel() for _, b in got])])
    assert np.linalg.norm(Pg - P) / np.linalg.norm(P - P0) < 1e-3


def test_learned_residual_beats_nominal_on_drag_plant(rtn, orc):
    # train 17-64-64-3 on drag residuals, then track figure-8s on the drag
    # plant: the learned model must track better than the nominal model
    n = 1 << 16
    X, U = W.training_samples(n, 7)
    Xd, Ud = dev(X), dev(U)
    layers = [(f32(w), f32(b)) for w, b in W.xavier_mlp([17, 64, 64, 3], 3)]
    B, steps = 32, 150
    prob = W.make_problem("cfg2_fp32_batch", seed=4, B=B)
    learn = rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], quad=QUAD, layers=layers)
    Yd = learn.drag_targets(Xd)
    losses = learn.train(Xd, Ud, Yd, epochs=20, batch=512, lr=1e-3)
    assert losses[-20:].mean() < 0.1 * losses[:20].mean()
    nominal = rtn.Controller(prob["N"], prob["dt"], prob["Q"], prob["R"], quad=QUAD)
    xrt, urt = W.trajectory_refs(prob, steps)
    rmse = {}
    for name, c in (("learned", learn), ("nominal", nominal)):
        x0 = xrt[:, 0].copy()
        c.reset(dev(x0))
        xp = torch.as_tensor(x0, dtype=torch.float64, device="cuda")
        traj, _ = c.closed_loop(steps, dev(xrt), dev(urt), xp, plant="drag")
        p = traj[:, :, :3].double().cpu().numpy()
        err = np.linalg.norm(p - xrt[:, 1:steps + 1, :3].transpose(1, 0, 2), axis=2)
        rmse[name] = np.sqrt((err[steps // 3:] ** 2).mean())
    assert rmse["learned"] < 0.7 * rmse["nominal"], rmse
